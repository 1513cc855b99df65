// g4_internal.cuh -- internal types and helpers of the sm_103a gravity library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "g4.h"

#define G4_KEYBITS 21
#define G4_MAXLEVEL 21
#define G4_NLEVELS 22
#define G4_WALK_QCAP 4096            // walk frontier ring per warp (power of two)
#define G4_WALK_BLOCKS_PER_SM 8      // persistent walk: 4-warp blocks launched per SM
#define G4_ITEM_SPLIT_MAX 8          // largest number of source parts of a split walk group

// -------------------------------------------------------------------------------------------
// error reporting (thread-local last error, status codes)
// -------------------------------------------------------------------------------------------
g4_status g4_fail(g4_status st, const char *fmt, ...);
g4_status g4_cuda_check(cudaError_t e, const char *what);
g4_status g4_launch_check(const char *what, int launches);
int g4_num_sms();

// device-side error flags of a tree handle
enum : int { G4_FLAG_CAPACITY = 1, G4_FLAG_TIMEOUT = 2, G4_FLAG_LISTCAP = 4 };

// -------------------------------------------------------------------------------------------
// node record (64 bytes, depth-first order).  The walk reads one record per visited node.
// -------------------------------------------------------------------------------------------
struct __align__(16) G4Node {
    uint32_t cx, cy, cz;  // geometric centre, integer units
    uint32_t meta;        // bits 0-4: level, bit 5: leaf
    float sx, sy, sz;     // centre of mass minus geometric centre (physical units)
    float mass;
    int32_t first, count, next, parent;
    float amin;           // minimum |a_old| of the node's particles (FMM criterion)
    float hmax;           // 2.8 * largest softening among the node's particles
    float hmin;           // 2.8 * smallest softening among the node's particles
    int32_t nchild;       // number of daughters (0 for a leaf)
};
static_assert(sizeof(G4Node) == 64, "node record must be 64 bytes");

__host__ __device__ constexpr int g4_nmono(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }
// number of stored moment components of orders 2..p, padded to a multiple of 4
__host__ __device__ constexpr int g4_nq_raw(int p) { return p < 2 ? 0 : g4_nmono(p) - 4; }
__host__ __device__ constexpr int g4_nq(int p) { return (g4_nq_raw(p) + 3) & ~3; }

// multi-index (a,b,c) -> position among all monomials of orders 0..n (order, then a desc,
// then b desc).  Moments of orders >= 2 are stored at position - 4.
__host__ __device__ constexpr int g4_midx(int a, int b, int c)
{
    return (a + b + c) * (a + b + c + 1) * (a + b + c + 2) / 6 +
           (b + c) * (b + c + 1) / 2 + c;
}

// -------------------------------------------------------------------------------------------
// tree handle
// -------------------------------------------------------------------------------------------
struct g4_tree_s {
    int64_t n_max = 0, cap = 0;
    int device = 0;
    // level-ordered (breadth-first) build arrays, capacity `cap`
    int32_t *b_first = nullptr, *b_count = nullptr, *b_child = nullptr, *b_nchild = nullptr;
    int32_t *b_size = nullptr, *b_dfs = nullptr, *b_parent = nullptr;
    int32_t *lvl = nullptr;       // [0..G4_NLEVELS]: offsets, [G4_NLEVELS+1 ..]: counts
    int32_t *d_flags = nullptr;   // device error flags
    // depth-first node arrays
    G4Node *node = nullptr;
    float *q = nullptr;           // cap x g4_nq(G4_MAX_ORDER) FP32 moments (orders 2..p)
    void *walk_queue = nullptr;   // walk frontier rings (allocated on the first walk)
    int walk_qcap = 0;            // their capacity per warp
    // walk copies (allocated on the first walk): node records in level order with
    // next = first daughter (level order) and parent = depth-first index, and the particles
    // as 16-byte records (x, y, z, mass bits)
    G4Node *wnode = nullptr;
    uint4 *wpart = nullptr;
    int64_t moments_stamp = 0, wnode_stamp = -1;
    double *qd = nullptr;         // FP64 mirror (precision 1 only): cap x (4 + nq)
    int built_n = -1;
    // forest (several independent systems in one handle); n_sys = 0 for a single system
    int n_sys = 0;
    const int32_t *sys_first = nullptr;   // caller device array [n_sys + 1], sorted-order offsets
    const double *sys_box = nullptr;      // caller device array [n_sys], box size per system
    int32_t *sys_goff = nullptr;          // library: walk-group offsets per system [n_sys + 1]
    int sys_cap = 0;
    // optional walk schedule: order in which the 32-sink groups are handed out
    const int32_t *group_order = nullptr;
    int64_t group_order_n = 0;
    // optional cost-partitioned work items: (first sink, count) pairs, count on the device
    const int32_t *items = nullptr;
    const int32_t *n_items = nullptr;
    int64_t items_cap = 0, items_n_sinks = -1;
    float *part_buf = nullptr;    // partial sums of split groups (see g4_tree_set_work_items)
    int32_t *part_cnt = nullptr;
    int part_cap = 0;
    int moments_order = -1;
    int moments_fp64 = 0;
    // Ewald correction grid of the pure periodic tree (built on first use, see g4_ewald.cu)
    double *ew64 = nullptr;
    float *ew32 = nullptr;
    double ew_L = 0.0;
    int ew_nt = -1;
    // host copies filled by g4_tree_status
    int64_t n_nodes_host = -1;
};

// -------------------------------------------------------------------------------------------
// small device helpers
// -------------------------------------------------------------------------------------------
__device__ __forceinline__ float g4_isep(uint32_t a, uint32_t b, float scale)
{
    // signed integer difference a - b: the two's complement gives the nearest periodic image
    // (Sec. 2.10); for isolated sets all differences are below 2^31 by construction.
    return (float)(int32_t)(a - b) * scale;
}
__device__ __forceinline__ double g4_isep_d(uint32_t a, uint32_t b, double scale)
{
    return (double)(int32_t)(a - b) * scale;
}

// launch helpers
static inline int g4_blocks_for(int64_t work, int threads, int per_sm = 8)
{
    int64_t b = (work + threads - 1) / threads;
    int64_t cap = (int64_t)g4_num_sms() * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// system of sorted particle j in a forest (binary search over the systems' first indices)
__device__ __forceinline__ int g4_system_of(const int32_t *sys_first, int n_sys, int j)
{
    int lo = 0, hi = n_sys - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sys_first[mid] <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// internal entry points shared between translation units
g4_status g4_sort_pairs_u64(const uint64_t *keys_in, uint64_t *keys_out, int32_t *vals_out,
                            int64_t n, void *workspace, size_t ws_bytes, int key_bits,
                            cudaStream_t st);
size_t g4_sort_workspace_bytes(int64_t n);
g4_status g4_particle_records(struct g4_tree_s *t, const uint32_t *pos_sorted, const float *mass_sorted,
                              int n, cudaStream_t st);
