// g4_fmm_args.cuh -- launch arguments of the FMM dual walk, shared by the entry points
// (g4_fmm.cu) and the kernel variants (g4_fmm_variant.cu).
#pragma once
#include "g4_internal.cuh"
#include "g4_kernels.cuh"
#include "g4_ewald.cuh"

namespace g4fmm {

using g4k::PairF;

constexpr int FMM_THREADS = 128;
constexpr int FMM_WARPS = FMM_THREADS / 32;
constexpr int FMM_STACK = 512;      // per-warp stack of the particle walk at leaf sinks
constexpr int FMM_P2PBUF = 96;      // per-warp buffer of particle-pair entries (one chunk)

enum : int { D_DROP = 0, D_ACCEPT = 1, D_P2P = 2, D_OPEN = 3, D_SELF = 4 };

struct FmmArgs {
    const uint32_t *pos;
    const float *mass;
    const uint8_t *cls;
    const float *aold;         // |a_old| per sorted particle (nullable: 0)
    int n;
    const int32_t *lvl;
    const int32_t *b_dfs;
    const G4Node *node;
    const int32_t *kids;       // per depth-first node: its daughters' depth-first indices (8)
    const float *q;
    const double *qd;          // FP64 node data (precision 1): (4 + nq) doubles per node --
                               // centre-of-mass offset, mass, the moments of q
    int nq;
    void *T_own, *T_tot;       // field tensors, float or double (the interaction type)
    int2 *D0, *D1;             // pass-down candidate lists, by level parity: (node, 0) or
                               // (-(first particle) - 1, particle mask)
    int64_t dcap;
    int32_t *dcount;           // [2] list fill counters
    int32_t *Doff, *Dlen;      // per node: its pass-down list
    uint32_t *m2l_own, *m2l_cum;
    int32_t *flags;
    float *acc, *pot;
    uint32_t *counts;          // 3 x n: particle pairs, particle-node terms, node-node fields
    double *momentum;
    double scale, G, alpha, theta2, rcut2, as, box;
    float h_cls[G4_MAX_EPS_CLASSES];
    int exclusion, pp_cut, keep_qp;
    int soft_nodes;            // 1: softened multipoles under the rule of Sec. 2.7
    int ewald;                 // pure periodic FMM with the Ewald correction (Sec. 2.2.4)
    int periodic;
    G4EwaldView ew;
    // particle-particle phase (shared with the tree walk)
    const uint4 *wpart;        // particles as (x, y, z, mass bits)
    float rcut2f, asf, figs, rc2i;
    PairF pf;
    // deferred particle pairs: chunks of (first, count, lane mask, -) entries per sink leaf,
    // chained in the order the sink's warp found them; lane mask 0 = every particle of the
    // sink leaf, otherwise the lanes of the 32-particle sink chunk named in the chunk header
    int4 *p2p_src;             // entries
    int4 *p2p_chunk;           // (offset, count, next chunk, sink chunk)
    int32_t *p2p_head;         // per node: first chunk of a sink leaf, -1 if none
    int32_t *p2p_sinks;        // sink leaves with particle pairs
    int32_t *p2p_fill;         // [0] list entries, [1] chunks, [2] sink leaves
    int64_t p2p_cap, chunk_cap;
};

// one (order, TreePM, interaction type) variant of the dual walk, defined in
// g4_fmm_variant.cu; R = double is the FP64 reference mode (decisions as in FP32, every
// expansion, field and particle pair in FP64 from the FP64 node data)
template <int P, bool TREEPM, typename R> void run_variant(const FmmArgs &A, bool geom, cudaStream_t st);

}  // namespace g4fmm
