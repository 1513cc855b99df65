// g4_walk.cu -- one-sided tree walk (Sec. 2.2.3) with the relative opening criterion
// (Eq. eqnrelcriterion) and the TreePM short-range kernel (Sec. 2.3), plus a GPU direct sum.
//
// Work decomposition: a warp owns a group of 32 PH-consecutive sinks (one per lane) and walks
// the tree breadth-first for the whole group (TreePM: runs of UNION_G consecutive groups share
// one walk where that gives each group exactly its own leaves, see union_walk).  The frontier holds (node, mask of the lanes
// still walking there) entries in a per-warp ring; each step takes 32 entries, one per lane
// (coalesced 64-byte records of the level-ordered node copy).  Group-level tests are
// conservative (a cube beyond r_cut of the group's bounding box is skipped for all lanes); a
// node some sink could use as a multipole gets the exact per-lane decision of the
// single-particle walk (skip, open, or accept: particle-node term, the lane leaves the
// subtree).  A lane's cutoff skip is hereditary and treated as "open" (the pair cutoff
// removes the leaves below), so every lane's interaction set is exactly that of a
// single-particle walk.  Leaves collect in a pending list; the particle-particle phase
// (g4_pp.cuh) evaluates them.  Groups -- or, with a cost-model schedule, parts of groups --
// come from a device work counter, so warps that finish early pull more (persistent kernel).
#include <cuda_fp16.h>

#include "g4_internal.cuh"
#include "g4_kernels.cuh"
#include "g4_ewald.cuh"
#include "g4_pp.cuh"

namespace {

using namespace g4k;

struct WalkArgs {
    const uint32_t *pos;
    const float *mass;
    const uint8_t *cls;
    const float *aold;
    const int32_t *active;
    int n, n_sinks;
    const int32_t *lvl;        // lvl[G4_NLEVELS] = node count
    const G4Node *node;        // depth-first records
    const G4Node *wnode;       // level-ordered copy: next = first daughter, parent = depth-first index
    const uint4 *wpart;        // particles as (x, y, z, mass bits)
    const float *q;
    const double *qd;          // FP64 node data (precision 1)
    int nq;
    float *acc, *pot;
    uint32_t *counts;
    int *work;                 // group counter
    int32_t *flags;            // tree error flags
    int2 *queue;               // per-warp frontier rings (level-ordered node, lane mask)
    int qcap;                  // ring capacity per warp (a power of two)
    int4 *ul_cube;             // per-warp union leaf lists: cube centre, level / meta
    int2 *ul_fc;               //   and (first particle, count); null: no union walks
    const int32_t *sys_first, *sys_goff;
    const double *sys_box;
    int n_sys;
    const int32_t *group_order;   // optional schedule (longest predicted cost first)
    const int32_t *operm;         // optional output order: acc/pot of sorted sink i go to operm[i]
    long long watchdog;           // > 0: a warp stops taking work after this many SM cycles
    const int4 *items;            // optional work items (first sink, count, part | parts << 8,
    const int32_t *n_items;       //   split slot); their number on the device
    int gs;                       // sinks per group (8, 16 or 32)
    float *part_buf;              // partial sums of split groups: [slot][part][lane][6]
    int32_t *part_cnt;            // arrivals per split slot (zero between walks)
    int part_cap;                 // split slots available
    double scale;
    double G, alpha, theta2, rcut2, as;
    double box;
    float Gf, alphaf, theta2f, rcut2f, asf;   // FP32 copies (no FP64 conversions in the loops)
    double inv_as, igs;                      // 1 / as; integer units per length unit (box)
    float h_cls[G4_MAX_EPS_CLASSES];
    int exclusion, pp_cut;
    int soft_nodes;               // GADGET-4 softened-node rule (Sec. 2.7)
    int ewald;                    // pure periodic tree with the Ewald correction (Sec. 2.2.4)
    G4EwaldView ew;
};


enum : int { ACT_NONE = 0, ACT_SKIP = 1, ACT_OPEN = 2, ACT_ACCEPT = 3, ACT_LEAF = 4 };

template <int P, typename T> __device__ __forceinline__ T ipow(T x)
{
    T r = T(1);
#pragma unroll
    for (int i = 0; i < P; i++) r *= x;
    return r;
}

constexpr int WALK_THREADS = 128;
constexpr int WALK_WARPS = WALK_THREADS / 32;
constexpr int LEAF_BUF = 256;   // pending leaves: a whole group's leaves usually fit (one flush)
constexpr int QCAP = G4_WALK_QCAP;   // frontier capacity per warp with the TreePM cutoff
constexpr int QCAP_TREE = 4 * QCAP;  // without a cutoff (large sets: the frontier is wider)
// minimum resident blocks per SM requested from the compiler for the FP32 walks of order <= 3
// (caps their registers; other instances keep the compiler's choice)
#ifndef G4_WALK_MIN_BLOCKS
#define G4_WALK_MIN_BLOCKS 4
#endif
// consecutive groups that share one union walk (1: every group walks on its own)
#ifndef G4_WALK_UNION
#define G4_WALK_UNION 4
#endif
constexpr int UNION_G = G4_WALK_UNION;
constexpr int ULCAP = 2048;     // union leaves per warp

// per-warp shared state: the pending leaf list of the group, the staged sources, the sinks
struct WalkSmem : PPSmem<LEAF_BUF> {
    float4 sink[32];            // sinks relative to the group centre, opening threshold
    int ul_n, ub;               // union leaf list: length (-1: none), next entry to take
    int rg, rn, rq, rul;        // current run of groups: first, count, next, its union list
};

// Per-lane decision for an internal node (the single-particle walk's rule): skip beyond the
// TreePM cutoff, open when inside the node / its exclusion zone / the softening range or
// when the opening criterion fails, otherwise accept the multipole.
template <int P, typename T, bool TREEPM, bool GEOM>
__device__ __forceinline__ int exact_decision(const WalkArgs &A, const G4Node &nd, int k,
                                              uint32_t xi, uint32_t yi, uint32_t zi, T hi, T crit,
                                              double gscale, double gbox)
{
    const T scale = (T)gscale;
    const T side = ldexp((T)gbox, -(int)(nd.meta & 31u)), half = T(0.5) * side;
    const T dcx = (T)(int32_t)(nd.cx - xi) * scale;
    const T dcy = (T)(int32_t)(nd.cy - yi) * scale;
    const T dcz = (T)(int32_t)(nd.cz - zi) * scale;
    if (TREEPM) {
        const T ex = fmax(fabs(dcx) - half, T(0));
        const T ey = fmax(fabs(dcy) - half, T(0));
        const T ez = fmax(fabs(dcz) - half, T(0));
        if (ex * ex + ey * ey + ez * ez > par<T>(A.rcut2, A.rcut2f)) return ACT_SKIP;
    }
    T ox, oy, oz, M;
    if (sizeof(T) == 8 && A.qd) {
        const double *dd = A.qd + (size_t)k * (4 + A.nq);
        ox = (T)dd[0]; oy = (T)dd[1]; oz = (T)dd[2]; M = (T)dd[3];
    } else {
        ox = (T)nd.sx; oy = (T)nd.sy; oz = (T)nd.sz; M = (T)nd.mass;
    }
    const T rx = dcx + ox, ry = dcy + oy, rz = dcz + oz;
    const T r2 = rx * rx + ry * ry + rz * rz;
    const T dmax = fmax(fabs(dcx), fmax(fabs(dcy), fabs(dcz)));
    const T h = fmax(hi, (T)nd.hmax);   // 2.8 eps_ij
    // closer than 2.8 eps_ij: GADGET-3 opens; GADGET-4 opens only a node that mixes smaller
    // softenings when the particle's own is smaller too, else uses the softened multipole
    const bool soft_open = r2 < h * h && (!A.soft_nodes || (hi < h && (T)nd.hmin < h));
    bool open = (dmax <= half) || (A.exclusion && dmax < side) || soft_open;
    if (!open) {
        if (GEOM) open = side * side >= par<T>(A.theta2, A.theta2f) * r2;
        else open = !(par<T>(A.G, A.Gf) * M * ipow<P>(side) < crit * ipow<P + 2>(sqrt(r2)));
    }
    return open ? ACT_OPEN : ACT_ACCEPT;
}

// Union walk for a run of consecutive groups (TreePM with the pair cutoff, plain sink order):
// one breadth-first walk for the bounding box of all their sinks collects the leaves within
// reach, with the single-group tests made slightly more conservative (cutoff slack 2e-4
// instead of 1e-4, the multipole tests' margins doubled), so that whatever a group's own walk
// would skip or find unusable the union walk skips or finds unusable too.  If no node could
// serve any of the sinks as a multipole, a group's own walk expands every node it reaches and
// keeps the leaves that pass its cutoff test, in breadth-first order; each group then takes
// the union's leaves that pass its own cutoff test, in the union's (the same) order, instead
// of walking.  Returns the number of leaves, or -1 if some node needs per-sink decisions or a
// buffer would overflow (the groups then walk on their own).
template <int P, bool GEOM>
__device__ __noinline__ int union_walk(const WalkArgs &A, int2 *Q, int4 *UC, int2 *UF, int lane, int s0,
                          int s_end)
{
    const unsigned lt = (1u << lane) - 1u;
    const double gscale = A.box * (1.0 / 4294967296.0);
    const float fscale = (float)gscale, fbox = (float)A.box;
    const uint4 p0 = A.wpart[s0];
    int lox = 0x7fffffff, hix = -0x7fffffff - 1, loy = lox, hiy = hix, loz = lox, hiz = hix;
    float critmax = 0.f;
    for (int s = s0 + lane; s < s_end; s += 32) {
        const uint4 p = A.wpart[s];
        const int ox = (int32_t)(p.x - p0.x), oy = (int32_t)(p.y - p0.y), oz = (int32_t)(p.z - p0.z);
        lox = min(lox, ox);
        hix = max(hix, ox);
        loy = min(loy, oy);
        hiy = max(hiy, oy);
        loz = min(loz, oz);
        hiz = max(hiz, oz);
        if (!GEOM) critmax = fmaxf(critmax, A.alphaf * (A.aold ? A.aold[s] : 0.f));
    }
    lox = __reduce_min_sync(0xffffffffu, lox);
    hix = __reduce_max_sync(0xffffffffu, hix);
    loy = __reduce_min_sync(0xffffffffu, loy);
    hiy = __reduce_max_sync(0xffffffffu, hiy);
    loz = __reduce_min_sync(0xffffffffu, loz);
    hiz = __reduce_max_sync(0xffffffffu, hiz);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) critmax = fmaxf(critmax, __shfl_xor_sync(0xffffffffu, critmax, o));
    critmax *= 1.002f;
    const uint32_t gcx = p0.x + (uint32_t)(int)(((long long)lox + hix) >> 1);
    const uint32_t gcy = p0.y + (uint32_t)(int)(((long long)loy + hiy) >> 1);
    const uint32_t gcz = p0.z + (uint32_t)(int)(((long long)loz + hiz) >> 1);
    const float ghx = (0.5f * (float)((long long)hix - lox) + 2.f) * fscale;
    const float ghy = (0.5f * (float)((long long)hiy - loy) + 2.f) * fscale;
    const float ghz = (0.5f * (float)((long long)hiz - loz) + 2.f) * fscale;
    int head = 0, tail = 1, nl = 0;
    if (lane == 0) Q[0] = make_int2(0, -1);
    __syncwarp();
    while (head < tail) {
        const int cnt = min(32, tail - head);
        const bool ve = lane < cnt;
        int d = 0;
        if (ve) d = Q[(head + lane) & (A.qcap - 1)].x;
        head += cnt;
        __syncwarp();
        G4Node nd;
        if (ve) nd = load_node(A.wnode + d);
        const bool leaf = ve && (nd.meta & 32u);
        bool gskip = !ve, maybe = false;
        if (ve) {
            const float side = ldexpf(fbox, -(int)(nd.meta & 31u)), half = 0.5f * side;
            const float dcx = (float)(int32_t)(nd.cx - gcx) * fscale;
            const float dcy = (float)(int32_t)(nd.cy - gcy) * fscale;
            const float dcz = (float)(int32_t)(nd.cz - gcz) * fscale;
            const float ex = fmaxf(fabsf(dcx) - half - ghx, 0.f);
            const float ey = fmaxf(fabsf(dcy) - half - ghy, 0.f);
            const float ez = fmaxf(fabsf(dcz) - half - ghz, 0.f);
            gskip = ex * ex + ey * ey + ez * ez > 1.0002f * A.rcut2f;
            if (!gskip && !leaf) {
                bool none = false;
                if (A.exclusion && fmaxf(fabsf(dcx) + ghx, fmaxf(fabsf(dcy) + ghy, fabsf(dcz) + ghz)) < 0.998f * side)
                    none = true;
                const float fx = fabsf(dcx + nd.sx) + ghx, fy = fabsf(dcy + nd.sy) + ghy,
                            fz = fabsf(dcz + nd.sz) + ghz;
                const float rmax2 = (fx * fx + fy * fy + fz * fz) * 1.002f;
                if (!A.soft_nodes && rmax2 < nd.hmax * nd.hmax) none = true;
                // a sink can use the node only within r_cut of its cube, so its distance to the
                // centre of mass is below r_cut + the cube's diagonal
                const float rlim = fminf(sqrtf(rmax2), (sqrtf(A.rcut2f) + 1.7320509f * side) * 1.002f);
                if (GEOM) {
                    if (side * side >= A.theta2f * rlim * rlim) none = true;
                } else {
                    if (!(A.Gf * nd.mass * ipow<P>(side) < critmax * ipow<P + 2>(rlim))) none = true;
                }
                maybe = !none;
            }
        }
        if (__any_sync(0xffffffffu, maybe)) return -1;
        const bool addleaf = leaf && !gskip;
        const unsigned lm = __ballot_sync(0xffffffffu, addleaf);
        if (nl + __popc(lm) > ULCAP) return -1;
        if (addleaf) {
            const int pos = nl + __popc(lm & lt);
            UC[pos] = make_int4((int)nd.cx, (int)nd.cy, (int)nd.cz, (int)nd.meta);
            UF[pos] = make_int2(nd.first, nd.count);
        }
        nl += __popc(lm);
        const bool expand = ve && !leaf && !gskip;
        const int nch = expand ? nd.nchild : 0;
        int pre = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += y;
        }
        const int tot = __shfl_sync(0xffffffffu, pre, 31);
        pre -= nch;
        if (tail + tot - head > A.qcap) return -1;
        for (int c = 0; c < nch; c++) Q[(tail + pre + c) & (A.qcap - 1)] = make_int2(nd.next + c, -1);
        tail += tot;
        __syncwarp();
    }
    return nl;
}

// The group walk.  Nodes are scanned in depth-first order in windows of 32 (one node per lane,
// coalesced loads).  A node is visited unless an earlier node of the window that the group
// skipped covers it (prefix maximum of the skipped subtrees' ends).  Group-level tests are
// conservative: a node is skipped only if its cube is beyond r_cut of the group's bounding
// box, and it needs per-lane decisions ("maybe") only if some sink could possibly accept its
// multipole.  Leaves go to the pending list with the mask of lanes that reach them; "maybe"
// nodes get the exact per-lane decision, and a lane that accepts or skips one resumes after
// its subtree, exactly as a single-particle walk would.
template <int P, typename T, bool TREEPM, bool GEOM>
__global__ void __launch_bounds__(WALK_THREADS, (sizeof(T) == 4 && P <= 3) ? G4_WALK_MIN_BLOCKS : 1)
k_walk(const WalkArgs A)
{
    __shared__ WalkSmem smem[WALK_WARPS];
    WalkSmem &S = smem[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    if (*A.flags & G4_FLAG_CAPACITY) return;   // incomplete tree: outputs left untouched
    int2 *Q = A.queue + (size_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * A.qcap;
    const int ngroups = A.items ? *A.n_items
                                : (A.n_sys ? A.sys_goff[A.n_sys] : (A.n_sinks + A.gs - 1) / A.gs);
    // a run of UNION_G consecutive groups shares one union walk where that is exact (see
    // union_walk); ul_n >= 0: the group takes its leaves from that walk's list
    const bool uni = UNION_G > 1 && TREEPM && A.ul_cube && !A.items && !A.group_order && !A.n_sys &&
                     !A.active && A.gs == 32 && A.pp_cut;
    auto group = [&](int g, int ul_n) {
        // the group's sinks, node range and box (a forest walks only its own system's tree)
        int s0 = g * A.gs, s_end = min(A.n_sinks, s0 + A.gs), k = 0;   // k: root, level-ordered
        int kp = 0, Kp = 1, pslot = -1;               // part of a split group
        if (A.items) {
            const int4 it = A.items[g];
            s0 = it.x;
            s_end = min(A.n_sinks, s0 + it.y);
            kp = it.z & 255;
            Kp = it.z >> 8;
            pslot = it.w;
            if (s0 < 0 || s0 >= s_end || it.y > 32 || Kp < 1 || Kp > G4_ITEM_SPLIT_MAX ||
                kp >= Kp || (Kp > 1 && (pslot < 0 || pslot >= A.part_cap))) {
                if (lane == 0) atomicOr(A.flags, G4_FLAG_LISTCAP);   // malformed item: reported
                return;
            }
        }
        double gbox = A.box;
        if (A.n_sys) {
            int lo = 0, hi_ = A.n_sys - 1;
            while (lo < hi_) {
                const int mid = (lo + hi_ + 1) >> 1;
                if (A.sys_goff[mid] <= g) lo = mid;
                else hi_ = mid - 1;
            }
            s0 = A.sys_first[lo] + (g - A.sys_goff[lo]) * 32;
            s_end = A.sys_first[lo + 1];
            k = lo;   // forest roots are the first n_sys level-ordered nodes
            gbox = A.sys_box[lo];
        }
        const double gscale = gbox * (1.0 / 4294967296.0);
        const float fscale = (float)gscale, fbox = (float)gbox;
        const int s = s0 + lane;
        const bool valid = s < s_end;
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        const int i = valid ? (A.active ? A.active[s] : s) : (A.active ? A.active[s0] : s0);
        const uint4 pi_ = A.wpart[i];
        const uint32_t xi = pi_.x, yi = pi_.y, zi = pi_.z;
        const T hi = (T)A.h_cls[A.cls ? A.cls[i] : 0];
        const T crit = GEOM ? T(0) : par<T>(A.alpha, A.alphaf) * (T)(A.aold ? A.aold[i] : 0.f);
        // group bounding box, in integer offsets from lane 0's sink
        const uint32_t x0 = __shfl_sync(0xffffffffu, xi, 0), y0 = __shfl_sync(0xffffffffu, yi, 0),
                       z0 = __shfl_sync(0xffffffffu, zi, 0);
        const int ox = (int32_t)(xi - x0), oy = (int32_t)(yi - y0), oz = (int32_t)(zi - z0);
        const int lox = __reduce_min_sync(0xffffffffu, ox), hix = __reduce_max_sync(0xffffffffu, ox);
        const int loy = __reduce_min_sync(0xffffffffu, oy), hiy = __reduce_max_sync(0xffffffffu, oy);
        const int loz = __reduce_min_sync(0xffffffffu, oz), hiz = __reduce_max_sync(0xffffffffu, oz);
        const uint32_t gcx = x0 + (uint32_t)(int)(((long long)lox + hix) >> 1);
        const uint32_t gcy = y0 + (uint32_t)(int)(((long long)loy + hiy) >> 1);
        const uint32_t gcz = z0 + (uint32_t)(int)(((long long)loz + hiz) >> 1);
        const float xr = (float)(int32_t)(xi - gcx) * fscale, yr = (float)(int32_t)(yi - gcy) * fscale,
                    zr = (float)(int32_t)(zi - gcz) * fscale;
        const float ghx = (0.5f * (float)((long long)hix - lox) + 2.f) * fscale;
        const float ghy = (0.5f * (float)((long long)hiy - loy) + 2.f) * fscale;
        const float ghz = (0.5f * (float)((long long)hiz - loz) + 2.f) * fscale;
        S.sink[lane] = make_float4(xr, yr, zr, valid ? (GEOM ? 1.f : (float)crit) : -1.f);
        __syncwarp();
        float critmax = (float)crit;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) critmax = fmaxf(critmax, __shfl_xor_sync(0xffffffffu, critmax, o));
        critmax *= 1.001f;

        // FP32 TreePM: particle-particle sums in integer-grid length units (see pair_treepm_fast)
        constexpr bool INTU = TREEPM && sizeof(T) == 4;
        const double igs = A.n_sys ? 4294967296.0 / gbox : A.igs;   // integer units per length unit
        const float figs = (float)igs;
        const PairF pf = make_pairf(A.as * gscale, A.inv_as * igs);
        const float rc2i = (float)(A.rcut2 * igs * igs);
        T ax = T(0), ay = T(0), az = T(0), ap = T(0);     // particle-particle sums
        T bx = T(0), by = T(0), bz = T(0), bp = T(0);     // particle-node sums
        uint32_t npp = 0, npn = 0;
        if (!TREEPM && A.ewald && kp == 0) {
            // the sink's own periodic images: + G m_i psi(0) in the potential, no force
            T D0[1];
            ewald_dpsi<0, T>(A.ew, T(0), T(0), T(0), D0);
            bp -= (T)__uint_as_float(pi_.w) * D0[0];
        }
        // breadth-first frontier of (node, lanes still walking there), 32 entries per step
        int head = 0, tail = ul_n >= 0 ? 0 : 1, nleaf = 0;
        if (lane == 0) {
            if (ul_n < 0) Q[0] = make_int2(k, (int)vmask);
            S.ul_n = ul_n;
            S.ub = 0;
        }
        __syncwarp();
        for (;;) {
            // (the union list's state lives in shared memory, not in registers)
            const int uln = S.ul_n, ub = S.ub;
            const bool more = uln >= 0 ? ub < uln : head < tail;
            // a step adds at most 32 leaves: flush before the list could overflow, and at the end
            if (nleaf > LEAF_BUF - 32 || (!more && nleaf > 0)) {
                pp_flush<T, TREEPM>(A, S, nleaf, lane, i, xi, yi, zi, gcx, gcy, gcz, xr, yr, zr, vmask,
                                    INTU ? hi * (T)figs : hi, ax, ay, az, ap, npp, gscale, figs, pf, rc2i,
                                    kp, Kp);
                nleaf = 0;
            }
            if (!more) break;
            if (uln >= 0) {
                // the union walk's leaves that pass this group's cutoff test (the test of the
                // breadth-first walk below, on the same leaf records)
                const size_t w0 = (size_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * ULCAP;
                const int e = ub + lane;
                __syncwarp();
                if (lane == 0) S.ub = ub + 32;
                bool keep = false;
                int2 fc = make_int2(0, 0);
                if (e < uln) {
                    const int4 c = A.ul_cube[w0 + e];
                    fc = A.ul_fc[w0 + e];
                    const float side = ldexpf(fbox, -(int)((uint32_t)c.w & 31u)), half = 0.5f * side;
                    const float dcx = (float)(int32_t)((uint32_t)c.x - gcx) * fscale;
                    const float dcy = (float)(int32_t)((uint32_t)c.y - gcy) * fscale;
                    const float dcz = (float)(int32_t)((uint32_t)c.z - gcz) * fscale;
                    const float ex = fmaxf(fabsf(dcx) - half - ghx, 0.f);
                    const float ey = fmaxf(fabsf(dcy) - half - ghy, 0.f);
                    const float ez = fmaxf(fabsf(dcz) - half - ghz, 0.f);
                    keep = !(ex * ex + ey * ey + ez * ez > 1.0001f * A.rcut2f);
                }
                const unsigned lm = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int pos = nleaf + __popc(lm & lt);
                    S.first[pos] = fc.x;
                    S.count[pos] = fc.y;
                    S.mask[pos] = vmask;
                }
                nleaf += __popc(lm);
                __syncwarp();
                continue;
            }
            const int cnt = min(32, tail - head);
            const bool ve = lane < cnt;
            int d = 0;
            unsigned m = 0u;
            if (ve) {
                const int2 qe = Q[(head + lane) & (A.qcap - 1)];
                d = qe.x;
                m = (unsigned)qe.y;
            }
            head += cnt;
            __syncwarp();
            G4Node nd;
            if (ve) nd = load_node(A.wnode + d);
            const bool leaf = ve && (nd.meta & 32u);
            bool gskip = !ve, maybe = false;
            if (ve) {
                const float side = ldexpf(fbox, -(int)(nd.meta & 31u)), half = 0.5f * side;
                const float dcx = (float)(int32_t)(nd.cx - gcx) * fscale;
                const float dcy = (float)(int32_t)(nd.cy - gcy) * fscale;
                const float dcz = (float)(int32_t)(nd.cz - gcz) * fscale;
                if (TREEPM) {
                    const float ex = fmaxf(fabsf(dcx) - half - ghx, 0.f);
                    const float ey = fmaxf(fabsf(dcy) - half - ghy, 0.f);
                    const float ez = fmaxf(fabsf(dcz) - half - ghz, 0.f);
                    gskip = ex * ex + ey * ey + ez * ez > 1.0001f * A.rcut2f;
                }
                if (!gskip && !leaf) {
                    // can any sink of the group use this node's multipole?
                    bool none = false;
                    if (A.exclusion && fmaxf(fabsf(dcx) + ghx, fmaxf(fabsf(dcy) + ghy, fabsf(dcz) + ghz)) < 0.999f * side)
                        none = true;
                    const float fx = fabsf(dcx + nd.sx) + ghx, fy = fabsf(dcy + nd.sy) + ghy,
                                fz = fabsf(dcz + nd.sz) + ghz;
                    const float rmax2 = (fx * fx + fy * fy + fz * fz) * 1.001f;
                    if (!A.soft_nodes && rmax2 < nd.hmax * nd.hmax) none = true;
                    // TreePM: a sink uses the node only within r_cut of its cube, so its distance
                    // to the centre of mass is below r_cut + the cube's diagonal
                    const float rlim = TREEPM ? fminf(sqrtf(rmax2), (sqrtf(A.rcut2f) + 1.7320509f * side) * 1.001f)
                                              : sqrtf(rmax2);
                    if (GEOM) {
                        if (side * side >= A.theta2f * rlim * rlim) none = true;
                    } else {
                        if (!(A.Gf * nd.mass * ipow<P>(side) < critmax * ipow<P + 2>(rlim))) none = true;
                    }
                    maybe = !none;
                }
            }
            if (__any_sync(0xffffffffu, maybe)) {
                // necessary condition for a sink to use the multipole: its own opening criterion
                // (exclusion, softening and inside-node tests can only open the node)
                bool any = false;
                if (maybe) {
                    const float side = ldexpf(fbox, -(int)(nd.meta & 31u));
                    const float cx = (float)(int32_t)(nd.cx - gcx) * fscale + nd.sx;
                    const float cy = (float)(int32_t)(nd.cy - gcy) * fscale + nd.sy;
                    const float cz = (float)(int32_t)(nd.cz - gcz) * fscale + nd.sz;
                    const float lhs = 0.999f * (GEOM ? side * side : A.Gf * nd.mass * ipow<P>(side));
                    for (int u = 0; u < 32 && !any; u++) {
                        if (!((m >> u) & 1u)) continue;
                        const float4 sk = S.sink[u];
                        const float dx = cx - sk.x, dy = cy - sk.y, dz = cz - sk.z;
                        const float r2 = (dx * dx + dy * dy + dz * dz) * 1.001f;
                        if (GEOM) any = lhs < sk.w * A.theta2f * r2;
                        else any = lhs < sk.w * ipow<P + 2>(sqrtf(r2));
                    }
                }
                maybe = any;
            }
            // exact per-lane decisions for the nodes some sink may use (rare in the TreePM
            // regime): a lane that uses the multipole leaves the node's subtree; a lane beyond
            // the cutoff keeps walking (the cutoff is hereditary, nothing below can be used and
            // the pair cutoff removes the leaves)
            unsigned mev = __ballot_sync(0xffffffffu, maybe);
            while (mev) {
                const int src = __ffs(mev) - 1;
                mev &= mev - 1u;
                const int jj = __shfl_sync(0xffffffffu, d, src);
                const unsigned mm = __shfl_sync(0xffffffffu, m, src);
                const G4Node n2 = load_node(A.wnode + jj);
                const int jd = n2.parent;   // depth-first index: moments
                int act = ACT_NONE;
                if ((mm >> lane) & 1u)
                    act = exact_decision<P, T, TREEPM, GEOM>(A, n2, jd, xi, yi, zi, hi, crit, gscale, gbox);
                const unsigned accm = __ballot_sync(0xffffffffu, act == ACT_ACCEPT);
                if (accm && act == ACT_ACCEPT && kp == 0) {   // multipoles: part 0 of a split group
                    T Qs[g4_nq(P) > 0 ? g4_nq(P) : 1];
                    T mx, my, mz, M;
                    if (sizeof(T) == 8 && A.qd) {
                        const double *dd = A.qd + (size_t)jd * (4 + A.nq);
                        mx = (T)dd[0]; my = (T)dd[1]; mz = (T)dd[2]; M = (T)dd[3];
#pragma unroll
                        for (int c = 0; c < g4_nq_raw(P); c++) Qs[c] = (T)dd[4 + c];
                    } else {
                        mx = (T)n2.sx; my = (T)n2.sy; mz = (T)n2.sz; M = (T)n2.mass;
                        const float *qq = A.q + (size_t)jd * A.nq;
#pragma unroll
                        for (int c = 0; c < g4_nq_raw(P); c++) Qs[c] = (T)__ldg(qq + c);
                    }
                    T rx = (T)(int32_t)(n2.cx - xi) * (T)gscale + mx;
                    T ry = (T)(int32_t)(n2.cy - yi) * (T)gscale + my;
                    T rz = (T)(int32_t)(n2.cz - zi) * (T)gscale + mz;
                    if (!TREEPM && A.ewald) {
                        // the Newtonian term plus the correction is the periodic potential,
                        // the same at every image of the centre of mass: take the one in the
                        // primary cell, which the correction grid covers
                        const T Lb = (T)gbox;
                        rx -= Lb * rint(rx / Lb);
                        ry -= Lb * rint(ry / Lb);
                        rz -= Lb * rint(rz / Lb);
                    }
                    const T hs = A.soft_nodes ? fmax(hi, (T)n2.hmax) : T(0);
                    pn_term<P, T, TREEPM>(Qs, M, rx, ry, rz, par<T>(A.as, A.asf), bx, by, bz, bp, hs);
                    if (!TREEPM && A.ewald) pn_ewald<P, T>(A.ew, Qs, M, rx, ry, rz, bx, by, bz, bp);
                    npn++;
                }
                if (lane == src) m &= ~accm;
            }
            // leaves go to the pending list, internal nodes push their daughters
            const bool addleaf = leaf && !gskip && m != 0u;
            const unsigned lm = __ballot_sync(0xffffffffu, addleaf);
            if (addleaf) {
                const int pos = nleaf + __popc(lm & lt);
                S.first[pos] = nd.first;
                S.count[pos] = nd.count;
                S.mask[pos] = m;
            }
            nleaf += __popc(lm);
            const bool expand = ve && !leaf && !gskip && m != 0u;
            const int nch = expand ? nd.nchild : 0;
            int pre = nch;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, pre, o);
                if (lane >= o) pre += y;
            }
            const int tot = __shfl_sync(0xffffffffu, pre, 31);
            pre -= nch;
            if (tail + tot - head > A.qcap) {
                if (lane == 0) atomicOr(A.flags, G4_FLAG_LISTCAP);
            } else if (nch > 0) {
                for (int c = 0; c < nch; c++)   // daughters are consecutive in level order
                    Q[(tail + pre + c) & (A.qcap - 1)] = make_int2(nd.next + c, (int)m);
            }
            if (tail + tot - head <= A.qcap) tail += tot;
            __syncwarp();
        }
        if (INTU) {
            const T ca = (T)figs * (T)figs, cp = (T)figs;
            ax *= ca;
            ay *= ca;
            az *= ca;
            ap *= cp;
        }
        if (Kp == 1) {
            if (valid) {
                const T G = par<T>(A.G, A.Gf);
                const int o = A.operm ? __ldg(A.operm + i) : i;
                A.acc[o] = (float)(-G * (ax + bx));
                A.acc[A.n + o] = (float)(-G * (ay + by));
                A.acc[2 * A.n + o] = (float)(-G * (az + bz));
                if (A.pot) A.pot[o] = (float)(-G * (ap + bp));
                if (A.counts) {
                    A.counts[i] = npp;
                    A.counts[A.n + i] = npn;
                }
            }
        } else {
            // split group: store this part's sums; the last part to arrive adds the parts in
            // part order (deterministic) and writes the outputs
            float *pb = A.part_buf + (((size_t)pslot * G4_ITEM_SPLIT_MAX + kp) * 32 + lane) * 6;
            pb[0] = (float)(ax + bx);
            pb[1] = (float)(ay + by);
            pb[2] = (float)(az + bz);
            pb[3] = (float)(ap + bp);
            pb[4] = __uint_as_float(npp);
            pb[5] = __uint_as_float(npn);
            __threadfence();
            __syncwarp();
            int last = 0;
            if (lane == 0) last = atomicAdd(A.part_cnt + pslot, 1) == Kp - 1;
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence();
                float sx = 0.f, sy = 0.f, sz = 0.f, sp = 0.f;
                uint32_t cp = 0, cn = 0;
                for (int q = 0; q < Kp; q++) {
                    const float *qb = A.part_buf + (((size_t)pslot * G4_ITEM_SPLIT_MAX + q) * 32 + lane) * 6;
                    sx += __ldcg(qb);
                    sy += __ldcg(qb + 1);
                    sz += __ldcg(qb + 2);
                    sp += __ldcg(qb + 3);
                    cp += __float_as_uint(__ldcg(qb + 4));
                    cn += __float_as_uint(__ldcg(qb + 5));
                }
                if (valid) {
                    const float G = A.Gf;
                    const int o = A.operm ? __ldg(A.operm + i) : i;
                    A.acc[o] = -G * sx;
                    A.acc[A.n + o] = -G * sy;
                    A.acc[2 * A.n + o] = -G * sz;
                    if (A.pot) A.pot[o] = -G * sp;
                    if (A.counts) {
                        A.counts[i] = cp;
                        A.counts[A.n + i] = cn;
                    }
                }
                if (lane == 0) A.part_cnt[pslot] = 0;   // ready for the next walk
            }
        }
    };
    const long long t_start = clock64();
    for (;;) {
        int g = 0;
        if (lane == 0) {
            if (A.watchdog > 0 && clock64() - t_start > A.watchdog) {
                atomicOr(A.flags, G4_FLAG_TIMEOUT);   // reported by g4_tree_status
                g = ngroups;
            } else {
                g = atomicAdd(A.work, uni ? UNION_G : 1);
            }
        }
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ngroups) break;
        int ng = 1, ul_n = -1;
        if (uni) {
            const size_t w0 = (size_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * ULCAP;
            ng = min(UNION_G, ngroups - g);
            ul_n = union_walk<P, GEOM>(A, Q, A.ul_cube + w0, A.ul_fc + w0, lane, g * 32,
                                       min(A.n_sinks, (g + ng) * 32));
        } else if (A.group_order) {
            g = A.group_order[g];
        }
        // the run's state lives in shared memory while its groups walk (register pressure)
        if (lane == 0) {
            S.rg = g;
            S.rn = ng;
            S.rq = 0;
            S.rul = ul_n;
        }
        __syncwarp();
        for (;;) {
            const int q = S.rq;
            if (q >= S.rn) break;
            group(S.rg + q, S.rul);
            __syncwarp();
            if (lane == 0) S.rq = q + 1;
            __syncwarp();
        }
    }
}

// -------------------------------------------------------------------------------------------
// direct summation on the GPU (validation helper): one thread per sink, sources through
// shared memory tiles.
// -------------------------------------------------------------------------------------------
struct DirectArgs {
    const uint32_t *pos;
    const float *mass;
    const uint8_t *cls;
    int n;
    const int32_t *sinks;
    int n_sinks;
    float *acc, *pot;
    double scale, G, rcut2, as;
    float h_cls[G4_MAX_EPS_CLASSES];
    int pp_cut;
};

template <typename T, bool TREEPM>
__global__ void __launch_bounds__(256) k_direct(const DirectArgs A)
{
    __shared__ uint32_t sxp[256], syp[256], szp[256];
    __shared__ float sm[256], sh[256];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = s < A.n_sinks;
    const int i = valid ? (A.sinks ? A.sinks[s] : s) : 0;
    const uint32_t xi = A.pos[i], yi = A.pos[A.n + i], zi = A.pos[2 * A.n + i];
    const T hi = (T)A.h_cls[A.cls ? A.cls[i] : 0];
    const T scale = (T)A.scale, as = (T)A.as, rcut2 = (T)A.rcut2;
    T ax = 0, ay = 0, az = 0, ph = 0;
    for (int base = 0; base < A.n; base += 256) {
        int j = base + threadIdx.x;
        if (j < A.n) {
            sxp[threadIdx.x] = A.pos[j];
            syp[threadIdx.x] = A.pos[A.n + j];
            szp[threadIdx.x] = A.pos[2 * A.n + j];
            sm[threadIdx.x] = A.mass[j];
            sh[threadIdx.x] = A.h_cls[A.cls ? A.cls[j] : 0];
        }
        __syncthreads();
        const int m = min(256, A.n - base);
        if (valid)
            for (int t = 0; t < m; t++) {
                if (base + t == i) continue;
                const T dx = (T)(int32_t)(sxp[t] - xi) * scale;
                const T dy = (T)(int32_t)(syp[t] - yi) * scale;
                const T dz = (T)(int32_t)(szp[t] - zi) * scale;
                const T r2 = dx * dx + dy * dy + dz * dz;
                if (TREEPM && A.pp_cut && r2 >= rcut2) continue;
                T g0, g1;
                pair_kernel<T, TREEPM>(r2, fmax(hi, (T)sh[t]), as, g0, g1);
                const T mj = (T)sm[t];
                ax += mj * g1 * dx;
                ay += mj * g1 * dy;
                az += mj * g1 * dz;
                ph += mj * g0;
            }
        __syncthreads();
    }
    if (valid) {
        const T G = (T)A.G;
        A.acc[i] = (float)(-G * ax);
        A.acc[A.n + i] = (float)(-G * ay);
        A.acc[2 * A.n + i] = (float)(-G * az);
        if (A.pot) A.pot[i] = (float)(-G * ph);
    }
}

__global__ void k_zero_int(int *p) { *p = 0; }

// Walk copies.  Node records in level order, so that a node's daughters are consecutive
// (the frontier pushes them without index look-ups); next = first daughter (level order),
// parent = depth-first index (position of the node's moments).
__global__ void k_walk_nodes(const int32_t *__restrict__ lvl, const int32_t *__restrict__ flags,
                             const int32_t *__restrict__ b_dfs,
                             const int32_t *__restrict__ b_child, const G4Node *__restrict__ node,
                             G4Node *__restrict__ wnode)
{
    if (*flags & G4_FLAG_CAPACITY) return;   // incomplete tree (the walk does not run either)
    const int nn = lvl[G4_NLEVELS];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nn; b += gridDim.x * blockDim.x) {
        const int d = b_dfs[b];
        if ((unsigned)d >= (unsigned)nn) continue;
        G4Node r = node[d];
        r.next = r.nchild > 0 ? b_child[b] : -1;
        r.parent = d;
        wnode[b] = r;
    }
}

// particles as one 16-byte record each (one load per staged source)
__global__ void k_walk_parts(const uint32_t *__restrict__ pos, const float *__restrict__ mass,
                             int n, uint4 *__restrict__ wp)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        wp[j] = make_uint4(pos[j], pos[n + j], pos[2 * n + j], __float_as_uint(mass[j]));
}

template <int P, typename T, bool TREEPM, bool GEOM>
void launch_walk(const WalkArgs &A, cudaStream_t st)
{
    // persistent: G4_WALK_BLOCKS_PER_SM 4-warp blocks per SM; groups come from the work counter
    int nb = g4_num_sms() * G4_WALK_BLOCKS_PER_SM;
#ifdef G4_WALK_CARVEOUT
    // preferred shared-memory carveout (percent of the unified L1/shared array)
    static bool carve_set = false;
    if (!carve_set) {
        cudaFuncSetAttribute(k_walk<P, T, TREEPM, GEOM>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             G4_WALK_CARVEOUT);
        carve_set = true;
    }
#endif
    k_walk<P, T, TREEPM, GEOM><<<nb, WALK_THREADS, 0, st>>>(A);
}

template <int P, typename T>
void dispatch_walk2(const WalkArgs &A, bool treepm, bool geom, cudaStream_t st)
{
    if (treepm) {
        if (geom) launch_walk<P, T, true, true>(A, st);
        else launch_walk<P, T, true, false>(A, st);
    } else {
        if (geom) launch_walk<P, T, false, true>(A, st);
        else launch_walk<P, T, false, false>(A, st);
    }
}

template <typename T>
void dispatch_walk(int p, const WalkArgs &A, bool treepm, bool geom, cudaStream_t st)
{
    switch (p) {
    case 1: dispatch_walk2<1, T>(A, treepm, geom, st); break;
    case 2: dispatch_walk2<2, T>(A, treepm, geom, st); break;
    case 3: dispatch_walk2<3, T>(A, treepm, geom, st); break;
    case 4: dispatch_walk2<4, T>(A, treepm, geom, st); break;
    default: dispatch_walk2<5, T>(A, treepm, geom, st); break;
    }
}

}  // namespace

double g4_r_cut(const g4_params *P)
{
    double emax = 0.0;
    for (int k = 0; k < P->n_eps_classes; k++) emax = fmax(emax, P->eps_table[k]);
    return fmax(P->r_cut_factor * P->r_s, 2.8 * emax);
}

g4_status g4_check_params(const g4_params *P, const char *who)
{
    if (!P) return g4_fail(G4_ERR_INVALID_ARG, "%s: NULL params", who);
    if (!(P->box_size > 0)) return g4_fail(G4_ERR_INVALID_ARG, "%s: box_size must be > 0", who);
    if (P->order_p < 1 || P->order_p > G4_MAX_ORDER)
        return g4_fail(G4_ERR_INVALID_ARG, "%s: order_p=%d out of [1,5]", who, P->order_p);
    if (P->n_eps_classes < 1 || P->n_eps_classes > G4_MAX_EPS_CLASSES)
        return g4_fail(G4_ERR_INVALID_ARG, "%s: n_eps_classes=%d", who, P->n_eps_classes);
    if (P->criterion != 0 && P->criterion != 1)
        return g4_fail(G4_ERR_INVALID_ARG, "%s: criterion=%d", who, P->criterion);
    if (P->precision != 0 && P->precision != 1)
        return g4_fail(G4_ERR_INVALID_ARG, "%s: precision=%d", who, P->precision);
    if (P->group_size != 0 && P->group_size != 8 && P->group_size != 16 && P->group_size != 32)
        return g4_fail(G4_ERR_INVALID_ARG, "%s: group_size=%d (8, 16 or 32)", who, P->group_size);
    if (P->ewald && (!P->periodic || P->r_s > 0.0 || P->order_p > 5))
        return g4_fail(G4_ERR_INVALID_ARG, "%s: the Ewald correction needs periodic=1, r_s=0", who);
    if (P->watchdog_cycles < 0)
        return g4_fail(G4_ERR_INVALID_ARG, "%s: watchdog_cycles=%lld", who, P->watchdog_cycles);
    return G4_OK;
}

// 16-byte particle records (x, y, z, mass bits) of the sorted particles in the handle's
// buffer, allocated on first use (outside graph capture), rewritten on every call
g4_status g4_particle_records(g4_tree t, const uint32_t *pos_sorted, const float *mass_sorted,
                              int n, cudaStream_t st)
{
    if (!t->wpart) {
        if (cudaMalloc(&t->wpart, sizeof(uint4) * (size_t)(t->n_max > 0 ? t->n_max : 1)) != cudaSuccess) {
            cudaGetLastError();
            t->wpart = nullptr;
            return g4_fail(G4_ERR_OOM, "particle records (%lld)", (long long)t->n_max);
        }
    }
    if (n > 0) k_walk_parts<<<g4_blocks_for(n, 256), 256, 0, st>>>(pos_sorted, mass_sorted, n, t->wpart);
    return g4_launch_check("particle records", n > 0 ? 1 : 0);
}

static g4_status gravity_tree(g4_tree t, const uint32_t *pos_sorted, const float *mass_sorted,
                              const uint8_t *cls_sorted, const float *aold_sorted,
                              const int32_t *active, int64_t n_active, const g4_params *P,
                              const int32_t *out_perm, float *acc, float *pot, uint32_t *counts,
                              void *stream)
{
    g4_status s = g4_check_params(P, "g4_gravity_tree");
    if (s != G4_OK) return s;
    if (!t || !pos_sorted || !mass_sorted || !acc)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_tree: NULL argument");
    if (t->built_n < 0 || t->moments_order < 0)
        return g4_fail(G4_ERR_STATE, "g4_gravity_tree: build and multipoles must run first");
    if (t->moments_order != P->order_p)
        return g4_fail(G4_ERR_STATE, "g4_gravity_tree: moments of order %d, walk order %d",
                       t->moments_order, P->order_p);
    if (P->precision == 1 && !t->moments_fp64)
        return g4_fail(G4_ERR_STATE, "g4_gravity_tree: FP64 walk needs FP64 multipoles");
    if (P->criterion == 0 && !aold_sorted)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_tree: relative criterion needs a_old");
    const int n = t->built_n;
    if (active && (n_active < 0 || n_active > n))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_tree: n_active=%lld", (long long)n_active);
    const int ns = active ? (int)n_active : n;
    if (n == 0 || ns == 0) return G4_OK;
    cudaStream_t st = (cudaStream_t)stream;
    WalkArgs A;
    A.pos = pos_sorted;
    A.mass = mass_sorted;
    A.cls = cls_sorted;
    A.aold = aold_sorted;
    A.active = active;
    A.n = n;
    A.n_sinks = ns;
    A.lvl = t->lvl;
    A.node = t->node;
    A.q = t->q;
    A.qd = P->precision == 1 ? t->qd : nullptr;
    A.nq = g4_nq(P->order_p);
    A.acc = acc;
    A.pot = pot;
    A.counts = counts;
    A.operm = out_perm;
    A.watchdog = P->watchdog_cycles;
    A.work = t->d_flags + 1;
    A.flags = t->d_flags;
    A.sys_first = t->sys_first;
    A.sys_goff = t->sys_goff;
    A.sys_box = t->sys_box;
    A.n_sys = t->n_sys;
    A.gs = (P->group_size == 0 || t->n_sys) ? 32 : P->group_size;
    A.group_order = (t->group_order && !active && !t->n_sys && A.gs == 32 &&
                     t->group_order_n == (ns + 31) / 32) ? t->group_order : nullptr;
    const bool use_items = t->items && !active && !t->n_sys && t->items_n_sinks == ns &&
                           P->precision == 0 && A.gs == 32;
    A.items = use_items ? (const int4 *)t->items : nullptr;
    A.n_items = use_items ? t->n_items : nullptr;
    A.part_buf = t->part_buf;
    A.part_cnt = t->part_cnt;
    A.part_cap = t->part_cap;
    if (use_items) A.group_order = nullptr;
    if (t->n_sys && active)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_tree: active subsets are not supported for forests");
    A.scale = P->box_size / 4294967296.0;
    A.G = P->G;
    A.alpha = P->alpha;
    A.theta2 = P->theta * P->theta;
    const bool treepm = P->r_s > 0.0;
    const double rc = treepm ? g4_r_cut(P) : 0.0;
    A.rcut2 = rc * rc;
    A.as = treepm ? 0.5 / P->r_s : 0.0;
    A.Gf = (float)A.G;
    A.alphaf = (float)A.alpha;
    A.theta2f = (float)A.theta2;
    A.rcut2f = (float)A.rcut2;
    A.asf = (float)A.as;
    A.inv_as = treepm ? 2.0 * P->r_s : 0.0;
    A.igs = 4294967296.0 / P->box_size;
    A.box = P->box_size;
    for (int k = 0; k < G4_MAX_EPS_CLASSES; k++)
        A.h_cls[k] = k < P->n_eps_classes ? (float)(2.8 * P->eps_table[k]) : 0.f;
    A.exclusion = P->exclusion_zone;
    A.pp_cut = P->pp_cut;
    A.soft_nodes = P->soft_nodes;
    A.ewald = P->ewald;
    if (P->ewald) {
        s = g4_ewald_ensure(t, P->box_size, P->order_p + 1 + 3, (cudaStream_t)stream, &A.ew);
        if (s != G4_OK) return s;
    }
    // per-warp frontier rings and union leaf lists, allocated on the handle's first walk
    // (outside any graph capture)
    // (the rings are four times wider for walks without the TreePM cutoff on large sets,
    // whose breadth-first frontier is wider; a handle grows its rings when first asked)
    const int qcap = (!treepm && n > (1 << 16)) ? QCAP_TREE : QCAP;
    const size_t nwarps = (size_t)g4_num_sms() * G4_WALK_BLOCKS_PER_SM * (WALK_THREADS / 32);
    const size_t qbytes = sizeof(int2) * (size_t)qcap * nwarps;
    const size_t ubytes = (sizeof(int4) + sizeof(int2)) * (size_t)ULCAP * nwarps;
    if (t->walk_queue && t->walk_qcap < qcap) {
        cudaFree(t->walk_queue);
        t->walk_queue = nullptr;
    }
    if (!t->walk_queue) {
        const size_t bytes = qbytes + ubytes;
        if (cudaMalloc(&t->walk_queue, bytes) != cudaSuccess) {
            cudaGetLastError();
            t->walk_queue = nullptr;
            return g4_fail(G4_ERR_OOM, "g4_gravity_tree: frontier buffers (%zu bytes)", bytes);
        }
        t->walk_qcap = qcap;
    }
    A.queue = (int2 *)t->walk_queue;
    A.qcap = t->walk_qcap;
    const size_t qoff = sizeof(int2) * (size_t)t->walk_qcap * nwarps;   // the rings as allocated
    A.ul_cube = (int4 *)((char *)t->walk_queue + qoff);
    A.ul_fc = (int2 *)((char *)t->walk_queue + qoff + sizeof(int4) * (size_t)ULCAP * nwarps);
    if (!t->wnode) {
        if (cudaMalloc(&t->wnode, sizeof(G4Node) * (size_t)t->cap) != cudaSuccess) {
            cudaGetLastError();
            t->wnode = nullptr;
            return g4_fail(G4_ERR_OOM, "g4_gravity_tree: level-ordered node copy");
        }
        t->wnode_stamp = -1;
    }
    int extra = 0;
    if (t->wnode_stamp != t->moments_stamp) {
        k_walk_nodes<<<g4_blocks_for(t->cap, 256), 256, 0, st>>>(t->lvl, t->d_flags, t->b_dfs, t->b_child,
                                                                t->node, t->wnode);
        t->wnode_stamp = t->moments_stamp;
        extra++;
    }
    s = g4_particle_records(t, pos_sorted, mass_sorted, n, st);
    if (s != G4_OK) return s;
    A.wnode = t->wnode;
    A.wpart = t->wpart;
    k_zero_int<<<1, 1, 0, st>>>(A.work);
    const bool geom = P->criterion == 1;
    if (P->precision == 1) dispatch_walk<double>(P->order_p, A, treepm, geom, st);
    else dispatch_walk<float>(P->order_p, A, treepm, geom, st);
    return g4_launch_check("tree walk", 2 + extra);
}

extern "C" g4_status g4_gravity_tree(g4_tree t, const uint32_t *pos_sorted,
                                     const float *mass_sorted, const uint8_t *cls_sorted,
                                     const float *aold_sorted, const int32_t *active,
                                     int64_t n_active, const g4_params *P, float *acc, float *pot,
                                     uint32_t *counts, void *stream)
{
    return gravity_tree(t, pos_sorted, mass_sorted, cls_sorted, aold_sorted, active, n_active, P,
                        nullptr, acc, pot, counts, stream);
}

extern "C" g4_status g4_gravity_tree_perm(g4_tree t, const uint32_t *pos_sorted,
                                          const float *mass_sorted, const uint8_t *cls_sorted,
                                          const float *aold_sorted, const int32_t *active,
                                          int64_t n_active, const g4_params *P,
                                          const int32_t *perm, float *acc, float *pot,
                                          uint32_t *counts, void *stream)
{
    if (!perm) return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_tree_perm: NULL perm");
    return gravity_tree(t, pos_sorted, mass_sorted, cls_sorted, aold_sorted, active, n_active, P,
                        perm, acc, pot, counts, stream);
}

extern "C" g4_status g4_direct(const uint32_t *pos, const float *mass, const uint8_t *cls,
                               int64_t n, const int32_t *sinks, int64_t n_sinks,
                               const g4_params *P, float *acc, float *pot, void *stream)
{
    g4_status s = g4_check_params(P, "g4_direct");
    if (s != G4_OK) return s;
    if (n < 0 || n >= ((int64_t)1 << 31) || !pos || !mass || !acc || (sinks && n_sinks < 0))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_direct: bad arguments");
    const int ns = sinks ? (int)n_sinks : (int)n;
    if (n == 0 || ns == 0) return G4_OK;
    DirectArgs A;
    A.pos = pos;
    A.mass = mass;
    A.cls = cls;
    A.n = (int)n;
    A.sinks = sinks;
    A.n_sinks = ns;
    A.acc = acc;
    A.pot = pot;
    A.scale = P->box_size / 4294967296.0;
    A.G = P->G;
    const bool treepm = P->r_s > 0.0;
    const double rc = treepm ? g4_r_cut(P) : 0.0;
    A.rcut2 = rc * rc;
    A.as = treepm ? 0.5 / P->r_s : 0.0;
    for (int k = 0; k < G4_MAX_EPS_CLASSES; k++)
        A.h_cls[k] = k < P->n_eps_classes ? (float)(2.8 * P->eps_table[k]) : 0.f;
    A.pp_cut = P->pp_cut;
    cudaStream_t st = (cudaStream_t)stream;
    int nb = (ns + 255) / 256;
    if (P->precision == 1) {
        if (treepm) k_direct<double, true><<<nb, 256, 0, st>>>(A);
        else k_direct<double, false><<<nb, 256, 0, st>>>(A);
    } else {
        if (treepm) k_direct<float, true><<<nb, 256, 0, st>>>(A);
        else k_direct<float, false><<<nb, 256, 0, st>>>(A);
    }
    return g4_launch_check("direct sum", 1);
}
