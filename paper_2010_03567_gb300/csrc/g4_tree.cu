// g4_tree.cu -- oct-tree construction over PH-sorted keys (Sec. 2.2.1) and the tree handle.
//
// Build, level by level (one launch per level, no host synchronisation):
//   expand(l):   every level-l node holding more than leaf_max particles finds the 8 daughter
//                ranges by binary search on the digit of level l+1 in its sorted key range and
//                appends its non-empty daughters (in PH order, contiguous) to level l+1;
//   subtree(l):  bottom-up subtree sizes;
//   dfs(l):      top-down depth-first pre-order numbers (daughters in PH order);
//   emit:        node records in depth-first order, `next` = index after the subtree.
// The depth-first numbering is fixed by the tree's structure, so the result is bit-exact and
// independent of the order in which atomics hand out the level slots.
#include "g4_internal.cuh"

namespace {

constexpr int BUILD_THREADS = 256;

__global__ void k_build_init(int32_t *lvl, int32_t *flags, int32_t *b_first, int32_t *b_count,
                             int32_t *b_parent, int32_t *b_dfs, int n)
{
    int t = threadIdx.x;
    if (t < 2 * (G4_NLEVELS + 1)) lvl[t] = 0;
    __syncthreads();
    if (t == 0) {
        lvl[G4_NLEVELS + 1 + 0] = n > 0 ? 1 : 0;  // count of level 0
        b_first[0] = 0;
        b_count[0] = n;
        b_parent[0] = -1;
        b_dfs[0] = 0;
        *flags = 0;
    }
}

// forest: level 0 holds one root per system, system s covering sorted particles
// [sys_first[s], sys_first[s+1])
__global__ void k_build_init_forest(int32_t *lvl, int32_t *flags, int32_t *b_first, int32_t *b_count,
                                    int32_t *b_parent, const int32_t *__restrict__ sys_first,
                                    int n_sys)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0) {
        if (t < 2 * (G4_NLEVELS + 1)) lvl[t] = 0;
        __syncthreads();
        if (t == 0) {
            lvl[G4_NLEVELS + 1 + 0] = n_sys;
            *flags = 0;
        }
    }
    for (int s = t; s < n_sys; s += gridDim.x * blockDim.x) {
        b_first[s] = sys_first[s];
        b_count[s] = sys_first[s + 1] - sys_first[s];
        b_parent[s] = -1;
    }
}

// forest: depth-first numbers of the roots (prefix sums of the subtree sizes) and the walk
// group offsets of the systems (prefix sums of ceil(n_s / 32)); one block
__global__ void __launch_bounds__(1024) k_forest_roots(const int32_t *__restrict__ b_size,
                                                       const int32_t *__restrict__ sys_first,
                                                       int n_sys, int32_t *__restrict__ b_dfs,
                                                       int32_t *__restrict__ goff)
{
    __shared__ int ws[2][32];
    __shared__ int carry[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry[0] = carry[1] = 0;
    __syncthreads();
    for (int base = 0; base < n_sys; base += 1024) {
        const int s = base + threadIdx.x;
        int a = s < n_sys ? b_size[s] : 0;
        int g = s < n_sys ? (sys_first[s + 1] - sys_first[s] + 31) / 32 : 0;
        int xa = a, xg = g;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ya = __shfl_up_sync(0xffffffffu, xa, o), yg = __shfl_up_sync(0xffffffffu, xg, o);
            if (lane >= o) { xa += ya; xg += yg; }
        }
        if (lane == 31) { ws[0][w] = xa; ws[1][w] = xg; }
        __syncthreads();
        int pa = carry[0], pg = carry[1];
        for (int k = 0; k < w; k++) { pa += ws[0][k]; pg += ws[1][k]; }
        if (s < n_sys) {
            b_dfs[s] = pa + xa - a;
            goff[s] = pg + xg - g;
        }
        __syncthreads();
        if (threadIdx.x == 1023) { carry[0] = pa + xa; carry[1] = pg + xg; }
        __syncthreads();
    }
    if (threadIdx.x == 0) goff[n_sys] = carry[1];
}

__device__ __forceinline__ int lower_bound_digit(const uint64_t *__restrict__ keys, int lo, int hi,
                                                 int shift, uint32_t d)
{
    // first index in [lo, hi) whose digit at `shift` is >= d (digits are sorted in range)
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        uint32_t v = (uint32_t)(keys[mid] >> shift) & 7u;
        if (v < d) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Splits the nodes [o, o + c) of one level with 8 * G lanes per node: lane group g (G lanes)
// finds, for digit g >= 1, the first key of the node whose digit is >= g by a (G + 1)-ary
// search over the whole node (the digits of a node's keys are non-decreasing), so the seven
// boundaries are searched at once and each needs about log_{G+1}(n) dependent loads instead
// of the seven chained binary searches of a thread per node. Group 0 stands for digit 0,
// whose boundary is the node's first key. Children are numbered in digit order, as below.
template <int G>
__device__ __forceinline__ void expand_grouped(
    const uint64_t *__restrict__ keys, int o, int c, int nbase, int level, int leaf_max,
    int64_t cap, int shift, int32_t *__restrict__ cnt, int32_t *__restrict__ flags,
    int32_t *__restrict__ b_first, int32_t *__restrict__ b_count, int32_t *__restrict__ b_child,
    int32_t *__restrict__ b_nchild, int32_t *__restrict__ b_parent, int warp, int nwarps,
    int lane)
{
    constexpr unsigned FULL = 0xffffffffu, GMASK = (1u << G) - 1u;
    constexpr int L = 8 * G, NPW = 32 / L;
    const int base = lane - lane % L, g = (lane - base) / G, j = lane % G, gb = lane - j;
    for (int b0 = warp * NPW; b0 < c; b0 += nwarps * NPW) {   // uniform within the warp
        const int b = b0 + (lane / L);
        const bool ok = b < c;
        const int node = o + b;
        int f = 0, n = 0;
        if (ok) {
            f = b_first[node];
            n = b_count[node];
        }
        const bool split = ok && n > leaf_max && level < G4_MAXLEVEL;
        const bool act = split && g >= 1;
        const uint32_t d = (uint32_t)g;
        int lo = f, hi = f + n;   // the boundary lies in [lo, hi]
        while (__any_sync(FULL, act && hi - lo > G)) {
            const bool go = act && hi - lo > G;
            int p = lo;
            bool below = false;
            if (go) {
                // G strictly increasing probes inside (lo, hi)
                p = lo + (int)((int64_t)(hi - lo) * (j + 1) / (G + 1));
                below = ((uint32_t)(keys[p] >> shift) & 7u) < d;
            }
            const int cb = __popc((__ballot_sync(FULL, below) >> gb) & GMASK);
            const int pl = __shfl_sync(FULL, p, gb + (cb > 0 ? cb - 1 : 0));
            const int ph = __shfl_sync(FULL, p, gb + (cb < G ? cb : G - 1));
            if (go) {
                if (cb > 0) lo = pl + 1;
                if (cb < G) hi = ph;
            }
        }
        const int q = lo + j;
        const bool below = act && q < hi && ((uint32_t)(keys[q] >> shift) & 7u) < d;
        const int bound = lo + __popc((__ballot_sync(FULL, below) >> gb) & GMASK);
        int nch = 0, before = 0, my_lo = f, my_hi = f;
        int prev = __shfl_sync(FULL, bound, base);
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int nxt = k < 7 ? __shfl_sync(FULL, bound, base + (k + 1) * G) : f + n;
            const int ne = nxt > prev;
            nch += ne;
            if (k < g) before += ne;
            if (k == g) {
                my_lo = prev;
                my_hi = nxt;
            }
            prev = nxt;
        }
        if (!split) nch = 0;
        int slot = 0;
        if (lane == base && nch > 0) slot = atomicAdd(&cnt[level + 1], nch);
        slot = nbase + __shfl_sync(FULL, slot, base);
        if (!ok) continue;
        if (nch == 0 || (int64_t)slot + nch > cap) {
            if (lane == base) {
                if (nch > 0) atomicOr(flags, G4_FLAG_CAPACITY);
                b_child[node] = -1;
                b_nchild[node] = 0;
            }
            continue;
        }
        if (lane == base) {
            b_child[node] = slot;
            b_nchild[node] = nch;
        }
        if (j == 0 && my_hi > my_lo) {
            const int k = slot + before;
            b_first[k] = my_lo;
            b_count[k] = my_hi - my_lo;
            b_parent[k] = node;
        }
    }
}

__global__ void __launch_bounds__(BUILD_THREADS) k_build_expand(
    const uint64_t *__restrict__ keys, int level, int leaf_max, int64_t cap,
    int32_t *__restrict__ lvl, int32_t *__restrict__ flags, int32_t *__restrict__ b_first,
    int32_t *__restrict__ b_count, int32_t *__restrict__ b_child, int32_t *__restrict__ b_nchild,
    int32_t *__restrict__ b_parent)
{
    int32_t *off = lvl, *cnt = lvl + G4_NLEVELS + 1;
    const int o = off[level], c_raw = cnt[level];
    const int nbase = o + c_raw;   // first slot of level + 1
    if (blockIdx.x == 0 && threadIdx.x == 0) off[level + 1] = nbase;
    // after a capacity overflow the slots an overflowing warp reserved below the capacity are
    // never written, so no later level reads them: the build stops here (tree invalid)
    if (*flags & G4_FLAG_CAPACITY) return;
    // after a capacity overflow only the slots inside the arrays are touched
    const int c = (int)min((int64_t)c_raw, cap - o > 0 ? cap - o : (int64_t)0);
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int shift = 3 * (G4_KEYBITS - level - 1);
    // few, large nodes: several lanes per node; many small nodes: a thread per node
    if (c <= nwarps) {
        expand_grouped<4>(keys, o, c, nbase, level, leaf_max, cap, shift, cnt, flags, b_first,
                          b_count, b_child, b_nchild, b_parent, warp, nwarps, lane);
        return;
    }
    if (c <= 16 * nwarps) {
        expand_grouped<1>(keys, o, c, nbase, level, leaf_max, cap, shift, cnt, flags, b_first,
                          b_count, b_child, b_nchild, b_parent, warp, nwarps, lane);
        return;
    }
    for (int wb = warp * 32; wb < c; wb += nwarps * 32) {
        int b = wb + lane;
        bool ok = b < c;
        int node = o + b;
        int f = 0, n = 0, bounds[9];
        int nch = 0;
        if (ok) {
            f = b_first[node];
            n = b_count[node];
            if (n > leaf_max && level < G4_MAXLEVEL) {
                bounds[0] = f;
                bounds[8] = f + n;
#pragma unroll
                for (int d = 1; d < 8; d++)
                    bounds[d] = lower_bound_digit(keys, bounds[d - 1], f + n, shift, (uint32_t)d);
#pragma unroll
                for (int d = 0; d < 8; d++) nch += bounds[d + 1] > bounds[d];
            }
        }
        // warp-aggregated slot allocation in level + 1
        int incl = nch;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, s);
            if (lane >= s) incl += y;
        }
        int tot = __shfl_sync(0xffffffffu, incl, 31);
        int start = 0;
        if (lane == 31 && tot > 0) start = atomicAdd(&cnt[level + 1], tot);
        start = __shfl_sync(0xffffffffu, start, 31);
        int slot = nbase + start + incl - nch;
        if (!ok) continue;
        if (nch == 0) {
            b_child[node] = -1;
            b_nchild[node] = 0;
            continue;
        }
        if ((int64_t)slot + nch > cap) {
            atomicOr(flags, G4_FLAG_CAPACITY);
            b_child[node] = -1;
            b_nchild[node] = 0;
            continue;
        }
        b_child[node] = slot;
        b_nchild[node] = nch;
        int k = slot;
#pragma unroll
        for (int d = 0; d < 8; d++)
            if (bounds[d + 1] > bounds[d]) {
                b_first[k] = bounds[d];
                b_count[k] = bounds[d + 1] - bounds[d];
                b_parent[k] = node;
                k++;
            }
    }
}

// level 21 (key resolution): every node is a leaf; also fixes the capacity-clipped count
__global__ void k_build_last(int32_t *__restrict__ lvl, int64_t cap, int32_t *__restrict__ b_child,
                             int32_t *__restrict__ b_nchild)
{
    int32_t *off = lvl, *cnt = lvl + G4_NLEVELS + 1;
    int o = off[G4_MAXLEVEL], c = cnt[G4_MAXLEVEL];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < c; b += gridDim.x * blockDim.x)
        if (o + b < cap) {
            b_child[o + b] = -1;
            b_nchild[o + b] = 0;
        }
}

// clip level counts to the capacity (after an overflow the tree is reported as invalid)
__global__ void k_build_clip(int32_t *lvl, int64_t cap)
{
    if (threadIdx.x != 0) return;
    int32_t *off = lvl, *cnt = lvl + G4_NLEVELS + 1;
    for (int l = 0; l < G4_NLEVELS; l++) {
        int64_t e = (int64_t)off[l] + cnt[l];
        if (e > cap) cnt[l] = (int32_t)(cap - off[l] > 0 ? cap - off[l] : 0);
        if (l + 1 < G4_NLEVELS && off[l + 1] < off[l] + cnt[l]) off[l + 1] = off[l] + cnt[l];
    }
    off[G4_NLEVELS] = off[G4_NLEVELS - 1] + cnt[G4_NLEVELS - 1];   // total node count
}

__global__ void k_build_subtree(int level, const int32_t *__restrict__ lvl,
                                const int32_t *__restrict__ flags,
                                const int32_t *__restrict__ b_child,
                                const int32_t *__restrict__ b_nchild, int32_t *__restrict__ b_size)
{
    if (*flags & G4_FLAG_CAPACITY) return;   // invalid tree: links may be unset
    const int32_t *off = lvl, *cnt = lvl + G4_NLEVELS + 1;
    int o = off[level], c = cnt[level];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < c; b += gridDim.x * blockDim.x) {
        int node = o + b, s = 1, ch = b_child[node], nc = b_nchild[node];
        for (int j = 0; j < nc; j++) s += b_size[ch + j];
        b_size[node] = s;
    }
}

__global__ void k_build_dfs(int level, const int32_t *__restrict__ lvl,
                            const int32_t *__restrict__ flags,
                            const int32_t *__restrict__ b_child, const int32_t *__restrict__ b_nchild,
                            const int32_t *__restrict__ b_size, int32_t *__restrict__ b_dfs)
{
    if (*flags & G4_FLAG_CAPACITY) return;
    const int32_t *off = lvl, *cnt = lvl + G4_NLEVELS + 1;
    int o = off[level], c = cnt[level];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < c; b += gridDim.x * blockDim.x) {
        int node = o + b, ch = b_child[node], nc = b_nchild[node];
        int run = b_dfs[node] + 1;
        for (int j = 0; j < nc; j++) {
            b_dfs[ch + j] = run;
            run += b_size[ch + j];
        }
    }
}

__global__ void k_build_emit(const int32_t *__restrict__ lvl, const int32_t *__restrict__ flags,
                             const uint32_t *__restrict__ pos,
                             int n, const int32_t *__restrict__ b_first,
                             const int32_t *__restrict__ b_count, const int32_t *__restrict__ b_child,
                             const int32_t *__restrict__ b_nchild,
                             const int32_t *__restrict__ b_size, const int32_t *__restrict__ b_dfs,
                             const int32_t *__restrict__ b_parent, G4Node *__restrict__ node)
{
    if (*flags & G4_FLAG_CAPACITY) return;
    const int32_t *off = lvl, *cnt = lvl + G4_NLEVELS + 1;
    const int total = off[G4_NLEVELS];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < total; b += gridDim.x * blockDim.x) {
        // level of BFS slot b
        int l = 0;
        while (l + 1 < G4_NLEVELS && b >= off[l + 1]) l++;
        (void)cnt;
        int d = b_dfs[b], f = b_first[b];
        if ((unsigned)d >= (unsigned)total) continue;   // invalid tree
        if (b_count[b] == 0 || (unsigned)f >= (unsigned)n) f = 0;   // empty system root
        G4Node nd;
        uint32_t x[3] = {pos[f], pos[n + f], pos[2 * n + f]};
        uint32_t mask = (l == 0) ? 0u : ~((1u << (32 - l)) - 1u);
        uint32_t half = (l == 0) ? 0x80000000u : (1u << (31 - l));
        nd.cx = (x[0] & mask) + half;
        nd.cy = (x[1] & mask) + half;
        nd.cz = (x[2] & mask) + half;
        bool leaf = b_child[b] < 0;
        nd.meta = (uint32_t)l | (leaf ? 32u : 0u);
        nd.sx = nd.sy = nd.sz = 0.f;
        nd.mass = 0.f;
        nd.first = b_count[b] == 0 ? 0 : f;
        nd.count = b_count[b];
        nd.next = d + b_size[b];
        nd.parent = b_parent[b] >= 0 ? b_dfs[b_parent[b]] : -1;
        nd.amin = 0.f;
        nd.hmax = 0.f;
        nd.hmin = 0.f;
        nd.nchild = b_child[b] < 0 ? 0 : b_nchild[b];
        node[d] = nd;
    }
}

__global__ void k_tree_nodes(const G4Node *__restrict__ node, const int32_t *__restrict__ lvl,
                             int32_t *level, int32_t *first, int32_t *count, int32_t *next,
                             uint32_t *center)
{
    int total = lvl[G4_NLEVELS];
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < total; d += gridDim.x * blockDim.x) {
        G4Node nd = node[d];
        if (level) level[d] = nd.meta & 31;
        if (first) first[d] = nd.first;
        if (count) count[d] = nd.count;
        if (next) next[d] = nd.next;
        if (center) {
            center[3 * d] = nd.cx;
            center[3 * d + 1] = nd.cy;
            center[3 * d + 2] = nd.cz;
        }
    }
}

}  // namespace

// -------------------------------------------------------------------------------------------
// host side
// -------------------------------------------------------------------------------------------
extern "C" g4_status g4_tree_create(int64_t n_max, int64_t node_capacity, g4_tree *out)
{
    if (!out || n_max < 0 || n_max >= ((int64_t)1 << 31) || node_capacity < 0)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_tree_create: bad arguments");
    *out = nullptr;
    int64_t cap = node_capacity;
    if (cap == 0) cap = 4096 + n_max + n_max / 2;   // ample for leaf_max >= 2
    if (cap >= ((int64_t)1 << 31)) cap = ((int64_t)1 << 31) - 1;
    g4_tree t = new g4_tree_s();
    t->n_max = n_max;
    t->cap = cap;
    cudaGetDevice(&t->device);
    size_t c = (size_t)cap;
    cudaError_t e = cudaSuccess;
    auto A = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes > 0 ? bytes : 16);
    };
    // largest arrays first: an impossible request fails before anything else is taken
    A((void **)&t->q, sizeof(float) * g4_nq(G4_MAX_ORDER) * c);
    A((void **)&t->node, sizeof(G4Node) * c);
    A((void **)&t->b_first, 4 * c);
    A((void **)&t->b_count, 4 * c);
    A((void **)&t->b_child, 4 * c);
    A((void **)&t->b_nchild, 4 * c);
    A((void **)&t->b_size, 4 * c);
    A((void **)&t->b_dfs, 4 * c);
    A((void **)&t->b_parent, 4 * c);
    A((void **)&t->lvl, 4 * (2 * (G4_NLEVELS + 1) + 2));
    A((void **)&t->d_flags, 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g4_tree_free(t);
        return g4_fail(G4_ERR_OOM, "g4_tree_create: cudaMalloc failed for %lld nodes (%s)",
                       (long long)cap, cudaGetErrorString(e));
    }
    cudaMemset(t->d_flags, 0, 16);
    cudaMemset(t->lvl, 0, 4 * (2 * (G4_NLEVELS + 1) + 2));
    *out = t;
    return G4_OK;
}

extern "C" void g4_tree_free(g4_tree t)
{
    if (!t) return;
    cudaDeviceSynchronize();
    cudaFree(t->b_first);
    cudaFree(t->b_count);
    cudaFree(t->b_child);
    cudaFree(t->b_nchild);
    cudaFree(t->b_size);
    cudaFree(t->b_dfs);
    cudaFree(t->b_parent);
    cudaFree(t->lvl);
    cudaFree(t->d_flags);
    cudaFree(t->node);
    cudaFree(t->q);
    if (t->qd) cudaFree(t->qd);
    if (t->sys_goff) cudaFree(t->sys_goff);
    if (t->walk_queue) cudaFree(t->walk_queue);
    if (t->ew64) cudaFree(t->ew64);
    if (t->ew32) cudaFree(t->ew32);
    if (t->wnode) cudaFree(t->wnode);
    if (t->wpart) cudaFree(t->wpart);
    if (t->part_buf) cudaFree(t->part_buf);
    if (t->part_cnt) cudaFree(t->part_cnt);
    delete t;
}

extern "C" g4_status g4_tree_build(g4_tree t, const uint64_t *keys_sorted,
                                   const uint32_t *pos_sorted, int64_t n, const g4_params *P,
                                   void *stream)
{
    if (!t || !P || n < 0 || n > t->n_max || (n > 0 && (!keys_sorted || !pos_sorted)))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_tree_build: bad arguments");
    if (P->leaf_max < 1 || P->leaf_max > 64)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_tree_build: leaf_max=%d out of [1,64]", P->leaf_max);
    cudaStream_t st = (cudaStream_t)stream;
    k_build_init<<<1, 64, 0, st>>>(t->lvl, t->d_flags, t->b_first, t->b_count, t->b_parent,
                                   t->b_dfs, (int)n);
    int nb = g4_num_sms() * 4;
    for (int l = 0; l < G4_MAXLEVEL; l++)
        k_build_expand<<<nb, BUILD_THREADS, 0, st>>>(keys_sorted, l, P->leaf_max, t->cap, t->lvl,
                                                     t->d_flags, t->b_first, t->b_count,
                                                     t->b_child, t->b_nchild, t->b_parent);
    k_build_last<<<nb, BUILD_THREADS, 0, st>>>(t->lvl, t->cap, t->b_child, t->b_nchild);
    k_build_clip<<<1, 32, 0, st>>>(t->lvl, t->cap);
    for (int l = G4_MAXLEVEL; l >= 0; l--)
        k_build_subtree<<<nb, BUILD_THREADS, 0, st>>>(l, t->lvl, t->d_flags, t->b_child, t->b_nchild, t->b_size);
    for (int l = 0; l <= G4_MAXLEVEL; l++)
        k_build_dfs<<<nb, BUILD_THREADS, 0, st>>>(l, t->lvl, t->d_flags, t->b_child, t->b_nchild, t->b_size,
                                                  t->b_dfs);
    k_build_emit<<<nb, BUILD_THREADS, 0, st>>>(t->lvl, t->d_flags, pos_sorted, (int)n, t->b_first, t->b_count,
                                               t->b_child, t->b_nchild, t->b_size, t->b_dfs,
                                               t->b_parent, t->node);
    t->built_n = (int)n;
    t->moments_order = -1;
    t->n_sys = 0;
    t->sys_first = nullptr;
    t->sys_box = nullptr;
    return g4_launch_check("tree build", 4 + G4_MAXLEVEL + 2 * (G4_MAXLEVEL + 1));
}

extern "C" g4_status g4_tree_build_forest(g4_tree t, const uint64_t *keys_sorted,
                                          const uint32_t *pos_sorted, int64_t n,
                                          const int32_t *sys_first, const double *sys_box,
                                          int32_t n_sys, const g4_params *P, void *stream)
{
    if (!t || !P || n < 0 || n > t->n_max || n_sys < 1 || !sys_first || !sys_box ||
        (n > 0 && (!keys_sorted || !pos_sorted)))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_tree_build_forest: bad arguments");
    if (P->leaf_max < 1 || P->leaf_max > 64)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_tree_build_forest: leaf_max=%d", P->leaf_max);
    if ((int64_t)n_sys > t->cap)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_tree_build_forest: more systems than node capacity");
    if (n_sys > t->sys_cap) {
        // grows only when a larger batch arrives; steady-state calls allocate nothing
        if (t->sys_goff) cudaFree(t->sys_goff);
        t->sys_goff = nullptr;
        t->sys_cap = 0;
        if (cudaMalloc(&t->sys_goff, sizeof(int32_t) * (n_sys + 1)) != cudaSuccess) {
            cudaGetLastError();
            return g4_fail(G4_ERR_OOM, "g4_tree_build_forest: group offsets");
        }
        t->sys_cap = n_sys;
    }
    cudaStream_t st = (cudaStream_t)stream;
    k_build_init_forest<<<g4_blocks_for(n_sys, 256, 4), 256, 0, st>>>(
        t->lvl, t->d_flags, t->b_first, t->b_count, t->b_parent, sys_first, n_sys);
    int nb = g4_num_sms() * 4;
    for (int l = 0; l < G4_MAXLEVEL; l++)
        k_build_expand<<<nb, BUILD_THREADS, 0, st>>>(keys_sorted, l, P->leaf_max, t->cap, t->lvl,
                                                     t->d_flags, t->b_first, t->b_count,
                                                     t->b_child, t->b_nchild, t->b_parent);
    k_build_last<<<nb, BUILD_THREADS, 0, st>>>(t->lvl, t->cap, t->b_child, t->b_nchild);
    k_build_clip<<<1, 32, 0, st>>>(t->lvl, t->cap);
    for (int l = G4_MAXLEVEL; l >= 0; l--)
        k_build_subtree<<<nb, BUILD_THREADS, 0, st>>>(l, t->lvl, t->d_flags, t->b_child, t->b_nchild, t->b_size);
    k_forest_roots<<<1, 1024, 0, st>>>(t->b_size, sys_first, n_sys, t->b_dfs, t->sys_goff);
    for (int l = 0; l <= G4_MAXLEVEL; l++)
        k_build_dfs<<<nb, BUILD_THREADS, 0, st>>>(l, t->lvl, t->d_flags, t->b_child, t->b_nchild, t->b_size,
                                                  t->b_dfs);
    k_build_emit<<<nb, BUILD_THREADS, 0, st>>>(t->lvl, t->d_flags, pos_sorted, (int)n, t->b_first, t->b_count,
                                               t->b_child, t->b_nchild, t->b_size, t->b_dfs,
                                               t->b_parent, t->node);
    t->built_n = (int)n;
    t->moments_order = -1;
    t->n_sys = n_sys;
    t->sys_first = sys_first;
    t->sys_box = sys_box;
    return g4_launch_check("forest build", 5 + G4_MAXLEVEL + 2 * (G4_MAXLEVEL + 1));
}

extern "C" g4_status g4_tree_status(g4_tree t, int64_t *n_nodes, int32_t *max_level, void *stream)
{
    if (!t) return g4_fail(G4_ERR_INVALID_ARG, "g4_tree_status: NULL tree");
    int32_t h[2 * (G4_NLEVELS + 1)];
    int32_t flags = 0;
    cudaStream_t st = (cudaStream_t)stream;
    g4_status s = g4_cuda_check(cudaMemcpyAsync(h, t->lvl, sizeof(h), cudaMemcpyDeviceToHost, st),
                                "tree status");
    if (s != G4_OK) return s;
    s = g4_cuda_check(cudaMemcpyAsync(&flags, t->d_flags, 4, cudaMemcpyDeviceToHost, st), "flags");
    if (s != G4_OK) return s;
    s = g4_cuda_check(cudaStreamSynchronize(st), "tree status sync");
    if (s != G4_OK) return s;
    int32_t *off = h, *cnt = h + G4_NLEVELS + 1;
    int64_t total = t->built_n < 0 ? 0 : off[G4_NLEVELS];
    int ml = 0;
    for (int l = 0; l < G4_NLEVELS; l++)
        if (cnt[l] > 0) ml = l;
    t->n_nodes_host = total;
    if (n_nodes) *n_nodes = total;
    if (max_level) *max_level = ml;
    if (flags & (G4_FLAG_CAPACITY | G4_FLAG_LISTCAP))
        return g4_fail(G4_ERR_CAPACITY, "node or list capacity exceeded (flags=%d)", flags);
    if (flags & G4_FLAG_TIMEOUT) return g4_fail(G4_ERR_TIMEOUT, "device wait ran out");
    return G4_OK;
}

extern "C" g4_status g4_tree_nodes(g4_tree t, int32_t *level, int32_t *first, int32_t *count,
                                   int32_t *next, uint32_t *center, void *stream)
{
    if (!t || t->built_n < 0) return g4_fail(G4_ERR_STATE, "g4_tree_nodes: tree not built");
    k_tree_nodes<<<g4_num_sms() * 4, 256, 0, (cudaStream_t)stream>>>(t->node, t->lvl, level, first,
                                                                      count, next, center);
    return g4_launch_check("tree nodes", 1);
}
