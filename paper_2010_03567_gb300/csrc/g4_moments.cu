// g4_moments.cu -- upward pass (Sec. 2.2.2, Sec. 2.4 phase 1): node mass M, centre of mass s,
// multipole moments Q_n = sum m (x - s)^(n) for n = 2..p (Q_1 = 0 about s), largest softening
// and smallest |a_old| per node.
//
// One launch per level, deepest level first.  Leaves sum their particles; internal nodes
// combine their daughters with the binomial (parallel-axis) shift
//   Q^P_{abc} = sum_C sum_{a'<=a,b'<=b,c'<=c} C(a,a')C(b,b')C(c,c') Q^C_{a'b'c'} d_x^{a-a'}
//               d_y^{b-b'} d_z^{c-c'},   d = s_C - s_P,
// evaluated as three one-axis passes.
// Nodes holding >= fp64_count particles accumulate in FP64 (top of the tree), the rest in
// FP32; positions enter only as exact integer offsets from the node's geometric centre.
#include "g4_internal.cuh"

namespace {

__host__ __device__ constexpr int binom(int n, int k)
{
    int r = 1;
    for (int i = 0; i < k; i++) r = r * (n - i) / (i + 1);
    return r;
}

template <int P, typename T>
__device__ __forceinline__ void powers(T *px, T *py, T *pz, T dx, T dy, T dz)
{
    px[0] = py[0] = pz[0] = T(1);
#pragma unroll
    for (int k = 1; k <= P; k++) {
        px[k] = px[k - 1] * dx;
        py[k] = py[k - 1] * dy;
        pz[k] = pz[k - 1] * dz;
    }
}

// out += moments of `in` (orders 0..P about a point) re-expressed about a point displaced by
// -d (i.e. monomials of (x + d)); in[1..3] (first moments) are taken as zero.  The shift is
// separable: it is applied one axis at a time, (x+d)^a = sum_a' C(a,a') x^a' d^(a-a').
template <int P, typename T>
__device__ __forceinline__ void shift_add(T *__restrict__ out, const T *__restrict__ in, T dx, T dy,
                                          T dz)
{
    constexpr int NM = g4_nmono(P);
    T px[P + 1], py[P + 1], pz[P + 1];
    powers<P, T>(px, py, pz, dx, dy, dz);
    T u[NM], v[NM];
#pragma unroll
    for (int k = 0; k < NM; k++) u[k] = (k >= 1 && k <= 3) ? T(0) : in[k];
    // x pass: v_{abc} = sum_{a'<=a} C(a,a') u_{a'bc} dx^(a-a')
#pragma unroll
    for (int n = 0; n <= P; n++)
#pragma unroll
        for (int bc = 0; bc <= n; bc++)
#pragma unroll
            for (int c = 0; c <= bc; c++) {
                const int a = n - bc, b = bc - c;
                T s = T(0);
#pragma unroll
                for (int a2 = 0; a2 <= a; a2++)
                    s += T(binom(a, a2)) * u[g4_midx(a2, b, c)] * px[a - a2];
                v[g4_midx(a, b, c)] = s;
            }
    // y pass
#pragma unroll
    for (int n = 0; n <= P; n++)
#pragma unroll
        for (int bc = 0; bc <= n; bc++)
#pragma unroll
            for (int c = 0; c <= bc; c++) {
                const int a = n - bc, b = bc - c;
                T s = T(0);
#pragma unroll
                for (int b2 = 0; b2 <= b; b2++)
                    s += T(binom(b, b2)) * v[g4_midx(a, b2, c)] * py[b - b2];
                u[g4_midx(a, b, c)] = s;
            }
    // z pass, accumulated into out
#pragma unroll
    for (int n = 0; n <= P; n++)
#pragma unroll
        for (int bc = 0; bc <= n; bc++)
#pragma unroll
            for (int c = 0; c <= bc; c++) {
                const int a = n - bc, b = bc - c;
                T s = T(0);
#pragma unroll
                for (int c2 = 0; c2 <= c; c2++)
                    s += T(binom(c, c2)) * u[g4_midx(a, b, c2)] * pz[c - c2];
                out[g4_midx(a, b, c)] += s;
            }
}

template <int P, typename T>
__device__ __forceinline__ void mono_add(T *__restrict__ q, T m, T dx, T dy, T dz)
{
    T px[P + 1], py[P + 1], pz[P + 1];
    powers<P, T>(px, py, pz, dx, dy, dz);
#pragma unroll
    for (int n = 2; n <= P; n++)
#pragma unroll
        for (int bc = 0; bc <= n; bc++)
#pragma unroll
            for (int c = 0; c <= bc; c++) {
                const int a = n - bc, b = bc - c;
                q[g4_midx(a, b, c)] += m * px[a] * py[b] * pz[c];
            }
}

struct MomArgs {
    const uint32_t *pos;
    const float *mass;
    const uint8_t *cls;
    const float *aold;
    int n;
    const int32_t *lvl;
    const int32_t *b_dfs;
    const int32_t *b_child;   // first daughter's level-order slot per level-order slot
    G4Node *node;
    float *q;        // nq floats per node
    double *qd;      // precision 1: (4 + nq) doubles per node, or nullptr
    int nq;
    double scale;    // L / 2^32
    float h_cls[G4_MAX_EPS_CLASSES];   // 2.8 eps per class
    int fp64_count;
    int all_fp64;
    const int32_t *flags;
    const int32_t *sys_first;    // forest: per-system box sizes (n_sys = 0: one system)
    const double *sys_box;
    int n_sys;
};

template <int P, typename T>
__device__ void node_moments(const MomArgs &A, int d, const G4Node &nd, int slot)
{
    constexpr int NM = g4_nmono(P);
    T q[NM];
#pragma unroll
    for (int k = 0; k < NM; k++) q[k] = T(0);
    const T scale = A.n_sys ? (T)(A.sys_box[g4_system_of(A.sys_first, A.n_sys, nd.first)] *
                                  (1.0 / 4294967296.0))
                            : (T)A.scale;
    T M = T(0), sx = T(0), sy = T(0), sz = T(0);
    float hmax = 0.f, hmin = 3.0e38f, amin = 3.0e38f;
    const bool leaf = nd.meta & 32u;
    if (leaf) {
        const int f = nd.first, e = nd.first + nd.count;
#pragma unroll 4
        for (int j = f; j < e; j++) {
            T m = (T)A.mass[j];
            M += m;
            sx += m * ((T)(int32_t)(A.pos[j] - nd.cx) * scale);
            sy += m * ((T)(int32_t)(A.pos[A.n + j] - nd.cy) * scale);
            sz += m * ((T)(int32_t)(A.pos[2 * A.n + j] - nd.cz) * scale);
            const float hj = A.h_cls[A.cls ? A.cls[j] : 0];
            hmax = fmaxf(hmax, hj);
            hmin = fminf(hmin, hj);
            amin = fminf(amin, A.aold ? A.aold[j] : 0.f);
        }
        const T inv = M > T(0) ? T(1) / M : T(0);
        sx *= inv;
        sy *= inv;
        sz *= inv;
#pragma unroll 4
        for (int j = f; j < e; j++) {
            T dx = (T)(int32_t)(A.pos[j] - nd.cx) * scale - sx;
            T dy = (T)(int32_t)(A.pos[A.n + j] - nd.cy) * scale - sy;
            T dz = (T)(int32_t)(A.pos[2 * A.n + j] - nd.cz) * scale - sz;
            mono_add<P, T>(q, (T)A.mass[j], dx, dy, dz);
        }
    } else {
        // daughters in key order, from the level-ordered child slots (independent loads)
        const int c0 = A.b_child[slot], nch = min(nd.nchild, 8);
        int chs[8];
#pragma unroll
        for (int k = 0; k < 8; k++) chs[k] = k < nch ? A.b_dfs[c0 + k] : 0;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if (k >= nch) break;
            const int ch = chs[k];
            const G4Node &c = A.node[ch];
            T mc = (T)c.mass, ox = (T)c.sx, oy = (T)c.sy, oz = (T)c.sz;
            if (A.all_fp64 && A.qd) {
                const double *src = A.qd + (size_t)ch * (4 + A.nq);
                mc = (T)src[3];
                ox = (T)src[0];
                oy = (T)src[1];
                oz = (T)src[2];
            }
            M += mc;
            sx += mc * ((T)(int32_t)(c.cx - nd.cx) * scale + ox);
            sy += mc * ((T)(int32_t)(c.cy - nd.cy) * scale + oy);
            sz += mc * ((T)(int32_t)(c.cz - nd.cz) * scale + oz);
            hmax = fmaxf(hmax, c.hmax);
            hmin = fminf(hmin, c.hmin);
            amin = fminf(amin, c.amin);
        }
        const T inv = M > T(0) ? T(1) / M : T(0);
        sx *= inv;
        sy *= inv;
        sz *= inv;
#pragma unroll 1
        for (int k = 0; k < nch; k++) {
            const int ch = chs[k];
            const G4Node &c = A.node[ch];
            T qc[NM];
            qc[0] = (T)c.mass;
            qc[1] = qc[2] = qc[3] = T(0);
            if (A.all_fp64 && A.qd) {
                const double *src = A.qd + (size_t)ch * (4 + A.nq);
                qc[0] = (T)src[3];
#pragma unroll
                for (int k = 4; k < NM; k++) qc[k] = (T)src[4 + k - 4];
            } else {
#pragma unroll
                for (int k = 4; k < NM; k++) qc[k] = (T)A.q[(size_t)ch * A.nq + k - 4];
            }
            T dx, dy, dz;
            if (A.all_fp64 && A.qd) {
                const double *src = A.qd + (size_t)ch * (4 + A.nq);
                dx = (T)(int32_t)(c.cx - nd.cx) * scale + (T)src[0] - sx;
                dy = (T)(int32_t)(c.cy - nd.cy) * scale + (T)src[1] - sy;
                dz = (T)(int32_t)(c.cz - nd.cz) * scale + (T)src[2] - sz;
            } else {
                dx = (T)(int32_t)(c.cx - nd.cx) * scale + (T)c.sx - sx;
                dy = (T)(int32_t)(c.cy - nd.cy) * scale + (T)c.sy - sy;
                dz = (T)(int32_t)(c.cz - nd.cz) * scale + (T)c.sz - sz;
            }
            shift_add<P, T>(q, qc, dx, dy, dz);
        }
    }
    G4Node &o = A.node[d];
    o.sx = (float)sx;
    o.sy = (float)sy;
    o.sz = (float)sz;
    o.mass = (float)M;
    o.hmax = hmax;
    o.hmin = hmin;
    o.amin = amin;
    float *dst = A.q + (size_t)d * A.nq;
#pragma unroll
    for (int k = 4; k < NM; k++) dst[k - 4] = (float)q[k];
    if (A.qd) {
        double *dd = A.qd + (size_t)d * (4 + A.nq);
        dd[0] = (double)sx;
        dd[1] = (double)sy;
        dd[2] = (double)sz;
        dd[3] = (double)M;
#pragma unroll
        for (int k = 4; k < NM; k++) dd[4 + k - 4] = (double)q[k];
    }
}

// sum over lanes 0..7 (the others hold zero); the result is valid in lanes 0..7
template <typename T>
__device__ __forceinline__ T octet_sum(T v)
{
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

// The internal-node combination of node_moments with one lane per daughter (at most eight):
// each lane shifts its daughter's moments to the node's centre of mass and the eight
// contributions are summed across lanes, so a large node costs one daughter's shift instead
// of eight in a row (this matters in FP64, where one thread's chain of products is slow).
// Only the order of the sums over daughters differs from node_moments.
template <int P, typename T>
__device__ void node_moments_warp(const MomArgs &A, int d, const G4Node &nd, int slot, int lane)
{
    constexpr int NM = g4_nmono(P);
    const T scale = A.n_sys ? (T)(A.sys_box[g4_system_of(A.sys_first, A.n_sys, nd.first)] *
                                  (1.0 / 4294967296.0))
                            : (T)A.scale;
    const bool has = lane < nd.nchild;
    T mc = T(0), ex = T(0), ey = T(0), ez = T(0);
    T qc[NM];
#pragma unroll
    for (int k = 0; k < NM; k++) qc[k] = T(0);
    float hmax = 0.f, hmin = 3.0e38f, amin = 3.0e38f;
    if (has) {
        const int ch = A.b_dfs[A.b_child[slot] + lane];
        const G4Node c = A.node[ch];
        T ox = (T)c.sx, oy = (T)c.sy, oz = (T)c.sz;
        mc = (T)c.mass;
        if (A.all_fp64 && A.qd) {
            const double *src = A.qd + (size_t)ch * (4 + A.nq);
            mc = (T)src[3];
            ox = (T)src[0];
            oy = (T)src[1];
            oz = (T)src[2];
#pragma unroll
            for (int k = 4; k < NM; k++) qc[k] = (T)src[4 + k - 4];
        } else {
#pragma unroll
            for (int k = 4; k < NM; k++) qc[k] = (T)A.q[(size_t)ch * A.nq + k - 4];
        }
        qc[0] = mc;
        // daughter's centre of mass relative to the node's geometric centre
        ex = (T)(int32_t)(c.cx - nd.cx) * scale + ox;
        ey = (T)(int32_t)(c.cy - nd.cy) * scale + oy;
        ez = (T)(int32_t)(c.cz - nd.cz) * scale + oz;
        hmax = c.hmax;
        hmin = c.hmin;
        amin = c.amin;
    }
    const T M = octet_sum(mc);
    const T inv = M > T(0) ? T(1) / M : T(0);
    const T sx = octet_sum(mc * ex) * inv, sy = octet_sum(mc * ey) * inv,
            sz = octet_sum(mc * ez) * inv;
    T q[NM];
#pragma unroll
    for (int k = 0; k < NM; k++) q[k] = T(0);
    if (has) shift_add<P, T>(q, qc, ex - sx, ey - sy, ez - sz);
#pragma unroll
    for (int k = 4; k < NM; k++) q[k] = octet_sum(q[k]);
#pragma unroll
    for (int s = 4; s >= 1; s >>= 1) {
        hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, s));
        hmin = fminf(hmin, __shfl_xor_sync(0xffffffffu, hmin, s));
        amin = fminf(amin, __shfl_xor_sync(0xffffffffu, amin, s));
    }
    if (lane != 0) return;
    G4Node &o = A.node[d];
    o.sx = (float)sx;
    o.sy = (float)sy;
    o.sz = (float)sz;
    o.mass = (float)M;
    o.hmax = hmax;
    o.hmin = hmin;
    o.amin = amin;
    float *dst = A.q + (size_t)d * A.nq;
#pragma unroll
    for (int k = 4; k < NM; k++) dst[k - 4] = (float)q[k];
    if (A.qd) {
        double *dd = A.qd + (size_t)d * (4 + A.nq);
        dd[0] = (double)sx;
        dd[1] = (double)sy;
        dd[2] = (double)sz;
        dd[3] = (double)M;
#pragma unroll
        for (int k = 4; k < NM; k++) dd[4 + k - 4] = (double)q[k];
    }
}

template <int P>
__global__ void __launch_bounds__(128) k_moments_level(const MomArgs A, int level)
{
    const int32_t *off = A.lvl, *cnt = A.lvl + G4_NLEVELS + 1;
    const int o = off[level], c = cnt[level];
    if (*A.flags & G4_FLAG_CAPACITY) return;   // the tree is incomplete: leave it untouched
    const int total = off[G4_NLEVELS];
    if (c <= (int)((gridDim.x * blockDim.x) >> 5)) {
        // few (large) nodes: a warp per node, a lane per daughter
        const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
        if (b >= c) return;
        const int d = A.b_dfs[o + b];
        if ((unsigned)d >= (unsigned)total) return;
        const G4Node nd = A.node[d];
        const bool fp64 = A.all_fp64 || nd.count >= A.fp64_count;
        if (nd.meta & 32u) {
            if (lane == 0) {
                if (fp64) node_moments<P, double>(A, d, nd, o + b);
                else node_moments<P, float>(A, d, nd, o + b);
            }
        } else if (fp64) {
            node_moments_warp<P, double>(A, d, nd, o + b, lane);
        } else {
            node_moments_warp<P, float>(A, d, nd, o + b, lane);
        }
        return;
    }
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < c; b += gridDim.x * blockDim.x) {
        const int d = A.b_dfs[o + b];
        if ((unsigned)d >= (unsigned)total) continue;
        const G4Node nd = A.node[d];
        if (A.all_fp64 || nd.count >= A.fp64_count) node_moments<P, double>(A, d, nd, o + b);
        else node_moments<P, float>(A, d, nd, o + b);
    }
}

__global__ void k_export_moments(const G4Node *__restrict__ node, const float *__restrict__ q,
                                 const double *__restrict__ qd, int nq, int nmono,
                                 const int32_t *__restrict__ lvl, double scale, double *mass,
                                 double *com, double *mono)
{
    int total = lvl[G4_NLEVELS];
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < total; d += gridDim.x * blockDim.x) {
        const G4Node nd = node[d];
        const double *dd = qd ? qd + (size_t)d * (4 + nq) : nullptr;
        double m = dd ? dd[3] : nd.mass;
        if (mass) mass[d] = m;
        if (com) {
            com[3 * d] = dd ? dd[0] : nd.sx;
            com[3 * d + 1] = dd ? dd[1] : nd.sy;
            com[3 * d + 2] = dd ? dd[2] : nd.sz;
        }
        if (mono) {
            double *o = mono + (size_t)d * nmono;
            o[0] = m;
            o[1] = o[2] = o[3] = 0.0;
            for (int k = 4; k < nmono; k++) o[k] = dd ? dd[k] : (double)q[(size_t)d * nq + k - 4];
        }
    }
}

}  // namespace

extern "C" g4_status g4_multipoles(g4_tree t, const uint32_t *pos_sorted, const float *mass_sorted,
                                   const uint8_t *cls_sorted, const float *aold_sorted,
                                   const g4_params *P, void *stream)
{
    if (!t || !P || !pos_sorted || !mass_sorted)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_multipoles: bad arguments");
    if (t->built_n < 0) return g4_fail(G4_ERR_STATE, "g4_multipoles: tree not built");
    if (P->order_p < 1 || P->order_p > G4_MAX_ORDER)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_multipoles: order_p=%d", P->order_p);
    if (P->n_eps_classes < 1 || P->n_eps_classes > G4_MAX_EPS_CLASSES)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_multipoles: n_eps_classes=%d", P->n_eps_classes);
    cudaStream_t st = (cudaStream_t)stream;
    const int p = P->order_p;
    MomArgs A;
    A.pos = pos_sorted;
    A.mass = mass_sorted;
    A.cls = cls_sorted;
    A.aold = aold_sorted;
    A.n = t->built_n;
    A.lvl = t->lvl;
    A.b_dfs = t->b_dfs;
    A.b_child = t->b_child;
    A.node = t->node;
    A.q = t->q;
    A.nq = g4_nq(p);
    A.scale = P->box_size / 4294967296.0;
    for (int k = 0; k < G4_MAX_EPS_CLASSES; k++)
        A.h_cls[k] = k < P->n_eps_classes ? (float)(2.8 * P->eps_table[k]) : 0.f;
    A.fp64_count = P->fp64_count > 0 ? P->fp64_count : 4096;
    A.all_fp64 = P->precision == 1;
    A.flags = t->d_flags;
    A.sys_first = t->sys_first;
    A.sys_box = t->sys_box;
    A.n_sys = t->n_sys;
    A.qd = nullptr;
    if (P->precision == 1) {
        if (!t->qd) {
            if (cudaMalloc(&t->qd, sizeof(double) * (4 + g4_nq(G4_MAX_ORDER)) * (size_t)t->cap) !=
                cudaSuccess) {
                cudaGetLastError();
                t->qd = nullptr;
                return g4_fail(G4_ERR_OOM, "g4_multipoles: FP64 moment arrays");
            }
        }
        A.qd = t->qd;
    }
    int nb = g4_num_sms() * 8;
    for (int l = G4_MAXLEVEL; l >= 0; l--) {
        switch (p) {
        case 1: k_moments_level<1><<<nb, 128, 0, st>>>(A, l); break;
        case 2: k_moments_level<2><<<nb, 128, 0, st>>>(A, l); break;
        case 3: k_moments_level<3><<<nb, 128, 0, st>>>(A, l); break;
        case 4: k_moments_level<4><<<nb, 128, 0, st>>>(A, l); break;
        default: k_moments_level<5><<<nb, 128, 0, st>>>(A, l); break;
        }
    }
    t->moments_order = p;
    t->moments_stamp++;
    t->moments_fp64 = P->precision == 1;
    return g4_launch_check("multipoles", G4_MAXLEVEL + 1);
}

extern "C" g4_status g4_tree_moments(g4_tree t, double *mass, double *com, double *mono,
                                     void *stream)
{
    if (!t || t->moments_order < 0) return g4_fail(G4_ERR_STATE, "g4_tree_moments: no moments");
    const int p = t->moments_order;
    k_export_moments<<<g4_num_sms() * 4, 256, 0, (cudaStream_t)stream>>>(
        t->node, t->q, t->moments_fp64 ? t->qd : nullptr, g4_nq(p), g4_nmono(p), t->lvl, 0.0, mass,
        com, mono);
    return g4_launch_check("export moments", 1);
}
