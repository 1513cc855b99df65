// g4_fmm.cu -- entry points of the symmetric Cartesian FMM (Sec. 2.4, Sec. 2.5): workspace
// layout, argument checks and the launch sequence.  The dual walk's kernels are in g4_fmm.cuh;
// g4_fmm_variant.cu compiles them once per (order, TreePM) variant.
#include "g4_fmm_args.cuh"

using g4fmm::FmmArgs;

namespace {

__global__ void k_fmm_reset(int32_t *dcount, double *mom)
{
    if (threadIdx.x < 2) dcount[threadIdx.x] = 0;
    if (mom && threadIdx.x < 3) mom[threadIdx.x] = 0.0;
}

// kids[8 d + c]: depth-first index of daughter c of the node with depth-first index d (-1
// past its daughters); the level-ordered build keeps a node's daughters consecutive
__global__ void k_fmm_kids(const int32_t *__restrict__ lvl, const int32_t *__restrict__ b_dfs,
                           const int32_t *__restrict__ b_child, const int32_t *__restrict__ b_nchild,
                           int64_t cap, int32_t *__restrict__ kids)
{
    const int64_t nn = lvl[G4_NLEVELS];
    for (int64_t lo = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; lo < nn && lo < cap;
         lo += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = b_dfs[lo], nc = b_nchild[lo], c0 = b_child[lo];
        for (int c = 0; c < 8; c++) kids[(size_t)d * 8 + c] = c < nc ? b_dfs[c0 + c] : -1;
    }
}

__global__ void k_momentum(const float *__restrict__ mass, const float *__restrict__ acc, int n,
                           double *__restrict__ mom)
{
    double s[3] = {0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double m = mass[i];
        s[0] += m * acc[i];
        s[1] += m * acc[n + i];
        s[2] += m * acc[2 * n + i];
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
        if ((threadIdx.x & 31) == 0) atomicAdd(mom + k, s[k]);
    }
}


template <int P, typename R>
void dispatch_fmm(const FmmArgs &A, bool treepm, bool geom, cudaStream_t st)
{
    if (treepm) g4fmm::run_variant<P, true, R>(A, geom, st);
    else g4fmm::run_variant<P, false, R>(A, geom, st);
}

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct FmmLayout {
    size_t T_own, T_tot, Doff, Dlen, m2l_own, m2l_cum, dcount, p2p_src, p2p_chunk, p2p_head,
        p2p_sinks, p2p_fill, kids, D0, D1, total;
    int64_t dcap, p2p_cap, chunk_cap;
};

// deferred particle-pair lists: 16 entries (16 bytes each) and 1.25 chunks per particle of the
// handle (plus a floor for small sets); overflowing chunks are evaluated by the dual walk itself
FmmLayout fmm_layout(int64_t nodes, int64_t n_max, int nt, size_t ws_bytes, int per_particle,
                     size_t tbytes)
{
    FmmLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += al256(bytes); return r; };
    L.T_own = take(tbytes * nt * nodes);   // field tensors: float, or double (FP64 mode)
    L.T_tot = take(tbytes * nt * nodes);
    L.Doff = take(4 * nodes);
    L.Dlen = take(4 * nodes);
    L.m2l_own = take(4 * nodes);
    L.m2l_cum = take(4 * nodes);
    L.dcount = take(16);
    const int64_t nm = n_max > 0 ? n_max : 1;
    if (per_particle <= 0) {
        L.p2p_cap = 16 * nm + ((int64_t)1 << 20);
        L.chunk_cap = nm + nm / 4 + ((int64_t)1 << 14);
    } else {   // explicit budget (small values exercise the in-walk evaluation)
        L.p2p_cap = (int64_t)per_particle * nm;
        L.chunk_cap = L.p2p_cap / 8 + 1;
    }
    L.p2p_src = take(16 * (size_t)L.p2p_cap);
    L.p2p_chunk = take(16 * (size_t)L.chunk_cap);
    L.p2p_head = take(4 * nodes);
    L.p2p_sinks = take(4 * nodes);
    L.p2p_fill = take(16);
    L.kids = take(32 * nodes);
    size_t fixed = o;
    int64_t dcap = 0;
    if (ws_bytes == 0) dcap = (int64_t)1 << 20 > 48 * nodes ? (int64_t)1 << 20 : 48 * nodes;
    else dcap = ws_bytes > fixed + 1024 ? (int64_t)((ws_bytes - fixed - 1024) / 16) : 0;
    if (dcap > ((int64_t)1 << 31) - 1) dcap = ((int64_t)1 << 31) - 1;
    L.D0 = take(8 * dcap);
    L.D1 = take(8 * dcap);
    L.dcap = dcap;
    L.total = o;
    return L;
}

}  // namespace

double g4_r_cut(const g4_params *P);
g4_status g4_check_params(const g4_params *P, const char *who);

extern "C" g4_status g4_fmm_workspace(g4_tree t, const g4_params *P, size_t *bytes)
{
    g4_status s = g4_check_params(P, "g4_fmm_workspace");
    if (s != G4_OK) return s;
    if (!t || !bytes) return g4_fail(G4_ERR_INVALID_ARG, "g4_fmm_workspace: NULL argument");
    // sized for the handle's node capacity, so no host synchronisation is needed
    *bytes = fmm_layout(t->cap, t->n_max, g4_nmono(P->order_p), 0, P->fmm_p2p_per_particle,
                        P->precision == 1 ? sizeof(double) : sizeof(float)).total;
    return G4_OK;
}

extern "C" g4_status g4_gravity_fmm(g4_tree t, const uint32_t *pos_sorted, const float *mass_sorted,
                                    const uint8_t *cls_sorted, const float *aold_sorted,
                                    const g4_params *P, float *acc, float *pot, uint32_t *counts,
                                    double *momentum_out, void *workspace, size_t workspace_bytes,
                                    void *stream)
{
    g4_status s = g4_check_params(P, "g4_gravity_fmm");
    if (s != G4_OK) return s;
    if (!t || !pos_sorted || !mass_sorted || !acc || !workspace)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_fmm: NULL argument");
    if (P->criterion == 0 && !aold_sorted)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_fmm: relative criterion needs a_old");
    if (((uintptr_t)workspace & 255) != 0)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_fmm: workspace not 256-byte aligned");
    if (t->built_n < 0 || t->moments_order < 0)
        return g4_fail(G4_ERR_STATE, "g4_gravity_fmm: build and multipoles must run first");
    if (t->moments_order != P->order_p)
        return g4_fail(G4_ERR_STATE, "g4_gravity_fmm: moments of order %d, FMM order %d",
                       t->moments_order, P->order_p);
    if (P->order_p < 2 || P->order_p > 5)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_fmm: order_p must be in [2,5]");
    if (P->precision == 1 && P->order_p != 4)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_fmm: the FP64 mode is built for order_p 4");
    if (P->precision == 1 && !t->moments_fp64)
        return g4_fail(G4_ERR_STATE, "g4_gravity_fmm: FP64 mode needs FP64 multipoles");
    const int n = t->built_n;
    if (n == 0) return G4_OK;
    const int nt = g4_nmono(P->order_p);
    // node count bound: the handle's capacity (no host synchronisation here)
    const bool fp64 = P->precision == 1;
    FmmLayout L = fmm_layout(t->cap, t->n_max, nt, workspace_bytes, P->fmm_p2p_per_particle,
                             fp64 ? sizeof(double) : sizeof(float));
    if (L.dcap < 1024 || L.total > workspace_bytes)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_fmm: workspace too small (%zu bytes)",
                       workspace_bytes);
    char *w = (char *)workspace;
    FmmArgs A;
    A.pos = pos_sorted;
    A.mass = mass_sorted;
    A.cls = cls_sorted;
    A.aold = aold_sorted;
    A.n = n;
    A.lvl = t->lvl;
    A.b_dfs = t->b_dfs;
    A.node = t->node;
    A.q = t->q;
    A.qd = fp64 ? t->qd : nullptr;
    A.nq = g4_nq(P->order_p);
    A.T_own = (void *)(w + L.T_own);
    A.T_tot = (void *)(w + L.T_tot);
    A.Doff = (int32_t *)(w + L.Doff);
    A.Dlen = (int32_t *)(w + L.Dlen);
    A.m2l_own = (uint32_t *)(w + L.m2l_own);
    A.m2l_cum = (uint32_t *)(w + L.m2l_cum);
    A.dcount = (int32_t *)(w + L.dcount);
    A.D0 = (int2 *)(w + L.D0);
    A.D1 = (int2 *)(w + L.D1);
    A.dcap = L.dcap;
    A.p2p_src = (int4 *)(w + L.p2p_src);
    A.p2p_chunk = (int4 *)(w + L.p2p_chunk);
    A.p2p_head = (int32_t *)(w + L.p2p_head);
    A.p2p_sinks = (int32_t *)(w + L.p2p_sinks);
    A.p2p_fill = (int32_t *)(w + L.p2p_fill);
    A.kids = (const int32_t *)(w + L.kids);
    A.p2p_cap = L.p2p_cap;
    A.chunk_cap = L.chunk_cap;
    A.flags = t->d_flags;
    A.acc = acc;
    A.pot = pot;
    A.counts = counts;
    A.momentum = momentum_out;
    A.scale = P->box_size / 4294967296.0;
    A.G = P->G;
    A.alpha = P->alpha;
    A.theta2 = P->theta * P->theta;
    const bool treepm = P->r_s > 0.0;
    const double rc = treepm ? g4_r_cut(P) : 0.0;
    A.rcut2 = rc * rc;
    A.as = treepm ? 0.5 / P->r_s : 0.0;
    A.box = P->box_size;
    for (int k = 0; k < G4_MAX_EPS_CLASSES; k++)
        A.h_cls[k] = k < P->n_eps_classes ? (float)(2.8 * P->eps_table[k]) : 0.f;
    A.exclusion = P->exclusion_zone;
    A.pp_cut = P->pp_cut;
    A.keep_qp = P->keep_qp;
    A.soft_nodes = P->soft_nodes;
    A.ewald = P->ewald;
    A.periodic = P->periodic;
    A.ew = G4EwaldView{nullptr, nullptr, 0, 1, 1.0};
    A.rcut2f = (float)A.rcut2;
    A.asf = (float)A.as;
    const double igs = 4294967296.0 / P->box_size;
    A.figs = (float)igs;
    A.rc2i = (float)(A.rcut2 * igs * igs);
    A.pf = g4k::make_pairf(A.as * A.scale, treepm ? 2.0 * P->r_s * igs : 0.0);
    cudaStream_t st = (cudaStream_t)stream;
    if (P->ewald) {
        s = g4_ewald_ensure(t, P->box_size, P->order_p + 3, st, &A.ew);
        if (s != G4_OK) return s;
    }
    s = g4_particle_records(t, pos_sorted, mass_sorted, n, st);
    if (s != G4_OK) return s;
    A.wpart = t->wpart;
    k_fmm_reset<<<1, 32, 0, st>>>(A.dcount, momentum_out);
    // each node's daughters by depth-first index (daughters are consecutive in level order)
    k_fmm_kids<<<g4_blocks_for(t->cap, 256), 256, 0, st>>>(t->lvl, t->b_dfs, t->b_child,
                                                          t->b_nchild, t->cap,
                                                          (int32_t *)(w + L.kids));
    if (cudaMemsetAsync(A.p2p_fill, 0, 16, st) != cudaSuccess)
        return g4_cuda_check(cudaGetLastError(), "g4_gravity_fmm: clear P2P counters");
    const bool geom = P->criterion == 1;
    if (fp64) {
        dispatch_fmm<4, double>(A, treepm, geom, st);
    } else {
        switch (P->order_p) {
        case 2: dispatch_fmm<2, float>(A, treepm, geom, st); break;
        case 3: dispatch_fmm<3, float>(A, treepm, geom, st); break;
        case 4: dispatch_fmm<4, float>(A, treepm, geom, st); break;
        default: dispatch_fmm<5, float>(A, treepm, geom, st); break;
        }
    }
    if (momentum_out) k_momentum<<<g4_num_sms() * 4, 256, 0, st>>>(mass_sorted, acc, n, momentum_out);
    return g4_launch_check("fmm", 3 + 2 * (G4_MAXLEVEL + 1) + (momentum_out ? 1 : 0));
}
