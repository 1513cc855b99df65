// g4_fmm.cu -- symmetric Cartesian fast multipole method (Sec. 2.4, Sec. 2.5).
//
// The paper's dual tree walk visits unordered node pairs.  Its decisions are symmetric in the
// two nodes, so the same interactions are found by visiting ordered pairs (A, B) -- sink A,
// source B -- where pair (A, B) and pair (B, A) receive the same decision.  That makes the
// walk sink-centric and free of write conflicts:
//
//   level by level, top-down, one warp per sink node A:
//     candidates of A = the list its parent passed down (the root starts with itself);
//     for each candidate B (lanes in parallel):
//       B == A        : internal -> pass A's daughters down; leaf -> P2P within A
//       gap > r_cut   : drop
//       accepted      : field of B's multipoles at A's centre of mass (M2L, one direction)
//       A, B leaves   : P2P, A's particles from B's
//       A leaf        : B is opened in place (its daughters become candidates of A)
//       otherwise     : passed down to A's daughters (B itself if B is a leaf, else its
//                       daughters), i.e. both nodes are opened ("open both", Sec. 2.4)
//   then level by level, top-down: L2L shift of the parent's field, L2P at the leaves.
//
// The field tensor of A from source B is, with r = s_B - s_A (multi-index form),
//   T^A_k = -G (-1)^|k| sum_n Q^B_n D_{k+n}(r) / n!      (|k| + |n| <= p, |n| != 1, |n| != p)
// and the potential near A's centre of mass is Phi(s_A + a) = sum_k T_k a^k / k!.
#include "g4_internal.cuh"
#include "g4_kernels.cuh"
#include "g4_pp.cuh"

namespace {

using namespace g4k;

constexpr int FMM_THREADS = 128;
constexpr int FMM_WARPS = FMM_THREADS / 32;
constexpr int FMM_STACK = 1024;     // per-warp stack of opened sources for leaf sinks
constexpr int FMM_P2PBUF = 128;     // per-warp buffer of P2P source leaves (one deferred chunk)

enum : int { D_DROP = 0, D_ACCEPT = 1, D_P2P = 2, D_OPEN = 3, D_SELF = 4 };

struct FmmArgs {
    const uint32_t *pos;
    const float *mass;
    const uint8_t *cls;
    int n;
    const int32_t *lvl;
    const int32_t *b_dfs;
    const G4Node *node;
    const float *q;
    int nq;
    float *T_own, *T_tot;
    int32_t *D0, *D1;          // pass-down candidate lists, by level parity
    int64_t dcap;
    int32_t *dcount;           // [2] list fill counters
    int32_t *Doff, *Dlen;      // per node: its pass-down list
    uint32_t *m2l_own, *m2l_cum;
    int32_t *flags;
    float *acc, *pot;
    uint32_t *counts;
    double *momentum;
    double scale, G, alpha, theta2, rcut2, as, box;
    float h_cls[G4_MAX_EPS_CLASSES];
    int exclusion, pp_cut, keep_qp;
    // particle-particle phase (shared with the tree walk)
    const uint4 *wpart;        // particles as (x, y, z, mass bits)
    float rcut2f, asf, figs, rc2i;
    PairF pf;
    // deferred leaf-leaf work: chunks of source leaves per sink leaf, chained in the order the
    // sink's warp found them; evaluated after the dual walk by k_fmm_p2p
    int32_t *p2p_src;          // source leaf (depth-first index) lists
    int4 *p2p_chunk;           // (offset, count, next chunk, -)
    int32_t *p2p_head;         // per node: first chunk of a sink leaf, -1 if none
    int32_t *p2p_sinks;        // sink leaves with P2P work
    int32_t *p2p_fill;         // [0] list entries, [1] chunks, [2] sink leaves
    int64_t p2p_cap, chunk_cap;
};

template <int P> struct FT { static constexpr int NT = g4_nmono(P); };

__device__ __forceinline__ float fside(double box, int lv) { return ldexpf((float)box, -lv); }

// decision for the ordered pair (A <- B), identical to the symmetric rule of the dual walk
template <int P, bool TREEPM, bool GEOM>
__device__ __forceinline__ int fmm_decide(const FmmArgs &A, const G4Node &na, int da,
                                          const G4Node &nb, int db, float &rx, float &ry, float &rz)
{
    const bool la = na.meta & 32u, lb = nb.meta & 32u;
    if (da == db) return la ? D_SELF : D_OPEN;
    const float scale = (float)A.scale;
    const float lA = fside(A.box, na.meta & 31u), lB = fside(A.box, nb.meta & 31u);
    const float hl = 0.5f * (lA + lB);
    const float dcx = (float)(int32_t)(nb.cx - na.cx) * scale;
    const float dcy = (float)(int32_t)(nb.cy - na.cy) * scale;
    const float dcz = (float)(int32_t)(nb.cz - na.cz) * scale;
    if (TREEPM) {
        const float ex = fmaxf(fabsf(dcx) - hl, 0.f), ey = fmaxf(fabsf(dcy) - hl, 0.f),
                    ez = fmaxf(fabsf(dcz) - hl, 0.f);
        if (ex * ex + ey * ey + ez * ez > (float)A.rcut2) return D_DROP;
    }
    rx = dcx + (nb.sx - na.sx);
    ry = dcy + (nb.sy - na.sy);
    rz = dcz + (nb.sz - na.sz);
    const float r2 = rx * rx + ry * ry + rz * rz;
    bool accept = true;
    const float dmax = fmaxf(fabsf(dcx), fmaxf(fabsf(dcy), fabsf(dcz)));
    if (A.exclusion && dmax <= hl) accept = false;   // touching nodes never interact
    if (dmax < hl) accept = false;                   // overlapping cubes
    const float h = fmaxf(na.hmax, nb.hmax);
    if (r2 < h * h) accept = false;                  // multipoles are unsoftened
    if (accept) {
        if (GEOM) {
            accept = (lA + lB) * (lA + lB) < (float)A.theta2 * r2;
        } else {
            const float r = sqrtf(r2);
            const float lmax = fmaxf(lA, lB), mmax = fmaxf(na.mass, nb.mass);
            float lp = 1.f, rp = r2;
#pragma unroll
            for (int i = 0; i < P - 1; i++) {
                lp *= lmax;
                rp *= r;
            }
            const float amin = fminf(na.amin, nb.amin);
            accept = (float)A.G * mmax * lp < (float)A.alpha * amin * rp;
        }
    }
    if (accept) return D_ACCEPT;
    if (la && lb) return D_P2P;
    return D_OPEN;
}

// lane-private M2L: T += field of node B at A's centre of mass (r = s_B - s_A)
template <int P, bool TREEPM>
__device__ __forceinline__ void m2l_add(const FmmArgs &A, float *T, int db, const G4Node &nb,
                                        float rx, float ry, float rz)
{
    constexpr int NT = FT<P>::NT;
    const float r2 = rx * rx + ry * ry + rz * rz;
    float g[P + 1];
    gn_kernel<P, float, TREEPM>(r2, (float)A.as, g);
    float D[NT];
    dtensors<P, float>(rx, ry, rz, g, D);
    float Q[NT];
    Q[0] = nb.mass;
    const float *qq = A.q + (size_t)db * A.nq;
#pragma unroll
    for (int k = 4; k < NT; k++) Q[k] = __ldg(qq + k - 4);
    const float mG = -(float)A.G;
#pragma unroll
    for (int kn = 0; kn <= P; kn++)
#pragma unroll
        for (int kbc = 0; kbc <= kn; kbc++)
#pragma unroll
            for (int kc = 0; kc <= kbc; kc++) {
                const int ka = kn - kbc, kb = kbc - kc;
                float s = Q[0] * D[g4_midx(ka, kb, kc)];
#pragma unroll
                for (int nn = 2; nn <= P - kn; nn++) {
                    if (nn == P && !A.keep_qp) continue;   // Q_p only shifts the potential
#pragma unroll
                    for (int nbc = 0; nbc <= nn; nbc++)
#pragma unroll
                        for (int nc = 0; nc <= nbc; nc++) {
                            const int na_ = nn - nbc, nb_ = nbc - nc;
                            s += Q[g4_midx(na_, nb_, nc)] * D[g4_midx(ka + na_, kb + nb_, kc + nc)] *
                                 (1.0f / (float)(fact(na_) * fact(nb_) * fact(nc)));
                        }
                }
                T[g4_midx(ka, kb, kc)] += ((kn & 1) ? -mG : mG) * s;
            }
}

__device__ __forceinline__ int warp_sum_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_excl_i(int v, int lane)
{
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x - v;
}

// P2P: particles of leaf A (owned by this warp) from the particles of the buffered leaves.
// Leaf-leaf (P2P) interactions of sink leaf A with the buffered source leaves, 32 sinks at a
// time (one per lane): the tree walk's particle-particle phase (staged sources, packed FP16x2
// candidate tests, exact evaluation of each lane's candidates; in integer-grid units for
// TreePM), the results added to the sinks' outputs.
template <bool TREEPM>
__device__ void p2p_flush(const FmmArgs &A, PPSmem<FMM_P2PBUF> &S, const G4Node &na, const int *buf,
                          int nbuf, int lane)
{
    const double gscale = A.scale;
    const float fscale = (float)gscale, figs = A.figs;
    const int nA = na.count;
    for (int ic = 0; ic < nA; ic += 32) {
        const int nac = min(32, nA - ic);
        const bool valid = lane < nac;
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        const int i = na.first + ic + (valid ? lane : 0);
        const uint4 pi_ = A.wpart[i];
        const uint32_t xi = pi_.x, yi = pi_.y, zi = pi_.z;
        // centre of the sinks' bounding box (integer offsets from lane 0's sink)
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
        for (int k = lane; k < nbuf; k += 32) {
            const G4Node nb = load_node(A.node + buf[k]);
            S.first[k] = nb.first;
            S.count[k] = nb.count;
            S.mask[k] = vmask;
        }
        __syncwarp();
        const float hi = A.h_cls[A.cls ? A.cls[i] : 0];
        float ax = 0.f, ay = 0.f, az = 0.f, ap = 0.f;
        uint32_t npp = 0;
        pp_flush<float, TREEPM>(A, S, nbuf, lane, i, xi, yi, zi, gcx, gcy, gcz, xr, yr, zr, vmask,
                                TREEPM ? hi * figs : hi, ax, ay, az, ap, npp, gscale, figs, A.pf,
                                A.rc2i, 0, 1);
        if (TREEPM) {
            const float ca = figs * figs;
            ax *= ca;
            ay *= ca;
            az *= ca;
            ap *= figs;
        }
        if (valid) {
            const float mG = -(float)A.G;
            A.acc[i] += mG * ax;
            A.acc[A.n + i] += mG * ay;
            A.acc[2 * A.n + i] += mG * az;
            if (A.pot) A.pot[i] += mG * ap;
            if (A.counts) A.counts[i] += npp;
        }
        __syncwarp();
    }
}

// Append the buffered source leaves of sink leaf da to the deferred P2P lists as one chunk,
// chained after the sink's previous chunk (tail); the first chunk registers the sink.
// Returns false when the lists are full: the caller then evaluates the chunk at once (same
// interactions; which chunks overflow depends on the warps' timing, so only the rounding of
// such sinks can differ from run to run).
__device__ bool defer_p2p(const FmmArgs &A, int da, const int *buf, int nbuf, int lane, int &tail)
{
    int off = 0, cid = 0;
    if (lane == 0) {
        off = atomicAdd(A.p2p_fill, nbuf);
        cid = atomicAdd(A.p2p_fill + 1, 1);
    }
    off = __shfl_sync(0xffffffffu, off, 0);
    cid = __shfl_sync(0xffffffffu, cid, 0);
    if ((int64_t)off + nbuf > A.p2p_cap || (int64_t)cid >= A.chunk_cap) return false;
    for (int k = lane; k < nbuf; k += 32) A.p2p_src[off + k] = buf[k];
    if (lane == 0) {
        A.p2p_chunk[cid] = make_int4(off, nbuf, -1, 0);
        if (tail < 0) {
            A.p2p_head[da] = cid;
            A.p2p_sinks[atomicAdd(A.p2p_fill + 2, 1)] = da;
        } else {
            A.p2p_chunk[tail].z = cid;
        }
    }
    tail = cid;
    __syncwarp();
    return true;
}

// Deferred leaf-leaf interactions: one warp per sink leaf, its chunks in the order they were
// found; the results are added to the sink particles' outputs (zeroed by the dual walk)
template <bool TREEPM>
__global__ void __launch_bounds__(FMM_THREADS, 5) k_fmm_p2p(const FmmArgs A)
{
    __shared__ PPSmem<FMM_P2PBUF> s_pp[FMM_WARPS];
    if (*A.flags & G4_FLAG_CAPACITY) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nsink = A.p2p_fill[2];
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int w = gw; w < nsink; w += nw) {
        const int da = A.p2p_sinks[w];
        const G4Node na = load_node(A.node + da);
        for (int c = A.p2p_head[da]; c >= 0;) {
            const int4 ch = A.p2p_chunk[c];
            p2p_flush<TREEPM>(A, s_pp[wib], na, A.p2p_src + ch.x, ch.y, lane);
            c = ch.z;
        }
    }
}

// minimum resident blocks per SM requested from the compiler for the dual walk
#ifndef G4_FMM_MIN_BLOCKS
#define G4_FMM_MIN_BLOCKS 1
#endif

template <int P, bool TREEPM, bool GEOM>
__global__ void __launch_bounds__(FMM_THREADS, G4_FMM_MIN_BLOCKS) k_fmm_level(const FmmArgs A, int level)
{
    constexpr int NT = FT<P>::NT;
    __shared__ int s_stack[FMM_WARPS][FMM_STACK];
    __shared__ int s_p2p[FMM_WARPS][FMM_P2PBUF];
    __shared__ PPSmem<FMM_P2PBUF> s_pp[FMM_WARPS];   // overflow of the deferred lists only
    if (*A.flags & G4_FLAG_CAPACITY) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int32_t *off = A.lvl, *cnt = A.lvl + G4_NLEVELS + 1;
    const int o = off[level], c = cnt[level];
    const int total_nodes = off[G4_NLEVELS];
    int32_t *Din = (level & 1) ? A.D0 : A.D1;
    int32_t *Dout = (level & 1) ? A.D1 : A.D0;
    int32_t *dcnt = A.dcount + (level & 1);
    int *stack = s_stack[wib];
    int *p2p = s_p2p[wib];
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int b = gw; b < c; b += nw) {
        const int da = A.b_dfs[o + b];
        if ((unsigned)da >= (unsigned)total_nodes) continue;
        const G4Node na = load_node(A.node + da);
        const bool leafA = na.meta & 32u;
        const int32_t *cand = nullptr;
        int ncand = 1;
        if (level > 0) {
            cand = Din + A.Doff[na.parent];
            ncand = A.Dlen[na.parent];
        }
        float T[NT];
#pragma unroll
        for (int k = 0; k < NT; k++) T[k] = 0.f;
        int nm2l = 0;
        if (!leafA) {
            // pass 1: size of the list passed down to the daughters
            int total = 0;
            for (int base = 0; base < ncand; base += 32) {
                const int j = base + lane;
                int e = 0;
                if (j < ncand) {
                    const int db = cand ? cand[j] : da;
                    const G4Node nb = load_node(A.node + db);
                    float rx, ry, rz;
                    if (fmm_decide<P, TREEPM, GEOM>(A, na, da, nb, db, rx, ry, rz) == D_OPEN)
                        e = (nb.meta & 32u) ? 1 : nb.nchild;
                }
                total += warp_sum_i(e);
            }
            int wbase = 0;
            if (lane == 0) wbase = atomicAdd(dcnt, total);
            wbase = __shfl_sync(0xffffffffu, wbase, 0);
            const bool fits = (int64_t)wbase + total <= A.dcap;
            if (!fits && lane == 0) atomicOr(A.flags, G4_FLAG_LISTCAP);
            // pass 2: M2L for accepted candidates, write the pass-down list
            int w = wbase;
            for (int base = 0; base < ncand; base += 32) {
                const int j = base + lane;
                int e = 0, dec = D_DROP, db = 0;
                G4Node nb;
                float rx = 0.f, ry = 0.f, rz = 0.f;
                if (j < ncand) {
                    db = cand ? cand[j] : da;
                    nb = load_node(A.node + db);
                    dec = fmm_decide<P, TREEPM, GEOM>(A, na, da, nb, db, rx, ry, rz);
                    if (dec == D_OPEN) e = (nb.meta & 32u) ? 1 : nb.nchild;
                }
                if (dec == D_ACCEPT) {
                    m2l_add<P, TREEPM>(A, T, db, nb, rx, ry, rz);
                    nm2l++;
                }
                const int pre = warp_excl_i(e, lane);
                if (e > 0 && fits) {
                    if (nb.meta & 32u) {
                        Dout[w + pre] = db;
                    } else {
                        int k = 0;
                        for (int ch = db + 1; ch < nb.next && k < e; k++) {
                            Dout[w + pre + k] = ch;
                            ch = max(A.node[ch].next, ch + 1);
                        }
                    }
                }
                w += warp_sum_i(e);
            }
            if (lane == 0) {
                A.Doff[da] = fits ? wbase : 0;
                A.Dlen[da] = fits ? total : 0;
            }
        } else {
            // leaf sink: zero its particles' outputs, then walk the candidates; opened
            // internal sources are expanded in place on a per-warp stack
            for (int i = na.first + lane; i < na.first + na.count; i += 32) {
                A.acc[i] = 0.f;
                A.acc[A.n + i] = 0.f;
                A.acc[2 * A.n + i] = 0.f;
                if (A.pot) A.pot[i] = 0.f;
                if (A.counts) A.counts[i] = 0u;
            }
            if (lane == 0) A.p2p_head[da] = -1;
            __syncwarp();
            int sp = 0, cursor = 0, nbuf = 0, tail = -1;
            for (;;) {
                int db = -1;
                int navail;
                if (cursor < ncand) {
                    navail = min(32, ncand - cursor);
                    if (lane < navail) db = cand ? cand[cursor + lane] : da;
                    cursor += navail;
                } else if (sp > 0) {
                    navail = min(32, sp);
                    if (lane < navail) db = stack[sp - navail + lane];
                    sp -= navail;
                } else {
                    break;
                }
                __syncwarp();
                int dec = D_DROP, e = 0;
                G4Node nb;
                float rx = 0.f, ry = 0.f, rz = 0.f;
                if (db >= 0) {
                    nb = load_node(A.node + db);
                    dec = fmm_decide<P, TREEPM, GEOM>(A, na, da, nb, db, rx, ry, rz);
                    if (dec == D_OPEN) e = nb.nchild;   // B internal (A is a leaf)
                }
                if (dec == D_ACCEPT) {
                    m2l_add<P, TREEPM>(A, T, db, nb, rx, ry, rz);
                    nm2l++;
                }
                // push daughters of opened sources
                const int pre = warp_excl_i(e, lane);
                const int tot = warp_sum_i(e);
                if (sp + tot > FMM_STACK) {
                    if (lane == 0) atomicOr(A.flags, G4_FLAG_LISTCAP);
                } else if (e > 0) {
                    int k = 0;
                    for (int ch = db + 1; ch < nb.next && k < e; k++) {
                        stack[sp + pre + k] = ch;
                        ch = max(A.node[ch].next, ch + 1);
                    }
                }
                if (sp + tot <= FMM_STACK) sp += tot;
                // P2P sources (including A itself)
                const bool isp = (dec == D_P2P || dec == D_SELF);
                const unsigned m = __ballot_sync(0xffffffffu, isp);
                const int ppre = __popc(m & ((1u << lane) - 1u));
                const int pcount = __popc(m);
                if (nbuf + pcount > FMM_P2PBUF) {
                    __syncwarp();
                    if (!defer_p2p(A, da, p2p, nbuf, lane, tail))
                        p2p_flush<TREEPM>(A, s_pp[wib], na, p2p, nbuf, lane);
                    nbuf = 0;
                }
                if (isp) p2p[nbuf + ppre] = db;
                nbuf += pcount;
                __syncwarp();
            }
            if (nbuf > 0 && !defer_p2p(A, da, p2p, nbuf, lane, tail))
                p2p_flush<TREEPM>(A, s_pp[wib], na, p2p, nbuf, lane);
        }
        // reduce the lane-private fields and store the node's own field
#pragma unroll
        for (int k = 0; k < NT; k++) {
            const float v = warp_sum_f(T[k]);
            if (lane == 0) A.T_own[(size_t)da * NT + k] = v;
        }
        nm2l = warp_sum_i(nm2l);
        if (lane == 0) A.m2l_own[da] = (uint32_t)nm2l;
    }
}

// downward pass: T_tot = T_own + shifted parent field (L2L); leaves evaluate at particles (L2P)
template <int P>
__global__ void __launch_bounds__(128) k_fmm_down(const FmmArgs A, int level)
{
    constexpr int NT = FT<P>::NT;
    if (*A.flags & G4_FLAG_CAPACITY) return;
    const int32_t *off = A.lvl, *cnt = A.lvl + G4_NLEVELS + 1;
    const int o = off[level], c = cnt[level];
    const int total_nodes = off[G4_NLEVELS];
    const float scale = (float)A.scale;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < c; b += gridDim.x * blockDim.x) {
        const int d = A.b_dfs[o + b];
        if ((unsigned)d >= (unsigned)total_nodes) continue;
        const G4Node nd = load_node(A.node + d);
        float T[NT];
#pragma unroll
        for (int k = 0; k < NT; k++) T[k] = A.T_own[(size_t)d * NT + k];
        uint32_t cum = A.m2l_own[d];
        if (nd.parent >= 0) {
            const G4Node np = load_node(A.node + nd.parent);
            const float dx = (float)(int32_t)(nd.cx - np.cx) * scale + (nd.sx - np.sx);
            const float dy = (float)(int32_t)(nd.cy - np.cy) * scale + (nd.sy - np.sy);
            const float dz = (float)(int32_t)(nd.cz - np.cz) * scale + (nd.sz - np.sz);
            float px[P + 1], py[P + 1], pz[P + 1];
            px[0] = py[0] = pz[0] = 1.f;
#pragma unroll
            for (int k = 1; k <= P; k++) {
                px[k] = px[k - 1] * dx;
                py[k] = py[k - 1] * dy;
                pz[k] = pz[k - 1] * dz;
            }
            const float *Tp = A.T_tot + (size_t)nd.parent * NT;
#pragma unroll
            for (int kn = 0; kn <= P; kn++)
#pragma unroll
                for (int kbc = 0; kbc <= kn; kbc++)
#pragma unroll
                    for (int kc = 0; kc <= kbc; kc++) {
                        const int ka = kn - kbc, kb = kbc - kc;
                        float s = 0.f;
#pragma unroll
                        for (int mn = 0; mn <= P - kn; mn++)
#pragma unroll
                            for (int mbc = 0; mbc <= mn; mbc++)
#pragma unroll
                                for (int mc = 0; mc <= mbc; mc++) {
                                    const int ma = mn - mbc, mb = mbc - mc;
                                    s += Tp[g4_midx(ka + ma, kb + mb, kc + mc)] * px[ma] * py[mb] *
                                         pz[mc] * (1.0f / (float)(fact(ma) * fact(mb) * fact(mc)));
                                }
                        T[g4_midx(ka, kb, kc)] += s;
                    }
            cum += A.m2l_cum[nd.parent];
        }
#pragma unroll
        for (int k = 0; k < NT; k++) A.T_tot[(size_t)d * NT + k] = T[k];
        A.m2l_cum[d] = cum;
        if (nd.meta & 32u) {
            for (int i = nd.first; i < nd.first + nd.count; i++) {
                const float ax = (float)(int32_t)(A.pos[i] - nd.cx) * scale - nd.sx;
                const float ay = (float)(int32_t)(A.pos[A.n + i] - nd.cy) * scale - nd.sy;
                const float az = (float)(int32_t)(A.pos[2 * A.n + i] - nd.cz) * scale - nd.sz;
                float px[P + 1], py[P + 1], pz[P + 1];
                px[0] = py[0] = pz[0] = 1.f;
#pragma unroll
                for (int k = 1; k <= P; k++) {
                    px[k] = px[k - 1] * ax;
                    py[k] = py[k - 1] * ay;
                    pz[k] = pz[k - 1] * az;
                }
                float phi = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
                for (int kn = 0; kn <= P; kn++)
#pragma unroll
                    for (int kbc = 0; kbc <= kn; kbc++)
#pragma unroll
                        for (int kc = 0; kc <= kbc; kc++) {
                            const int ka = kn - kbc, kb = kbc - kc;
                            const float w = px[ka] * py[kb] * pz[kc] *
                                            (1.0f / (float)(fact(ka) * fact(kb) * fact(kc)));
                            phi += T[g4_midx(ka, kb, kc)] * w;
                            if (kn < P) {
                                gx += T[g4_midx(ka + 1, kb, kc)] * w;
                                gy += T[g4_midx(ka, kb + 1, kc)] * w;
                                gz += T[g4_midx(ka, kb, kc + 1)] * w;
                            }
                        }
                A.acc[i] -= gx;
                A.acc[A.n + i] -= gy;
                A.acc[2 * A.n + i] -= gz;
                if (A.pot) A.pot[i] += phi;
                if (A.counts) A.counts[A.n + i] = cum;
            }
        }
    }
}

__global__ void k_fmm_reset(int32_t *dcount, double *mom)
{
    if (threadIdx.x < 2) dcount[threadIdx.x] = 0;
    if (mom && threadIdx.x < 3) mom[threadIdx.x] = 0.0;
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

template <int P, bool TREEPM, bool GEOM>
void run_fmm(const FmmArgs &A, cudaStream_t st)
{
    const int nb = g4_num_sms() * 8;
    for (int l = 0; l <= G4_MAXLEVEL; l++) {
        if (l >= 2) {
            // the list of level l-2 is no longer needed: its buffer is reused at level l
            cudaMemsetAsync(A.dcount + (l & 1), 0, sizeof(int32_t), st);
        }
        k_fmm_level<P, TREEPM, GEOM><<<nb, FMM_THREADS, 0, st>>>(A, l);
    }
    k_fmm_p2p<TREEPM><<<g4_num_sms() * 5, FMM_THREADS, 0, st>>>(A);
    for (int l = 0; l <= G4_MAXLEVEL; l++) k_fmm_down<P><<<nb, 128, 0, st>>>(A, l);
}

template <int P>
void dispatch_fmm(const FmmArgs &A, bool treepm, bool geom, cudaStream_t st)
{
    if (treepm) {
        if (geom) run_fmm<P, true, true>(A, st);
        else run_fmm<P, true, false>(A, st);
    } else {
        if (geom) run_fmm<P, false, true>(A, st);
        else run_fmm<P, false, false>(A, st);
    }
}

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct FmmLayout {
    size_t T_own, T_tot, Doff, Dlen, m2l_own, m2l_cum, dcount, p2p_src, p2p_chunk, p2p_head,
        p2p_sinks, p2p_fill, D0, D1, total;
    int64_t dcap, p2p_cap, chunk_cap;
};

// deferred P2P lists: 16 source-leaf entries and 1.25 chunks per particle of the handle (plus
// a floor for small sets); overflowing chunks are evaluated by the dual walk itself
FmmLayout fmm_layout(int64_t nodes, int64_t n_max, int nt, size_t ws_bytes, int per_particle)
{
    FmmLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += al256(bytes); return r; };
    L.T_own = take(sizeof(float) * nt * nodes);
    L.T_tot = take(sizeof(float) * nt * nodes);
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
    L.p2p_src = take(4 * (size_t)L.p2p_cap);
    L.p2p_chunk = take(16 * (size_t)L.chunk_cap);
    L.p2p_head = take(4 * nodes);
    L.p2p_sinks = take(4 * nodes);
    L.p2p_fill = take(16);
    size_t fixed = o;
    int64_t dcap = 0;
    if (ws_bytes == 0) dcap = (int64_t)1 << 20 > 48 * nodes ? (int64_t)1 << 20 : 48 * nodes;
    else dcap = ws_bytes > fixed + 1024 ? (int64_t)((ws_bytes - fixed - 1024) / 8) : 0;
    if (dcap > ((int64_t)1 << 31) - 1) dcap = ((int64_t)1 << 31) - 1;
    L.D0 = take(4 * dcap);
    L.D1 = take(4 * dcap);
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
    *bytes = fmm_layout(t->cap, t->n_max, g4_nmono(P->order_p), 0, P->fmm_p2p_per_particle).total;
    return G4_OK;
}

extern "C" g4_status g4_gravity_fmm(g4_tree t, const uint32_t *pos_sorted, const float *mass_sorted,
                                    const uint8_t *cls_sorted, const g4_params *P, float *acc,
                                    float *pot, uint32_t *counts, double *momentum_out,
                                    void *workspace, size_t workspace_bytes, void *stream)
{
    g4_status s = g4_check_params(P, "g4_gravity_fmm");
    if (s != G4_OK) return s;
    if (!t || !pos_sorted || !mass_sorted || !acc || !workspace)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_fmm: NULL argument");
    if (((uintptr_t)workspace & 255) != 0)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_fmm: workspace not 256-byte aligned");
    if (t->built_n < 0 || t->moments_order < 0)
        return g4_fail(G4_ERR_STATE, "g4_gravity_fmm: build and multipoles must run first");
    if (t->moments_order != P->order_p)
        return g4_fail(G4_ERR_STATE, "g4_gravity_fmm: moments of order %d, FMM order %d",
                       t->moments_order, P->order_p);
    if (P->order_p < 2 || P->order_p > 5)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_fmm: order_p must be in [2,5]");
    if (P->precision != 0)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_fmm: only FP32 interactions (precision 0)");
    const int n = t->built_n;
    if (n == 0) return G4_OK;
    const int nt = g4_nmono(P->order_p);
    // node count bound: the handle's capacity (no host synchronisation here)
    FmmLayout L = fmm_layout(t->cap, t->n_max, nt, workspace_bytes, P->fmm_p2p_per_particle);
    if (L.dcap < 1024 || L.total > workspace_bytes)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gravity_fmm: workspace too small (%zu bytes)",
                       workspace_bytes);
    char *w = (char *)workspace;
    FmmArgs A;
    A.pos = pos_sorted;
    A.mass = mass_sorted;
    A.cls = cls_sorted;
    A.n = n;
    A.lvl = t->lvl;
    A.b_dfs = t->b_dfs;
    A.node = t->node;
    A.q = t->q;
    A.nq = g4_nq(P->order_p);
    A.T_own = (float *)(w + L.T_own);
    A.T_tot = (float *)(w + L.T_tot);
    A.Doff = (int32_t *)(w + L.Doff);
    A.Dlen = (int32_t *)(w + L.Dlen);
    A.m2l_own = (uint32_t *)(w + L.m2l_own);
    A.m2l_cum = (uint32_t *)(w + L.m2l_cum);
    A.dcount = (int32_t *)(w + L.dcount);
    A.D0 = (int32_t *)(w + L.D0);
    A.D1 = (int32_t *)(w + L.D1);
    A.dcap = L.dcap;
    A.p2p_src = (int32_t *)(w + L.p2p_src);
    A.p2p_chunk = (int4 *)(w + L.p2p_chunk);
    A.p2p_head = (int32_t *)(w + L.p2p_head);
    A.p2p_sinks = (int32_t *)(w + L.p2p_sinks);
    A.p2p_fill = (int32_t *)(w + L.p2p_fill);
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
    A.rcut2f = (float)A.rcut2;
    A.asf = (float)A.as;
    const double igs = 4294967296.0 / P->box_size;
    A.figs = (float)igs;
    A.rc2i = (float)(A.rcut2 * igs * igs);
    A.pf = make_pairf(A.as * A.scale, treepm ? 2.0 * P->r_s * igs : 0.0);
    cudaStream_t st = (cudaStream_t)stream;
    s = g4_particle_records(t, pos_sorted, mass_sorted, n, st);
    if (s != G4_OK) return s;
    A.wpart = t->wpart;
    k_fmm_reset<<<1, 32, 0, st>>>(A.dcount, momentum_out);
    if (cudaMemsetAsync(A.p2p_fill, 0, 16, st) != cudaSuccess)
        return g4_cuda_check(cudaGetLastError(), "g4_gravity_fmm: clear P2P counters");
    const bool geom = P->criterion == 1;
    switch (P->order_p) {
    case 2: dispatch_fmm<2>(A, treepm, geom, st); break;
    case 3: dispatch_fmm<3>(A, treepm, geom, st); break;
    case 4: dispatch_fmm<4>(A, treepm, geom, st); break;
    default: dispatch_fmm<5>(A, treepm, geom, st); break;
    }
    if (momentum_out) k_momentum<<<g4_num_sms() * 4, 256, 0, st>>>(mass_sorted, acc, n, momentum_out);
    return g4_launch_check("fmm", 2 + 2 * (G4_MAXLEVEL + 1) + (momentum_out ? 1 : 0));
}
