// g4_fmm.cuh -- symmetric Cartesian fast multipole method (Sec. 2.4, Sec. 2.5).
//
// The paper's dual tree walk visits unordered pairs of cells, a cell being a node or a single
// particle (Sec. 2.4).  A particle is a cell of side 0 whose only moment is Q_0 = m.  A pair
// either interacts through the symmetric expansion, or fails and is opened: both cells if both
// can be (Sec. 2.4 opens both), a leaf into its particles, a particle never.  Two particles
// always interact directly.  The decisions are symmetric in
// the two cells, so the same interactions are found by visiting ordered pairs (X, Y) -- sink X,
// source Y -- where (X, Y) and (Y, X) receive the same decision.  That makes the walk
// sink-centric and free of write conflicts:
//
//   level by level, top-down, one warp per sink node A; the candidates of A are the entries
//   its parent passed down (the root starts with itself): nodes, or chunks of up to 32
//   particles of one leaf with a mask of the particles still interacting;
//   internal A, node candidate B:
//       B == A        : pass A's daughters down
//       gap > r_cut   : drop
//       accepted      : field of B's multipoles at A's centre of mass (M2L, one direction)
//       otherwise     : pass B's daughters down (B's particles, in chunks, if B is a leaf)
//   internal A, particle candidate y: drop, accept (field of the point mass y at A: P2L), or
//       pass y down to A's daughters;
//   leaf A (its particles are the daughters it opens into):
//       node B == A, or B a leaf that fails : particle pairs with all of A's particles
//       node B internal that fails : each particle x of A against B's daughters -- a per-lane
//           walk (one particle per lane): accept (B's field at x: M2P), drop, open (daughters,
//           or particle pairs of x with a leaf's particles)
//       accepted node B or particle y : field at A's centre of mass (M2L / P2L)
//       particle y that fails : particle pairs of y with all of A's particles
//   then level by level, top-down: L2L shift of the parent's field, L2P at the leaves.
// Particle pairs are recorded during the dual walk as chained per-sink-leaf lists of
// (first particle, count, lane mask) entries and evaluated afterwards by k_fmm_p2p with the tree
// walk's particle-particle phase (g4_pp.cuh).
//
// The field tensor of A from source B is, with r = s_B - s_A (multi-index form),
//   T^A_k = -G (-1)^|k| sum_n Q^B_n D_{k+n}(r) / n!      (|k| + |n| <= p, |n| != 1, |n| != p)
// and the potential near A's centre of mass is Phi(s_A + a) = sum_k T_k a^k / k!.
#pragma once
#include "g4_internal.cuh"
#include "g4_kernels.cuh"
#include "g4_pp.cuh"
#include "g4_fmm_args.cuh"



namespace {

using namespace g4k;
using namespace g4fmm;

template <int P> struct FT { static constexpr int NT = g4_nmono(P); };

__device__ __forceinline__ float fside(double box, int lv) { return ldexpf((float)box, -lv); }

// a particle as a cell: integer position, mass, softening 2.8 eps, |a_old|
struct PCell {
    uint32_t x, y, z;
    float m, h, a;
};

__device__ __forceinline__ PCell load_pcell(const FmmArgs &A, int j)
{
    const uint4 w = __ldg(A.wpart + j);
    PCell c;
    c.x = w.x;
    c.y = w.y;
    c.z = w.z;
    c.m = __uint_as_float(w.w);
    c.h = A.h_cls[A.cls ? __ldg(A.cls + j) : 0];
    c.a = A.aold ? __ldg(A.aold + j) : 0.f;
    return c;
}

// Periodic box: the nearest image of a centre-of-mass separation.  The centres' separation
// is already the nearest image, but with the centres of mass it can pass half the box; taking
// the separation's own nearest image keeps the two directions of a pair mirror images
// (centres exactly half a box apart get the same image sign from both sides), so both take
// the same decision.  Without a cutoff only: within r_cut it changes nothing.
template <typename R>
__device__ __forceinline__ void periodic_wrap(const FmmArgs &A, R &rx, R &ry, R &rz)
{
    if (!A.periodic) return;
    const R L = (R)A.box;
    rx -= L * rint(rx / L);
    ry -= L * rint(ry / L);
    rz -= L * rint(rz / L);
}

// FP64 node data of node d (precision 1): centre-of-mass offset [0..2], mass [3], moments [4..]
__device__ __forceinline__ const double *node_fp64(const FmmArgs &A, int d)
{
    return A.qd + (size_t)d * (4 + A.nq);
}

// decision for the node pair (A <- B), identical to the symmetric rule of the dual walk
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
    if (!TREEPM) periodic_wrap(A, rx, ry, rz);   // (a no-op within r_cut)
    const float r2 = rx * rx + ry * ry + rz * rz;
    bool accept = true;
    const float dmax = fmaxf(fabsf(dcx), fmaxf(fabsf(dcy), fabsf(dcz)));
    if (A.exclusion && dmax <= fmaxf(lA, lB)) accept = false;   // touching nodes never interact
    if (dmax < hl) accept = false;                              // overlapping cubes
    // closer than 2.8 eps_ij: opened (GADGET-3 rule), or under the rule of Sec. 2.7 only if
    // both nodes hold particles with softenings below eps_ij (else a softened interaction)
    const float h = fmaxf(na.hmax, nb.hmax);
    if (r2 < h * h && (!A.soft_nodes || (na.hmin < h && nb.hmin < h))) accept = false;
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

// Decision for a node Z and a particle x, the same whichever of the two is the sink: a cell of
// side 0 at x with x's mass, softening and |a_old|.  (rx, ry, rz) = s_Z - x.  Returns D_DROP,
// D_ACCEPT or D_OPEN (Z is opened; a particle cannot be).
template <int P, bool TREEPM, bool GEOM>
__device__ __forceinline__ int fmm_decide_pn(const FmmArgs &A, const G4Node &nz, const PCell &x,
                                             float &rx, float &ry, float &rz)
{
    const float scale = (float)A.scale;
    const float l = fside(A.box, nz.meta & 31u), hl = 0.5f * l;
    const float dcx = (float)(int32_t)(nz.cx - x.x) * scale;
    const float dcy = (float)(int32_t)(nz.cy - x.y) * scale;
    const float dcz = (float)(int32_t)(nz.cz - x.z) * scale;
    if (TREEPM) {
        const float ex = fmaxf(fabsf(dcx) - hl, 0.f), ey = fmaxf(fabsf(dcy) - hl, 0.f),
                    ez = fmaxf(fabsf(dcz) - hl, 0.f);
        if (ex * ex + ey * ey + ez * ez > (float)A.rcut2) return D_DROP;
    }
    rx = dcx + nz.sx;
    ry = dcy + nz.sy;
    rz = dcz + nz.sz;
    if (!TREEPM) periodic_wrap(A, rx, ry, rz);   // (a no-op within r_cut)
    const float r2 = rx * rx + ry * ry + rz * rz;
    bool accept = true;
    const float dmax = fmaxf(fabsf(dcx), fmaxf(fabsf(dcy), fabsf(dcz)));
    if (A.exclusion && dmax <= l) accept = false;   // inside the node's exclusion cube
    if (dmax < hl) accept = false;                  // inside the node
    const float h = fmaxf(nz.hmax, x.h);
    if (r2 < h * h && (!A.soft_nodes || (nz.hmin < h && x.h < h))) accept = false;
    if (accept) {
        if (GEOM) {
            accept = l * l < (float)A.theta2 * r2;
        } else {
            const float r = sqrtf(r2);
            float lp = 1.f, rp = r2;
#pragma unroll
            for (int i = 0; i < P - 1; i++) {
                lp *= l;
                rp *= r;
            }
            const float amin = fminf(nz.amin, x.a), mmax = fmaxf(nz.mass, x.m);
            accept = (float)A.G * mmax * lp < (float)A.alpha * amin * rp;
        }
    }
    return accept ? D_ACCEPT : D_OPEN;
}

// g_0..g_P of the interaction kernel: the softened one (h = 2.8 eps_ij) inside h when the
// rule of Sec. 2.7 is in force (hs = h), the unsoftened one otherwise (hs = 0)
template <int P, bool TREEPM, typename R>
__device__ __forceinline__ void fmm_gn(const FmmArgs &A, R r2, R hs, R *g)
{
    if (hs > R(0) && r2 < hs * hs) gn_soft<P, R, TREEPM>(r2, hs, (R)A.as, g);
    else gn_kernel<P, R, TREEPM>(r2, (R)A.as, g);
}

// lane-private M2L: T += field of node B at A's centre of mass (r = s_B - s_A)
// Pure periodic FMM (Sec. 2.2.4): the separation moved to its image in the primary cell (the
// periodic kernel 1/r - psi is the same at every image), and the correction tensors D_n[psi]
// subtracted from the Newtonian ones there.
template <typename R>
__device__ __forceinline__ void ewald_wrap(const FmmArgs &A, R &rx, R &ry, R &rz)
{
    if (!A.ewald) return;
    const R L = (R)A.box;
    rx -= L * rint(rx / L);
    ry -= L * rint(ry / L);
    rz -= L * rint(rz / L);
}
template <int P, typename R>
__device__ __forceinline__ void ewald_sub(const FmmArgs &A, R rx, R ry, R rz, R *D)
{
    if (!A.ewald) return;
    R Dp[g4_nmono(P)];
    ewald_dpsi<P, R>(A.ew, rx, ry, rz, Dp);
#pragma unroll
    for (int k = 0; k < g4_nmono(P); k++) D[k] -= Dp[k];
}

template <int P, bool TREEPM, typename R>
__device__ __forceinline__ void m2l_add(const FmmArgs &A, R *T, int db, const G4Node &nb,
                                        R rx, R ry, R rz, R hs)
{
    constexpr int NT = FT<P>::NT;
    if (!TREEPM) ewald_wrap(A, rx, ry, rz);
    const R r2 = rx * rx + ry * ry + rz * rz;
    R g[P + 1];
    fmm_gn<P, TREEPM>(A, r2, hs, g);
    R D[NT];
    dtensors<P, R>(rx, ry, rz, g, D);
    if (!TREEPM) ewald_sub<P>(A, rx, ry, rz, D);
    R Q[NT];
    if (sizeof(R) == 8) {
        const double *dd = node_fp64(A, db);
        Q[0] = (R)dd[3];
#pragma unroll
        for (int k = 4; k < NT; k++) Q[k] = (R)dd[k];
    } else {
        Q[0] = nb.mass;
        const float *qq = A.q + (size_t)db * A.nq;
#pragma unroll
        for (int k = 4; k < NT; k++) Q[k] = __ldg(qq + k - 4);
    }
    const R mG = -(R)A.G;
#pragma unroll
    for (int kn = 0; kn <= P; kn++)
#pragma unroll
        for (int kbc = 0; kbc <= kn; kbc++)
#pragma unroll
            for (int kc = 0; kc <= kbc; kc++) {
                const int ka = kn - kbc, kb = kbc - kc;
                R s = Q[0] * D[g4_midx(ka, kb, kc)];
#pragma unroll
                for (int nn = 2; nn <= P - kn; nn++) {
                    if (nn == P && !A.keep_qp) continue;   // Q_p only shifts the potential
#pragma unroll
                    for (int nbc = 0; nbc <= nn; nbc++)
#pragma unroll
                        for (int nc = 0; nc <= nbc; nc++) {
                            const int na_ = nn - nbc, nb_ = nbc - nc;
                            s += Q[g4_midx(na_, nb_, nc)] * D[g4_midx(ka + na_, kb + nb_, kc + nc)] *
                                 (R(1) / (R)(fact(na_) * fact(nb_) * fact(nc)));
                        }
                }
                T[g4_midx(ka, kb, kc)] += ((kn & 1) ? -mG : mG) * s;
            }
}

// lane-private P2L: T += field of a point mass m at A's centre of mass, r = x - s_A
// (the M2L with Q_0 = m only): T_k += -G (-1)^|k| m D_k(r)
template <int P, bool TREEPM, typename R>
__device__ __forceinline__ void p2l_add(const FmmArgs &A, R *T, R m, R rx, R ry, R rz, R hs)
{
    constexpr int NT = FT<P>::NT;
    if (!TREEPM) ewald_wrap(A, rx, ry, rz);
    const R r2 = rx * rx + ry * ry + rz * rz;
    R g[P + 1];
    fmm_gn<P, TREEPM>(A, r2, hs, g);
    R D[NT];
    dtensors<P, R>(rx, ry, rz, g, D);
    if (!TREEPM) ewald_sub<P>(A, rx, ry, rz, D);
    const R mG = -(R)A.G * m;
#pragma unroll
    for (int kn = 0; kn <= P; kn++)
#pragma unroll
        for (int kbc = 0; kbc <= kn; kbc++)
#pragma unroll
            for (int kc = 0; kc <= kbc; kc++) {
                const int k = g4_midx(kn - kbc, kbc - kc, kc);
                T[k] += ((kn & 1) ? -mG : mG) * D[k];
            }
}

// M2P: field of node Z at particle x, r = s_Z - x (the mutual expansion evaluated on a cell of
// side 0): sacc += sum_{n<P} Q_n . D_{n+1} / n!,  spot += sum_{n<P} Q_n . D_n / n! (plus Q_P
// when keep_qp); the caller multiplies both by -G.
template <int P, bool TREEPM, typename R>
__device__ __forceinline__ void m2p_add(const FmmArgs &A, int dz, const G4Node &nz, R x, R y, R z,
                                        R hs, R &sx, R &sy, R &sz, R &sp)
{
    if (!TREEPM) ewald_wrap(A, x, y, z);
    const R r2 = x * x + y * y + z * z;
    R g[P + 1];
    fmm_gn<P, TREEPM>(A, r2, hs, g);
    R D[g4_nmono(P)];
    dtensors<P, R>(x, y, z, g, D);
    if (!TREEPM) ewald_sub<P>(A, x, y, z, D);
    const double *dd = sizeof(R) == 8 ? node_fp64(A, dz) : nullptr;
    const R M = sizeof(R) == 8 ? (R)dd[3] : (R)nz.mass;
    R ax = M * D[g4_midx(1, 0, 0)], ay = M * D[g4_midx(0, 1, 0)], az = M * D[g4_midx(0, 0, 1)];
    R ph = M * D[0];
    const float *qq = A.q + (size_t)dz * A.nq;
#pragma unroll
    for (int n = 2; n <= P; n++)
#pragma unroll
        for (int bc = 0; bc <= n; bc++)
#pragma unroll
            for (int c = 0; c <= bc; c++) {
                const int a = n - bc, b = bc - c;
                const R qn = sizeof(R) == 8 ? (R)dd[g4_midx(a, b, c)] : (R)__ldg(qq + g4_midx(a, b, c) - 4);
                const R w = qn * (R(1) / (R)(fact(a) * fact(b) * fact(c)));
                if (n <= P - 1) {
                    ph += w * D[g4_midx(a, b, c)];
                    ax += w * D[g4_midx(a + 1, b, c)];
                    ay += w * D[g4_midx(a, b + 1, c)];
                    az += w * D[g4_midx(a, b, c + 1)];
                } else if (A.keep_qp) {
                    ph += w * D[g4_midx(a, b, c)];
                }
            }
    sx += ax;
    sy += ay;
    sz += az;
    sp += ph;
}

__device__ __forceinline__ int warp_sum_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename R>
__device__ __forceinline__ R warp_sum_f(R v)
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

// Particle pairs of sink leaf A with the buffered entries (first, count, lane mask), 32 sinks
// at a time (one per lane): the tree walk's particle-particle phase (staged sources, packed
// FP16x2 candidate tests, exact evaluation of each lane's candidates; in integer-grid units
// for TreePM), the results added to the sinks' outputs.  An entry with lane mask 0 reaches
// every sink of A; any other entry only the lanes of sink chunk `ic`.
template <bool TREEPM, typename R>
__device__ void p2p_flush(const FmmArgs &A, PPSmem<FMM_P2PBUF> &S, const G4Node &na, const int4 *buf,
                          int nbuf, int ic, int lane)
{
    constexpr bool INTU = TREEPM && sizeof(R) == 4;   // FP32 TreePM: integer-grid units
    const double gscale = A.scale;
    const float fscale = (float)gscale, figs = A.figs;
    const int nA = na.count;
    for (int jc = 0; 32 * jc < nA; jc++) {
        const int c0 = 32 * jc;
        const int nac = min(32, nA - c0);
        const bool valid = lane < nac;
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        bool any = false;
        for (int k = lane; k < nbuf; k += 32) {
            const int4 e = buf[k];
            const unsigned m = e.z == 0 ? vmask : (jc == ic ? ((unsigned)e.z & vmask) : 0u);
            S.first[k] = e.x;
            S.count[k] = e.y;
            S.mask[k] = m;
            any |= m != 0u;
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        const int i = na.first + c0 + (valid ? lane : 0);
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
        __syncwarp();
        const float hi = A.h_cls[A.cls ? A.cls[i] : 0];
        R ax = R(0), ay = R(0), az = R(0), ap = R(0);
        uint32_t npp = 0;
        pp_flush<R, TREEPM>(A, S, nbuf, lane, i, xi, yi, zi, gcx, gcy, gcz, xr, yr, zr, vmask,
                            INTU ? (R)(hi * figs) : (R)hi, ax, ay, az, ap, npp, gscale, figs, A.pf,
                            A.rc2i, 0, 1);
        if (INTU) {
            const float ca = figs * figs;
            ax *= ca;
            ay *= ca;
            az *= ca;
            ap *= figs;
        }
        if (valid) {
            const R mG = -(R)A.G;
            A.acc[i] = (float)((R)A.acc[i] + mG * ax);
            A.acc[A.n + i] = (float)((R)A.acc[A.n + i] + mG * ay);
            A.acc[2 * A.n + i] = (float)((R)A.acc[2 * A.n + i] + mG * az);
            if (A.pot) A.pot[i] = (float)((R)A.pot[i] + mG * ap);
            if (A.counts) A.counts[i] += npp;
        }
        __syncwarp();
    }
}

// Append the buffered entries of sink leaf da (sink chunk ic) to the deferred lists as one
// chunk, chained after the sink's previous chunk (tail); the first chunk registers the sink.
// Returns false when the lists are full: the caller then evaluates the chunk at once (same
// interactions; which chunks overflow depends on the warps' timing, so only the rounding of
// such sinks can differ from run to run).
__device__ bool defer_p2p(const FmmArgs &A, int da, const int4 *buf, int nbuf, int ic, int lane,
                          int &tail)
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
        A.p2p_chunk[cid] = make_int4(off, nbuf, -1, ic);
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

// Deferred particle pairs: one warp per sink leaf, its chunks in the order they were found;
// the results are added to the sink particles' outputs (zeroed by the dual walk)
// resident blocks per SM of the deferred particle-pair pass (FP32: 6, 80 registers with a few
// bytes of spills, 1.4% faster per FMM call than 5 at 96 registers; FP64: 5)
#ifndef G4_FMM_P2P_MIN_BLOCKS
#define G4_FMM_P2P_MIN_BLOCKS 6
#endif
template <typename R> constexpr int fmm_p2p_blocks() { return sizeof(R) == 4 ? G4_FMM_P2P_MIN_BLOCKS : 5; }
template <bool TREEPM, typename R>
__global__ void __launch_bounds__(FMM_THREADS, fmm_p2p_blocks<R>()) k_fmm_p2p(const FmmArgs A)
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
            p2p_flush<TREEPM, R>(A, s_pp[wib], na, A.p2p_src + ch.x, ch.y, ch.w, lane);
            c = ch.z;
        }
    }
}

// minimum resident blocks per SM requested from the compiler for the FP32 dual walk: 3 caps
// its registers at 168 (from 207 at order 4; 2 blocks per SM), with a few bytes of spills and
// 9% less time per FMM call at 256^3; the FP64 reference mode keeps the compiler's choice
#ifndef G4_FMM_MIN_BLOCKS
#define G4_FMM_MIN_BLOCKS 3
#endif
template <typename R> constexpr int fmm_level_min_blocks() { return sizeof(R) == 4 ? G4_FMM_MIN_BLOCKS : 1; }

// per-warp state of a leaf sink: pending particle-pair entries, the particle walk's stack
struct LeafSmem {
    int4 pp[FMM_P2PBUF];
    int2 stack[FMM_STACK];
};

// Separations for the expansions.  FP32: the ones the decisions computed.  FP64 (R = double):
// recomputed from the integer centres and the FP64 centre-of-mass offsets.
template <bool TREEPM, typename R>
__device__ __forceinline__ void sep_nodes(const FmmArgs &A, const G4Node &na, int da, const G4Node &nb,
                                          int db, float fx, float fy, float fz, R &rx, R &ry, R &rz)
{
    if (sizeof(R) == 4) {
        rx = fx; ry = fy; rz = fz;
        return;
    }
    const double *a = node_fp64(A, da), *b = node_fp64(A, db);
    rx = (R)((double)(int32_t)(nb.cx - na.cx) * A.scale + (b[0] - a[0]));
    ry = (R)((double)(int32_t)(nb.cy - na.cy) * A.scale + (b[1] - a[1]));
    rz = (R)((double)(int32_t)(nb.cz - na.cz) * A.scale + (b[2] - a[2]));
    if (!TREEPM) periodic_wrap(A, rx, ry, rz);
}
// s_Z - x for node Z and particle x (fx.. = the decision's FP32 separation)
template <bool TREEPM, typename R>
__device__ __forceinline__ void sep_node_particle(const FmmArgs &A, const G4Node &nz, int dz,
                                                  const PCell &x, float fx, float fy, float fz,
                                                  R &rx, R &ry, R &rz)
{
    if (sizeof(R) == 4) {
        rx = fx; ry = fy; rz = fz;
        return;
    }
    const double *z = node_fp64(A, dz);
    rx = (R)((double)(int32_t)(nz.cx - x.x) * A.scale + z[0]);
    ry = (R)((double)(int32_t)(nz.cy - x.y) * A.scale + z[1]);
    rz = (R)((double)(int32_t)(nz.cz - x.z) * A.scale + z[2]);
    if (!TREEPM) periodic_wrap(A, rx, ry, rz);
}

template <int P, bool TREEPM, bool GEOM, typename R>
__global__ void __launch_bounds__(FMM_THREADS, fmm_level_min_blocks<R>()) k_fmm_level(const FmmArgs A, int level)
{
    constexpr int NT = FT<P>::NT;
    __shared__ LeafSmem s_leaf[FMM_WARPS];
    __shared__ PPSmem<FMM_P2PBUF> s_pp[FMM_WARPS];   // overflow of the deferred lists only
    if (*A.flags & G4_FLAG_CAPACITY) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int32_t *off = A.lvl, *cnt = A.lvl + G4_NLEVELS + 1;
    const int o = off[level], c = cnt[level];
    const int total_nodes = off[G4_NLEVELS];
    int2 *Din = (level & 1) ? A.D0 : A.D1;
    int2 *Dout = (level & 1) ? A.D1 : A.D0;
    int32_t *dcnt = A.dcount + (level & 1);
    LeafSmem &L = s_leaf[wib];
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int b = gw; b < c; b += nw) {
        const int da = A.b_dfs[o + b];
        if ((unsigned)da >= (unsigned)total_nodes) continue;
        const G4Node na = load_node(A.node + da);
        const bool leafA = na.meta & 32u;
        const int2 *cand = nullptr;
        int ncand = 1;
        if (level > 0) {
            cand = Din + A.Doff[na.parent];
            ncand = A.Dlen[na.parent];
        }
        R T[NT];
#pragma unroll
        for (int k = 0; k < NT; k++) T[k] = R(0);
        int nm2l = 0;
        if (!leafA) {
            // pass 1: size of the list passed down to the daughters (a particle chunk always
            // takes one entry, possibly with an empty mask)
            int total = 0;
            for (int base = 0; base < ncand; base += 32) {
                const int j = base + lane;
                int e = 0;
                if (j < ncand) {
                    const int2 ce = cand ? cand[j] : make_int2(da, 0);
                    if (ce.x < 0) {
                        e = 1;
                    } else {
                        const G4Node nb = load_node(A.node + ce.x);
                        float rx, ry, rz;
                        if (fmm_decide<P, TREEPM, GEOM>(A, na, da, nb, ce.x, rx, ry, rz) == D_OPEN)
                            e = (nb.meta & 32u) ? (nb.count + 31) >> 5 : nb.nchild;
                    }
                }
                total += warp_sum_i(e);
            }
            int wbase = 0;
            if (lane == 0) wbase = atomicAdd(dcnt, total);
            wbase = __shfl_sync(0xffffffffu, wbase, 0);
            const bool fits = (int64_t)wbase + total <= A.dcap;
            if (!fits && lane == 0) atomicOr(A.flags, G4_FLAG_LISTCAP);
            // pass 2: M2L / P2L for accepted candidates, write the pass-down list
            int w = wbase;
            for (int base = 0; base < ncand; base += 32) {
                const int j = base + lane;
                int e = 0, dec = D_DROP;
                int2 ce = make_int2(0, 0);
                G4Node nb;
                float rx = 0.f, ry = 0.f, rz = 0.f;
                if (j < ncand) {
                    ce = cand ? cand[j] : make_int2(da, 0);
                    if (ce.x < 0) {
                        // particles of one leaf: each is dropped, accepted (P2L) or passed on
                        const int p0 = -ce.x - 1;
                        unsigned keep = 0u;
                        for (unsigned m = (unsigned)ce.y; m; m &= m - 1u) {
                            const int bit = __ffs(m) - 1;
                            const PCell x = load_pcell(A, p0 + bit);
                            const int d = fmm_decide_pn<P, TREEPM, GEOM>(A, na, x, rx, ry, rz);
                            if (d == D_ACCEPT) {
                                R qx, qy, qz;
                                sep_node_particle<TREEPM, R>(A, na, da, x, rx, ry, rz, qx, qy, qz);
                                p2l_add<P, TREEPM, R>(A, T, (R)x.m, -qx, -qy, -qz,
                                                      (R)(A.soft_nodes ? fmaxf(na.hmax, x.h) : 0.f));
                            } else if (d == D_OPEN) {
                                keep |= 1u << bit;
                            }
                        }
                        ce.y = (int)keep;
                        e = 1;
                    } else {
                        nb = load_node(A.node + ce.x);
                        dec = fmm_decide<P, TREEPM, GEOM>(A, na, da, nb, ce.x, rx, ry, rz);
                        if (dec == D_OPEN) e = (nb.meta & 32u) ? (nb.count + 31) >> 5 : nb.nchild;
                    }
                }
                if (dec == D_ACCEPT) {
                    R qx, qy, qz;
                    sep_nodes<TREEPM, R>(A, na, da, nb, ce.x, rx, ry, rz, qx, qy, qz);
                    m2l_add<P, TREEPM, R>(A, T, ce.x, nb, qx, qy, qz,
                                          (R)(A.soft_nodes ? fmaxf(na.hmax, nb.hmax) : 0.f));
                    nm2l++;
                }
                const int pre = warp_excl_i(e, lane);
                if (e > 0 && fits) {
                    if (ce.x < 0) {
                        Dout[w + pre] = ce;
                    } else if (nb.meta & 32u) {
                        // a leaf opens into its particles, 32 to an entry
                        for (int k = 0; k < e; k++) {
                            const int nk = min(32, nb.count - 32 * k);
                            Dout[w + pre + k] = make_int2(-(nb.first + 32 * k) - 1,
                                                          (int)(nk >= 32 ? 0xffffffffu : ((1u << nk) - 1u)));
                        }
                    } else {
                        for (int k = 0; k < e; k++)
                            Dout[w + pre + k] = make_int2(__ldg(A.kids + (size_t)ce.x * 8 + k), 0);
                    }
                }
                w += warp_sum_i(e);
            }
            if (lane == 0) {
                A.Doff[da] = fits ? wbase : 0;
                A.Dlen[da] = fits ? total : 0;
            }
        } else {
            // leaf sink: zero its particles' outputs; then, for each chunk of 32 of its
            // particles (one per lane): the leaf-level decisions on the candidates (fields at
            // A's centre of mass and particle pairs with all of A's particles -- taken once,
            // with the first chunk), and the per-particle walk into the internal nodes A opens
            for (int i = na.first + lane; i < na.first + na.count; i += 32) {
                A.acc[i] = 0.f;
                A.acc[A.n + i] = 0.f;
                A.acc[2 * A.n + i] = 0.f;
                if (A.pot) {
                    // each particle's own periodic images: + G m_i psi(0) (pure periodic FMM)
                    float p0 = 0.f;
                    if (!TREEPM && A.ewald) {
                        R D0[1];
                        ewald_dpsi<0, R>(A.ew, R(0), R(0), R(0), D0);
                        p0 = (float)((R)A.G * (R)A.mass[i] * D0[0]);
                    }
                    A.pot[i] = p0;
                }
                if (A.counts) {
                    A.counts[i] = 0u;
                    A.counts[A.n + i] = 0u;
                }
            }
            if (lane == 0) A.p2p_head[da] = -1;
            __syncwarp();
            int tail = -1;
            for (int ic = 0; 32 * ic < na.count; ic++) {
                const int nac = min(32, na.count - 32 * ic);
                const bool valid = lane < nac;
                const unsigned vmask = __ballot_sync(0xffffffffu, valid);
                const int i = na.first + 32 * ic + (valid ? lane : 0);
                const PCell xs = load_pcell(A, i);
                R bx = R(0), by = R(0), bz = R(0), bp = R(0);
                uint32_t npn = 0;
                int sp = 0, nbuf = 0;
                // appends one particle-pair entry per lane that has one
                auto push_pp = [&](bool has, int4 ent) {
                    const unsigned bm = __ballot_sync(0xffffffffu, has);
                    const int k = __popc(bm);
                    if (k == 0) return;
                    if (nbuf + k > FMM_P2PBUF) {
                        __syncwarp();
                        if (!defer_p2p(A, da, L.pp, nbuf, ic, lane, tail))
                            p2p_flush<TREEPM, R>(A, s_pp[wib], na, L.pp, nbuf, ic, lane);
                        nbuf = 0;
                    }
                    if (has) L.pp[nbuf + __popc(bm & lt)] = ent;
                    nbuf += k;
                    __syncwarp();
                };
                for (int cursor = 0; cursor < ncand; cursor += 32) {
                    const int j = cursor + lane;
                    int2 ce = make_int2(0, 0);
                    bool has = j < ncand;
                    if (has) ce = cand ? cand[j] : make_int2(da, 0);
                    // node candidates
                    int dec = D_DROP, e = 0;
                    G4Node nb;
                    float rx = 0.f, ry = 0.f, rz = 0.f;
                    if (has && ce.x >= 0) {
                        nb = load_node(A.node + ce.x);
                        dec = fmm_decide<P, TREEPM, GEOM>(A, na, da, nb, ce.x, rx, ry, rz);
                        if (dec == D_OPEN && !(nb.meta & 32u)) e = nb.nchild;   // B internal
                    }
                    if (ic == 0 && dec == D_ACCEPT) {
                        R qx, qy, qz;
                        sep_nodes<TREEPM, R>(A, na, da, nb, ce.x, rx, ry, rz, qx, qy, qz);
                        m2l_add<P, TREEPM, R>(A, T, ce.x, nb, qx, qy, qz,
                                              (R)(A.soft_nodes ? fmaxf(na.hmax, nb.hmax) : 0.f));
                        nm2l++;
                    }
                    // leaf pairs (A itself, or a leaf B that fails): all of A's particles
                    const bool lp = ic == 0 && (dec == D_SELF || dec == D_P2P ||
                                                (dec == D_OPEN && (nb.meta & 32u)));
                    push_pp(lp, make_int4(nb.first, nb.count, 0, 0));
                    // internal B that fails: its daughters start A's particle walk
                    const int pre = warp_excl_i(e, lane);
                    const int tot = warp_sum_i(e);
                    if (sp + tot > FMM_STACK) {
                        if (lane == 0) atomicOr(A.flags, G4_FLAG_LISTCAP);
                    } else {
                        for (int k = 0; k < e; k++)
                            L.stack[sp + pre + k] =
                                make_int2(__ldg(A.kids + (size_t)ce.x * 8 + k), (int)vmask);
                        sp += tot;
                    }
                    // particle candidates (taken once): accepted ones add to A's field, the
                    // others that fail meet all of A's particles
                    const bool pc = ic == 0 && has && ce.x < 0;
                    if (__any_sync(0xffffffffu, pc && ce.y != 0)) {
                        const int p0 = -ce.x - 1;
                        const unsigned pm = pc ? (unsigned)ce.y : 0u;
                        for (int bit = 0; bit < 32; bit++) {
                            bool op = false;
                            int y = 0;
                            if ((pm >> bit) & 1u) {
                                y = p0 + bit;
                                const PCell x = load_pcell(A, y);
                                float qx, qy, qz;
                                const int d = fmm_decide_pn<P, TREEPM, GEOM>(A, na, x, qx, qy, qz);
                                if (d == D_ACCEPT) {
                                    R ux, uy, uz;
                                    sep_node_particle<TREEPM, R>(A, na, da, x, qx, qy, qz, ux, uy, uz);
                                    p2l_add<P, TREEPM, R>(A, T, (R)x.m, -ux, -uy, -uz,
                                                          (R)(A.soft_nodes ? fmaxf(na.hmax, x.h) : 0.f));
                                }
                                op = d == D_OPEN;
                            }
                            push_pp(op, make_int4(y, 1, 0, 0));
                        }
                    }
                    __syncwarp();
                    // the particle walk: one stack entry at a time, every lane decides for its
                    // own particle (drop, field of the node at the particle, or open)
                    while (sp > 0) {
                        sp--;
                        const int2 se = L.stack[sp];
                        __syncwarp();
                        const G4Node nz = load_node(A.node + se.x);
                        int d = D_DROP;
                        float qx = 0.f, qy = 0.f, qz = 0.f;
                        if (((unsigned)se.y >> lane) & 1u)
                            d = fmm_decide_pn<P, TREEPM, GEOM>(A, nz, xs, qx, qy, qz);
                        if (d == D_ACCEPT) {
                            R ux, uy, uz;
                            sep_node_particle<TREEPM, R>(A, nz, se.x, xs, qx, qy, qz, ux, uy, uz);
                            m2p_add<P, TREEPM, R>(A, se.x, nz, ux, uy, uz,
                                                  (R)(A.soft_nodes ? fmaxf(nz.hmax, xs.h) : 0.f), bx,
                                                  by, bz, bp);
                            npn++;
                        }
                        const unsigned om = __ballot_sync(0xffffffffu, d == D_OPEN);
                        if (om) {
                            if (nz.meta & 32u) {
                                push_pp(lane == 0, make_int4(nz.first, nz.count, (int)om, 0));
                            } else if (sp + nz.nchild > FMM_STACK) {
                                if (lane == 0) atomicOr(A.flags, G4_FLAG_LISTCAP);
                            } else {
                                if (lane < nz.nchild)   // one daughter per lane
                                    L.stack[sp + lane] =
                                        make_int2(__ldg(A.kids + (size_t)se.x * 8 + lane), (int)om);
                                sp += nz.nchild;
                                __syncwarp();
                            }
                        }
                    }
                }
                if (nbuf > 0 && !defer_p2p(A, da, L.pp, nbuf, ic, lane, tail))
                    p2p_flush<TREEPM, R>(A, s_pp[wib], na, L.pp, nbuf, ic, lane);
                if (valid) {
                    const R mG = -(R)A.G;
                    A.acc[i] = (float)((R)A.acc[i] + mG * bx);
                    A.acc[A.n + i] = (float)((R)A.acc[A.n + i] + mG * by);
                    A.acc[2 * A.n + i] = (float)((R)A.acc[2 * A.n + i] + mG * bz);
                    if (A.pot) A.pot[i] = (float)((R)A.pot[i] + mG * bp);
                    if (A.counts) A.counts[A.n + i] = npn;
                }
                __syncwarp();
            }
        }
        // reduce the lane-private fields and store the node's own field
#pragma unroll
        for (int k = 0; k < NT; k++) {
            const R v = warp_sum_f(T[k]);
            if (lane == 0) ((R *)A.T_own)[(size_t)da * NT + k] = v;
        }
        nm2l = warp_sum_i(nm2l);
        if (lane == 0) A.m2l_own[da] = (uint32_t)nm2l;
    }
}

// downward pass: T_tot = T_own + shifted parent field (L2L); leaves evaluate at particles (L2P)
template <int P, typename R>
__global__ void __launch_bounds__(128) k_fmm_down(const FmmArgs A, int level)
{
    constexpr int NT = FT<P>::NT;
    if (*A.flags & G4_FLAG_CAPACITY) return;
    const int32_t *off = A.lvl, *cnt = A.lvl + G4_NLEVELS + 1;
    const int o = off[level], c = cnt[level];
    const int total_nodes = off[G4_NLEVELS];
    const R scale = (R)A.scale;
    const R *Town = (const R *)A.T_own;
    R *Ttot = (R *)A.T_tot;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < c; b += gridDim.x * blockDim.x) {
        const int d = A.b_dfs[o + b];
        if ((unsigned)d >= (unsigned)total_nodes) continue;
        const G4Node nd = load_node(A.node + d);
        // centre-of-mass offset (FP64 node data in the FP64 mode)
        R ndx = nd.sx, ndy = nd.sy, ndz = nd.sz;
        if (sizeof(R) == 8) {
            const double *dd = node_fp64(A, d);
            ndx = (R)dd[0]; ndy = (R)dd[1]; ndz = (R)dd[2];
        }
        R T[NT];
#pragma unroll
        for (int k = 0; k < NT; k++) T[k] = Town[(size_t)d * NT + k];
        uint32_t cum = A.m2l_own[d];
        if (nd.parent >= 0) {
            const G4Node np = load_node(A.node + nd.parent);
            R npx = np.sx, npy = np.sy, npz = np.sz;
            if (sizeof(R) == 8) {
                const double *dp = node_fp64(A, nd.parent);
                npx = (R)dp[0]; npy = (R)dp[1]; npz = (R)dp[2];
            }
            const R dx = (R)(int32_t)(nd.cx - np.cx) * scale + (ndx - npx);
            const R dy = (R)(int32_t)(nd.cy - np.cy) * scale + (ndy - npy);
            const R dz = (R)(int32_t)(nd.cz - np.cz) * scale + (ndz - npz);
            R px[P + 1], py[P + 1], pz[P + 1];
            px[0] = py[0] = pz[0] = R(1);
#pragma unroll
            for (int k = 1; k <= P; k++) {
                px[k] = px[k - 1] * dx;
                py[k] = py[k - 1] * dy;
                pz[k] = pz[k - 1] * dz;
            }
            const R *Tp = Ttot + (size_t)nd.parent * NT;
#pragma unroll
            for (int kn = 0; kn <= P; kn++)
#pragma unroll
                for (int kbc = 0; kbc <= kn; kbc++)
#pragma unroll
                    for (int kc = 0; kc <= kbc; kc++) {
                        const int ka = kn - kbc, kb = kbc - kc;
                        R s = R(0);
#pragma unroll
                        for (int mn = 0; mn <= P - kn; mn++)
#pragma unroll
                            for (int mbc = 0; mbc <= mn; mbc++)
#pragma unroll
                                for (int mc = 0; mc <= mbc; mc++) {
                                    const int ma = mn - mbc, mb = mbc - mc;
                                    s += Tp[g4_midx(ka + ma, kb + mb, kc + mc)] * px[ma] * py[mb] *
                                         pz[mc] * (R(1) / (R)(fact(ma) * fact(mb) * fact(mc)));
                                }
                        T[g4_midx(ka, kb, kc)] += s;
                    }
            cum += A.m2l_cum[nd.parent];
        }
#pragma unroll
        for (int k = 0; k < NT; k++) Ttot[(size_t)d * NT + k] = T[k];
        A.m2l_cum[d] = cum;
        if (nd.meta & 32u) {
            for (int i = nd.first; i < nd.first + nd.count; i++) {
                const R ax = (R)(int32_t)(A.pos[i] - nd.cx) * scale - ndx;
                const R ay = (R)(int32_t)(A.pos[A.n + i] - nd.cy) * scale - ndy;
                const R az = (R)(int32_t)(A.pos[2 * A.n + i] - nd.cz) * scale - ndz;
                R px[P + 1], py[P + 1], pz[P + 1];
                px[0] = py[0] = pz[0] = R(1);
#pragma unroll
                for (int k = 1; k <= P; k++) {
                    px[k] = px[k - 1] * ax;
                    py[k] = py[k - 1] * ay;
                    pz[k] = pz[k - 1] * az;
                }
                R phi = R(0), gx = R(0), gy = R(0), gz = R(0);
#pragma unroll
                for (int kn = 0; kn <= P; kn++)
#pragma unroll
                    for (int kbc = 0; kbc <= kn; kbc++)
#pragma unroll
                        for (int kc = 0; kc <= kbc; kc++) {
                            const int ka = kn - kbc, kb = kbc - kc;
                            const R w = px[ka] * py[kb] * pz[kc] *
                                        (R(1) / (R)(fact(ka) * fact(kb) * fact(kc)));
                            phi += T[g4_midx(ka, kb, kc)] * w;
                            if (kn < P) {
                                gx += T[g4_midx(ka + 1, kb, kc)] * w;
                                gy += T[g4_midx(ka, kb + 1, kc)] * w;
                                gz += T[g4_midx(ka, kb, kc + 1)] * w;
                            }
                        }
                A.acc[i] = (float)((R)A.acc[i] - gx);
                A.acc[A.n + i] = (float)((R)A.acc[A.n + i] - gy);
                A.acc[2 * A.n + i] = (float)((R)A.acc[2 * A.n + i] - gz);
                if (A.pot) A.pot[i] = (float)((R)A.pot[i] + phi);
                if (A.counts) A.counts[2 * A.n + i] = cum;
            }
        }
    }
}

template <int P, bool TREEPM, bool GEOM, typename R>
void run_fmm(const FmmArgs &A, cudaStream_t st)
{
    const int nb = g4_num_sms() * 8;
    for (int l = 0; l <= G4_MAXLEVEL; l++) {
        if (l >= 2) {
            // the list of level l-2 is no longer needed: its buffer is reused at level l
            cudaMemsetAsync(A.dcount + (l & 1), 0, sizeof(int32_t), st);
        }
        k_fmm_level<P, TREEPM, GEOM, R><<<nb, FMM_THREADS, 0, st>>>(A, l);
    }
    k_fmm_p2p<TREEPM, R><<<g4_num_sms() * fmm_p2p_blocks<R>(), FMM_THREADS, 0, st>>>(A);
    for (int l = 0; l <= G4_MAXLEVEL; l++) k_fmm_down<P, R><<<nb, 128, 0, st>>>(A, l);
}

}  // namespace

// The variant's launches: the dual walk level by level, the deferred particle pairs, the
// downward pass.
template <int P, bool TREEPM, typename R>
void g4fmm::run_variant(const FmmArgs &A, bool geom, cudaStream_t st)
{
    if (geom) run_fmm<P, TREEPM, true, R>(A, st);
    else run_fmm<P, TREEPM, false, R>(A, st);
}
