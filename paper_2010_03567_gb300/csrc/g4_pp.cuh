// g4_pp.cuh -- the particle-particle phase shared by the tree walk and the FMM's leaf-leaf
// interactions: for up to 32 sinks (one per lane) and a list of source leaves (with the mask of
// the lanes that may see each), stage the sources, test them against every sink in packed
// FP16x2, and evaluate each lane's candidates exactly (Eqs. eqnsoft, eqnpo4; Sec. 2.3).
#pragma once
#include <cuda_fp16.h>

#include "g4_kernels.cuh"
#include "g4_ewald.cuh"
#include "g4_pp_fp16.h"

namespace g4k {

constexpr int PP_STAGE = 128;   // sources staged per pass
// FP16x2 candidate test.  For a group whose sinks lie within R r_cut of the group centre (per
// axis), FP16 positions relative to the centre in units of r_cut err by at most e = (2 R + 2)
// 2^-11 per axis (sink, source, difference), so a pair inside r_cut has a computed r^2 of at
// most 1 + 2 sqrt(3) e + 3 e^2, plus ~0.0016 of rounding in the FP16 sums.  The threshold is
// that bound (with slack, rounded up), so no pair inside r_cut is missed: ~1.012 r_cut^2 for
// compact groups, wider for spread ones.  Beyond PP_FP16_RMAX (where the threshold reaches 20)
// every staged source is a candidate.  The constants are in g4_pp_fp16.h.
constexpr float PP_FP16_RMAX = G4_PP_FP16_RMAX;

// pending source leaves and the staged sources of one warp
template <int LB> struct PPSmem {
    int first[LB], count[LB], pref[LB];
    unsigned mask[LB];
    uint4 ipos[PP_STAGE];          // source integer position, softening length h (bits)
    float2 mj[PP_STAGE];           // source mass, particle index (bits)
    unsigned smask[PP_STAGE];      // lane mask of the source's leaf
    __align__(16) __half hx[PP_STAGE];   // source position / r_cut relative to the group centre
    __align__(16) __half hy[PP_STAGE];
    __align__(16) __half hz[PP_STAGE];
};

// a launch parameter in the arithmetic type of the caller
template <typename T> __device__ __forceinline__ T par(double d, float f);
template <> __device__ __forceinline__ float par<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double par<double>(double d, float) { return d; }

// largest power of two <= n; a binary search over n + 1 pending leaves starts with that step,
// so that every index up to n is reachable
__host__ __device__ constexpr int pow2_floor(int n) { return n < 2 ? 1 : 2 * pow2_floor(n / 2); }

// Slot of staged source u in the candidate masks.  The FP16x2 test handles sources 2j, 2j+1
// of a 32-source block together and sets bits j and 16 + j of the block's mask word, so the
// per-source arrays used by the evaluation are stored at that bit position.
__device__ __forceinline__ int cand_bit(int u)
{
    return (u & ~31) | ((u & 1) << 4) | ((u & 31) >> 1);
}

// Particle-particle phase for the pending leaves of a group.
// Sources are staged 128 at a time.  TreePM with the pair cutoff: every lane first tests all
// staged sources against its own sink in packed FP16x2 (two sources per instruction;
// positions relative to the group centre in units of r_cut, threshold from the group's FP16
// error bound, so no pair inside r_cut is missed) and keeps a candidate bit per source; then
// each lane evaluates only its own candidates with exact integer separations, the exact
// cutoff and the full kernel.  Without the pair cutoff, for a group spread wider than
// PP_FP16_RMAX, or for one reaching within r_cut of half the periodic box from its centre,
// every staged source is a candidate.  Leaf masks (lanes that used an
// ancestor's multipole must not see the leaf) are applied per source when a staged leaf does
// not reach the whole group.  INTU (FP32 TreePM): the pair terms are summed in integer-grid
// length units with the fast kernel; the caller rescales the sums.  Part kp of Kp (a group
// split by the cost-model schedule) takes list positions kp, kp + Kp, ...; Kp = 1: all.
// A lane's sums follow its staging order (deterministic for a given leaf list).
// Args provides: wpart (16-byte particle records), cls, h_cls, pp_cut, rcut2/rcut2f, as/asf.
template <typename T, bool TREEPM, int LB, class Args>
__device__ __forceinline__ void pp_flush(const Args &A, PPSmem<LB> &S, int nleaf, int lane, int i,
                                         uint32_t xi, uint32_t yi, uint32_t zi, uint32_t gcx,
                                         uint32_t gcy, uint32_t gcz, float xr, float yr, float zr,
                                         unsigned vmask, T hi, T &ax, T &ay, T &az, T &ap,
                                         uint32_t &npp, double gscale, float figs, const PairF &pf,
                                         float rc2i, int kp, int Kp)
{
    constexpr bool INTU = TREEPM && sizeof(T) == 4;
    const float fscale = (float)gscale;
    const T scale = (T)gscale, as = par<T>(A.as, A.asf), rcut2 = par<T>(A.rcut2, A.rcut2f);
    const float hconv = INTU ? figs : 1.f;   // staged softening length unit
    // drop leaves nobody reaches; prefix sums of the particle counts
    int nk = 0, total = 0;
    for (int b = 0; b < nleaf; b += 32) {
        const int e = b + lane;
        const bool ok = e < nleaf;
        int f = 0, c = 0;
        unsigned m = 0;
        if (ok) {
            f = S.first[e];
            c = S.count[e];
            m = S.mask[e];
        }
        const bool keep = ok && m != 0u;
        const unsigned km = __ballot_sync(0xffffffffu, keep);
        const int cc = keep ? c : 0;
        int pre = cc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += y;
        }
        __syncwarp();
        if (keep) {
            const int pos = nk + __popc(km & ((1u << lane) - 1u));
            S.first[pos] = f;
            S.count[pos] = c;
            S.mask[pos] = m;
            S.pref[pos] = total + pre - cc;
        }
        __syncwarp();
        nk += __popc(km);
        total += __shfl_sync(0xffffffffu, pre, 31);
    }
    const float inv_rc = TREEPM ? rsqrtf(A.rcut2f) : 0.f;
    // group radius R in units of r_cut (non-negative floats order like their bit patterns)
    const float R = __uint_as_float(__reduce_max_sync(
        0xffffffffu, __float_as_uint(fmaxf(fabsf(xr), fmaxf(fabsf(yr), fabsf(zr))) * inv_rc)));
    // The FP16 positions are nearest-image offsets from the group centre, so a source within
    // r_cut of a sink keeps its true offset only while R + 1 stays below half the box (in r_cut
    // units); a group reaching that far in a periodic box (a sparse subset, say) would see
    // such sources wrapped to the other side, so it skips the FP16 test.
    const float half_box = 2147483648.f * fscale * inv_rc;
    const bool test16 = TREEPM && A.pp_cut && R <= PP_FP16_RMAX && R + 1.01f < half_box;
    const float e16 = (G4_PP_FP16_EA * R + G4_PP_FP16_EB) * (1.f / G4_PP_FP16_ULP);
    const __half2 nlim = __half2half2(__float2half_rd(
        -((1.f + G4_PP_FP16_C1 * e16 + G4_PP_FP16_C2 * e16 * e16) * G4_PP_FP16_SLACK_MUL +
          G4_PP_FP16_SLACK_ADD)));
    const __half2 sx2 = __float2half2_rn(xr * inv_rc), sy2 = __float2half2_rn(yr * inv_rc),
                  sz2 = __float2half2_rn(zr * inv_rc);
    // Staged sources farther than r_cut from the sinks' bounding box (half extents gbx, gby,
    // gbz about the centre) cannot pair with any sink: they are dropped before the per-lane
    // tests (about half of the staged sources in a clustered box, whose leaves overhang the
    // cutoff sphere).  Offsets and extents are rounded alike, and their FP32 error at
    // R <= G4_PP_PRUNE_RMAX (64) is below 1e-5 r_cut, inside the G4_PP_PRUNE_MARGIN (2e-4)
    // on r_cut^2.  Same nearest-image guard as the FP16 test.
    const bool prune = TREEPM && A.pp_cut && R <= G4_PP_PRUNE_RMAX && R + 1.01f < half_box;
    const float gbx = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(xr))));
    const float gby = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(yr))));
    const float gbz = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(zr))));
    const float plim = A.rcut2f * G4_PP_PRUNE_MARGIN;
    // Batch bb takes sources bb, bb + nbat, bb + 2 nbat, ...: every batch samples the whole
    // neighbourhood, so each lane's candidates spread evenly over the batches and the per-lane
    // evaluation loops below stay balanced across the warp.
    // part kp of Kp takes list positions kp, kp + Kp, kp + 2 Kp, ... (a split group's parts
    // share the list; Kp = 1: the whole list)
    const int tv = total > kp ? (total - kp + Kp - 1) / Kp : 0;
    const int nbat = (tv + PP_STAGE - 1) / PP_STAGE;
    // slot q of this lane stages virtual position bb + (32 q + lane) nbat in batch bb, list
    // position t = kp + Kp * (that); its leaf lq: a fixed-step binary search for bb = 0, then
    // it only moves forward
    int lq[PP_STAGE / 32], tq[PP_STAGE / 32];
#pragma unroll
    for (int q = 0; q < PP_STAGE / 32; q++) {
        lq[q] = 0;
        tq[q] = kp + Kp * ((q * 32 + lane) * nbat);
    }
#pragma unroll
    for (int step = pow2_floor(LB - 1); step >= 1; step >>= 1)
#pragma unroll
        for (int q = 0; q < PP_STAGE / 32; q++) {
            const int c = lq[q] + step;
            if (c < nk && S.pref[c] <= tq[q]) lq[q] = c;
        }
    for (int bb = 0; bb < nbat; bb++) {
        const int nb = (tv - bb + nbat - 1) / nbat;
        bool partial = false;
        if (bb > 0) {
#pragma unroll
            for (int q = 0; q < PP_STAGE / 32; q++) {
                tq[q] += Kp;
                while (lq[q] + 1 < nk && S.pref[lq[q] + 1] <= tq[q]) lq[q]++;
            }
        }
        uint4 pq[PP_STAGE / 32];
        int jq[PP_STAGE / 32];
#pragma unroll
        for (int q = 0; q < PP_STAGE / 32; q++) {
            const int u = q * 32 + lane;
            jq[q] = S.first[lq[q]] + (tq[q] - S.pref[lq[q]]);
            pq[q] = u < nb ? __ldg(A.wpart + jq[q]) : make_uint4(gcx, gcy, gcz, 0u);
        }
        // staged sources kept (all of them without the prune), packed in staging order
        int ns = 0;
#pragma unroll
        for (int q = 0; q < PP_STAGE / 32; q++) {
            const int u = q * 32 + lane;
            const uint32_t px = pq[q].x, py = pq[q].y, pz = pq[q].z;
            const float ox = (float)(int32_t)(px - gcx) * fscale;
            const float oy = (float)(int32_t)(py - gcy) * fscale;
            const float oz = (float)(int32_t)(pz - gcz) * fscale;
            bool keep = u < nb;
            if (prune && keep) {
                const float ex = fmaxf(fabsf(ox) - gbx, 0.f), ey = fmaxf(fabsf(oy) - gby, 0.f),
                            ez = fmaxf(fabsf(oz) - gbz, 0.f);
                keep = fmaf(ez, ez, fmaf(ey, ey, ex * ex)) <= plim;
            }
            const unsigned km = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int us = ns + __popc(km & ((1u << lane) - 1u)), v = cand_bit(us);
                const int j = jq[q];
                const float hj = A.h_cls[A.cls ? __ldg(A.cls + j) : 0] * hconv;
                const unsigned mk = S.mask[lq[q]];
                S.ipos[v] = make_uint4(px, py, pz, __float_as_uint(hj));
                S.mj[v] = make_float2(__uint_as_float(pq[q].w), __int_as_float(j));
                S.smask[v] = mk;
                S.hx[us] = __float2half_rn(ox * inv_rc);
                S.hy[us] = __float2half_rn(oy * inv_rc);
                S.hz[us] = __float2half_rn(oz * inv_rc);
                partial |= (mk != vmask);
            }
            ns += __popc(km);
        }
        {
            // pad the last block of 32 with sources no test accepts
            const int us = ns + lane;
            if (us < ((ns + 31) & ~31)) {
                S.hx[us] = S.hy[us] = S.hz[us] = __float2half_rn(100.f);
                S.smask[cand_bit(us)] = 0xffffffffu;
            }
        }
        partial = __any_sync(0xffffffffu, partial);
        __syncwarp();
        const int nw = (ns + 31) >> 5;
        uint32_t w0 = 0u, w1 = 0u, w2 = 0u, w3 = 0u;
        if (test16) {
            const uint4 *X = reinterpret_cast<const uint4 *>(S.hx);
            const uint4 *Y = reinterpret_cast<const uint4 *>(S.hy);
            const uint4 *Z = reinterpret_cast<const uint4 *>(S.hz);
            for (int w = 0; w < nw; w++) {
                uint32_t m = 0u;
#pragma unroll
                for (int qd = 0; qd < 4; qd++) {
                    const uint4 x4 = X[4 * w + qd], y4 = Y[4 * w + qd], z4 = Z[4 * w + qd];
                    const uint32_t xs[4] = {x4.x, x4.y, x4.z, x4.w};
                    const uint32_t ys[4] = {y4.x, y4.y, y4.z, y4.w};
                    const uint32_t zs[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        const __half2 dx = __hsub2(*reinterpret_cast<const __half2 *>(&xs[c]), sx2);
                        const __half2 dy = __hsub2(*reinterpret_cast<const __half2 *>(&ys[c]), sy2);
                        const __half2 dz = __hsub2(*reinterpret_cast<const __half2 *>(&zs[c]), sz2);
                        // r^2 - threshold: a set sign bit marks a candidate; the low / high
                        // halves' sign bits (15, 31) move to bits k, 16 + k
                        const __half2 d2 = __hfma2(dz, dz, __hfma2(dy, dy, __hfma2(dx, dx, nlim)));
                        const int k = 4 * qd + c;   // a constant once unrolled
                        m |= (*reinterpret_cast<const uint32_t *>(&d2) >> (15 - k)) &
                             (0x00010001u << k);
                    }
                }
                w0 = w == 0 ? m : w0;
                w1 = w == 1 ? m : w1;
                w2 = w == 2 ? m : w2;
                w3 = w == 3 ? m : w3;
            }
        } else {
            // every kept source is a candidate; bit positions of sources u < ns
#pragma unroll
            for (int w = 0; w < 4; w++) {
                const int r = min(max(ns - 32 * w, 0), 32);   // valid sources in block w
                const int ev = (r + 1) >> 1, od = r >> 1;      // even / odd ones
                const uint32_t m = (ev >= 16 ? 0xffffu : ((1u << ev) - 1u)) |
                                   ((od >= 16 ? 0xffffu : ((1u << od) - 1u)) << 16);
                if (w == 0) w0 = m;
                else if (w == 1) w1 = m;
                else if (w == 2) w2 = m;
                else w3 = m;
            }
        }
        if (partial) {
            for (int v = 0; v < 32 * nw; v++)
                if (!((S.smask[v] >> lane) & 1u)) {
                    const uint32_t clr = ~(1u << (v & 31));
                    if (v < 32) w0 &= clr;
                    else if (v < 64) w1 &= clr;
                    else if (v < 96) w2 &= clr;
                    else w3 &= clr;
                }
        }
        // the lane's nonempty candidate words packed to the front (cw first), with their slot
        // offsets in the bytes of `bases`; popping a candidate is then a bit scan and a clear
        uint32_t cw = 0u, n1 = 0u, n2 = 0u, n3 = 0u, bases = 0u;
#pragma unroll
        for (int w = 3; w >= 0; w--) {
            const uint32_t x = w == 0 ? w0 : (w == 1 ? w1 : (w == 2 ? w2 : w3));
            const bool e = x != 0u;
            n3 = e ? n2 : n3;
            n2 = e ? n1 : n2;
            n1 = e ? cw : n1;
            cw = e ? x : cw;
            bases = e ? (bases << 8) | (uint32_t)(32 * w) : bases;
        }
        // exact evaluation of the lane's own candidates
        while (cw) {
            const int v = (int)(bases & 0xffu) + __clz(__brev(cw));
            cw &= cw - 1u;
            const bool e = cw == 0u;
            cw = e ? n1 : cw;
            n1 = e ? n2 : n1;
            n2 = e ? n3 : n2;
            n3 = e ? 0u : n3;
            bases = e ? bases >> 8 : bases;
            const uint4 ip = S.ipos[v];
            const float2 mj = S.mj[v];
            if (INTU) {
                // branch-free: the sink itself and pairs beyond the cutoff get mass 0 at a
                // harmless separation, so the lanes of the warp stay in step
                const float dx = (float)(int32_t)(ip.x - xi);
                const float dy = (float)(int32_t)(ip.y - yi);
                const float dz = (float)(int32_t)(ip.z - zi);
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const bool use = __float_as_int(mj.y) != i && !(A.pp_cut && r2 >= rc2i);
                float g0, g1;
                pair_treepm_fast(use ? r2 : rc2i, fmaxf((float)hi, __uint_as_float(ip.w)), pf, g0, g1);
                const float m_ = use ? mj.x : 0.f;
                const float mg1 = m_ * g1;
                ax = fmaf(mg1, dx, (float)ax);
                ay = fmaf(mg1, dy, (float)ay);
                az = fmaf(mg1, dz, (float)az);
                ap = fmaf(m_, g0, (float)ap);
                npp += use;
                continue;
            } else {
                if (__float_as_int(mj.y) == i) continue;
                const T dx = (T)(int32_t)(ip.x - xi) * scale;
                const T dy = (T)(int32_t)(ip.y - yi) * scale;
                const T dz = (T)(int32_t)(ip.z - zi) * scale;
                const T r2 = dx * dx + dy * dy + dz * dz;
                if (TREEPM && A.pp_cut && r2 >= rcut2) continue;
                T g0, g1;
                pair_kernel<T, TREEPM>(r2, fmax(hi, (T)__uint_as_float(ip.w)), as, g0, g1);
                const T m_ = (T)mj.x;
                const T mg1 = m_ * g1;
                ax += mg1 * dx;
                ay += mg1 * dy;
                az += mg1 * dz;
                ap += m_ * g0;
                if (!TREEPM && A.ewald) {
                    // Ewald correction of the pair (Sec. 2.2.4): + G m psi(d) in the
                    // potential, + G m grad psi(d) in the acceleration (sums carry -G)
                    T Dp[4];
                    ewald_dpsi<1, T>(A.ew, dx, dy, dz, Dp);
                    ap -= m_ * Dp[0];
                    ax -= m_ * Dp[g4_midx(1, 0, 0)];
                    ay -= m_ * Dp[g4_midx(0, 1, 0)];
                    az -= m_ * Dp[g4_midx(0, 0, 1)];
                }
            }
            npp++;
        }
        __syncwarp();
    }
}

}  // namespace g4k
