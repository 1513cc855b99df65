// g4_ewald.cuh -- Ewald correction of the pure periodic tree (Sec. 2.2.4): the derivative
// tensors D_n of the correction potential psi (Eq. eqnewal) at an arbitrary separation, by a
// third-order Taylor expansion about the nearest point of a precomputed grid of the tensors
// up to order n + 3 (the paper's scheme; the grid is built by g4_ewald.cu).
//
// Grid: G^3 cells covering one octant [0, L/2]^3 of the primary cell, values at the cell
// centres ((i + 1/2) h, h = L / (2G)), all monomial components D_abc, a + b + c <= nt, at
// g4_midx(a, b, c).  psi is even in each coordinate, so for a separation x the expansion is
// taken at |x| and component D_abc changes sign with each reflected axis counted a, b, c
// times.  Valid for separations in the primary cell, as nearest images are.
#pragma once
#include "g4_internal.cuh"
#include "g4_kernels.cuh"

struct G4EwaldView {
    const float *t32;     // FP32 grid (cells x nmono(nt))
    const double *t64;    // FP64 grid
    int nt;               // highest tabulated order
    int G;                // cells per axis
    double h;             // cell size L / (2G)
};

namespace g4k {

template <typename T> __device__ __forceinline__ const T *ew_tab(const G4EwaldView &E);
template <> __device__ __forceinline__ const float *ew_tab<float>(const G4EwaldView &E) { return E.t32; }
template <> __device__ __forceinline__ const double *ew_tab<double>(const G4EwaldView &E) { return E.t64; }

// D[g4_midx(a,b,c)] = D_abc[psi](x, y, z) for a + b + c <= N (N + 3 <= E.nt).
template <int N, typename T>
__device__ __forceinline__ void ewald_dpsi(const G4EwaldView &E, T x, T y, T z, T *D)
{
    const T ax = fabs(x), ay = fabs(y), az = fabs(z);
    const T h = (T)E.h, hinv = T(1) / h;
    const int ix = max(0, min((int)(ax * hinv), E.G - 1)), iy = max(0, min((int)(ay * hinv), E.G - 1)),
              iz = max(0, min((int)(az * hinv), E.G - 1));
    const T dx = ax - (T(ix) + T(0.5)) * h, dy = ay - (T(iy) + T(0.5)) * h,
            dz = az - (T(iz) + T(0.5)) * h;
    const T *c = ew_tab<T>(E) + ((size_t)(ix * E.G + iy) * E.G + iz) * g4_nmono(E.nt);
    // dx^i / i!, i <= 3
    const T px[4] = {T(1), dx, dx * dx * T(0.5), dx * dx * dx * T(1.0 / 6.0)};
    const T py[4] = {T(1), dy, dy * dy * T(0.5), dy * dy * dy * T(1.0 / 6.0)};
    const T pz[4] = {T(1), dz, dz * dz * T(0.5), dz * dz * dz * T(1.0 / 6.0)};
    const bool fx = x < T(0), fy = y < T(0), fz = z < T(0);
#pragma unroll
    for (int n = 0; n <= N; n++)
#pragma unroll
        for (int bc = 0; bc <= n; bc++)
#pragma unroll
            for (int cc = 0; cc <= bc; cc++) {
                const int a = n - bc, b = bc - cc;
                T s = T(0);
#pragma unroll
                for (int m = 0; m <= 3; m++)
#pragma unroll
                    for (int jk = 0; jk <= m; jk++)
#pragma unroll
                        for (int k = 0; k <= jk; k++) {
                            const int i = m - jk, j = jk - k;
                            s += c[g4_midx(a + i, b + j, cc + k)] * px[i] * py[j] * pz[k];
                        }
                const bool neg = ((a & 1) && fx) ^ ((b & 1) && fy) ^ ((cc & 1) && fz);
                D[g4_midx(a, b, cc)] = neg ? -s : s;
            }
}

// Ewald correction of an accepted node with moments (M, Qs) about its centre of mass at
// r = s - x (nearest image): the correction potential psi expanded like the Newtonian term,
// with the opposite sign (it enters the potential as +G sum m psi):
// sacc -= sum_{n<P} Q_n . D_{n+1}[psi] / n!,  spot -= sum_{n<=P} Q_n . D_n[psi] / n!.
template <int P, typename T>
__device__ __forceinline__ void pn_ewald(const G4EwaldView &E, const T *Qs, T M, T x, T y, T z,
                                         T &sx, T &sy, T &sz, T &sp)
{
    T D[g4_nmono(P)];
    ewald_dpsi<P, T>(E, x, y, z, D);
    T cx = T(0), cy = T(0), cz = T(0), cp = T(0);
    pn_contract<P, T>(Qs, M, D, cx, cy, cz, cp);
    sx -= cx;
    sy -= cy;
    sz -= cz;
    sp -= cp;
}

}  // namespace g4k

// the grid for box size L with orders up to nt (built or reused; see g4_ewald.cu)
g4_status g4_ewald_ensure(struct g4_tree_s *t, double L, int nt, cudaStream_t st,
                          G4EwaldView *view);
