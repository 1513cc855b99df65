// g4_ewald.cu -- the grid of Ewald correction tensors for the pure periodic tree
// (Sec. 2.2.4): D_abc[psi] at the cell centres of one octant of the primary cell, computed in
// FP64 from the Ewald sums of Eq. (eqnewal), term by term:
//   psi = pi/(a^2 V) + erf(a|x|)/|x| - sum_{n != 0} erfc(a|x+q_n|)/|x+q_n|
//         - (4 pi / V) sum_{k != 0} exp(-k^2/(4 a^2))/k^2 cos(k . x),
// radial terms through g_n = (r^-1 d/dr)^n and the tensor formula of D_abc, Fourier terms
// through d/dx_i cos(k.x + phase) = k_i cos(k.x + phase + pi/2) (k and -k together).  Split
// a = 3.5 / L with images |n_i| <= 1 (the first one left out lies beyond 1.5 L from any point
// of the primary cell: erfc(5.25) ~ 1e-13) and wave vectors |m_i| <= 7 (k = 2 pi m / L:
// exp(-pi^2 m^2 / (a L)^2) ~ 1e-17 at m = 7).  For erf(a r)/r at a r < 1.5 the g_n come from
// its power series (1/r and erfc/r would cancel there).
#include "g4_internal.cuh"
#include "g4_kernels.cuh"
#include "g4_ewald.cuh"

namespace {

using namespace g4k;

constexpr int EW_G = 32;             // cells per axis of the octant
constexpr int EW_NK = 7;             // wave vectors |m_i| <= EW_NK
constexpr double EW_ALPHA_L = 3.5;   // a L
constexpr int EW_THREADS = 224;      // one thread per component (nmono(9) = 220)
constexpr int EW_NMAX = 9;           // highest tabulated order
constexpr int EW_KSIDE = 2 * EW_NK + 1;

// g_n of erf(a r)/r, n = 0..EW_NMAX
__device__ void ew_gn_erf(double r, double a, double *g)
{
    const double x = a * r;
    if (x < 1.5) {
        // g_n = (-1)^n (2/sqrt(pi)) 2^n a^(2n+1) sum_j (-1)^j x^(2j) / (j! (2j + 2n + 1))
        double pre = 1.1283791670955126 * a;
        for (int n = 0; n <= EW_NMAX; n++) {
            double s = 0.0, term = 1.0;
            for (int j = 0; j < 48; j++) {
                s += term / (2.0 * j + 2.0 * n + 1.0);
                term *= -x * x / (j + 1.0);
            }
            g[n] = ((n & 1) ? -pre : pre) * s;
            pre *= 2.0 * a * a;
        }
        return;
    }
    double gN[EW_NMAX + 1], gE[EW_NMAX + 1];
    gn_kernel<EW_NMAX, double, false>(r * r, 0.0, gN);
    gn_kernel<EW_NMAX, double, true>(r * r, a, gE);
    for (int n = 0; n <= EW_NMAX; n++) g[n] = gN[n] - gE[n];
}

// D_abc of a radial function with derivatives g at separation d
__device__ double ew_component(int a, int b, int c, const double *d, const double *g)
{
    const int n = a + b + c;
    double s = 0.0;
    for (int i = 0; 2 * i <= a; i++)
        for (int j = 0; 2 * j <= b; j++)
            for (int k = 0; 2 * k <= c; k++) {
                double t = (double)pairk(a, i) * pairk(b, j) * pairk(c, k) * g[n - i - j - k];
                for (int u = 0; u < a - 2 * i; u++) t *= d[0];
                for (int u = 0; u < b - 2 * j; u++) t *= d[1];
                for (int u = 0; u < c - 2 * k; u++) t *= d[2];
                s += t;
            }
    return s;
}

// one block per cell, one thread per component of orders 0..nt
__global__ void __launch_bounds__(EW_THREADS) k_ewald_grid(double L, int nt, double *t64, float *t32)
{
    __shared__ double sk[EW_THREADS][5];   // kx, ky, kz, w cos(k.x0), w sin(k.x0)
    const int cell = blockIdx.x, tid = threadIdx.x;
    const int nm = g4_nmono(nt);
    const double pi = 3.14159265358979323846, V = L * L * L, al = EW_ALPHA_L / L;
    const double h = L / (2.0 * EW_G);
    const int ci = cell / (EW_G * EW_G), cj = (cell / EW_G) % EW_G, ck = cell % EW_G;
    const double x0[3] = {(ci + 0.5) * h, (cj + 0.5) * h, (ck + 0.5) * h};
    // this thread's component (a, b, c) of order n
    int a = 0, b = 0, c = 0, n = 0;
    const bool active = tid < nm;
    if (active) {
        while (g4_nmono(n) <= tid) n++;
        const int r = tid - (n > 0 ? g4_nmono(n - 1) : 0);
        int bc = 0;
        while ((bc + 1) * (bc + 2) / 2 <= r) bc++;
        c = r - bc * (bc + 1) / 2;
        b = bc - c;
        a = n - bc;
    }
    double D = (active && n == 0) ? pi / (al * al * V) : 0.0;
    // real-space images
    if (active) {
        double g[EW_NMAX + 1];
        for (int ia = -1; ia <= 1; ia++)
            for (int ib = -1; ib <= 1; ib++)
                for (int ic = -1; ic <= 1; ic++) {
                    const double d[3] = {x0[0] + ia * L, x0[1] + ib * L, x0[2] + ic * L};
                    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    if (ia == 0 && ib == 0 && ic == 0) {
                        ew_gn_erf(r, al, g);
                        D += ew_component(a, b, c, d, g);
                    } else {
                        gn_kernel<EW_NMAX, double, true>(r * r, al, g);
                        D -= ew_component(a, b, c, d, g);
                    }
                }
    }
    // Fourier terms, EW_THREADS wave-vector slots at a time (half of the integer triplets)
    const int ntrip = EW_KSIDE * EW_KSIDE * EW_KSIDE;
    for (int base = 0; base < ntrip; base += EW_THREADS) {
        const int t = base + tid;
        double kx = 0.0, ky = 0.0, kz = 0.0, wc = 0.0, ws = 0.0;
        if (t < ntrip) {
            const int mx = t / (EW_KSIDE * EW_KSIDE) - EW_NK, my = (t / EW_KSIDE) % EW_KSIDE - EW_NK,
                      mz = t % EW_KSIDE - EW_NK;
            if (mx > 0 || (mx == 0 && (my > 0 || (my == 0 && mz > 0)))) {
                kx = 2 * pi * mx / L;
                ky = 2 * pi * my / L;
                kz = 2 * pi * mz / L;
                const double k2 = kx * kx + ky * ky + kz * kz;
                const double w = 2.0 * 4.0 * pi / V * exp(-k2 / (4.0 * al * al)) / k2;
                double sn, cs;
                sincos(kx * x0[0] + ky * x0[1] + kz * x0[2], &sn, &cs);
                wc = w * cs;
                ws = w * sn;
            }
        }
        __syncthreads();
        sk[tid][0] = kx;
        sk[tid][1] = ky;
        sk[tid][2] = kz;
        sk[tid][3] = wc;
        sk[tid][4] = ws;
        __syncthreads();
        if (active) {
            for (int q = 0; q < EW_THREADS; q++) {
                const double wcq = sk[q][3], wsq = sk[q][4];
                if (wcq == 0.0 && wsq == 0.0) continue;
                // w cos(k.x0 + n pi / 2) = w cos, -w sin, -w cos, w sin
                const double cm = (n & 1) ? ((n & 2) ? wsq : -wsq) : ((n & 2) ? -wcq : wcq);
                double p = cm;
                for (int u = 0; u < a; u++) p *= sk[q][0];
                for (int u = 0; u < b; u++) p *= sk[q][1];
                for (int u = 0; u < c; u++) p *= sk[q][2];
                D -= p;
            }
        }
    }
    if (active) {
        t64[(size_t)cell * nm + tid] = D;
        t32[(size_t)cell * nm + tid] = (float)D;
    }
}

template <int N>
__global__ void k_ewald_eval(G4EwaldView E, const double *__restrict__ x, int64_t n,
                             double *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double D[g4_nmono(N)];
        ewald_dpsi<N, double>(E, x[3 * i], x[3 * i + 1], x[3 * i + 2], D);
        for (int c = 0; c < g4_nmono(N); c++) out[(size_t)i * g4_nmono(N) + c] = D[c];
    }
}

}  // namespace

// The grid for box size L with orders up to nt (<= 9), kept in the handle; rebuilt when L
// changes or a higher order is asked for.  Allocates on first use (outside graph capture).
g4_status g4_ewald_ensure(g4_tree t, double L, int nt, cudaStream_t st, G4EwaldView *view)
{
    if (nt < 3 || nt > EW_NMAX) return g4_fail(G4_ERR_INVALID_ARG, "Ewald grid: order %d", nt);
    if (!(L > 0)) return g4_fail(G4_ERR_INVALID_ARG, "Ewald grid: box size");
    int launches = 0;
    if (!t->ew64 || t->ew_L != L || t->ew_nt < nt) {
        const int ntb = EW_NMAX;   // always the full set: one grid serves every order
        const size_t cells = (size_t)EW_G * EW_G * EW_G, nm = (size_t)g4_nmono(ntb);
        if (!t->ew64) {
            if (cudaMalloc(&t->ew64, sizeof(double) * cells * nm) != cudaSuccess ||
                cudaMalloc(&t->ew32, sizeof(float) * cells * nm) != cudaSuccess) {
                cudaGetLastError();
                if (t->ew64) cudaFree(t->ew64);
                t->ew64 = nullptr;
                t->ew32 = nullptr;
                return g4_fail(G4_ERR_OOM, "Ewald grid (%zu cells)", cells);
            }
        }
        k_ewald_grid<<<(unsigned)cells, EW_THREADS, 0, st>>>(L, ntb, t->ew64, t->ew32);
        t->ew_L = L;
        t->ew_nt = ntb;
        launches = 1;
    }
    view->t32 = t->ew32;
    view->t64 = t->ew64;
    view->nt = t->ew_nt;
    view->G = EW_G;
    view->h = L / (2.0 * EW_G);
    return g4_launch_check("Ewald grid", launches);
}

extern "C" g4_status g4_ewald_eval(g4_tree t, const double *x, int64_t n, int nmax, double box,
                                   double *out, void *stream)
{
    if (!t || (n > 0 && (!x || !out)) || n < 0 || nmax < 0 || nmax > 6)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_ewald_eval: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    G4EwaldView E;
    g4_status s = g4_ewald_ensure(t, box, nmax + 3, st, &E);
    if (s != G4_OK || n == 0) return s;
    const int nb = g4_blocks_for(n, 128);
    switch (nmax) {
    case 0: k_ewald_eval<0><<<nb, 128, 0, st>>>(E, x, n, out); break;
    case 1: k_ewald_eval<1><<<nb, 128, 0, st>>>(E, x, n, out); break;
    case 2: k_ewald_eval<2><<<nb, 128, 0, st>>>(E, x, n, out); break;
    case 3: k_ewald_eval<3><<<nb, 128, 0, st>>>(E, x, n, out); break;
    case 4: k_ewald_eval<4><<<nb, 128, 0, st>>>(E, x, n, out); break;
    case 5: k_ewald_eval<5><<<nb, 128, 0, st>>>(E, x, n, out); break;
    default: k_ewald_eval<6><<<nb, 128, 0, st>>>(E, x, n, out); break;
    }
    return g4_launch_check("Ewald evaluation", 1);
}
