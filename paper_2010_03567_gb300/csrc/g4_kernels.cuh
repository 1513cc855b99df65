// g4_kernels.cuh -- interaction kernels shared by the walk, FMM and direct-sum kernels:
//   * pair kernel of the short-range potential (Eq. eqnpo4) with cubic-spline softening
//     (Eq. eqnsoft), g = g_soft - erf(r / 2 r_s) / r, returning g0 = g and g1 = g'/r;
//   * g_n = (r^-1 d/dr)^n g for the unsoftened multipole kernel (1/r or erfc(r/2r_s)/r),
//     from the upward recursion B_n = ((2n-1) B_{n-1} + (2a^2)^(n-1) t) / r^2, g_n = (-1)^n B_n
//     (a = 1/(2 r_s), t = (2a/sqrt(pi)) exp(-a^2 r^2); t = 0 for the Newtonian kernel);
//   * Cartesian derivative tensors D_{abc} = d^a_x d^b_y d^c_z g(|r|) for a symmetric
//     multi-index, D_{abc} = sum_{i,j,k} K(a,i) K(b,j) K(c,k) g_{n-i-j-k} x^(a-2i) y^(b-2j)
//     z^(c-2k) with K(a,i) = a! / (2^i i! (a-2i)!) -- the count of ways to pair 2i of the a
//     equal index slots by Kronecker deltas (Eqs. eqngderiv0-eqngderiv).
#pragma once
#include "g4_erfcx.cuh"
#include "g4_internal.cuh"

namespace g4k {

// one 64-byte node record through the read-only path (4 x 16-byte loads)
__device__ __forceinline__ G4Node load_node(const G4Node *p)
{
    const int4 *v = reinterpret_cast<const int4 *>(p);
    const int4 a = __ldg(v), b = __ldg(v + 1), c = __ldg(v + 2), d = __ldg(v + 3);
    G4Node nd;
    nd.cx = (uint32_t)a.x;
    nd.cy = (uint32_t)a.y;
    nd.cz = (uint32_t)a.z;
    nd.meta = (uint32_t)a.w;
    nd.sx = __int_as_float(b.x);
    nd.sy = __int_as_float(b.y);
    nd.sz = __int_as_float(b.z);
    nd.mass = __int_as_float(b.w);
    nd.first = c.x;
    nd.count = c.y;
    nd.next = c.z;
    nd.parent = c.w;
    nd.amin = __int_as_float(d.x);
    nd.hmax = __int_as_float(d.y);
    nd.hmin = __int_as_float(d.z);
    nd.nchild = d.w;
    return nd;
}

__host__ __device__ constexpr int fact(int n) { return n <= 1 ? 1 : n * fact(n - 1); }
__host__ __device__ constexpr int pairk(int a, int i)
{
    // a! / (2^i i! (a-2i)!)
    return fact(a) / ((1 << i) * fact(i) * fact(a - 2 * i));
}

template <typename T> struct Math;
template <> struct Math<float> {
    static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float sqrt(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float erfc(float x) { return erfcf(x); }
    static __device__ __forceinline__ float erf(float x) { return erff(x); }
    static __device__ __forceinline__ float exp(float x) { return expf(x); }
};
template <> struct Math<double> {
    static __device__ __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double erfc(double x) { return ::erfc(x); }
    static __device__ __forceinline__ double erf(double x) { return ::erf(x); }
    static __device__ __forceinline__ double exp(double x) { return ::exp(x); }
};

// Pair kernel.  r2: squared separation, h: 2.8 eps_ij, as = 1/(2 r_s) (TREEPM only).
// Returns g0 = g(r), g1 = g'(r)/r.  At r = 0 (coincident particles) g1 is irrelevant.
template <typename T, bool TREEPM>
__device__ __forceinline__ void pair_kernel(T r2, T h, T as, T &g0, T &g1)
{
    const T two_over_sqrtpi = T(1.1283791670955126);
    if (r2 >= h * h) {
        const T rinv = Math<T>::rsqrt(r2);
        if (TREEPM) {
            const T r = r2 * rinv, x = r * as;
            const T e = Math<T>::erfc(x);
            const T t = two_over_sqrtpi * as * Math<T>::exp(-x * x);
            g0 = e * rinv;
            g1 = -(g0 + t) * rinv * rinv;
        } else {
            g0 = rinv;
            g1 = -rinv * rinv * rinv;
        }
        return;
    }
    const T r = Math<T>::sqrt(r2);
    const T hinv = T(1) / h;
    const T u = r * hinv, u2 = u * u;
    T W, dWu;   // W_2(u) and W_2'(u)/u of the cubic-spline potential
    if (u < T(0.5)) {
        W = u2 * (T(16.0 / 3.0) + u2 * (T(-48.0 / 5.0) + u * T(32.0 / 5.0))) - T(14.0 / 5.0);
        dWu = T(32.0 / 3.0) + u2 * (T(-192.0 / 5.0) + u * T(32.0));
    } else {
        const T uinv = T(1) / u;
        W = T(1.0 / 15.0) * uinv +
            u2 * (T(32.0 / 3.0) + u * (T(-16.0) + u * (T(48.0 / 5.0) + u * T(-32.0 / 15.0)))) -
            T(16.0 / 5.0);
        dWu = T(-1.0 / 15.0) * uinv * uinv * uinv + T(64.0 / 3.0) +
              u * (T(-48.0) + u * (T(192.0 / 5.0) + u * T(-32.0 / 3.0)));
    }
    g0 = -W * hinv;
    g1 = -dWu * hinv * hinv * hinv;
    if (TREEPM) {
        if (r2 > T(0)) {
            const T rinv = T(1) / r, x = r * as;
            const T ef = Math<T>::erf(x);
            const T t = two_over_sqrtpi * as * Math<T>::exp(-x * x);
            g0 -= ef * rinv;
            g1 += (ef * rinv - t) * rinv * rinv;
        } else {
            g0 -= two_over_sqrtpi * as;
        }
    }
}

// FP32 TreePM pair kernel with lengths in units of the integer grid (so separations need no
// scaling).  For r >= h and x = as r <= G4_ERFCX_XMAX:
//   exp(-x^2) = 2^(k2 r^2), k2 = -as^2 log2(e)          (ex2.approx),
//   erfc(x)   = exp(-x^2) erfcx(x)                      (fitted polynomial, g4_erfcx.cuh),
//   g0 = erfc(x) / r,  g1 = -(g0 + ct exp(-x^2)) / r^2,  ct = 2 as / sqrt(pi).
// Softened pairs and pairs beyond the fit take pair_kernel<float, true>.  The kernel is
// homogeneous in the length unit (g0 ~ 1/length, g1 ~ 1/length^3), so the caller converts
// the sums back with 1/scale and 1/scale^2.
struct PairF {
    float as, k2, ct, fit2;
};

__host__ __device__ inline PairF make_pairf(double as, double inv_as)
{
    PairF c;
    c.as = (float)as;
    c.k2 = (float)(-as * as * 1.4426950408889634);
    c.ct = (float)(1.1283791670955126 * as);
    c.fit2 = (float)((double)G4_ERFCX_XMAX * G4_ERFCX_XMAX * inv_as * inv_as);
    return c;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void pair_treepm_fast(float r2, float h, const PairF &c, float &g0,
                                                 float &g1)
{
    if (r2 < h * h || r2 > c.fit2) {
        pair_kernel<float, true>(r2, h, c.as, g0, g1);
        return;
    }
    const float rinv = rsqrt_approx(r2), r = r2 * rinv;   // r2 > 0 here, never subnormal
    const float e = ex2_approx(r2 * c.k2);
    const float t = rcp_approx(fmaf(G4_ERFCX_K * c.as, r, 1.f));
    const float ec = e * g4_erfcx_poly(fmaf(t, G4_ERFCX_U1, G4_ERFCX_U0));
    g0 = ec * rinv;
    g1 = -fmaf(c.ct, e, g0) * rinv * rinv;
}

// g_0..g_N of the unsoftened multipole kernel at squared distance r2 (r2 > 0).
template <int N, typename T, bool TREEPM>
__device__ __forceinline__ void gn_kernel(T r2, T as, T *g)
{
    const T rinv = Math<T>::rsqrt(r2), rinv2 = rinv * rinv;
    T B = rinv, t = T(0), tw = T(0);
    if (TREEPM) {
        const T r = r2 * rinv, x = r * as;
        B = Math<T>::erfc(x) * rinv;
        t = T(1.1283791670955126) * as * Math<T>::exp(-x * x);
        tw = T(2) * as * as;
    }
    g[0] = B;
#pragma unroll
    for (int n = 1; n <= N; n++) {
        B = (T(2 * n - 1) * B + t) * rinv2;
        if (TREEPM) t *= tw;
        g[n] = (n & 1) ? -B : B;
    }
}

// g_0..g_N of the softened kernel for a softened multipole (Sec. 2.7), r < h: the spline part
// -W_2(u)/h (u = r/h) differentiated term by term -- (r^-1 d/dr) u^k = (k / h^2) u^(k-2) --
// plus, for TreePM, -erf(r/2r_s)/r = erfc/r - 1/r (the unsoftened erfc kernel's g_n minus the
// Newtonian ones).  W_2 = sum c_k u^k on u < 1/2 and on 1/2 <= u < 1 (k = -1, 0, 2, 3, 4, 5).
template <int N, typename T, bool TREEPM>
__device__ __noinline__ void gn_soft(T r2, T h, T as, T *g)
{
    const T r = Math<T>::sqrt(r2), u = r / h, uinv = T(1) / u, hinv = T(1) / h, h2inv = hinv * hinv;
    const bool inner = u < T(0.5);
    const int kk[6] = {-1, 0, 2, 3, 4, 5};
    const T ci[6] = {T(0), T(-14.0 / 5.0), T(16.0 / 3.0), T(0), T(-48.0 / 5.0), T(32.0 / 5.0)};
    const T co[6] = {T(1.0 / 15.0), T(-16.0 / 5.0), T(32.0 / 3.0), T(-16.0), T(48.0 / 5.0),
                     T(-32.0 / 15.0)};
    T hp = hinv;   // h^-(2n+1)
    for (int n = 0; n <= N; n++) {
        T sum = T(0);
        for (int t = 0; t < 6; t++) {
            const T c = inner ? ci[t] : co[t];
            T f = T(1);
            for (int m = 0; m < n; m++) f *= T(kk[t] - 2 * m);
            if (c == T(0) || f == T(0)) continue;
            const int e = kk[t] - 2 * n;
            T up = T(1);
            for (int q = 0; q < (e > 0 ? e : -e); q++) up *= (e > 0 ? u : uinv);
            sum += c * f * up;
        }
        g[n] = -sum * hp;
        hp *= h2inv;
    }
    if (TREEPM) {
        T ge[N + 1], gn[N + 1];
        gn_kernel<N, T, true>(r2, as, ge);
        gn_kernel<N, T, false>(r2, as, gn);
        for (int n = 0; n <= N; n++) g[n] += ge[n] - gn[n];
    }
}

// All D_{abc} with a+b+c <= N into D[g4_midx(a,b,c)].
template <int N, typename T>
__device__ __forceinline__ void dtensors(T x, T y, T z, const T *g, T *D)
{
    T px[N + 1], py[N + 1], pz[N + 1];
    px[0] = py[0] = pz[0] = T(1);
#pragma unroll
    for (int k = 1; k <= N; k++) {
        px[k] = px[k - 1] * x;
        py[k] = py[k - 1] * y;
        pz[k] = pz[k - 1] * z;
    }
#pragma unroll
    for (int n = 0; n <= N; n++)
#pragma unroll
        for (int bc = 0; bc <= n; bc++)
#pragma unroll
            for (int c = 0; c <= bc; c++) {
                const int a = n - bc, b = bc - c;
                T s = T(0);
#pragma unroll
                for (int i = 0; 2 * i <= a; i++)
#pragma unroll
                    for (int j = 0; 2 * j <= b; j++)
#pragma unroll
                        for (int k = 0; 2 * k <= c; k++)
                            s += T(pairk(a, i) * pairk(b, j) * pairk(c, k)) * g[n - i - j - k] *
                                 px[a - 2 * i] * py[b - 2 * j] * pz[c - 2 * k];
                D[g4_midx(a, b, c)] = s;
            }
}

template <int P, typename T>
__device__ __forceinline__ void pn_contract(const T *Qs, T M, const T *D, T &sx, T &sy, T &sz,
                                            T &sp);

// Particle-node term of the one-sided expansion with r = s - x (Eqs. eqonesidetreepotential,
// eqonesidetreeacc): sacc += sum_{n<P} Q_n . D_{n+1} / n!,  spot += sum_{n<=P} Q_n . D_n / n!
// (the caller multiplies both by -G).  Qs holds moments of orders 2..P at g4_midx - 4.
// hs > 0 with r^2 < hs^2: the multipole of the softened kernel with h = hs (Sec. 2.7).
template <int P, typename T, bool TREEPM>
__device__ __forceinline__ void pn_term(const T *Qs, T M, T x, T y, T z, T as, T &sx, T &sy,
                                        T &sz, T &sp, T hs = T(0))
{
    const T r2 = x * x + y * y + z * z;
    T g[P + 1];
    if (hs > T(0) && r2 < hs * hs) gn_soft<P, T, TREEPM>(r2, hs, as, g);
    else gn_kernel<P, T, TREEPM>(r2, as, g);
    T D[g4_nmono(P)];
    dtensors<P, T>(x, y, z, g, D);
    pn_contract<P, T>(Qs, M, D, sx, sy, sz, sp);
}

// The contraction of pn_term for given derivative tensors D (a + b + c <= P):
// sacc += sum_{n<P} Q_n . D_{n+1} / n!,  spot += sum_{n<=P} Q_n . D_n / n!.
template <int P, typename T>
__device__ __forceinline__ void pn_contract(const T *Qs, T M, const T *D, T &sx, T &sy, T &sz,
                                            T &sp)
{
    T ax = M * D[g4_midx(1, 0, 0)], ay = M * D[g4_midx(0, 1, 0)], az = M * D[g4_midx(0, 0, 1)];
    T ph = M * D[0];
#pragma unroll
    for (int n = 2; n <= P; n++)
#pragma unroll
        for (int bc = 0; bc <= n; bc++)
#pragma unroll
            for (int c = 0; c <= bc; c++) {
                const int a = n - bc, b = bc - c;
                const T w = Qs[g4_midx(a, b, c) - 4] * T(1.0 / double(fact(a) * fact(b) * fact(c)));
                ph += w * D[g4_midx(a, b, c)];
                if (n <= P - 1) {
                    ax += w * D[g4_midx(a + 1, b, c)];
                    ay += w * D[g4_midx(a, b + 1, c)];
                    az += w * D[g4_midx(a, b, c + 1)];
                }
            }
    sx += ax;
    sy += ay;
    sz += az;
    sp += ph;
}

}  // namespace g4k
