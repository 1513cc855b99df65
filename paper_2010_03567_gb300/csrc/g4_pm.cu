// g4_pm.cu -- long-range particle-mesh force of the TreePM split (Sec. 2.3), hand-written:
//   1. clouds-in-cell (CIC) assignment of the particle masses to a periodic N^3 mesh (mesh
//      points at i * Delta, Delta = L / N; atomics into the real parts of a complex mesh);
//   2. forward 3-D FFT: three passes of batched 1-D radix-2 transforms in shared memory (a tile
//      of lines per block; the x pass over contiguous lines, the y and z passes over columns of
//      consecutive x, so every global access is coalesced along x);
//   3. multiplication by the Green's function -4 pi G exp(-k^2 r_s^2) / k^2, divided by the
//      CIC assignment and interpolation transforms prod_i sinc^4(k_i Delta / 2) and by N^3
//      (the inverse transform is unnormalised); zero at k = 0.  Everything but 1/k^2 factorises
//      over the axes: per-axis tables in FP64, one FP32 product and division per mesh cell;
//   4. inverse 3-D FFT: the long-range potential on the mesh (real parts);
//   5-6. at each sink, fourth-order differences of the potential at the 8 CIC mesh points,
//      weighted with the CIC weights: a = -grad phi, and phi itself.
// Positions are the uint32 integer coordinates of the tree code (unit L / 2^32) and N is a
// power of two, so the mesh cell and the CIC fraction of a particle are exact bit fields.
#include "g4_internal.cuh"

namespace {

constexpr int PM_THREADS = 256;
constexpr int PM_TILE = 4096;   // complex values per block tile (32 KB of shared memory)
// shared-memory slot of tile element i: one float2 of padding after every 16, so that the
// bit-reversed scatter of a warp (indices that differ by multiples of n/32) and the strided
// butterflies of the first stages spread over the banks
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
constexpr int PM_SMEM = PM_TILE + PM_TILE / 16;

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// twiddles w_j = exp(-2 pi i j / N), j < N/2, evaluated in FP64 and rounded
__global__ void k_pm_twiddles(float2 *__restrict__ tw, int n)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n / 2; j += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * j / n, &s, &c);
        tw[j] = make_float2((float)c, (float)s);
    }
}

__device__ __forceinline__ int bitrev(int j, int logn) { return (int)(__brev((unsigned)j) >> (32 - logn)); }

// In-place radix-2 decimation-in-time transforms of `lines` lines of length n held in shared
// memory in bit-reversed order: element j of line l at s[pad(l * ls + j * js)]; stage st joins
// blocks of 2^st with twiddles W_{2^(st+1)}^k = tw[k n / 2^(st+1)].  Contiguous lines (ls = n,
// js = 1) give consecutive threads consecutive butterflies of one line; interleaved columns
// (ls = 1, js = lines) give them the same butterfly of consecutive lines, so a warp's accesses
// stay on consecutive slots either way.  inverse: conjugate twiddles.
__device__ void fft_lines_smem(float2 *s, int lines, int n, int logn, int ls, int js,
                               const float2 *__restrict__ tw, bool inverse)
{
    const bool lfast = ls == 1;
    int st = 0;
    // pairs of radix-2 stages (st, st + 1) fused: each thread loads 4 elements, applies both
    // stages in registers (the same operations as two separate stages) and stores them back
    for (; st + 1 < logn; st += 2) {
        const int h = 1 << st;
        const int nq = n >> 2, nb = lines * nq;
        const int t1 = n >> (st + 1), t2 = n >> (st + 2);   // twiddle strides of both stages
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            int line, bb;
            if (lfast) {
                line = b % lines;
                bb = b / lines;
            } else {
                line = b / nq;
                bb = b - line * nq;
            }
            const int g = bb >> st, k = bb & (h - 1);
            const int j0 = g * 4 * h + k, base = line * ls;
            const int a0 = pad(base + j0 * js), a1 = pad(base + (j0 + h) * js);
            const int a2 = pad(base + (j0 + 2 * h) * js), a3 = pad(base + (j0 + 3 * h) * js);
            float2 w1 = __ldg(tw + k * t1), w2 = __ldg(tw + k * t2), w3 = __ldg(tw + (k + h) * t2);
            if (inverse) {
                w1.y = -w1.y;
                w2.y = -w2.y;
                w3.y = -w3.y;
            }
            float2 x0 = s[a0], x1 = s[a1], x2 = s[a2], x3 = s[a3];
            // stage st: (x0, x1) and (x2, x3) with W_{2h}^k
            float2 t = cmul(w1, x1);
            float2 y0 = make_float2(x0.x + t.x, x0.y + t.y), y1 = make_float2(x0.x - t.x, x0.y - t.y);
            t = cmul(w1, x3);
            float2 y2 = make_float2(x2.x + t.x, x2.y + t.y), y3 = make_float2(x2.x - t.x, x2.y - t.y);
            // stage st + 1: (y0, y2) with W_{4h}^k, (y1, y3) with W_{4h}^(k + h)
            t = cmul(w2, y2);
            s[a0] = make_float2(y0.x + t.x, y0.y + t.y);
            s[a2] = make_float2(y0.x - t.x, y0.y - t.y);
            t = cmul(w3, y3);
            s[a1] = make_float2(y1.x + t.x, y1.y + t.y);
            s[a3] = make_float2(y1.x - t.x, y1.y - t.y);
        }
        __syncthreads();
    }
    // a last single radix-2 stage when log2 n is odd
    for (; st < logn; st++) {
        const int half = 1 << st;
        const int tstep = n >> (st + 1);
        const int nh = n >> 1, nb = lines * nh;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            int line, bb;
            if (lfast) {
                line = b % lines;
                bb = b / lines;
            } else {
                line = b / nh;
                bb = b - line * nh;
            }
            const int g = bb >> st, k = bb & (half - 1);
            const int j0 = g * 2 * half + k;
            const int i0 = pad(line * ls + j0 * js), i1 = pad(line * ls + (j0 + half) * js);
            float2 w = __ldg(tw + k * tstep);
            if (inverse) w.y = -w.y;
            const float2 a = s[i0], t = cmul(w, s[i1]);
            s[i0] = make_float2(a.x + t.x, a.y + t.y);
            s[i1] = make_float2(a.x - t.x, a.y - t.y);
        }
        __syncthreads();
    }
}

// x pass: tiles of `lines` consecutive contiguous lines (lines = PM_TILE / n, all n^2 lines)
__global__ void __launch_bounds__(PM_THREADS) k_pm_fft_x(float2 *__restrict__ g, int n, int logn,
                                                         const float2 *__restrict__ tw, int inverse)
{
    __shared__ float2 s[PM_SMEM];
    const int lines = PM_TILE / n;
    const long long nlines = (long long)n * n;
    for (long long l0 = (long long)blockIdx.x * lines; l0 < nlines; l0 += (long long)gridDim.x * lines) {
        float2 *base = g + l0 * n;
        for (int e = threadIdx.x; e < lines * n; e += blockDim.x) {
            const int line = e / n, j = e - line * n;
            s[pad(line * n + bitrev(j, logn))] = base[e];
        }
        __syncthreads();
        fft_lines_smem(s, lines, n, logn, n, 1, tw, inverse != 0);
        for (int e = threadIdx.x; e < lines * n; e += blockDim.x) base[e] = s[pad(e)];
        __syncthreads();
    }
}

// y / z pass: tiles of `cols` consecutive x columns (cols = min(n, PM_TILE / n)), transform
// along the axis with element stride `stride` (n for y, n^2 for z); `outer` indexes the
// remaining axis with stride `ostride`.  The tile is kept column-interleaved in shared memory
// (element j of column c at j * cols + c), as it is in the mesh.
__global__ void __launch_bounds__(PM_THREADS) k_pm_fft_col(float2 *__restrict__ g, int n, int logn,
                                                           long long stride, long long ostride,
                                                           const float2 *__restrict__ tw, int inverse)
{
    __shared__ float2 s[PM_SMEM];
    const int cols = min(n, PM_TILE / n);
    const int ntx = n / cols;                       // column tiles per row of x
    const long long ntiles = (long long)ntx * n;    // times the other axis
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int xt = (int)(t % ntx);
        const long long o = t / ntx;
        float2 *base = g + o * ostride + (long long)xt * cols;
        for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {
            const int j = e / cols, c = e - j * cols;   // consecutive threads: consecutive x
            s[pad(bitrev(j, logn) * cols + c)] = base[(long long)j * stride + c];
        }
        __syncthreads();
        fft_lines_smem(s, cols, n, logn, 1, cols, tw, inverse != 0);
        for (int e = threadIdx.x; e < cols * n; e += blockDim.x) {
            const int j = e / cols, c = e - j * cols;
            base[(long long)j * stride + c] = s[pad(e)];
        }
        __syncthreads();
    }
}

// CIC: mesh cell and fraction of an integer coordinate (n = 2^logn)
__device__ __forceinline__ void cic_axis(uint32_t x, int logn, int &i, float &d)
{
    const int sh = 32 - logn;
    i = (int)(x >> sh);
    d = (float)(x & ((1u << sh) - 1u)) * __int_as_float((127 - sh) << 23);   // * 2^-sh
}

__global__ void k_pm_assign(const uint32_t *__restrict__ pos, const float *__restrict__ mass, int np,
                            float2 *__restrict__ g, int n, int logn, float inv_cell_vol)
{
    const int mask = n - 1;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        int ix, iy, iz;
        float dx, dy, dz;
        cic_axis(pos[p], logn, ix, dx);
        cic_axis(pos[np + p], logn, iy, dy);
        cic_axis(pos[2 * np + p], logn, iz, dz);
        const float m = mass[p] * inv_cell_vol;
#pragma unroll
        for (int oz = 0; oz < 2; oz++)
#pragma unroll
            for (int oy = 0; oy < 2; oy++)
#pragma unroll
                for (int ox = 0; ox < 2; ox++) {
                    const float w = (ox ? dx : 1.f - dx) * (oy ? dy : 1.f - dy) * (oz ? dz : 1.f - dz);
                    const long long c = (((long long)((iz + oz) & mask) * n + ((iy + oy) & mask)) * n) +
                                        ((ix + ox) & mask);
                    atomicAdd(&g[c].x, m * w);
                }
    }
}

// Per-axis factors of the Green's function (FP64, rounded to FP32), for wave number index i:
// k_i = 2 pi n_i / L with n_i = i for i < N/2, i - N otherwise;
//   kk[i] = k_i^2,  ew[i] = exp(-k_i^2 r_s^2) / sinc^4(k_i Delta / 2)
// (exp(-k^2 r_s^2) factorises over the axes, and so does the CIC deconvolution).
__global__ void k_pm_green_tables(float *__restrict__ kk, float *__restrict__ ew, int n,
                                  double two_pi_over_L, double rs2, double half_delta)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ni = i < n / 2 ? i : i - n;
        const double k = ni * two_pi_over_L, x = k * half_delta;
        const double sc = x == 0.0 ? 1.0 : sin(x) / x;
        kk[i] = (float)(k * k);
        ew[i] = (float)(exp(-k * k * rs2) / (sc * sc * sc * sc));
    }
}

// multiplication by the Green's function -4 pi G exp(-k^2 r_s^2) / k^2 with the CIC
// deconvolution and 1/N^3: scale * ew[ix] ew[iy] ew[iz] / (kk[ix] + kk[iy] + kk[iz])
__global__ void k_pm_green(float2 *__restrict__ g, int n, int logn, const float *__restrict__ kk,
                           const float *__restrict__ ew, float scale)
{
    const long long total = (long long)n * n * n;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
         c += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(c & (n - 1)), iy = (int)((c >> logn) & (n - 1)), iz = (int)(c >> (2 * logn));
        const float k2 = __ldg(kk + ix) + __ldg(kk + iy) + __ldg(kk + iz);
        const float f = (c == 0) ? 0.f : scale * __ldg(ew + ix) * __ldg(ew + iy) * __ldg(ew + iz) / k2;
        const float2 v = g[c];
        g[c] = make_float2(v.x * f, v.y * f);
    }
}

__device__ __forceinline__ float phi_at(const float2 *__restrict__ g, int n, int x, int y, int z)
{
    const int m = n - 1;
    return __ldg(&g[(((long long)(z & m) * n + (y & m)) * n) + (x & m)].x);
}

// fourth-order differences of the potential at the 8 CIC points of each sink, interpolated
__global__ void k_pm_interp(const float2 *__restrict__ g, int n, int logn, const uint32_t *__restrict__ pos,
                            int ns, float inv12delta, float *__restrict__ acc, float *__restrict__ pot,
                            int accumulate)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < ns; p += gridDim.x * blockDim.x) {
        int ix, iy, iz;
        float dx, dy, dz;
        cic_axis(pos[p], logn, ix, dx);
        cic_axis(pos[ns + p], logn, iy, dy);
        cic_axis(pos[2 * ns + p], logn, iz, dz);
        float ax = 0.f, ay = 0.f, az = 0.f, ph = 0.f;
#pragma unroll
        for (int oz = 0; oz < 2; oz++)
#pragma unroll
            for (int oy = 0; oy < 2; oy++)
#pragma unroll
                for (int ox = 0; ox < 2; ox++) {
                    const float w = (ox ? dx : 1.f - dx) * (oy ? dy : 1.f - dy) * (oz ? dz : 1.f - dz);
                    const int x = ix + ox, y = iy + oy, z = iz + oz;
                    const float gx = 8.f * (phi_at(g, n, x + 1, y, z) - phi_at(g, n, x - 1, y, z)) -
                                     (phi_at(g, n, x + 2, y, z) - phi_at(g, n, x - 2, y, z));
                    const float gy = 8.f * (phi_at(g, n, x, y + 1, z) - phi_at(g, n, x, y - 1, z)) -
                                     (phi_at(g, n, x, y + 2, z) - phi_at(g, n, x, y - 2, z));
                    const float gz = 8.f * (phi_at(g, n, x, y, z + 1) - phi_at(g, n, x, y, z - 1)) -
                                     (phi_at(g, n, x, y, z + 2) - phi_at(g, n, x, y, z - 2));
                    ax -= w * gx;
                    ay -= w * gy;
                    az -= w * gz;
                    ph += w * phi_at(g, n, x, y, z);
                }
        ax *= inv12delta;
        ay *= inv12delta;
        az *= inv12delta;
        if (accumulate) {
            acc[p] += ax;
            acc[ns + p] += ay;
            acc[2 * ns + p] += az;
            if (pot) pot[p] += ph;
        } else {
            acc[p] = ax;
            acc[ns + p] = ay;
            acc[2 * ns + p] = az;
            if (pot) pot[p] = ph;
        }
    }
}

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

bool pm_grid_ok(int32_t n) { return n >= 16 && n <= 1024 && (n & (n - 1)) == 0; }

int ilog2(int n)
{
    int l = 0;
    while ((1 << l) < n) l++;
    return l;
}

}  // namespace

g4_status g4_check_params(const g4_params *P, const char *who);

extern "C" g4_status g4_pm_workspace(int32_t n_grid, size_t *bytes)
{
    if (!bytes || !pm_grid_ok(n_grid))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_pm_workspace: n_grid=%d (a power of two in [16, 1024])", n_grid);
    const size_t n = (size_t)n_grid;
    *bytes = al256(sizeof(float2) * n * n * n) + al256(sizeof(float2) * (n / 2)) +
             2 * al256(sizeof(float) * n);
    return G4_OK;
}

extern "C" g4_status g4_pm_long_range(const uint32_t *pos, const float *mass, int64_t n,
                                      const uint32_t *pos_sinks, int64_t n_sinks,
                                      const g4_params *P, int32_t n_grid, float *acc, float *pot,
                                      int accumulate, void *workspace, size_t workspace_bytes,
                                      void *stream)
{
    g4_status s = g4_check_params(P, "g4_pm_long_range");
    if (s != G4_OK) return s;
    if (!P->periodic || !(P->r_s > 0.0))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_pm_long_range: needs a periodic box and r_s > 0");
    if (n < 0 || n >= ((int64_t)1 << 31) || n_sinks < 0 || n_sinks >= ((int64_t)1 << 31))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_pm_long_range: n=%lld n_sinks=%lld", (long long)n,
                       (long long)n_sinks);
    size_t need = 0;
    s = g4_pm_workspace(n_grid, &need);
    if (s != G4_OK) return s;
    if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255) != 0)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_pm_long_range: workspace (%zu bytes, need %zu, 256-byte aligned)",
                       workspace_bytes, need);
    if ((n > 0 && (!pos || !mass)) || (n_sinks > 0 && (!pos_sinks || !acc)))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_pm_long_range: NULL pointer");
    if (n_sinks == 0) return G4_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int N = n_grid, logn = ilog2(N);
    const size_t cells = (size_t)N * N * N;
    float2 *grid = (float2 *)workspace;
    float2 *tw = (float2 *)((char *)workspace + al256(sizeof(float2) * cells));
    float *kk = (float *)((char *)tw + al256(sizeof(float2) * (N / 2)));
    float *ew = (float *)((char *)kk + al256(sizeof(float) * N));
    const double L = P->box_size, delta = L / N;
    int launches = 0;
    if (cudaMemsetAsync(grid, 0, sizeof(float2) * cells, st) != cudaSuccess)
        return g4_cuda_check(cudaGetLastError(), "g4_pm_long_range: clear mesh");
    const double two_pi = 6.283185307179586;
    k_pm_twiddles<<<(N / 2 + 255) / 256, 256, 0, st>>>(tw, N);
    k_pm_green_tables<<<(N + 255) / 256, 256, 0, st>>>(kk, ew, N, two_pi / L, P->r_s * P->r_s, 0.5 * delta);
    launches += 2;
    if (n > 0) {
        k_pm_assign<<<g4_blocks_for(n, 256), 256, 0, st>>>(pos, mass, (int)n, grid, N, logn,
                                                            (float)(1.0 / (delta * delta * delta)));
        launches++;
    }
    const int gx = g4_num_sms() * 8;
    const long long n2 = (long long)N * N;
    for (int inv = 0; inv < 2; inv++) {
        k_pm_fft_x<<<gx, PM_THREADS, 0, st>>>(grid, N, logn, tw, inv);
        k_pm_fft_col<<<gx, PM_THREADS, 0, st>>>(grid, N, logn, N, n2, tw, inv);      // y
        k_pm_fft_col<<<gx, PM_THREADS, 0, st>>>(grid, N, logn, n2, N, tw, inv);      // z
        launches += 3;
        if (inv == 0) {
            k_pm_green<<<g4_blocks_for((int64_t)cells, 256), 256, 0, st>>>(
                grid, N, logn, kk, ew, (float)(-2.0 * two_pi * P->G / (double)cells));
            launches++;
        }
    }
    k_pm_interp<<<g4_blocks_for(n_sinks, 256), 256, 0, st>>>(grid, N, logn, pos_sinks, (int)n_sinks,
                                                             (float)(1.0 / (12.0 * delta)), acc, pot,
                                                             accumulate);
    launches++;
    return g4_launch_check("pm long range", launches);
}
