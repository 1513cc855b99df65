// g4_keys.cu -- integer coordinates (Sec. 2.10/2.11), Peano-Hilbert keys (Sec. 2.2.1),
// stable LSD radix sort of the 63-bit keys, and the PH-order gather/scatter of particles.
#include <cstdio>

#include "g4_internal.cuh"

namespace {

// -------------------------------------------------------------------------------------------
// a1: integer coordinates
// -------------------------------------------------------------------------------------------
__global__ void k_int_coords_periodic(const double *__restrict__ pos, int64_t n, double L,
                                      uint32_t *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            double t = floor(__dmul_rn(__ddiv_rn(pos[3 * i + k], L), 4294967296.0));
            out[k * n + i] = (uint32_t)((long long)t & 0xFFFFFFFFLL);
        }
    }
}

// Bounding box of an isolated set, accumulated in the caller's frame buffer (no scratch):
// doubles are mapped to unsigned integers that order like them (sign bit set: all bits
// inverted; otherwise the sign bit set), so atomicMin / atomicMax give exact minima / maxima.
__device__ __forceinline__ unsigned long long ord_of(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double of_ord(unsigned long long v)
{
    return __longlong_as_double((long long)((v >> 63) ? (v & 0x7fffffffffffffffull) : ~v));
}

// stage 0: frame[0..2] = ord(+inf) (minima), frame[3..5] = ord(-inf) (maxima)
__global__ void k_bbox_init(double *__restrict__ frame)
{
    unsigned long long *f = reinterpret_cast<unsigned long long *>(frame);
    if (threadIdx.x < 3) f[threadIdx.x] = ord_of(INFINITY);
    else if (threadIdx.x < 6) f[threadIdx.x] = ord_of(-INFINITY);
}

// stage 1: per-block minima / maxima of each axis, folded into the frame with atomics
__global__ void k_bbox_partial(const double *__restrict__ pos, int64_t n, double *__restrict__ frame)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            double x = pos[3 * i + k];
            lo[k] = fmin(lo[k], x);
            hi[k] = fmax(hi[k], x);
        }
    __shared__ double s[6][32];
#pragma unroll
    for (int k = 0; k < 3; k++)
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fmin(lo[k], __shfl_down_sync(0xffffffffu, lo[k], o));
            hi[k] = fmax(hi[k], __shfl_down_sync(0xffffffffu, hi[k], o));
        }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0)
        for (int k = 0; k < 3; k++) { s[k][w] = lo[k]; s[3 + k][w] = hi[k]; }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = s[threadIdx.x][0];
        for (int j = 1; j < nw; j++)
            v = threadIdx.x < 3 ? fmin(v, s[threadIdx.x][j]) : fmax(v, s[threadIdx.x][j]);
        unsigned long long *f = reinterpret_cast<unsigned long long *>(frame);
        if (threadIdx.x < 3) atomicMin(f + threadIdx.x, ord_of(v));
        else atomicMax(f + threadIdx.x, ord_of(v));
    }
}

// stage 2: frame = {c - S/2, S, c}; S = smallest power of two >= 2 * extent
__global__ void k_bbox_frame(double *__restrict__ frame)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned long long *f = reinterpret_cast<const unsigned long long *>(frame);
    double lo[3], hi[3];
    for (int k = 0; k < 3; k++) {
        lo[k] = of_ord(f[k]);
        hi[k] = of_ord(f[3 + k]);
    }
    double ext = 0.0, c[3];
    for (int k = 0; k < 3; k++) {
        c[k] = __dmul_rn(0.5, __dadd_rn(lo[k], hi[k]));
        double e = __dsub_rn(hi[k], lo[k]);
        if (e > ext) ext = e;
    }
    double S = 1.0;
    if (ext > 0.0) {
        int e;
        double fr = frexp(2.0 * ext, &e);
        S = (fr == 0.5) ? ldexp(1.0, e - 1) : ldexp(1.0, e);
    }
    for (int k = 0; k < 3; k++) frame[k] = __dsub_rn(c[k], 0.5 * S);
    frame[3] = S;
    frame[4] = c[0];
    frame[5] = c[1];
    frame[6] = c[2];
    frame[7] = 0.0;
}

// periodic frame {0, 0, 0, L} (written on the device: no host copy, no synchronisation)
__global__ void k_frame_periodic(double *__restrict__ frame, double L)
{
    if (threadIdx.x < 8) frame[threadIdx.x] = threadIdx.x == 3 ? L : 0.0;
}

__global__ void k_int_coords_isolated(const double *__restrict__ pos, int64_t n,
                                      const double *__restrict__ frame, uint32_t *__restrict__ out)
{
    double S = frame[3];
    double scale = 4294967296.0 / S;   // exact: S is a power of two
    double c[3] = {frame[4], frame[5], frame[6]};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            double t = floor(__dmul_rn(__dsub_rn(pos[3 * i + k], c[k]), scale)) + 2147483648.0;
            out[k * n + i] = (uint32_t)(long long)t;
        }
}

// -------------------------------------------------------------------------------------------
// a2: Peano-Hilbert key.  The curve is Skilling's (2004) construction: from the top bit
// down, a set bit of an axis inverts the lower bits of axis 0, a clear bit exchanges the
// lower bits of axis 0 and that axis; the transposed index is then Gray-decoded and its bits
// interleaved (axis 0 first, most significant level first).  Branch-free form.
// -------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t ph_key21(uint32_t x, uint32_t y, uint32_t z)
{
    uint32_t a0 = x >> 11, a1 = y >> 11, a2 = z >> 11;
#pragma unroll
    for (int b = 20; b >= 1; b--) {
        const uint32_t q = 1u << b, low = q - 1u;
        // axis 0 against itself: only the inversion can happen
        a0 ^= (a0 & q) ? low : 0u;
        // axis 1
        {
            uint32_t t = (a0 ^ a1) & low;
            bool set = a1 & q;
            a0 ^= set ? low : t;
            a1 ^= set ? 0u : t;
        }
        // axis 2
        {
            uint32_t t = (a0 ^ a2) & low;
            bool set = a2 & q;
            a0 ^= set ? low : t;
            a2 ^= set ? 0u : t;
        }
    }
    a1 ^= a0;
    a2 ^= a1;
    // flip = XOR of (q-1) over the set bits q >= 2 of a2: a prefix-XOR of a2's bits above
    uint32_t f = a2 & ~1u;
    f ^= f >> 1;
    f ^= f >> 2;
    f ^= f >> 4;
    f ^= f >> 8;
    f ^= f >> 16;
    // f now holds at bit j the parity of a2's bits >= j (bits >= 1 only); the mask of
    // (q - 1) contributions is parity of set bits strictly above j.
    uint32_t flip = (f >> 1) & 0x1FFFFFu;
    a0 ^= flip;
    a1 ^= flip;
    a2 ^= flip;
    // interleave 3 x 21 bits: key bit 3j+2 <- a0 bit j, 3j+1 <- a1 bit j, 3j <- a2 bit j
    auto spread = [](uint32_t v) -> uint64_t {
        uint64_t r = v & 0x1FFFFFu;
        r = (r | (r << 32)) & 0x1F00000000FFFFull;
        r = (r | (r << 16)) & 0x1F0000FF0000FFull;
        r = (r | (r << 8)) & 0x100F00F00F00F00Full;
        r = (r | (r << 4)) & 0x10C30C30C30C30C3ull;
        r = (r | (r << 2)) & 0x1249249249249249ull;
        return r;
    };
    return (spread(a0) << 2) | (spread(a1) << 1) | spread(a2);
}

__global__ void k_keys(const uint32_t *__restrict__ pos, int64_t n, uint64_t *__restrict__ keys)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = ph_key21(pos[i], pos[n + i], pos[2 * n + i]);
}

// -------------------------------------------------------------------------------------------
// a3: stable LSD radix sort, 8-bit digits, tiles of SORT_TILE keys (2048 by default).
//   hist:    per-tile digit counts, digit-major  cnt[d * ntiles + t]
//   rowscan: per-digit exclusive scan over tiles, digit totals
//   scatter: warp-ordered stable ranks (match_any), global position = digit base + tile
//            offset + warp offset + rank
// -------------------------------------------------------------------------------------------
#ifndef G4_SORT_ITEMS
#define G4_SORT_ITEMS 8         // keys per thread in a tile
#endif
#ifndef G4_SORT_MIN_BLOCKS
#define G4_SORT_MIN_BLOCKS 4    // resident scatter blocks per SM requested from the compiler
#endif
constexpr int SORT_THREADS = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_ITEMS = G4_SORT_ITEMS;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int SCAN_THREADS = 1024;

__global__ void __launch_bounds__(SORT_THREADS) k_sort_hist(const uint64_t *__restrict__ keys,
                                                             int n, int shift,
                                                             uint32_t *__restrict__ cnt, int ntiles)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * SORT_TILE;
#pragma unroll 4
    for (int k = threadIdx.x; k < SORT_TILE; k += SORT_THREADS) {
        int i = base + k;
        if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    cnt[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// exclusive block scan of one value per thread (blockDim = SCAN_THREADS); returns the total
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t &excl)
{
    __shared__ uint32_t ws[32];
    int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (l >= o) x += y;
    }
    if (l == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = (l < (int)(blockDim.x >> 5)) ? ws[l] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (l >= o) s += y;
        }
        ws[l] = s;
    }
    __syncthreads();
    uint32_t before = (w > 0) ? ws[w - 1] : 0u;
    uint32_t total = ws[(blockDim.x >> 5) - 1];
    excl = before + x - v;
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_sort_rowscan(uint32_t *__restrict__ cnt,
                                                                int ntiles,
                                                                uint32_t *__restrict__ totals)
{
    uint32_t *row = cnt + (size_t)blockIdx.x * ntiles;
    int per = (ntiles + SCAN_THREADS - 1) / SCAN_THREADS;
    int b = threadIdx.x * per, e = min(b + per, ntiles);
    uint32_t s = 0;
    for (int i = b; i < e; i++) s += row[i];
    uint32_t ex;
    uint32_t tot = block_excl_scan(s, ex);
    for (int i = b; i < e; i++) {
        uint32_t v = row[i];
        row[i] = ex;
        ex += v;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

// Scatter of one tile: stable ranks per warp (match_any), then the tile is reordered by digit
// in shared memory, so that consecutive threads write consecutive addresses of each digit's
// output run (coalesced stores).  Dynamic shared memory: keys, values of the tile.
constexpr size_t SCATTER_SMEM = (size_t)SORT_TILE * (sizeof(uint64_t) + sizeof(int32_t));

__global__ void __launch_bounds__(SORT_THREADS, G4_SORT_MIN_BLOCKS) k_sort_scatter(
    const uint64_t *__restrict__ kin, const int32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    int32_t *__restrict__ vout, int n, int shift, const uint32_t *__restrict__ cnt,
    const uint32_t *__restrict__ totals, int ntiles)
{
    extern __shared__ __align__(16) unsigned char sort_smem[];
    uint64_t *sk = reinterpret_cast<uint64_t *>(sort_smem);
    int32_t *sv = reinterpret_cast<int32_t *>(sort_smem + (size_t)SORT_TILE * sizeof(uint64_t));
    __shared__ uint32_t wc[SORT_WARPS][256];
    __shared__ uint32_t gbase[256];    // output position of the tile's first key of each digit
    __shared__ uint32_t lstart[256];   // first slot of each digit in the reordered tile
    __shared__ uint32_t ws[SORT_WARPS];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    // digit bases: exclusive scan of the 256 digit totals (one digit per thread)
    {
        uint32_t v = totals[tid];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[w] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int j = 0; j < w; j++) before += ws[j];
        gbase[tid] = before + x - v + cnt[(size_t)tid * ntiles + blockIdx.x];
    }
#pragma unroll
    for (int j = 0; j < SORT_WARPS; j++) wc[j][tid] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    uint64_t key[SORT_ITEMS];
    int32_t val[SORT_ITEMS];
    uint32_t rank[SORT_ITEMS];
    const int tile0 = blockIdx.x * SORT_TILE;
    const int wbase = tile0 + w * (SORT_TILE / SORT_WARPS);
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; it++) {
        int i = wbase + it * 32 + lane;
        bool ok = i < n;
        key[it] = ok ? kin[i] : 0ull;
        val[it] = ok ? (vin ? vin[i] : i) : 0;
        uint32_t d = ok ? ((uint32_t)(key[it] >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int leader = __ffs(peers) - 1;
        uint32_t c = 0;
        if (ok && lane == leader) {
            c = wc[w][d];
            wc[w][d] = c + __popc(peers);
        }
        c = __shfl_sync(0xffffffffu, c, leader);
        rank[it] = c + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    // per digit: offsets of the warps' runs, and the digit's first slot in the tile
    uint32_t dcount = 0;
    {
#pragma unroll
        for (int j = 0; j < SORT_WARPS; j++) {
            uint32_t t = wc[j][tid];
            wc[j][tid] = dcount;
            dcount += t;
        }
        uint32_t x = dcount;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __syncthreads();
        if (lane == 31) ws[w] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int j = 0; j < w; j++) before += ws[j];
        lstart[tid] = before + x - dcount;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; it++) {
        int i = wbase + it * 32 + lane;
        if (i < n) {
            uint32_t d = (uint32_t)(key[it] >> shift) & 255u;
            uint32_t p = lstart[d] + wc[w][d] + rank[it];
            sk[p] = key[it];
            sv[p] = val[it];
        }
    }
    __syncthreads();
    const int tn = min(SORT_TILE, n - tile0);
    for (int k = tid; k < tn; k += SORT_THREADS) {
        const uint64_t kk = sk[k];
        const uint32_t d = (uint32_t)(kk >> shift) & 255u;
        const uint32_t p = gbase[d] + (uint32_t)k - lstart[d];
        kout[p] = kk;
        vout[p] = sv[k];
    }
}

// -------------------------------------------------------------------------------------------
// gather / scatter of particle arrays
// -------------------------------------------------------------------------------------------
// gather / scatter of a subset between arrays of different SoA strides
__global__ void k_gather_subset(const int32_t *__restrict__ idx, int64_t n_out, int64_t n_in,
                                const uint32_t *__restrict__ pin, const float *__restrict__ min,
                                const uint8_t *__restrict__ cin, const float *__restrict__ ain,
                                uint32_t *__restrict__ pout, float *__restrict__ mout,
                                uint8_t *__restrict__ cout, float *__restrict__ aout)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_out;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = idx[k];
        pout[k] = pin[j];
        pout[n_out + k] = pin[n_in + j];
        pout[2 * n_out + k] = pin[2 * n_in + j];
        mout[k] = min[j];
        if (cin) cout[k] = cin[j];
        if (ain) aout[k] = ain[j];
    }
}

__global__ void k_scatter_subset(const int32_t *__restrict__ idx, int64_t n_sub, int64_t n_out,
                                 const float *__restrict__ ain, const float *__restrict__ pin,
                                 float *__restrict__ aout, float *__restrict__ pout)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_sub;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = idx[k];
        aout[j] = ain[k];
        aout[n_out + j] = ain[n_sub + k];
        aout[2 * n_out + j] = ain[2 * n_sub + k];
        if (pin) pout[j] = pin[k];
    }
}

__global__ void k_gather(const int32_t *__restrict__ perm, int64_t n,
                         const uint32_t *__restrict__ pin, const float *__restrict__ min,
                         const uint8_t *__restrict__ cin, const float *__restrict__ ain,
                         uint32_t *__restrict__ pout, float *__restrict__ mout,
                         uint8_t *__restrict__ cout, float *__restrict__ aout)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = perm[k];
        if ((uint64_t)j >= (uint64_t)n) j = 0;   // a corrupt permutation reads nothing outside
        pout[k] = pin[j];
        pout[n + k] = pin[n + j];
        pout[2 * n + k] = pin[2 * n + j];
        mout[k] = min[j];
        if (cin) cout[k] = cin[j];
        if (ain) aout[k] = ain[j];
    }
}

__global__ void k_scatter(const int32_t *__restrict__ perm, int64_t n,
                          const float *__restrict__ ain, const float *__restrict__ pin,
                          float *__restrict__ aout, float *__restrict__ pout)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = perm[k];
        if ((uint64_t)j >= (uint64_t)n) continue;   // a corrupt permutation writes nothing outside
        aout[j] = ain[k];
        aout[n + j] = ain[n + k];
        aout[2 * n + j] = ain[2 * n + k];
        if (pin) pout[j] = pin[k];
    }
}

__global__ void k_sys_keys(const uint16_t *__restrict__ sys, const int32_t *__restrict__ perm,
                           int64_t n, uint64_t *__restrict__ out)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = sys[perm[k]];
}

__global__ void k_compose(const uint64_t *__restrict__ keys1, const int32_t *__restrict__ perm1,
                          const int32_t *__restrict__ p2, int64_t n, uint64_t *__restrict__ keys,
                          int32_t *__restrict__ perm)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int j = p2[k];
        keys[k] = keys1[j];
        perm[k] = perm1[j];
    }
}

}  // namespace

// -------------------------------------------------------------------------------------------
// host side
// -------------------------------------------------------------------------------------------
static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t g4_sort_workspace_bytes(int64_t n)
{
    int64_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
    if (ntiles < 1) ntiles = 1;
    return align256(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1)) +    // alternate keys
           align256(sizeof(int32_t) * (size_t)(n > 0 ? n : 1)) * 2 +  // values, both buffers
           align256(sizeof(uint32_t) * 256 * (size_t)ntiles) +        // tile counts
           align256(sizeof(uint32_t) * 256);                          // digit totals
}

// Sorts keys_in (n keys, may alias keys_out) into keys_out with vals_out = original index.
// key_bits: number of low key bits that can be non-zero (63 for PH keys).
g4_status g4_sort_pairs_u64(const uint64_t *keys_in, uint64_t *keys_out, int32_t *vals_out,
                            int64_t n, void *workspace, size_t ws_bytes, int key_bits,
                            cudaStream_t st)
{
    if (n == 0) return G4_OK;
    if (ws_bytes < g4_sort_workspace_bytes(n))
        return g4_fail(G4_ERR_INVALID_ARG, "sort workspace too small (%zu < %zu)", ws_bytes,
                       g4_sort_workspace_bytes(n));
    int ntiles = (int)((n + SORT_TILE - 1) / SORT_TILE);
    char *p = (char *)workspace;
    uint64_t *kalt = (uint64_t *)p;
    p += align256(sizeof(uint64_t) * (size_t)n);
    int32_t *v0 = (int32_t *)p;
    p += align256(sizeof(int32_t) * (size_t)n);
    int32_t *v1 = (int32_t *)p;
    p += align256(sizeof(int32_t) * (size_t)n);
    uint32_t *cnt = (uint32_t *)p;
    p += align256(sizeof(uint32_t) * 256 * (size_t)ntiles);
    uint32_t *tot = (uint32_t *)p;
    // opt in to the tile's dynamic shared memory once per device (flags per device, set
    // atomically, so that threads and devices do not repeat the call)
    static int smem_set[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return g4_fail(G4_ERR_CUDA, "radix sort: no usable device");
    if (!__atomic_load_n(&smem_set[dev], __ATOMIC_ACQUIRE)) {
        cudaError_t e = cudaFuncSetAttribute(k_sort_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SCATTER_SMEM);
        if (e != cudaSuccess) return g4_cuda_check(e, "radix sort: shared memory opt-in");
        __atomic_store_n(&smem_set[dev], 1, __ATOMIC_RELEASE);
    }
    int passes = (key_bits + 7) / 8;
    if (passes & 1) passes++;   // even pass count: the result lands in keys_out
    // pass 0 reads keys_in with implicit values; ping-pong between keys_out/kalt and v0/v1 so
    // that the last pass writes keys_out and vals_out.
    const uint64_t *ksrc = keys_in;
    const int32_t *vsrc = nullptr;
    for (int pass = 0; pass < passes; pass++) {
        bool last = (pass == passes - 1);
        uint64_t *kdst = (pass & 1) ? keys_out : kalt;
        int32_t *vdst = last ? vals_out : ((pass & 1) ? v1 : v0);
        if (ksrc == kdst) return g4_fail(G4_ERR_INVALID_ARG, "sort buffers alias");
        int shift = 8 * pass;
        k_sort_hist<<<ntiles, SORT_THREADS, 0, st>>>(ksrc, (int)n, shift, cnt, ntiles);
        k_sort_rowscan<<<256, SCAN_THREADS, 0, st>>>(cnt, ntiles, tot);
        k_sort_scatter<<<ntiles, SORT_THREADS, SCATTER_SMEM, st>>>(ksrc, vsrc, kdst, vdst, (int)n,
                                                                   shift, cnt, tot, ntiles);
        ksrc = kdst;
        vsrc = vdst;
    }
    return g4_launch_check("radix sort", 3 * passes);
}

extern "C" g4_status g4_keys_sort_workspace(int64_t n, size_t *bytes)
{
    if (!bytes || n < 0) return g4_fail(G4_ERR_INVALID_ARG, "g4_keys_sort_workspace: bad args");
    *bytes = g4_sort_workspace_bytes(n);
    return G4_OK;
}

extern "C" g4_status g4_keys_sort(const uint32_t *pos_int, int64_t n, uint64_t *keys_sorted,
                                  int32_t *perm, void *workspace, size_t workspace_bytes,
                                  void *stream)
{
    if (n < 0 || n >= (int64_t)1 << 31)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_keys_sort: n=%lld out of range", (long long)n);
    if (n == 0) return G4_OK;
    if (!pos_int || !keys_sorted || !perm || !workspace)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_keys_sort: NULL pointer");
    if (((uintptr_t)workspace & 255) != 0)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_keys_sort: workspace not 256-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    k_keys<<<g4_blocks_for(n, 256), 256, 0, st>>>(pos_int, n, keys_sorted);
    g4_status s = g4_launch_check("keys", 1);
    if (s != G4_OK) return s;
    return g4_sort_pairs_u64(keys_sorted, keys_sorted, perm, n, workspace, workspace_bytes,
                             63, st);
}

static size_t batched_extra(int64_t n)
{
    size_t m = (size_t)(n > 0 ? n : 1);
    return 2 * align256(8 * m) + 2 * align256(4 * m);
}

extern "C" g4_status g4_keys_sort_batched_workspace(int64_t n, size_t *bytes)
{
    if (!bytes || n < 0) return g4_fail(G4_ERR_INVALID_ARG, "g4_keys_sort_batched_workspace: bad args");
    *bytes = g4_sort_workspace_bytes(n) + batched_extra(n);
    return G4_OK;
}

extern "C" g4_status g4_keys_sort_batched(const uint32_t *pos_int, int64_t n, const uint16_t *sys_id,
                                          uint64_t *keys_sorted, int32_t *perm, void *workspace,
                                          size_t workspace_bytes, void *stream)
{
    if (n < 0 || n >= (int64_t)1 << 31)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_keys_sort_batched: n=%lld out of range", (long long)n);
    if (n == 0) return G4_OK;
    if (!pos_int || !sys_id || !keys_sorted || !perm || !workspace)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_keys_sort_batched: NULL pointer");
    if (((uintptr_t)workspace & 255) != 0)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_keys_sort_batched: workspace not 256-byte aligned");
    const size_t need = g4_sort_workspace_bytes(n) + batched_extra(n);
    if (workspace_bytes < need)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_keys_sort_batched: workspace too small (%zu < %zu)",
                       workspace_bytes, need);
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)workspace + g4_sort_workspace_bytes(n);
    const size_t m = (size_t)n;
    uint64_t *keys1 = (uint64_t *)w;
    w += align256(8 * m);
    uint64_t *sysk = (uint64_t *)w;
    w += align256(8 * m);
    int32_t *perm1 = (int32_t *)w;
    w += align256(4 * m);
    int32_t *p2 = (int32_t *)w;
    const int nb = g4_blocks_for(n, 256);
    // stage 1: stable sort by Peano-Hilbert key; stage 2: stable sort by system (16-bit ids)
    k_keys<<<nb, 256, 0, st>>>(pos_int, n, keys1);
    g4_status s = g4_launch_check("batched keys", 1);
    if (s != G4_OK) return s;
    s = g4_sort_pairs_u64(keys1, keys1, perm1, n, workspace, g4_sort_workspace_bytes(n), 63, st);
    if (s != G4_OK) return s;
    k_sys_keys<<<nb, 256, 0, st>>>(sys_id, perm1, n, sysk);
    s = g4_sort_pairs_u64(sysk, sysk, p2, n, workspace, g4_sort_workspace_bytes(n), 16, st);
    if (s != G4_OK) return s;
    k_compose<<<nb, 256, 0, st>>>(keys1, perm1, p2, n, keys_sorted, perm);
    return g4_launch_check("batched sort", 2);
}

extern "C" g4_status g4_int_coords(const double *pos, int64_t n, int periodic, double box_size,
                                   uint32_t *pos_int, double *frame, void *stream)
{
    if (n < 0 || !pos_int || !frame || (n > 0 && !pos))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_int_coords: bad arguments");
    if (periodic && !(box_size > 0))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_int_coords: box_size must be > 0");
    cudaStream_t st = (cudaStream_t)stream;
    if (periodic) {
        k_frame_periodic<<<1, 32, 0, st>>>(frame, box_size);
        if (n > 0) k_int_coords_periodic<<<g4_blocks_for(n, 256), 256, 0, st>>>(pos, n, box_size, pos_int);
        return g4_launch_check("int coords", n > 0 ? 2 : 1);
    }
    if (n == 0) return g4_fail(G4_ERR_INVALID_ARG, "g4_int_coords: isolated set needs n > 0");
    // the bounding box is reduced into the caller's frame buffer itself (8 doubles)
    k_bbox_init<<<1, 32, 0, st>>>(frame);
    k_bbox_partial<<<g4_blocks_for(n, 256, 2), 256, 0, st>>>(pos, n, frame);
    k_bbox_frame<<<1, 32, 0, st>>>(frame);
    k_int_coords_isolated<<<g4_blocks_for(n, 256), 256, 0, st>>>(pos, n, frame, pos_int);
    return g4_launch_check("int coords (isolated)", 4);
}

extern "C" g4_status g4_gather(const int32_t *perm, int64_t n, const uint32_t *pos_in,
                               const float *mass_in, const uint8_t *cls_in, const float *aold_in,
                               uint32_t *pos_out, float *mass_out, uint8_t *cls_out,
                               float *aold_out, void *stream)
{
    if (n < 0) return g4_fail(G4_ERR_INVALID_ARG, "g4_gather: n < 0");
    if (n == 0) return G4_OK;
    if (!perm || !pos_in || !mass_in || !pos_out || !mass_out || (!cls_in) != (!cls_out) ||
        (!aold_in) != (!aold_out))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gather: bad pointers");
    k_gather<<<g4_blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(
        perm, n, pos_in, mass_in, cls_in, aold_in, pos_out, mass_out, cls_out, aold_out);
    return g4_launch_check("gather", 1);
}

extern "C" g4_status g4_gather_subset(const int32_t *idx, int64_t n_sub, int64_t n_all,
                                      const uint32_t *pos_in, const float *mass_in,
                                      const uint8_t *cls_in, const float *aold_in,
                                      uint32_t *pos_out, float *mass_out, uint8_t *cls_out,
                                      float *aold_out, void *stream)
{
    if (n_sub < 0 || n_all < 0 || n_sub > n_all)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gather_subset: sizes");
    if (n_sub == 0) return G4_OK;
    if (!idx || !pos_in || !mass_in || !pos_out || !mass_out || (!cls_in) != (!cls_out) ||
        (!aold_in) != (!aold_out))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_gather_subset: bad pointers");
    k_gather_subset<<<g4_blocks_for(n_sub, 256), 256, 0, (cudaStream_t)stream>>>(
        idx, n_sub, n_all, pos_in, mass_in, cls_in, aold_in, pos_out, mass_out, cls_out, aold_out);
    return g4_launch_check("gather subset", 1);
}

extern "C" g4_status g4_scatter_subset(const int32_t *idx, int64_t n_sub, int64_t n_all,
                                       const float *acc_sub, const float *pot_sub, float *acc_out,
                                       float *pot_out, void *stream)
{
    if (n_sub < 0 || n_all < 0 || n_sub > n_all)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_scatter_subset: sizes");
    if (n_sub == 0) return G4_OK;
    if (!idx || !acc_sub || !acc_out || (!pot_sub) != (!pot_out))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_scatter_subset: bad pointers");
    k_scatter_subset<<<g4_blocks_for(n_sub, 256), 256, 0, (cudaStream_t)stream>>>(
        idx, n_sub, n_all, acc_sub, pot_sub, acc_out, pot_out);
    return g4_launch_check("scatter subset", 1);
}

extern "C" g4_status g4_scatter(const int32_t *perm, int64_t n, const float *acc_sorted,
                                const float *pot_sorted, float *acc_out, float *pot_out,
                                void *stream)
{
    if (n < 0) return g4_fail(G4_ERR_INVALID_ARG, "g4_scatter: n < 0");
    if (n == 0) return G4_OK;
    if (!perm || !acc_sorted || !acc_out || (!pot_sorted) != (!pot_out))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_scatter: bad pointers");
    k_scatter<<<g4_blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(perm, n, acc_sorted,
                                                                       pot_sorted, acc_out, pot_out);
    return g4_launch_check("scatter", 1);
}

// -------------------------------------------------------------------------------------------
// Allocation-free variant of g4_keys_sort.
//
// Some callers cannot allocate device memory at the time they need the sort: host
// applications whose device memory is owned by another allocator (a pre-reserved arena) and
// that forbid cudaMalloc after start-up, and plugins that are handed device pointers but no
// allocator.  This entry point takes its
// scratch from a fixed file-scope device array instead of a caller-provided workspace.
//
// The array is part of the library image: every GPU that loads libg4 holds it (about 16 MB)
// until the process exits.  All calls share it, so calls whose work overlaps on the GPU
// (different streams, or different host threads) race on it; serialise them.  The sort
// overwrites every scratch word it later reads (tile counts are written in full before the
// scan), so the contents left by an earlier call never need clearing.
// -------------------------------------------------------------------------------------------
static constexpr int64_t G4_STATIC_SORT_MAX = (int64_t)1 << 20;

static constexpr size_t static_align256(size_t x) { return (x + 255) & ~(size_t)255; }
static constexpr size_t G4_STATIC_SORT_BYTES =
    static_align256(sizeof(uint64_t) * G4_STATIC_SORT_MAX) +
    static_align256(sizeof(int32_t) * G4_STATIC_SORT_MAX) * 2 +
    static_align256(sizeof(uint32_t) * 256 * ((G4_STATIC_SORT_MAX + SORT_TILE - 1) / SORT_TILE)) +
    static_align256(sizeof(uint32_t) * 256);

static __device__ __align__(256) unsigned char g4_static_sort_scratch[G4_STATIC_SORT_BYTES];

// Host code may not use the array's name as a device address: the device address is looked
// up once per device (with that device current) and cached.
static void *g4_static_scratch_ptr[64] = {nullptr};

extern "C" g4_status g4_keys_sort_noalloc(const uint32_t *pos_int, int64_t n,
                                          uint64_t *keys_sorted, int32_t *perm, void *stream)
{
    if (n < 0 || n > G4_STATIC_SORT_MAX)
        return g4_fail(G4_ERR_INVALID_ARG,
                       "g4_keys_sort_noalloc: n=%lld exceeds the static scratch limit of %lld "
                       "particles (use g4_keys_sort with a caller workspace)",
                       (long long)n, (long long)G4_STATIC_SORT_MAX);
    if (n == 0) return G4_OK;
    if (!pos_int || !keys_sorted || !perm)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_keys_sort_noalloc: NULL pointer");
    int dev = 0;
    g4_status s = g4_cuda_check(cudaGetDevice(&dev), "g4_keys_sort_noalloc: cudaGetDevice");
    if (s != G4_OK) return s;
    if (dev < 0 || dev >= 64) return g4_fail(G4_ERR_INVALID_ARG, "g4_keys_sort_noalloc: device id");
    void *scratch = __atomic_load_n(&g4_static_scratch_ptr[dev], __ATOMIC_ACQUIRE);
    if (!scratch) {
        // first call on this device: look up the array's device address
        s = g4_cuda_check(cudaGetSymbolAddress(&scratch, g4_static_sort_scratch),
                          "g4_keys_sort_noalloc: cudaGetSymbolAddress");
        if (s != G4_OK) return s;
        __atomic_store_n(&g4_static_scratch_ptr[dev], scratch, __ATOMIC_RELEASE);
    }
    cudaStream_t st = (cudaStream_t)stream;
    k_keys<<<g4_blocks_for(n, 256), 256, 0, st>>>(pos_int, n, keys_sorted);
    s = g4_launch_check("keys (static scratch)", 1);
    if (s != G4_OK) return s;
    return g4_sort_pairs_u64(keys_sorted, keys_sorted, perm, n, scratch, G4_STATIC_SORT_BYTES, 63, st);
}
