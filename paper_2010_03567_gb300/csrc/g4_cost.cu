// g4_cost.cu -- learned cost model for scheduling the tree walk.
//
// The paper balances work with a cost factor q_i per particle: the number of interactions of
// its last force computation (Sec. 6.1).  Here a small MLP predicts that cost from cheap
// per-particle tree features, and the walk's 32-sink groups are handed out heaviest first
// (longest-processing-time order) through the walk's device work queue.  Forces do not depend
// on the order: every group's result is the same whichever warp computes it and whenever.
//
// Model: 6 -> 32 -> 32 -> 1, ReLU, weights and activations stored in BF16 with FP32
// accumulation; FP32 master weights trained by Adam on the mean squared error of
// log(1 + cost).  Parameter layout (1313 floats):
//   W1[32][6], b1[32], W2[32][32], b2[32], W3[32], b3.
#include <cuda_bf16.h>

#include "g4_internal.cuh"

namespace {

constexpr int F = 6, H = 32;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * F, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H, NPARAM = OFF_B3 + 1;
static_assert(NPARAM == 1313, "parameter count");
constexpr int MLP_THREADS = 256;

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16(x)); }

// ---- features --------------------------------------------------------------------------------

__global__ void k_leaf_of(const G4Node *__restrict__ node, const int32_t *__restrict__ lvl,
                          int32_t *__restrict__ leaf_of)
{
    const int total = lvl[G4_NLEVELS];
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < total; d += gridDim.x * blockDim.x) {
        const G4Node nd = node[d];
        if (nd.meta & 32u)
            for (int i = nd.first; i < nd.first + nd.count; i++) leaf_of[i] = d;
    }
}

// Six features per (sorted) particle: leaf occupancy / leaf_max, leaf depth / 21,
// log10 |a_old|, time bin / 8, log2 of the parent node's particle count / 24 (local node
// count), log2 of the grandparent's count / 24 (density of the PH-key prefix two levels up).
__global__ void k_features(const G4Node *__restrict__ node, const int32_t *__restrict__ leaf_of,
                           const float *__restrict__ aold, const uint8_t *__restrict__ bins, int n,
                           float inv_leaf, float *__restrict__ feat)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int d = leaf_of[i];
        const G4Node lf = node[d];
        const int p = lf.parent >= 0 ? lf.parent : d;
        const G4Node pn = node[p];
        const int gp = pn.parent >= 0 ? pn.parent : p;
        const int gc = node[gp].count;
        const float a = aold ? fmaxf(aold[i], 1e-30f) : 1.0f;
        float *f = feat + (size_t)i * F;
        f[0] = (float)lf.count * inv_leaf;
        f[1] = (float)(lf.meta & 31u) * (1.0f / 21.0f);
        f[2] = log10f(a);
        f[3] = bins ? (float)bins[i] * 0.125f : 0.0f;
        f[4] = log2f((float)pn.count + 1.0f) * (1.0f / 24.0f);
        f[5] = log2f((float)gc + 1.0f) * (1.0f / 24.0f);
    }
}

// cost label of the last walk: log(1 + PP + c_pn * PN)
__global__ void k_cost_label(const uint32_t *__restrict__ counts, int n, float c_pn,
                             float *__restrict__ y)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = log1pf((float)counts[i] + c_pn * (float)counts[n + i]);
}

// ---- MLP forward / backward --------------------------------------------------------------------

struct SW {
    __nv_bfloat16 w1[H * F], w2[H * H], w3[H];
    float b1[H], b2[H], b3;
};

__device__ __forceinline__ void load_weights(SW &s, const float *__restrict__ P)
{
    for (int k = threadIdx.x; k < H * F; k += blockDim.x) s.w1[k] = __float2bfloat16(P[OFF_W1 + k]);
    for (int k = threadIdx.x; k < H * H; k += blockDim.x) s.w2[k] = __float2bfloat16(P[OFF_W2 + k]);
    for (int k = threadIdx.x; k < H; k += blockDim.x) {
        s.w3[k] = __float2bfloat16(P[OFF_W3 + k]);
        s.b1[k] = P[OFF_B1 + k];
        s.b2[k] = P[OFF_B2 + k];
    }
    if (threadIdx.x == 0) s.b3 = P[OFF_B3];
}

// forward of one sample: BF16 inputs/weights/activations, FP32 sums
__device__ __forceinline__ float mlp_forward(const SW &s, const float *x_in, float *h1, float *h2)
{
    float x[F];
#pragma unroll
    for (int k = 0; k < F; k++) x[k] = bf(x_in[k]);
#pragma unroll 4
    for (int j = 0; j < H; j++) {
        float a = s.b1[j];
#pragma unroll
        for (int k = 0; k < F; k++) a += __bfloat162float(s.w1[j * F + k]) * x[k];
        h1[j] = bf(fmaxf(a, 0.f));
    }
#pragma unroll 2
    for (int j = 0; j < H; j++) {
        float a = s.b2[j];
#pragma unroll
        for (int k = 0; k < H; k++) a += __bfloat162float(s.w2[j * H + k]) * h1[k];
        h2[j] = bf(fmaxf(a, 0.f));
    }
    float y = s.b3;
#pragma unroll
    for (int k = 0; k < H; k++) y += __bfloat162float(s.w3[k]) * h2[k];
    return y;
}

__global__ void __launch_bounds__(MLP_THREADS) k_mlp_forward(const float *__restrict__ P,
                                                             const float *__restrict__ feat, int n,
                                                             float *__restrict__ out)
{
    __shared__ SW s;
    load_weights(s, P);
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float h1[H], h2[H];
        out[i] = mlp_forward(s, feat + (size_t)i * F, h1, h2);
    }
}

// Per-block gradient of the mean squared error over the block's samples (FP32), written to
// gpart[block][NPARAM]; the loss sum goes to gpart[block][NPARAM].  A fixed-order reduction
// follows, so training is deterministic.
__global__ void __launch_bounds__(MLP_THREADS) k_mlp_grad(const float *__restrict__ P,
                                                          const float *__restrict__ feat,
                                                          const float *__restrict__ y, int n,
                                                          float inv_n, float *__restrict__ gpart)
{
    __shared__ SW s;
    __shared__ float g[MLP_THREADS / 32][NPARAM + 1];   // one row per warp: no atomics
    load_weights(s, P);
    for (int k = threadIdx.x; k < (MLP_THREADS / 32) * (NPARAM + 1); k += blockDim.x)
        (&g[0][0])[k] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const int i = base + threadIdx.x;
        const bool ok = i < n;
        float x[F], h1[H], h2[H];
        float e = 0.f;
        if (ok) {
#pragma unroll
            for (int k = 0; k < F; k++) x[k] = bf(feat[(size_t)i * F + k]);
            const float out = mlp_forward(s, feat + (size_t)i * F, h1, h2);
            e = out - y[i];
        } else {
#pragma unroll
            for (int k = 0; k < F; k++) x[k] = 0.f;
#pragma unroll
            for (int k = 0; k < H; k++) h1[k] = h2[k] = 0.f;
        }
        const float dy = 2.f * e * inv_n;      // d(mean sq. error)/d(output)
        // layer 3
        float d2[H];
#pragma unroll
        for (int k = 0; k < H; k++) d2[k] = (h2[k] > 0.f) ? dy * __bfloat162float(s.w3[k]) : 0.f;
        // warp-reduce each gradient component, one shared atomic per warp
        auto acc = [&](int idx, float v) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) g[w][idx] += v;
        };
        for (int k = 0; k < H; k++) acc(OFF_W3 + k, dy * h2[k]);
        acc(OFF_B3, dy);
        acc(NPARAM, ok ? e * e * inv_n : 0.f);
        // layer 2
        float d1[H];
#pragma unroll
        for (int k = 0; k < H; k++) d1[k] = 0.f;
        for (int j = 0; j < H; j++) {
            acc(OFF_B2 + j, d2[j]);
            for (int k = 0; k < H; k++) {
                acc(OFF_W2 + j * H + k, d2[j] * h1[k]);
                d1[k] += d2[j] * __bfloat162float(s.w2[j * H + k]);
            }
        }
        // layer 1
        for (int j = 0; j < H; j++) {
            const float dj = (h1[j] > 0.f) ? d1[j] : 0.f;
            acc(OFF_B1 + j, dj);
#pragma unroll
            for (int k = 0; k < F; k++) acc(OFF_W1 + j * F + k, dj * x[k]);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k <= NPARAM; k += blockDim.x) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < MLP_THREADS / 32; q++) t += g[q][k];
        gpart[(size_t)blockIdx.x * (NPARAM + 1) + k] = t;
    }
}

// fixed-order reduction of the per-block gradients, then one Adam step on the FP32 masters
__global__ void k_mlp_adam(float *__restrict__ P, float *__restrict__ m, float *__restrict__ v,
                           const float *__restrict__ gpart, int nblocks, float lr, float b1,
                           float b2, float eps, int step, float *__restrict__ grad_out,
                           float *__restrict__ loss_out)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= NPARAM; k += gridDim.x * blockDim.x) {
        float gk = 0.f;
        for (int b = 0; b < nblocks; b++) gk += gpart[(size_t)b * (NPARAM + 1) + k];
        if (k == NPARAM) {
            if (loss_out) *loss_out = gk;
            continue;
        }
        if (grad_out) grad_out[k] = gk;
        if (lr > 0.f) {
            const float mk = b1 * m[k] + (1.f - b1) * gk;
            const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
            m[k] = mk;
            v[k] = vk;
            const float mh = mk / (1.f - powf(b1, (float)step));
            const float vh = vk / (1.f - powf(b2, (float)step));
            P[k] -= lr * mh / (sqrtf(vh) + eps);
        }
    }
}

// ---- longest-processing-time order of the walk groups ----------------------------------------

// predicted cost of chunks of `chunk` consecutive walk groups (32 sinks each), as sort keys
// for descending cost
__global__ void k_chunk_cost(const float *__restrict__ pred, int n, int chunk, int nchunks,
                             uint64_t *__restrict__ key)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += gridDim.x * blockDim.x) {
        float s = 0.f;
        const int b = c * chunk * 32, e = min(n, b + chunk * 32);
        for (int i = b; i < e; i++) s += expm1f(fmaxf(pred[i], 0.f));
        key[c] = (uint64_t)(0xFFFFFFFFu - __float_as_uint(fmaxf(s, 0.f)));
    }
}

// position of the (possibly short) last chunk in the sorted chunk order
__global__ void k_find_last(const int32_t *__restrict__ chunk_order, int nchunks, int32_t *pos)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nchunks; p += gridDim.x * blockDim.x)
        if (chunk_order[p] == nchunks - 1) *pos = p;
}

// group order: chunks by descending predicted cost, groups inside a chunk in PH order.  All
// chunks hold `chunk` groups except the last one; chunks placed after it start earlier by
// the difference.
__global__ void k_expand_chunks(const int32_t *__restrict__ chunk_order, int nchunks, int chunk,
                                int ngroups, const int32_t *__restrict__ pos_last,
                                int32_t *__restrict__ group_order)
{
    const int last = nchunks - 1;
    const int last_size = ngroups - last * chunk;
    const int pl = *pos_last;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nchunks; p += gridDim.x * blockDim.x) {
        const int c = chunk_order[p];
        const int start = p * chunk - (p > pl ? chunk - last_size : 0);
        const int size = (c == last) ? last_size : chunk;
        for (int t = 0; t < size; t++) group_order[start + t] = c * chunk + t;
    }
}

// ---- cost-partitioned work items of the walk ---------------------------------------------------
// A 32-sink group whose predicted cost exceeds the target item cost is split into K parts
// (K in {2, 4, 8}); part k of K walks the same tree for the same 32 sinks but evaluates only
// every K-th source of the group's source list (and, for k = 0, the multipoles).  Lanes stay
// full; the parts' sums are combined in part order by whichever part finishes last.

constexpr int ITEM_SPLIT_MAX = G4_ITEM_SPLIT_MAX;

// predicted cost of each 32-sink group (sequential sum: deterministic)
__global__ void k_group_cost(const float *__restrict__ pred, int n, int ngroups,
                             float *__restrict__ gcost)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += gridDim.x * blockDim.x) {
        float c = 0.f;
        const int b = 32 * g, e = min(n, b + 32);
        for (int i = b; i < e; i++) c += expm1f(fmaxf(pred[i], 0.f));
        gcost[g] = c;
    }
}

// total predicted cost, one block, fixed summation order
__global__ void __launch_bounds__(1024) k_cost_total(const float *__restrict__ gcost, int ngroups,
                                                     double *__restrict__ total)
{
    __shared__ double part[1024];
    double s = 0.0;
    for (int g = threadIdx.x; g < ngroups; g += 1024) s += (double)gcost[g];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = part[0];
}

// wanted number of parts of each group
__global__ void k_group_parts(const float *__restrict__ gcost, int ngroups,
                              const double *__restrict__ total, float target,
                              int32_t *__restrict__ kparts)
{
    const float T = (float)(*total / (double)target);
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += gridDim.x * blockDim.x) {
        const float c = gcost[g];
        int K = 1;
        while (K < ITEM_SPLIT_MAX && c > (float)K * T) K <<= 1;
        kparts[g] = K;
    }
}

// split slot of each group: exclusive count of split groups before it (one block, fixed
// order); groups beyond the capacity stay whole
__global__ void __launch_bounds__(1024) k_split_ids(int32_t *__restrict__ kparts, int ngroups,
                                                    int max_split, int32_t *__restrict__ sid)
{
    __shared__ int32_t cnt[1024];
    const int per = (ngroups + 1023) / 1024, b = threadIdx.x * per, e = min(ngroups, b + per);
    int c = 0;
    for (int g = b; g < e; g++) c += kparts[g] > 1;
    cnt[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int t = 0; t < 1024; t++) {
            const int v = cnt[t];
            cnt[t] = run;
            run += v;
        }
    }
    __syncthreads();
    int run = cnt[threadIdx.x];
    for (int g = b; g < e; g++) {
        if (kparts[g] > 1) {
            if (run < max_split) sid[g] = run;
            else {
                sid[g] = -1;
                kparts[g] = 1;
            }
            run++;
        } else {
            sid[g] = -1;
        }
    }
}

// sort keys of the item slots 8g .. 8g+7: descending part cost for the K parts, all-ones
// (last) for the unused slots
__global__ void k_item_slots(const float *__restrict__ gcost, const int32_t *__restrict__ kparts,
                             int ngroups, uint64_t *__restrict__ key, int32_t *__restrict__ nitems)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += gridDim.x * blockDim.x) {
        const int K = kparts[g];
        const uint32_t ck = 0xFFFFFFFEu - __float_as_uint(fmaxf(gcost[g] / (float)K, 0.f));
        for (int j = 0; j < ITEM_SPLIT_MAX; j++)
            key[(size_t)ITEM_SPLIT_MAX * g + j] = j < K ? (uint64_t)ck : 0xFFFFFFFFull;
        atomicAdd(nitems, K);
    }
}

// items in sorted slot order: (first sink, count, part | parts << 8, split slot), unused
// slots all zero
__global__ void k_items_out(const int32_t *__restrict__ slot_order, int nslots,
                            const int32_t *__restrict__ kparts, const int32_t *__restrict__ sid,
                            int n, int4 *__restrict__ items)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nslots; k += gridDim.x * blockDim.x) {
        const int slot = slot_order[k], g = slot / ITEM_SPLIT_MAX, j = slot % ITEM_SPLIT_MAX;
        const int K = kparts[g];
        items[k] = j < K ? make_int4(32 * g, min(32, n - 32 * g), j | (K << 8), sid[g])
                         : make_int4(0, 0, 0, 0);
    }
}

}  // namespace

static inline size_t al256c(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" int32_t g4_mlp_param_count(void) { return NPARAM; }

extern "C" g4_status g4_cost_features(g4_tree t, const float *aold_sorted, const uint8_t *bins_sorted,
                                      const g4_params *P, float *features, int32_t *leaf_scratch,
                                      void *stream)
{
    if (!t || !P || !features || !leaf_scratch)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_cost_features: NULL argument");
    if (t->built_n < 0) return g4_fail(G4_ERR_STATE, "g4_cost_features: tree not built");
    const int n = t->built_n;
    if (n == 0) return G4_OK;
    cudaStream_t st = (cudaStream_t)stream;
    k_leaf_of<<<g4_num_sms() * 4, 256, 0, st>>>(t->node, t->lvl, leaf_scratch);
    k_features<<<g4_blocks_for(n, 256), 256, 0, st>>>(t->node, leaf_scratch, aold_sorted, bins_sorted,
                                                     n, 1.0f / (float)P->leaf_max, features);
    return g4_launch_check("cost features", 2);
}

extern "C" g4_status g4_cost_labels(const uint32_t *counts, int64_t n, float c_pn, float *labels,
                                    void *stream)
{
    if (n < 0 || (n > 0 && (!counts || !labels)))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_cost_labels: bad arguments");
    if (n == 0) return G4_OK;
    k_cost_label<<<g4_blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(counts, (int)n, c_pn, labels);
    return g4_launch_check("cost labels", 1);
}

extern "C" g4_status g4_mlp_forward(const float *params, const float *features, int64_t n,
                                    float *out, void *stream)
{
    if (n < 0 || n >= ((int64_t)1 << 31) || !params || (n > 0 && (!features || !out)))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_mlp_forward: bad arguments");
    if (n == 0) return G4_OK;
    k_mlp_forward<<<g4_blocks_for(n, MLP_THREADS, 4), MLP_THREADS, 0, (cudaStream_t)stream>>>(
        params, features, (int)n, out);
    return g4_launch_check("mlp forward", 1);
}

extern "C" g4_status g4_mlp_train_workspace(int64_t n, size_t *bytes)
{
    if (!bytes || n < 0) return g4_fail(G4_ERR_INVALID_ARG, "g4_mlp_train_workspace: bad args");
    const int nb = g4_blocks_for(n > 0 ? n : 1, MLP_THREADS, 2);
    *bytes = al256c(sizeof(float) * (size_t)nb * (NPARAM + 1));
    return G4_OK;
}

extern "C" g4_status g4_mlp_train_step(float *params, float *adam_m, float *adam_v, int32_t step,
                                       const float *features, const float *labels, int64_t n,
                                       float lr, float *loss_out, float *grad_out, void *workspace,
                                       size_t workspace_bytes, void *stream)
{
    if (n <= 0 || n >= ((int64_t)1 << 31) || !params || !adam_m || !adam_v || !features ||
        !labels || !workspace || step < 1)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_mlp_train_step: bad arguments");
    const int nb = g4_blocks_for(n, MLP_THREADS, 2);
    if (workspace_bytes < sizeof(float) * (size_t)nb * (NPARAM + 1))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_mlp_train_step: workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    float *gpart = (float *)workspace;
    k_mlp_grad<<<nb, MLP_THREADS, 0, st>>>(params, features, labels, (int)n, 1.0f / (float)n, gpart);
    k_mlp_adam<<<(NPARAM + 256) / 256, 256, 0, st>>>(params, adam_m, adam_v, gpart, nb, lr, 0.9f,
                                                     0.999f, 1e-8f, step, grad_out, loss_out);
    return g4_launch_check("mlp train step", 2);
}

extern "C" g4_status g4_schedule_workspace(int64_t n, size_t *bytes)
{
    if (!bytes || n < 0) return g4_fail(G4_ERR_INVALID_ARG, "g4_schedule_workspace: bad args");
    const int64_t ng = (n + 31) / 32;
    *bytes = al256c(8 * (size_t)(ng > 0 ? ng : 1)) + al256c(4 * (size_t)(ng > 0 ? ng : 1)) +
             256 + g4_sort_workspace_bytes(ng);
    return G4_OK;
}

extern "C" g4_status g4_schedule_lpt(const float *pred_sorted, int64_t n, int32_t chunk,
                                     int32_t *group_order, void *workspace, size_t workspace_bytes,
                                     void *stream)
{
    if (n < 0 || n >= ((int64_t)1 << 31) || chunk < 1 ||
        (n > 0 && (!pred_sorted || !group_order || !workspace)))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_schedule_lpt: bad arguments");
    if (n == 0) return G4_OK;
    const int64_t ng = (n + 31) / 32;
    const int64_t nc = (ng + chunk - 1) / chunk;
    size_t need = 0;
    g4_schedule_workspace(n, &need);
    if (workspace_bytes < need) return g4_fail(G4_ERR_INVALID_ARG, "g4_schedule_lpt: workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t *key = (uint64_t *)workspace;
    int32_t *corder = (int32_t *)((char *)workspace + al256c(8 * (size_t)ng));
    int32_t *pos_last = (int32_t *)((char *)corder + al256c(4 * (size_t)ng));
    void *sws = (char *)pos_last + 256;
    k_chunk_cost<<<g4_blocks_for(nc, 256), 256, 0, st>>>(pred_sorted, (int)n, chunk, (int)nc, key);
    g4_status s = g4_launch_check("chunk cost", 1);
    if (s != G4_OK) return s;
    // stable sort by descending predicted cost; ties keep PH order
    s = g4_sort_pairs_u64(key, key, corder, nc, sws, g4_sort_workspace_bytes(nc), 32, st);
    if (s != G4_OK) return s;
    k_find_last<<<g4_blocks_for(nc, 256), 256, 0, st>>>(corder, (int)nc, pos_last);
    k_expand_chunks<<<g4_blocks_for(nc, 256), 256, 0, st>>>(corder, (int)nc, chunk, (int)ng, pos_last,
                                                           group_order);
    return g4_launch_check("expand chunks", 2);
}

extern "C" g4_status g4_schedule_items_workspace(int64_t n, size_t *bytes)
{
    if (!bytes || n < 0) return g4_fail(G4_ERR_INVALID_ARG, "g4_schedule_items_workspace: bad args");
    const size_t ng = (size_t)((n + 31) / 32 > 0 ? (n + 31) / 32 : 1);
    const size_t ns = ITEM_SPLIT_MAX * ng;
    *bytes = al256c(4 * ng) + al256c(8) + 2 * al256c(4 * ng) + al256c(8 * ns) + al256c(4 * ns) +
             g4_sort_workspace_bytes((int64_t)ns);
    return G4_OK;
}

extern "C" g4_status g4_schedule_items(const float *pred_sorted, int64_t n, int32_t target,
                                       int32_t max_split, int32_t *items, int32_t *n_items,
                                       void *workspace, size_t workspace_bytes, void *stream)
{
    if (n < 0 || n >= ((int64_t)1 << 28) || target < 1 || max_split < 0 || !items || !n_items ||
        !workspace || (n > 0 && !pred_sorted))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_schedule_items: bad arguments");
    size_t need = 0;
    g4_schedule_items_workspace(n, &need);
    if (workspace_bytes < need) return g4_fail(G4_ERR_INVALID_ARG, "g4_schedule_items: workspace too small");
    if (((uintptr_t)workspace & 255) != 0)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_schedule_items: workspace not 256-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(n_items, 0, sizeof(int32_t), st) != cudaSuccess)
        return g4_cuda_check(cudaGetLastError(), "g4_schedule_items: clear count");
    if (n == 0) return G4_OK;
    const int64_t ng = (n + 31) / 32, ns = ITEM_SPLIT_MAX * ng;
    char *p = (char *)workspace;
    float *gcost = (float *)p;
    p += al256c(4 * (size_t)ng);
    double *total = (double *)p;
    p += al256c(8);
    int32_t *kparts = (int32_t *)p;
    p += al256c(4 * (size_t)ng);
    int32_t *sid = (int32_t *)p;
    p += al256c(4 * (size_t)ng);
    uint64_t *key = (uint64_t *)p;
    p += al256c(8 * (size_t)ns);
    int32_t *slot_order = (int32_t *)p;
    p += al256c(4 * (size_t)ns);
    void *sws = p;
    k_group_cost<<<g4_blocks_for(ng, 256), 256, 0, st>>>(pred_sorted, (int)n, (int)ng, gcost);
    k_cost_total<<<1, 1024, 0, st>>>(gcost, (int)ng, total);
    k_group_parts<<<g4_blocks_for(ng, 256), 256, 0, st>>>(gcost, (int)ng, total, (float)target, kparts);
    k_split_ids<<<1, 1024, 0, st>>>(kparts, (int)ng, max_split, sid);
    k_item_slots<<<g4_blocks_for(ng, 256), 256, 0, st>>>(gcost, kparts, (int)ng, key, n_items);
    g4_status s = g4_launch_check("item slots", 5);
    if (s != G4_OK) return s;
    s = g4_sort_pairs_u64(key, key, slot_order, ns, sws, g4_sort_workspace_bytes(ns), 32, st);
    if (s != G4_OK) return s;
    k_items_out<<<g4_blocks_for(ns, 256), 256, 0, st>>>(slot_order, (int)ns, kparts, sid, (int)n,
                                                       (int4 *)items);
    return g4_launch_check("items", 1);
}

extern "C" g4_status g4_tree_set_work_items(g4_tree t, const int32_t *items, const int32_t *n_items,
                                            int64_t capacity, int64_t n_sinks, int32_t max_split)
{
    if (!t || capacity < 0 || n_sinks < 0 || max_split < 0 || (items && !n_items))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_tree_set_work_items: bad args");
    if (items && max_split > t->part_cap) {
        // partial sums of split groups: 8 parts x 32 lanes x (4 floats + 2 counts), plus one
        // arrival counter per split group (zero between walks)
        if (t->part_buf) cudaFree(t->part_buf);
        if (t->part_cnt) cudaFree(t->part_cnt);
        t->part_buf = nullptr;
        t->part_cnt = nullptr;
        t->part_cap = 0;
        const size_t bb = (size_t)max_split * ITEM_SPLIT_MAX * 32 * 6 * sizeof(float);
        if (cudaMalloc(&t->part_buf, bb) != cudaSuccess ||
            cudaMalloc(&t->part_cnt, sizeof(int32_t) * (size_t)max_split) != cudaSuccess) {
            cudaGetLastError();
            if (t->part_buf) cudaFree(t->part_buf);
            t->part_buf = nullptr;
            t->part_cnt = nullptr;
            return g4_fail(G4_ERR_OOM, "g4_tree_set_work_items: partial-sum buffers (%zu bytes)", bb);
        }
        if (cudaMemset(t->part_cnt, 0, sizeof(int32_t) * (size_t)max_split) != cudaSuccess)
            return g4_cuda_check(cudaGetLastError(), "g4_tree_set_work_items: clear counters");
        t->part_cap = max_split;
    }
    t->items = items;
    t->n_items = items ? n_items : nullptr;
    t->items_cap = items ? capacity : 0;
    t->items_n_sinks = items ? n_sinks : -1;
    return G4_OK;
}

extern "C" g4_status g4_tree_set_group_order(g4_tree t, const int32_t *group_order, int64_t ngroups)
{
    if (!t || ngroups < 0) return g4_fail(G4_ERR_INVALID_ARG, "g4_tree_set_group_order: bad args");
    t->group_order = group_order;
    t->group_order_n = group_order ? ngroups : 0;
    return G4_OK;
}
