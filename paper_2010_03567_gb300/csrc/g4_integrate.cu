// g4_integrate.cu -- kick, drift and timestep-bin kernels of the hierarchical time integration
// (Sec. 4.2): the kick operator K adds dt * a to the velocities of a particle set, the drift
// operator D moves the integer coordinates by v * dt (Sec. 2.10: positions stay exact integers,
// a periodic box wraps through the 32-bit overflow), and the timestep criterion
// dt_i = sqrt(2 eta eps_i / |a_i|) places every particle in the power-of-two bin k with
// dt_max / 2^k <= dt_i.  g4_translate shifts all integer coordinates by one vector (the random
// translation of Sec. 3.8).
#include "g4_internal.cuh"

namespace {

__global__ void k_kick(float *__restrict__ vel, const float *__restrict__ acc,
                       const int32_t *__restrict__ idx, int m, int n, float dt)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
        const int i = idx ? idx[t] : t;
        vel[i] = fmaf(dt, acc[i], vel[i]);
        vel[n + i] = fmaf(dt, acc[n + i], vel[n + i]);
        vel[2 * n + i] = fmaf(dt, acc[2 * n + i], vel[2 * n + i]);
    }
}

// x_int += rint(v dt 2^32 / L) modulo 2^32; isolated sets flag a step that would leave the
// central half of the integer cube (their frame keeps particles inside it)
__global__ void k_drift(uint32_t *__restrict__ pos, const float *__restrict__ vel,
                        const int32_t *__restrict__ idx, int m, int n, double dt_units,
                        int periodic, int32_t *__restrict__ flag)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
        const int i = idx ? idx[t] : t;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const long long d = __double2ll_rn((double)vel[a * n + i] * dt_units);
            const long long x = (long long)pos[a * n + i] + d;
            if (!periodic && (x < 0x40000000LL || x >= 0xC0000000LL)) {
                atomicOr(flag, 1);
                continue;
            }
            pos[a * n + i] = (uint32_t)(unsigned long long)x;
        }
    }
}

struct EpsTab {
    double e[G4_MAX_EPS_CLASSES];   // softening length eps_0 per class
};

__global__ void k_timebins(const float *__restrict__ acc, const uint8_t *__restrict__ cls,
                           const int32_t *__restrict__ idx, int m, int n, double two_eta,
                           const EpsTab eps_cls, double dt_max, int max_bin, uint8_t *__restrict__ bins)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
        const int i = idx ? idx[t] : t;
        const double ax = acc[i], ay = acc[n + i], az = acc[2 * n + i];
        const double a = sqrt(ax * ax + ay * ay + az * az);
        const double eps = eps_cls.e[cls ? cls[i] : 0];
        int k = 0;
        if (a > 0.0) {
            const double dti = sqrt(two_eta * eps / a);
            double dt = dt_max;
            while (k < max_bin && dt > dti) {
                dt *= 0.5;
                k++;
            }
        }
        bins[i] = (uint8_t)k;
    }
}

// out = in + shift (mod 2^32) per axis: the loss-less random translation of Sec. 3.8
__global__ void k_translate(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int n,
                            uint32_t sx, uint32_t sy, uint32_t sz)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        out[i] = in[i] + sx;
        out[n + i] = in[n + i] + sy;
        out[2 * n + i] = in[2 * n + i] + sz;
    }
}

}  // namespace

g4_status g4_check_params(const g4_params *P, const char *who);

extern "C" g4_status g4_translate(const uint32_t *pos_in, uint32_t *pos_out, int64_t n,
                                  const uint32_t *shift, void *stream)
{
    if (n < 0 || n >= ((int64_t)1 << 31) || !shift || (n > 0 && (!pos_in || !pos_out)))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_translate: bad arguments");
    if (n == 0) return G4_OK;
    k_translate<<<g4_blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(pos_in, pos_out, (int)n,
                                                                         shift[0], shift[1], shift[2]);
    return g4_launch_check("translate", 1);
}

extern "C" g4_status g4_kick(float *vel, const float *acc, const int32_t *idx, int64_t n_idx,
                             int64_t n, double dt, void *stream)
{
    if (n < 0 || n >= ((int64_t)1 << 31) || (idx && (n_idx < 0 || n_idx > n)) || !vel || !acc)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_kick: bad arguments");
    const int64_t m = idx ? n_idx : n;
    if (m == 0) return G4_OK;
    k_kick<<<g4_blocks_for(m, 256), 256, 0, (cudaStream_t)stream>>>(vel, acc, idx, (int)m, (int)n,
                                                                    (float)dt);
    return g4_launch_check("kick", 1);
}

extern "C" g4_status g4_drift(uint32_t *pos, const float *vel, const int32_t *idx, int64_t n_idx,
                              int64_t n, double dt, const g4_params *P, int32_t *flag, void *stream)
{
    if (!P || !(P->box_size > 0) || n < 0 || n >= ((int64_t)1 << 31) ||
        (idx && (n_idx < 0 || n_idx > n)) || !pos || !vel || (!P->periodic && !flag))
        return g4_fail(G4_ERR_INVALID_ARG, "g4_drift: bad arguments");
    const int64_t m = idx ? n_idx : n;
    if (m == 0) return G4_OK;
    k_drift<<<g4_blocks_for(m, 256), 256, 0, (cudaStream_t)stream>>>(
        pos, vel, idx, (int)m, (int)n, dt * 4294967296.0 / P->box_size, P->periodic, flag);
    return g4_launch_check("drift", 1);
}

extern "C" g4_status g4_timestep_bins(const float *acc, const uint8_t *cls, const int32_t *idx,
                                      int64_t n_idx, int64_t n, const g4_params *P, double eta,
                                      double dt_max, int32_t max_bin, uint8_t *bins, void *stream)
{
    g4_status s = g4_check_params(P, "g4_timestep_bins");
    if (s != G4_OK) return s;
    if (n < 0 || n >= ((int64_t)1 << 31) || (idx && (n_idx < 0 || n_idx > n)) || !acc || !bins ||
        !(eta > 0) || !(dt_max > 0) || max_bin < 0 || max_bin > 60)
        return g4_fail(G4_ERR_INVALID_ARG, "g4_timestep_bins: bad arguments");
    const int64_t m = idx ? n_idx : n;
    if (m == 0) return G4_OK;
    EpsTab tab;   // the softening table travels as a kernel argument
    for (int k = 0; k < G4_MAX_EPS_CLASSES; k++)
        tab.e[k] = k < P->n_eps_classes ? P->eps_table[k] : 0.0;
    k_timebins<<<g4_blocks_for(m, 256), 256, 0, (cudaStream_t)stream>>>(
        acc, cls, idx, (int)m, (int)n, 2.0 * eta, tab, dt_max, max_bin, bins);
    return g4_launch_check("timestep bins", 1);
}
