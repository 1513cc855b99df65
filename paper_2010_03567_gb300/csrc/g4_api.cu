// g4_api.cu -- error reporting, device queries and small host-side entry points of libg4.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "g4_internal.cuh"

static thread_local char g4_err_buf[512] = "";

g4_status g4_fail(g4_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g4_err_buf, sizeof(g4_err_buf), fmt, ap);
    va_end(ap);
    return st;
}

g4_status g4_cuda_check(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return G4_OK;
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation)
        return g4_fail(G4_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return g4_fail(G4_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static unsigned long long g4_launches = 0;

g4_status g4_launch_check(const char *what, int launches)
{
    __atomic_fetch_add(&g4_launches, (unsigned long long)launches, __ATOMIC_RELAXED);
    return g4_cuda_check(cudaGetLastError(), what);
}

extern "C" int64_t g4_launch_count(void)
{
    return (int64_t)__atomic_load_n(&g4_launches, __ATOMIC_RELAXED);
}

int g4_num_sms()
{
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 1;
        }
        cached[dev] = v;
    }
    return cached[dev];
}

extern "C" const char *g4_version(void) { return "g4-gb300 0.1 (sm_103a)"; }

extern "C" const char *g4_last_error(void) { return g4_err_buf; }

extern "C" g4_status g4_params_default(g4_params *p)
{
    if (!p) return g4_fail(G4_ERR_INVALID_ARG, "g4_params_default: NULL");
    memset(p, 0, sizeof(*p));
    p->box_size = 1.0;
    p->periodic = 0;
    p->r_s = 0.0;
    p->r_cut_factor = 4.5;
    p->pp_cut = 1;
    p->alpha = 0.0025;
    p->theta = 0.5;
    p->criterion = 0;
    p->order_p = 3;
    p->leaf_max = 8;
    p->exclusion_zone = 1;
    p->precision = 0;
    p->G = 1.0;
    p->n_eps_classes = 1;
    p->eps_table[0] = 0.01;
    p->group_size = 32;
    p->fp64_count = 4096;
    p->keep_qp = 0;
    p->fmm_p2p_per_particle = 0;
    p->soft_nodes = 0;
    p->ewald = 0;
    p->watchdog_cycles = 0;
    return G4_OK;
}
