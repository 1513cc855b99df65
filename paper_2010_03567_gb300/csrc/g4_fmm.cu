// g4_fmm.cu -- symmetric Cartesian FMM (Sec. 2.4).  (dual walk, M2L, L2L, L2P)
#include "g4_internal.cuh"

extern "C" g4_status g4_fmm_workspace(g4_tree tree, const g4_params *params, size_t *bytes)
{
    (void)tree; (void)params;
    if (bytes) *bytes = 0;
    return g4_fail(G4_ERR_STATE, "g4_fmm_workspace: FMM not available in this build");
}

extern "C" g4_status g4_gravity_fmm(g4_tree tree, const uint32_t *pos_sorted, const float *mass_sorted,
                                    const uint8_t *cls_sorted, const g4_params *params, float *acc,
                                    float *pot, uint32_t *counts, double *momentum_out, void *workspace,
                                    size_t workspace_bytes, void *stream)
{
    return g4_fail(G4_ERR_STATE, "g4_gravity_fmm: FMM not available in this build");
}
