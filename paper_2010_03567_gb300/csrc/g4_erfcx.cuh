// g4_erfcx.cuh -- written by fit_erfcx.py; do not edit.
// erfcx(x) = exp(x^2) erfc(x) on [0, G4_ERFCX_XMAX]: polynomial in
// u = t * G4_ERFCX_U1 + G4_ERFCX_U0 with t = 1 / (1 + G4_ERFCX_K x).
// Max relative error of the FP32 evaluation: 3.96e-07.
#pragma once
#define G4_ERFCX_XMAX 2.5f
#define G4_ERFCX_K 0.5f
#define G4_ERFCX_U1 3.600000000e+00f
#define G4_ERFCX_U0 -2.600000000e+00f
#define G4_ERFCX_DEG 7
static __device__ __forceinline__ float g4_erfcx_poly(float u)
{
    float a = 6.104947701e-06f;
    a = fmaf(a, u, 4.017611956e-05f);
    a = fmaf(a, u, -2.988271775e-04f);
    a = fmaf(a, u, -1.093416161e-03f);
    a = fmaf(a, u, 1.227572989e-02f);
    a = fmaf(a, u, 1.065106702e-01f);
    a = fmaf(a, u, 3.826138101e-01f);
    a = fmaf(a, u, 4.999457681e-01f);
    return a;
}
