// g4_erfcx.cuh -- written by fit_erfcx.py; do not edit.
// erfcx(x) = exp(x^2) erfc(x) on [0, G4_ERFCX_XMAX]: polynomial in
// u = t * G4_ERFCX_U1 + G4_ERFCX_U0 with t = 1 / (1 + G4_ERFCX_K x).
// Max relative error of the FP32 evaluation: 4.74e-07.
#pragma once
#define G4_ERFCX_XMAX 4.0f
#define G4_ERFCX_K 0.5f
#define G4_ERFCX_U1 3.000000000e+00f
#define G4_ERFCX_U0 -2.000000000e+00f
#define G4_ERFCX_DEG 8
static __device__ __forceinline__ float g4_erfcx_poly(float u)
{
    float a = -8.205137330e-06f;
    a = fmaf(a, u, 3.316561600e-05f);
    a = fmaf(a, u, 9.891978379e-05f);
    a = fmaf(a, u, -8.601173065e-04f);
    a = fmaf(a, u, -1.601501723e-03f);
    a = fmaf(a, u, 2.250917814e-02f);
    a = fmaf(a, u, 1.424269372e-01f);
    a = fmaf(a, u, 4.098180478e-01f);
    a = fmaf(a, u, 4.275835774e-01f);
    return a;
}
