"""Writes g4_erfcx.cuh: the scaled complementary error function erfcx(x) = exp(x^2) erfc(x)
on [0, XMAX] as a polynomial in u, where t = 1 / (1 + K x) and u = (2 t - 1 - t0) / (1 - t0),
t0 = 1 / (1 + K XMAX), so that u runs over [-1, 1].

The substitution t = 1/(1 + K x) (the variable of Abramowitz & Stegun 7.1.25-7.1.28) makes
erfcx a slowly varying function of t on the whole range; the polynomial is a Chebyshev
least-squares fit on Chebyshev points of t, converted to monomials in u.  erfc(x) is then
exp(-x^2) * erfcx(x).  The walk uses it for the TreePM short-range factor of Eq. (eqnpo4).

Run:  python fit_erfcx.py  (needs numpy, scipy; rewrites g4_erfcx.cuh beside this file)
"""
import os
import numpy as np
from numpy.polynomial import chebyshev as C
from scipy.special import erfcx

XMAX, K, DEG = 2.5, 0.5, 7


def fit():
    t0 = 1.0 / (1.0 + K * XMAX)
    u = np.cos(np.linspace(0.0, np.pi, 4001))
    t = 0.5 * (u * (1.0 - t0) + 1.0 + t0)
    x = (1.0 / t - 1.0) / K
    c = C.chebfit(u, erfcx(x), DEG)
    return t0, C.cheb2poly(c)


def eval_f32(x, t0, p):
    """The device evaluation in FP32 (rcp and Horner), for the accuracy check."""
    x = np.asarray(x, np.float32)
    t = np.float32(1) / (np.float32(1) + np.float32(K) * x)
    u = t * np.float32(2.0 / (1.0 - t0)) - np.float32((1.0 + t0) / (1.0 - t0))
    acc = np.float32(p[-1])
    for k in range(len(p) - 2, -1, -1):
        acc = acc * u + np.float32(p[k])
    return acc


def main():
    t0, p = fit()
    xs = np.linspace(0.0, XMAX, 400001)
    err = np.abs(eval_f32(xs, t0, p).astype(np.float64) / erfcx(xs) - 1.0).max()
    lines = [
        "// g4_erfcx.cuh -- written by fit_erfcx.py; do not edit.",
        "// erfcx(x) = exp(x^2) erfc(x) on [0, G4_ERFCX_XMAX]: polynomial in",
        "// u = t * G4_ERFCX_U1 + G4_ERFCX_U0 with t = 1 / (1 + G4_ERFCX_K x).",
        f"// Max relative error of the FP32 evaluation: {err:.2e}.",
        "#pragma once",
        f"#define G4_ERFCX_XMAX {XMAX:.1f}f",
        f"#define G4_ERFCX_K {K:.1f}f",
        f"#define G4_ERFCX_U1 {2.0 / (1.0 - t0):.9e}f",
        f"#define G4_ERFCX_U0 {-(1.0 + t0) / (1.0 - t0):.9e}f",
        f"#define G4_ERFCX_DEG {DEG}",
        "static __device__ __forceinline__ float g4_erfcx_poly(float u)",
        "{",
        f"    float a = {p[-1]:.9e}f;",
    ]
    for k in range(len(p) - 2, -1, -1):
        lines.append(f"    a = fmaf(a, u, {p[k]:.9e}f);")
    lines += ["    return a;", "}", ""]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "g4_erfcx.cuh")
    with open(out, "w") as f:
        f.write("\n".join(lines))
    print(f"wrote {out}; max relative error {err:.2e}")


if __name__ == "__main__":
    main()
