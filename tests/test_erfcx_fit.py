"""The FP32 short-range factor used by the walk: erfc(x) = exp(-x^2) erfcx(x) with erfcx from
the fitted polynomial in g4_erfcx.cuh (variable t = 1 / (1 + K x)).  Checked here, without a
GPU, by evaluating the header's coefficients in FP32 exactly as the device does (reciprocal,
one FMA for u, Horner) against math.erfc in FP64."""
import math
import pathlib
import re

import numpy as np

HDR = pathlib.Path(__file__).resolve().parents[1] / "paper_2010_03567_gb300" / "csrc" / "g4_erfcx.cuh"


def _header():
    txt = HDR.read_text()
    defs = {m.group(1): float(m.group(2)) for m in
            re.finditer(r"#define G4_ERFCX_(\w+) ([-+0-9.eE]+)f?", txt)}
    coef = [float(c) for c in re.findall(r"([-+]?[0-9.]+e[-+][0-9]+)f\);", txt)]
    first = float(re.search(r"float a = ([-+0-9.eE]+)f;", txt).group(1))
    return defs, [first] + coef   # highest degree first


def _erfcx_f32(x, defs, coef):
    x = np.asarray(x, np.float32)
    t = np.float32(1) / (np.float32(1) + np.float32(defs["K"]) * x)
    u = t * np.float32(defs["U1"]) + np.float32(defs["U0"])
    a = np.float32(coef[0])
    for c in coef[1:]:
        a = a * u + np.float32(c)
    return a


def test_erfcx_fit_relative_error():
    defs, coef = _header()
    assert len(coef) == int(defs["DEG"]) + 1
    xs = np.linspace(0.0, defs["XMAX"], 20001)
    got = _erfcx_f32(xs, defs, coef).astype(np.float64)
    want = np.array([math.erfc(x) * math.exp(x * x) for x in xs])
    assert np.max(np.abs(got / want - 1.0)) < 8e-7


def test_erfc_and_force_factor():
    # erfc(x) and erfc(x) + 2x/sqrt(pi) exp(-x^2) (the two factors of the short-range pair
    # force, Sec. 2.3) to 1e-6 relative over the cutoff range
    defs, coef = _header()
    xs = np.linspace(0.0, defs["XMAX"], 4001)
    e = np.exp(-xs * xs)
    ec = _erfcx_f32(xs, defs, coef).astype(np.float64) * e
    f1 = ec + 2.0 * xs / math.sqrt(math.pi) * e
    w0 = np.array([math.erfc(x) for x in xs])
    w1 = w0 + 2.0 * xs / math.sqrt(math.pi) * e
    assert np.max(np.abs(ec / w0 - 1.0)) < 1e-6
    assert np.max(np.abs(f1 / w1 - 1.0)) < 1e-6
