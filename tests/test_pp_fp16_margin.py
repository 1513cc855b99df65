"""The particle-particle phase first tests every staged source against each sink in packed FP16
(positions relative to the group centre in units of r_cut, threshold 1.05 r_cut^2) and then
evaluates only the candidates exactly.  Dropping a pair inside r_cut (Sec. 2.3: pairs are
summed up to r_cut) would change the interaction set, so the test may be used only where the
FP16 rounding stays inside the 5% margin: sinks within PP_FP16_RMAX r_cut of the group centre
(per axis).  Here the kernel's arithmetic (each FP16 operation rounded once from the exact
value) is emulated in numpy for pairs just inside r_cut at the edge of that range; beyond it
(a sparse group) pairs inside r_cut are lost, which is why wider groups skip the test."""
import pathlib
import re

import numpy as np
import pytest

HDR = pathlib.Path(__file__).resolve().parents[1] / "paper_2010_03567_gb300" / "csrc" / "g4_pp.cuh"


def _rmax():
    m = re.search(r"constexpr float PP_FP16_RMAX = ([0-9.]+)f;", HDR.read_text())
    assert m, "PP_FP16_RMAX not found"
    return float(m.group(1))


def _h(x):
    return np.asarray(x, np.float64).astype(np.float16)


def _candidates(sink, src):
    """sink, src: (n, 3) float64 positions in r_cut units relative to the group centre.
    Returns the FP16 candidate flags: sign of r^2 - 1.05 computed as the kernel does."""
    s16 = _h(sink.astype(np.float32))
    x16 = _h(src.astype(np.float32))
    d = _h(x16.astype(np.float64) - s16.astype(np.float64))          # HSUB2
    acc = _h(-1.05)
    for c in range(3):                                                  # HFMA2 chain
        dc = d[:, c].astype(np.float64)
        acc = _h(dc * dc + acc.astype(np.float64))
    return np.signbit(acc)


def _pairs(rng, n, R, rmin=0.95):
    """Sinks with coordinates in [-R, R] (half of them on the cube's corners, where the FP16
    spacing is widest), sources at distance in [rmin, 1) along random directions."""
    sink = rng.uniform(-R, R, size=(n, 3))
    corner = rng.integers(0, 2, size=(n // 2, 3)) * 2.0 - 1.0
    sink[: n // 2] = corner * R * (1.0 - 1e-6)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = rng.uniform(rmin, 1.0, size=(n, 1)) * (1.0 - 1e-7)
    return sink, sink + r * u


def test_fp16_test_keeps_every_pair_inside_rcut_within_rmax():
    R = _rmax()
    assert 1.0 <= R <= 16.0
    rng = np.random.Generator(np.random.PCG64(9101))
    for _ in range(4):
        sink, src = _pairs(rng, 200_000, R)
        assert np.all(_candidates(sink, src))


def test_fp16_test_alone_loses_pairs_in_wide_groups():
    """Negative control: at 100 r_cut from the centre the same test misses pairs inside
    r_cut, so the range check is needed (and this emulation can see a miss)."""
    rng = np.random.Generator(np.random.PCG64(9102))
    sink, src = _pairs(rng, 200_000, 100.0, rmin=0.99)
    assert not np.all(_candidates(sink, src))


@pytest.mark.parametrize("r", [0.5, 0.9, 0.999])
def test_fp16_test_near_the_centre(r):
    """Close to the group centre the FP16 test is essentially exact: inside r_cut always a
    candidate, beyond 1.1 r_cut never."""
    rng = np.random.Generator(np.random.PCG64(9103))
    sink = rng.uniform(-0.5, 0.5, size=(10_000, 3))
    u = rng.normal(size=(10_000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    assert np.all(_candidates(sink, sink + r * u))
    assert not np.any(_candidates(sink, sink + 1.1 * u))
