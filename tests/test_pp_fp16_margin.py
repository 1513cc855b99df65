"""The particle-particle phase first tests every staged source against each sink in packed FP16
(positions relative to the group centre in units of r_cut) and then evaluates only the
candidates exactly.  Dropping a pair inside r_cut (Sec. 2.3: pairs are summed up to r_cut)
would change the interaction set, so the test's threshold on r^2 / r_cut^2 follows the FP16
error bound for the group's radius R (sinks within R r_cut of the centre, per axis):
e = (2 R + 2) 2^-11 per axis, threshold (1 + 2 sqrt(3) e + 3 e^2) 1.002 + 0.002, rounded
up.  Here the kernel's arithmetic (each FP16 operation rounded once from the exact value) is
emulated in numpy for pairs just inside r_cut at the edge of that range."""
import pathlib
import re

import numpy as np
import pytest

HDR = pathlib.Path(__file__).resolve().parents[1] / "paper_2010_03567_gb300" / "csrc" / "g4_pp_fp16.h"


def _consts():
    """The candidate test's constants, read from the header the kernel includes."""
    c = dict(re.findall(r"#define G4_PP_FP16_(\w+) ([0-9.]+)f", HDR.read_text()))
    keys = ("RMAX", "EA", "EB", "ULP", "C1", "C2", "SLACK_MUL", "SLACK_ADD")
    assert all(k in c for k in keys), c
    return {k: np.float32(float(c[k])) for k in keys}


def _rmax():
    return float(_consts()["RMAX"])


def test_threshold_constants_cover_the_error_bound():
    """The slack terms are at least the bound's own coefficients: 2 sqrt(3) for e and 3 for
    e^2 (the rest of this file checks the rounded result on random pairs)."""
    c = _consts()
    assert c["C1"] >= 2 * np.sqrt(3.0) - 1e-4 and c["C2"] >= 3.0
    assert c["SLACK_MUL"] >= 1.0 and c["SLACK_ADD"] >= 0.0 and c["ULP"] == 2048.0


def _h(x):
    return np.asarray(x, np.float64).astype(np.float16)


def _threshold(R):
    """Negative FP16 threshold for radius R (the kernel's formula with the header's constants),
    rounded toward -inf as __float2half_rd does."""
    c = _consts()
    e = np.float32((c["EA"] * np.float32(R) + c["EB"]) / c["ULP"])
    lim = np.float32((np.float32(1.0) + c["C1"] * e + c["C2"] * e * e) * c["SLACK_MUL"]
                     + c["SLACK_ADD"])
    v = np.float16(-lim)
    if float(v) > -float(lim):
        v = np.nextafter(v, np.float16(-np.inf))
    return v


def _candidates(sink, src, nlim):
    """sink, src: (n, 3) float64 positions in r_cut units relative to the group centre.
    Returns the FP16 candidate flags: sign of r^2 - threshold computed as the kernel does."""
    s16 = _h(sink.astype(np.float32))
    x16 = _h(src.astype(np.float32))
    d = _h(x16.astype(np.float64) - s16.astype(np.float64))          # HSUB2
    acc = np.full(len(sink), nlim, np.float16)
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


@pytest.mark.parametrize("R", [0.25, 1.0, 4.0, 12.0, 50.0, 300.0, "rmax"])
def test_fp16_test_keeps_every_pair_inside_rcut(R):
    R = _rmax() if R == "rmax" else R
    rng = np.random.Generator(np.random.PCG64(9101))
    nlim = _threshold(R)
    for rmin in (0.95, 0.999):
        sink, src = _pairs(rng, 200_000, R, rmin)
        assert np.all(_candidates(sink, src, nlim)), R


def test_fixed_margin_loses_pairs_in_wide_groups():
    """Negative control: a fixed 5% margin at 100 r_cut from the centre misses pairs inside
    r_cut, so the threshold has to grow with R (and this emulation can see a miss)."""
    rng = np.random.Generator(np.random.PCG64(9102))
    sink, src = _pairs(rng, 200_000, 100.0, rmin=0.99)
    assert not np.all(_candidates(sink, src, np.float16(-1.05)))
    assert np.all(_candidates(sink, src, _threshold(100.0)))


@pytest.mark.parametrize("r", [0.5, 0.9, 0.999])
def test_fp16_test_compact_group(r):
    """A compact group (R <= 1) keeps every pair inside r_cut and rejects everything beyond
    1.03 r_cut: the threshold is about 1.012 r_cut^2 there."""
    assert -float(_threshold(1.0)) < 1.02
    rng = np.random.Generator(np.random.PCG64(9103))
    sink = rng.uniform(-1.0, 1.0, size=(10_000, 3))
    u = rng.normal(size=(10_000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    nlim = _threshold(1.0)
    assert np.all(_candidates(sink, sink + r * u, nlim))
    assert not np.any(_candidates(sink, sink + 1.03 * u, nlim))


def test_fp16_test_needs_groups_inside_half_the_box():
    """The FP16 positions are nearest-image offsets from the group centre.  A sink R r_cut from
    the centre and a source r_cut beyond it stay on the same side only while R + 1 < L / (2
    r_cut); past that, the source's offset wraps by a box length and the FP16 test would reject
    a pair inside r_cut -- so the kernel skips the test for such groups (R + 1.01 < half box)."""
    half_box = 10.0                      # L = 20 r_cut
    R = half_box - 0.5                   # a sink 9.5 r_cut from the group centre
    sink = np.array([[R, 0.0, 0.0]])
    true_src = sink + np.array([[0.99, 0.0, 0.0]])           # 10.49: across the boundary
    wrapped = true_src - np.array([[2 * half_box, 0.0, 0.0]])   # its nearest-image offset
    assert not np.all(_candidates(sink, wrapped, _threshold(R)))   # the pair would be lost
    assert np.all(_candidates(sink, true_src, _threshold(R)))
    assert not (R + 1.01 < half_box)     # the kernel's rule turns the FP16 test off here
    R_ok = half_box - 1.02
    assert R_ok + 1.01 < half_box        # ... and keeps it where no source can wrap
