"""Before the FP16 candidate test, the particle-particle phase drops staged sources farther than
r_cut from the bounding box of the group's sinks (Sec. 2.3: only pairs closer than r_cut are
summed, so such a source pairs with no sink).  The box is the sinks' largest |offset| from the
group centre per axis, offsets are FP32 (integer separation converted, times the length of one
integer unit), and a source is kept when its squared distance to the box is at most
r_cut^2 G4_PP_PRUNE_MARGIN; groups wider than G4_PP_PRUNE_RMAX r_cut skip the prune.  Here the
kernel's FP32 arithmetic is emulated in numpy on integer positions for pairs just inside
r_cut, at sinks on the box's faces and corners, up to the widest group that prunes."""
import pathlib
import re

import numpy as np
import pytest

HDR = pathlib.Path(__file__).resolve().parents[1] / "paper_2010_03567_gb300" / "csrc" / "g4_pp_fp16.h"


def _consts():
    c = dict(re.findall(r"#define G4_PP_PRUNE_(\w+) ([0-9.]+)f", HDR.read_text()))
    assert set(c) == {"RMAX", "MARGIN"}, c
    return np.float32(float(c["RMAX"])), np.float32(float(c["MARGIN"]))


L = 1000.0
FSCALE = np.float32(L / 2.0 ** 32)


def _off(p, gc):
    """(float)(int32)(p - gc) * fscale, as the kernel computes it."""
    d = ((p.astype(np.int64) - gc + 2 ** 31) % 2 ** 32 - 2 ** 31).astype(np.float32)
    return d * FSCALE


def _fma(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _kept(sinks, src, rcut):
    """sinks: (32, 3) integer positions; src: (n, 3).  The kernel's keep flags."""
    _, margin = _consts()
    x0 = sinks[0].astype(np.int64)
    o = (sinks.astype(np.int64) - x0 + 2 ** 31) % 2 ** 32 - 2 ** 31
    gc = (x0 + ((o.min(0) + o.max(0)) >> 1)) % 2 ** 32
    gb = np.abs(_off(sinks, gc)).max(0)
    so = _off(src, gc)
    e = np.maximum(np.abs(so) - gb, np.float32(0.0))
    d2 = _fma(e[:, 2], e[:, 2], _fma(e[:, 1], e[:, 1], (e[:, 0] * e[:, 0]).astype(np.float32)))
    return d2 <= np.float32(rcut * rcut) * margin


def _group(rng, R, rcut, corner):
    """32 sinks within R r_cut of a random centre (per axis); with corner, one sink at each
    extreme so that the box is as wide as R allows."""
    c = rng.uniform(0, 2 ** 32, 3)
    off = rng.uniform(-1, 1, (32, 3)) * R * rcut
    if corner:
        off[0] = R * rcut * 0.999999
        off[1] = -R * rcut * 0.999999
    return ((c + off / float(FSCALE)) % 2 ** 32).astype(np.int64)


@pytest.mark.parametrize("R", [0.05, 0.5, 2.0, 8.0, 32.0, "rmax"])
def test_prune_keeps_every_pair_inside_rcut(R):
    rmax, _ = _consts()
    R = float(rmax) if R == "rmax" else R
    rcut = 5.49
    rng = np.random.Generator(np.random.PCG64(9201))
    for trial in range(40):
        sinks = _group(rng, R, rcut, corner=trial % 2 == 0)
        # sources at true distance in [0.999, 1) r_cut from a sink, pointing away from the box
        k = rng.integers(0, 32, 4000)
        u = rng.normal(size=(4000, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        r = rng.uniform(0.999, 1.0, (4000, 1)) * rcut
        src = np.rint(sinks[k] + u * r / float(FSCALE)).astype(np.int64)
        d = ((src - sinks[k] + 2 ** 31) % 2 ** 32 - 2 ** 31) * float(FSCALE)
        inside = np.sum(d * d, axis=1) < rcut * rcut
        assert np.all(_kept(sinks, src % 2 ** 32, rcut)[inside]), (R, trial)


def test_prune_drops_sources_beyond_rcut_of_the_box():
    """Negative control: sources 1.01 r_cut outside the box along an axis are dropped, and so
    is half of a uniform shell around a compact group (the prune does work)."""
    rcut = 5.49
    rng = np.random.Generator(np.random.PCG64(9202))
    sinks = _group(rng, 0.6, rcut, corner=True)
    x0 = sinks[0]
    o = (sinks - x0 + 2 ** 31) % 2 ** 32 - 2 ** 31
    hi = x0 + o.max(0)
    src = hi[None, :] + np.array([[int(1.01 * rcut / float(FSCALE)), 0, 0]])
    src[0, 1:] = x0[1:] + (o.min(0)[1:] + o.max(0)[1:]) // 2
    assert not _kept(sinks, src % 2 ** 32, rcut)[0]
    u = rng.normal(size=(20000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    shell = np.rint(sinks[0] + u * rng.uniform(0, 3 * rcut, (20000, 1)) / float(FSCALE)).astype(np.int64)
    frac = _kept(sinks, shell % 2 ** 32, rcut).mean()
    assert 0.2 < frac < 0.9, frac
