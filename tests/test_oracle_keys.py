"""Pins for the oracle's integer coordinates, Peano-Hilbert keys and sort (CPU only).

The Hilbert curve is pinned by properties that any correct 3-D Hilbert curve has and that a
plausible coding mistake breaks: it is a bijection on the 2^(3b) cells, consecutive keys are
face-adjacent cells, and every 3l-bit key prefix is one aligned cube of the level-l grid
(Sec. 2.2.1: the curve is commensurate with the oct-tree)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2010_03567_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _all_keys(bits):
    n = 1 << bits
    cells = [(x, y, z) for x in range(n) for y in range(n) for z in range(n)]
    keys = np.array([oracle.hilbert_key(x, y, z, bits) for x, y, z in cells], np.uint64)
    return np.array(cells, np.int64), keys


@pytest.mark.parametrize("bits", [1, 2, 3, 4])
def test_hilbert_bijection_and_adjacency(bits):
    cells, keys = _all_keys(bits)
    n3 = 1 << (3 * bits)
    assert sorted(keys.tolist()) == list(range(n3))
    order = np.argsort(keys)
    walk = cells[order]
    step = np.abs(np.diff(walk, axis=0))
    assert np.all(step.sum(axis=1) == 1), "consecutive keys must be face-adjacent cells"


@pytest.mark.parametrize("bits", [2, 3, 4])
def test_hilbert_prefix_is_octree_cell(bits):
    cells, keys = _all_keys(bits)
    for level in range(1, bits + 1):
        pref = keys >> np.uint64(3 * (bits - level))
        cellpref = cells >> (bits - level)
        for p in np.unique(pref):
            sel = cellpref[pref == p]
            assert len(sel) == 8 ** (bits - level)
            assert np.all(sel == sel[0]), "a key prefix must be one aligned cube"


def test_hilbert_21bit_levels_are_hilbert_walks():
    # centres of all level-3 cells, keyed at full 21-bit resolution: the level-3 cells visited
    # in key order must again form a face-adjacent walk, and prefixes must map to cells
    n = 8
    c = [(x, y, z) for x in range(n) for y in range(n) for z in range(n)]
    half = 1 << 17
    keys = np.array([oracle.hilbert_key((x << 18) + half, (y << 18) + half, (z << 18) + half, 21)
                     for x, y, z in c], np.uint64)
    cells = np.array(c)
    walk = cells[np.argsort(keys)]
    assert np.all(np.abs(np.diff(walk, axis=0)).sum(axis=1) == 1)
    pref = keys >> np.uint64(3 * 18)
    assert len(np.unique(pref)) == 512


def test_hilbert_21bit_random_prefix_property():
    g = np.random.default_rng(7)
    pos = g.integers(0, 2 ** 32, size=(3, 20000), dtype=np.uint64).astype(np.uint32)
    keys = oracle.keys(pos)
    assert keys.max() < 2 ** 63
    for level in (1, 2, 3, 5, 8):
        kp = keys >> np.uint64(3 * (21 - level))
        cp = (pos >> np.uint32(32 - level)).astype(np.uint64)
        cid = (cp[0] << np.uint64(2 * level)) | (cp[1] << np.uint64(level)) | cp[2]
        # same key prefix <=> same cell
        pairs = set(zip(kp.tolist(), cid.tolist()))
        assert len(pairs) == len(np.unique(kp)) == len(np.unique(cid))


def test_sort_is_stable_and_a_permutation():
    g = np.random.default_rng(3)
    k = g.integers(0, 50, size=5000).astype(np.uint64)  # many equal keys
    ks, perm = oracle.sort(k)
    assert np.all(np.diff(ks.astype(np.int64)) >= 0)
    assert np.array_equal(np.sort(perm), np.arange(5000))
    assert np.array_equal(ks, k[perm])
    ref = np.lexsort((np.arange(5000), k))
    assert np.array_equal(perm, ref)


def test_integer_nearest_image_paper_example():
    e = GOLD["integer_nearest_image_example"]
    x1, x2 = np.uint8(e["x1"]), np.uint8(e["x2"])
    with np.errstate(over="ignore"):
        d = np.uint8(x1 - x2)
        assert int(d) == e["unsigned_diff"]
        assert int(d.view(np.int8)) == e["signed_diff"]
        assert int(np.uint8(x1 + np.uint8(e["shift"]))) == e["wrapped"]


def test_int_coords_periodic():
    L = 100.0
    pos = np.array([[0.0, 50.0, 99.999999], [25.0, -25.0, 125.0]])
    q = oracle.int_coords_periodic(pos, L)
    assert q[0, 0] == 0 and q[1, 0] == 2 ** 31
    assert q[0, 1] == 2 ** 30 and q[1, 1] == 3 * 2 ** 30 and q[2, 1] == 2 ** 30
    # nearest image of 99.999999 relative to 0 is a small negative separation
    d = np.int32(np.uint32(q[2, 0]) - np.uint32(q[0, 0]))
    assert -100 < d * L / 2 ** 32 < 0
    # positions are recovered to the integer resolution
    back = q.T.astype(np.float64) * L / 2 ** 32
    assert np.all(np.abs(back[0] - np.mod(pos[0], L)) <= L / 2 ** 32)


def test_int_coords_isolated_frame():
    ps = synth.plummer(2000, 11)
    q, frame = oracle.int_coords_isolated(ps.pos)
    S = frame[3]
    ext = float(np.max(ps.pos.max(0) - ps.pos.min(0)))
    assert S >= 2 * ext and S < 4 * ext and np.log2(S) == int(np.log2(S))
    # all particles in the central half, so integer differences never wrap
    assert q.min() >= 2 ** 30 and q.max() <= 3 * 2 ** 30
    back = frame[:3][None, :] + q.T.astype(np.float64) * S / 2 ** 32
    assert np.max(np.abs(back - ps.pos)) <= S / 2 ** 32
