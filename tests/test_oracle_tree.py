"""Pins for the oracle's oct-tree (Sec. 2.2.1) and node moments (Sec. 2.2.2), CPU only.

The tree is compared with a brute-force recursive subdivision that groups particles by
coordinate bits (not by keys), and checked for the invariants every oct-tree must satisfy.
Moments are pinned by exact dyadic mass sums and by the parallel-axis (binomial shift)
identity that links a node's moments to its daughters' moments -- an identity the oracle
never uses (it computes every node by definition)."""
import math

import numpy as np
import pytest

import oracle
from paper_2010_03567_gb300 import synth


def _prepare(ps, leaf_max, order=3, periodic=None):
    if ps.periodic:
        q = oracle.int_coords_periodic(ps.pos, ps.box_size)
        box = ps.box_size
    else:
        q, frame = oracle.int_coords_isolated(ps.pos)
        box = frame[3]
    P = oracle.OracleParams(box=box, periodic=ps.periodic, eps=ps.eps_table, order=order)
    run = oracle.prepare(q, ps.mass, ps.eps_class, None, P, leaf_max)
    return run, q


def _brute_tree(pos, keys, leaf_max):
    n = pos.shape[1]
    nodes = []

    def rec(level, idx):
        me = len(nodes)
        nodes.append([level, idx[0], len(idx), None])
        if len(idx) > leaf_max and level < 21:
            groups = {}
            for i in idx:
                o = tuple(int((pos[ax, i] >> (31 - level)) & 1) for ax in range(3))
                groups.setdefault(o, []).append(i)
            for grp in sorted(groups.values(), key=lambda g_: int(keys[g_[0]])):
                assert grp == list(range(grp[0], grp[0] + len(grp))), "cells contiguous in PH order"
                rec(level + 1, grp)
        nodes[me][3] = len(nodes)

    rec(0, list(range(n)))
    return np.array(nodes, np.int64)


@pytest.mark.parametrize("leaf_max", [1, 4, 8])
def test_tree_matches_bruteforce_subdivision(leaf_max):
    ps = synth.plummer(1500, 21)
    run, _ = _prepare(ps, leaf_max)
    t = run.tree.export()
    ref = _brute_tree(run.tree.pos, run.keys_sorted, leaf_max)
    assert np.array_equal(t["level"], ref[:, 0])
    assert np.array_equal(t["first"], ref[:, 1])
    assert np.array_equal(t["count"], ref[:, 2])
    assert np.array_equal(t["next"], ref[:, 3])


def test_tree_invariants_periodic():
    ps = synth.zeldovich(16, 10.0, 0.5, 5)
    run, _ = _prepare(ps, 8)
    t = run.tree.export()
    pos = run.tree.pos
    nn = len(t["level"])
    leaf = t["next"] == np.arange(nn) + 1
    # every particle is in exactly one leaf
    cover = np.zeros(pos.shape[1], np.int64)
    for f, c in zip(t["first"][leaf], t["count"][leaf]):
        cover[f:f + c] += 1
    assert np.all(cover == 1)
    for k in range(nn):
        lv, f, c = t["level"][k], t["first"][k], t["count"][k]
        # the node cube contains its particles
        side = 2 ** (32 - int(lv))
        lo = t["center"][k].astype(np.int64) - side // 2
        pk = pos[:, f:f + c].astype(np.int64)
        assert np.all(pk >= lo[:, None]) and np.all(pk < lo[:, None] + side)
        if not leaf[k]:
            assert c > 8 and lv < 21
            ch, s = k + 1, 0
            while ch < t["next"][k]:
                assert t["level"][ch] == lv + 1 and t["first"][ch] == f + s
                s += t["count"][ch]
                ch = t["next"][ch]
            assert s == c and ch == t["next"][k]


def _shift_moments(mono, d, order):
    """Moments about a point displaced by -d: sum m (x + d)^(a,b,c) from sum m x^(a',b',c')."""
    out = np.zeros_like(mono)
    for n in range(order + 1):
        for a in range(n, -1, -1):
            for b in range(n - a, -1, -1):
                c = n - a - b
                s = 0.0
                for a2 in range(a + 1):
                    for b2 in range(b + 1):
                        for c2 in range(c + 1):
                            s += (math.comb(a, a2) * math.comb(b, b2) * math.comb(c, c2)
                                  * mono[oracle.mono_index(a2, b2, c2)]
                                  * d[0] ** (a - a2) * d[1] ** (b - b2) * d[2] ** (c - c2))
                out[oracle.mono_index(a, b, c)] = s
    return out


@pytest.mark.parametrize("order", [3, 5])
def test_moments_parallel_axis_identity(order):
    ps = synth.plummer(3000, 31)
    run, _ = _prepare(ps, 4, order=order)
    t = run.tree.export()
    m = run.tree.export_moments()
    nn = len(t["level"])
    box = run.params.box
    unit = box / 2 ** 32
    n_checked = 0
    for k in range(nn):
        if t["next"][k] == k + 1:
            continue
        acc = np.zeros(oracle.nmono(order))
        ch = k + 1
        while ch < t["next"][k]:
            # daughter COM relative to the parent COM
            d = ((t["center"][ch].astype(np.int64) - t["center"][k].astype(np.int64)) * unit
                 + m["com"][ch] - m["com"][k])
            acc += _shift_moments(m["mono"][ch], d, order)
            ch = t["next"][ch]
        scale = np.array([m["mass"][k] * (box / 2 ** t["level"][k]) ** (a + b + c)
                          for n in range(order + 1) for a in range(n, -1, -1)
                          for b in range(n - a, -1, -1) for c in [n - a - b]])
        assert np.allclose(acc, m["mono"][k], rtol=0, atol=1e-10 * scale.max())
        n_checked += 1
        if n_checked > 60:
            break
    assert n_checked > 10


def test_masses_exact_and_first_moment_zero():
    ps = synth.plummer_16k()          # m = 2^-14: every node mass is exact
    run, _ = _prepare(ps, 8)
    t = run.tree.export()
    m = run.tree.export_moments()
    assert m["mass"][0] == 1.0
    assert np.array_equal(m["mass"], t["count"] * 2.0 ** -14)
    side = run.params.box / 2.0 ** t["level"]
    for (a, b, c) in [(1, 0, 0), (0, 1, 0), (0, 0, 1)]:
        q1 = m["mono"][:, oracle.mono_index(a, b, c)]
        assert np.all(np.abs(q1) <= 1e-12 * m["mass"] * side)
    # second moments: trace = sum m |x - s|^2 >= 0 ; single-particle nodes have Q_n = 0
    tr = sum(m["mono"][:, oracle.mono_index(*e)] for e in [(2, 0, 0), (0, 2, 0), (0, 0, 2)])
    assert np.all(tr >= -1e-15)
    one = t["count"] == 1
    assert np.all(np.abs(m["mono"][one, 1:]) < 1e-30)
