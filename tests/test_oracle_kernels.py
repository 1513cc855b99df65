"""Pins for the oracle's interaction kernels (CPU only).

* spline softening (Eq. eqnsoft): zero-lag depth, C^1 continuity, Newtonian beyond h, and
  the enclosed mass of the cubic-spline density integrated numerically;
* TreePM short-range pair kernel (Eq. eqnpo4): the closed-form erfc force law;
* g_n (Appendix A): printed Newtonian values, finite differences for the erfc kernel;
* D_n (Eqs. eqngderiv0-eqngderiv): symmetry, tracelessness of the Newtonian tensors,
  finite differences of D_{n-1}, and the printed D_2 form.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.special import erfc

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _spline_density(r, h):
    u = r / h
    k = 8.0 / (math.pi * h ** 3)
    if u < 0.5:
        return k * (1 - 6 * u * u + 6 * u ** 3)
    if u < 1:
        return k * 2 * (1 - u) ** 3
    return 0.0


def test_softening_depth_and_edge():
    s = GOLD["softening"]
    for eps0 in (0.01, 0.3, 1.0):
        h = s["h_over_eps0"] * eps0
        g0, _ = oracle.soft_kernel(0.0, h)
        assert g0 == pytest.approx(s["potential_at_zero_lag_times_eps0"] / eps0, rel=1e-14)
        for r in (h, 1.5 * h, 10 * h):
            g0, g1 = oracle.soft_kernel(r, h)
            assert g0 == pytest.approx(1 / r, rel=1e-14)
            assert g1 == pytest.approx(-1 / r ** 3, rel=1e-14)


def test_softening_is_potential_of_cubic_spline_mass():
    h = 2.8
    for r in np.linspace(0.05, 1.2 * h, 25):
        _, g1 = oracle.soft_kernel(r, h)
        menc = integrate.quad(lambda s: 4 * math.pi * s * s * _spline_density(s, h), 0, r,
                              points=[0.5 * h, h], epsabs=1e-13, epsrel=1e-12)[0]
        # g' = -M(<r)/r^2 for unit mass, and g1 = g'/r
        assert -g1 * r ** 3 == pytest.approx(menc, rel=1e-9, abs=1e-12)


def test_softening_continuity_and_force_is_derivative():
    h = 1.0
    for u0 in (0.5, 1.0):
        a0, a1 = oracle.soft_kernel(u0 * h * (1 - 1e-12), h)
        b0, b1 = oracle.soft_kernel(u0 * h * (1 + 1e-12), h)
        assert a0 == pytest.approx(b0, rel=1e-9) and a1 == pytest.approx(b1, rel=1e-9)
    d = 1e-5
    for r in (0.1, 0.3, 0.49, 0.7, 0.95, 1.3):
        gp = (oracle.soft_kernel(r + d, h)[0] - oracle.soft_kernel(r - d, h)[0]) / (2 * d)
        assert oracle.soft_kernel(r, h)[1] == pytest.approx(gp / r, rel=1e-7)


def test_pair_kernel_erfc_closed_form():
    rs = 0.7
    h = 0.05
    for r in (0.06, 0.3, 1.0, 2.5, 4.0):
        g0, g1 = oracle.pair_kernel(r, h, rs)
        assert g0 == pytest.approx(erfc(r / (2 * rs)) / r, rel=1e-12)
        F = (erfc(r / (2 * rs)) + r / (rs * math.sqrt(math.pi)) * math.exp(-r * r / (4 * rs * rs))) / r ** 2
        assert -g1 * r == pytest.approx(F, rel=1e-12)


def test_pair_kernel_inside_softening_consistent():
    rs, h = 0.5, 0.4
    d = 1e-6
    for r in (1e-4, 2e-3, 0.05, 0.15, 0.25, 0.39):
        gp = (oracle.pair_kernel(r + d, h, rs)[0] - oracle.pair_kernel(r - d, h, rs)[0]) / (2 * d)
        assert oracle.pair_kernel(r, h, rs)[1] == pytest.approx(gp / r, rel=2e-5, abs=1e-8)
    # the small-argument series agrees with the direct branch at the switch point x = 1e-3
    r0 = 1e-3 * 2 * rs
    lo = oracle.pair_kernel(r0 * (1 - 1e-9), h, rs)
    hi = oracle.pair_kernel(r0 * (1 + 1e-9), h, rs)
    assert lo[0] == pytest.approx(hi[0], rel=1e-12) and lo[1] == pytest.approx(hi[1], rel=1e-7)


def test_cutoff_suppression_order_printed():
    e = GOLD["treepm_cutoff_suppression"]
    rs = 1.0
    r = e["R_cut"] * rs
    g0, g1 = oracle.pair_kernel(r, 1e-3, rs)
    force_ratio = (-g1 * r) * r * r        # relative to Newtonian 1/r^2
    pot_ratio = g0 * r
    for v in (force_ratio, pot_ratio):
        assert 0.05 * e["suppression_order"] < v < 5 * e["suppression_order"]


def test_gn_newtonian_printed_values():
    e = GOLD["newtonian_gn_at_r_equal_1"]
    g = oracle.gn(1.0, 0.0, 7)
    assert np.array_equal(g, np.array(e["values"], float))
    r = 2.5
    g = oracle.gn(r, 0.0, 7)
    ref = np.array(e["values"], float) / r ** np.array(e["radial_powers"], float)
    assert np.allclose(g, ref, rtol=1e-13)


@pytest.mark.parametrize("rs", [0.3, 1.0])
def test_gn_erfc_finite_differences(rs):
    for r in (0.2, 0.9, 2.1, 3.7):
        for n in range(1, 6):
            d = 1e-3 * r
            f = lambda x: oracle.gn(x, rs, n)[n - 1]
            der = (-f(r + 2 * d) + 8 * f(r + d) - 8 * f(r - d) + f(r - 2 * d)) / (12 * d)
            assert oracle.gn(r, rs, n)[n] == pytest.approx(der / r, rel=2e-7)


def test_gn_large_split_scale_is_newtonian():
    g = oracle.gn(1.3, 1e7, 5)
    assert np.allclose(g, oracle.gn(1.3, 0.0, 5), rtol=1e-6)


def _full_index(t, m):
    return [(t // 3 ** k) % 3 for k in range(m)]


@pytest.mark.parametrize("m", [2, 3, 4, 5])
def test_D_symmetry_and_newtonian_trace(m):
    rv = np.array([0.7, -1.1, 0.4])
    r = np.linalg.norm(rv)
    D = oracle.D_full(m, rv, oracle.gn(r, 0.0, m))
    # totally symmetric: equal on all index permutations
    for t in range(3 ** m):
        idx = _full_index(t, m)
        for perm in set(itertools.permutations(idx)):
            t2 = sum(v * 3 ** k for k, v in enumerate(perm))
            assert D[t2] == pytest.approx(D[t], rel=1e-13, abs=1e-14)
    # number of independent components, printed 6/10/15/21 for orders 2..5
    e = GOLD["symmetric_component_counts"]
    distinct = {tuple(sorted(_full_index(t, m))) for t in range(3 ** m)}
    assert len(distinct) == e["counts"][e["orders"].index(m)]
    # Newtonian D_m is trace-free (the potential is harmonic away from r = 0)
    scale = np.max(np.abs(D))
    for t in range(3 ** (m - 2)):
        tr = sum(D[a + 3 * a + 9 * t] for a in range(3))
        assert abs(tr) < 1e-12 * scale


@pytest.mark.parametrize("rs", [0.0, 0.8])
def test_D_finite_difference(rs):
    rv = np.array([0.9, 0.35, -0.6])
    for m in range(0, 5):
        g = lambda v: oracle.gn(np.linalg.norm(v), rs, m + 1)
        Dn1 = oracle.D_full(m + 1, rv, g(rv))
        for k in range(3):
            d = 1e-4
            e = np.zeros(3)
            e[k] = d
            fd = (oracle.D_full(m, rv + e, g(rv + e)) - oracle.D_full(m, rv - e, g(rv - e))) / (2 * d)
            got = Dn1[np.arange(3 ** m) + 3 ** m * k]
            assert np.allclose(got, fd, rtol=1e-6, atol=1e-7 * np.max(np.abs(Dn1)))


def test_D2_printed_form():
    rv = np.array([0.3, 0.5, -0.2])
    g = oracle.gn(np.linalg.norm(rv), 0.6, 3)
    D2 = oracle.D_full(2, rv, g).reshape(3, 3)
    ref = g[1] * np.eye(3) + g[2] * np.outer(rv, rv)
    assert np.allclose(D2, ref, rtol=1e-14)
    D3 = oracle.D_full(3, rv, g)
    for t in range(27):
        i, j, k = _full_index(t, 3)
        ref = g[2] * ((i == j) * rv[k] + (j == k) * rv[i] + (i == k) * rv[j]) + g[3] * rv[i] * rv[j] * rv[k]
        assert D3[t] == pytest.approx(ref, rel=1e-13, abs=1e-15)


def test_softened_gn_matches_pair_kernel_and_differences():
    """g_n of the softened kernel (softened multipoles, Sec. 2.7): g_0 and g_1 are the pair
    kernel's g and g'/r (both pieces of the spline, with and without the TreePM part); each
    g_(n+1) is (1/r) d g_n / dr by central differences; beyond h it is the unsoftened g_n;
    g_0..g_2 are continuous at u = 1/2 and u = 1 (the spline potential is C^2)."""
    h = 1.0
    for r_s in (0.0, 0.4):
        for r in (0.2, 0.35, 0.6, 0.85, 1.3):
            g = oracle.gn_soft(r, h, r_s, 5)
            g0, g1 = oracle.pair_kernel(r, h, r_s)
            assert abs(g[0] - g0) < 1e-12 * abs(g0) and abs(g[1] - g1) < 1e-11 * abs(g1)
            if r >= h:
                assert np.allclose(g, oracle.gn(r, r_s, 5), rtol=1e-12)
            for n in range(4):
                d = 1e-5
                fd = (oracle.gn_soft(r + d, h, r_s, n)[n] - oracle.gn_soft(r - d, h, r_s, n)[n]) / (2 * d) / r
                assert abs(fd - g[n + 1]) < 1e-5 * max(1.0, abs(g[n + 1])), (r_s, r, n, fd, g[n + 1])
        for ub in (0.5, 1.0):
            lo = oracle.gn_soft(ub - 1e-9, h, r_s, 2)
            hi = oracle.gn_soft(ub + 1e-9, h, r_s, 2)
            assert np.allclose(lo, hi, rtol=1e-6, atol=1e-6), (ub, lo, hi)


def test_softened_multipole_converges_inside_the_softening():
    """The particle-node term of the softened kernel approximates the softened direct sum of a
    small cluster at r < h, its error falling with the cluster size faster for higher order."""
    rng = np.random.default_rng(4)
    h, r_s = 1.0, 0.0
    x = rng.uniform(-0.5, 0.5, (24, 3))
    m = rng.uniform(0.5, 1.5, 24)
    target = np.array([0.62, 0.1, -0.05])              # inside h of the cluster centre
    errs = {}
    for p in (1, 3, 5):
        e = []
        for size in (0.16, 0.08, 0.04):
            pts = x * size
            com, mono = oracle.moments_points(pts, m, p)
            a_pn, _ = oracle.pn_soft(mono, com - target, p, r_s, h)
            a_d = np.zeros(3)
            for j in range(len(m)):
                dvec = pts[j] - target
                rr = np.linalg.norm(dvec)
                _, g1 = oracle.pair_kernel(rr, h, r_s)
                a_d += -m[j] * g1 * dvec
            e.append(np.linalg.norm(a_pn - a_d) / np.linalg.norm(a_d))
        errs[p] = e
    for p in (1, 3):
        assert errs[p][2] < errs[p][0]                   # shrinks with the cluster size
    assert errs[3][1] < errs[1][1] and errs[5][1] < errs[3][1], errs
