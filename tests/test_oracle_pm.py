"""Pins of the periodic Ewald reference and of the particle-mesh oracle (CPU only).

* Ewald (Sec. 2.1, Eq. eqnewal): the printed psi(0) L = 2.8372975; independence of the split
  parameter; zero force at the half-box symmetry points; the small-distance limit (Newtonian
  force plus the neutralising background's 4 pi r / 3V), i.e. the printed ~1e-5 deviation at
  1% of the box; the TreePM split: the erfc short-range force plus the k-space sum with
  alpha = 1/(2 r_s) add up to the full periodic force.
* PM (Sec. 2.3): the force of a point mass (PM long range + exact short range) against the
  Ewald force, with the ~1% maximum error at the matching scale the paper reports (Sec. 3.4),
  falling as A_smth grows; exact momentum conservation (same assignment and interpolation
  kernels, antisymmetric difference operator); zero force on a uniform lattice.
"""
import json
import os

import numpy as np
from scipy.special import erfc

import oracle
from oracle import pm

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_ewald_psi_at_origin_printed_value():
    for L in (1.0, 100.0):
        for alpha in (1.5 / L, 2.0 / L, 3.5 / L):
            v = oracle.ewald_psi([0.0, 0.0, 0.0], L, alpha, nr=4, nk=10) * L
            assert abs(v - GOLD["ewald_correction_at_origin"]["psi0_times_L"]) < 1e-7, v


def test_ewald_force_split_independent_and_symmetric():
    L = 1.0
    x = np.array([[0.31, 0.12, -0.07], [0.05, -0.41, 0.22]])
    f = [oracle.ewald_force(x, np.zeros((1, 3)), [1.0], L, a, 4, 10) for a in (1.5, 2.0, 3.0)]
    assert np.max(np.abs(f[0] - f[1])) < 1e-12 * np.max(np.abs(f[1]))
    assert np.max(np.abs(f[2] - f[1])) < 1e-12 * np.max(np.abs(f[1]))
    half = np.array([[0.5, 0, 0], [0.5, 0.5, 0], [0.5, 0.5, 0.5], [0, 0.5, 0]])
    assert np.max(np.abs(oracle.ewald_force(half, np.zeros((1, 3)), [1.0], L))) < 1e-12
    # translation by a box period and reflection symmetry
    g = oracle.ewald_force(x + np.array([1.0, -1.0, 0.0]), np.zeros((1, 3)), [1.0], L)
    assert np.max(np.abs(g - f[1])) < 1e-12 * np.max(np.abs(f[1]))
    h = oracle.ewald_force(-x, np.zeros((1, 3)), [1.0], L)
    assert np.max(np.abs(h + f[1])) < 1e-12 * np.max(np.abs(f[1]))


def test_ewald_small_distance_limit():
    L = 1.0
    for r in (0.003, 0.01, 0.03):
        u = np.array([0.3, -0.5, 0.81])
        u /= np.linalg.norm(u)
        a = oracle.ewald_force((r * u)[None, :], np.zeros((1, 3)), [1.0], L)[0]
        newton = -u / r ** 2
        model = newton + 4 * np.pi / 3 * r * u          # point mass + neutralising background
        assert np.linalg.norm(a - model) < 1e-6 * np.linalg.norm(a), r
        if r == 0.01:
            dev = np.linalg.norm(a - newton) / np.linalg.norm(newton)
            ref = GOLD["periodic_force_deviation_at_one_percent_of_box"]["deviation_about"]
            assert ref / 5 < dev < ref * 2, dev


def _grid_points(rng, n, L):
    x = rng.uniform(0, L, (n, 3))
    q = np.floor(x / L * 2 ** 32).astype(np.uint64).astype(np.uint32)
    return q.T.copy(), q.astype(np.float64) * L / 2 ** 32


def _point_mass_errors(N, A, seed=1, n_eval=3000):
    L = 1.0
    rs = A * L / N
    rng = np.random.default_rng(seed)
    qs, xs = _grid_points(rng, 1, L)
    qe, xe = _grid_points(rng, n_eval, L)
    a_pm, _ = pm.long_range(qs, np.array([1.0]), N, L, rs, sinks=qe)
    a_tot = oracle.ewald_force(xe, xs, [1.0], L, 2.0 / L, 4, 10)
    d = xe - xs[0]
    d -= L * np.round(d / L)
    r = np.linalg.norm(d, axis=1)
    x = r / (2 * rs)
    a_sr = (-(erfc(x) + 2 * x / np.sqrt(np.pi) * np.exp(-x * x)) / r ** 3)[:, None] * d
    nk = int(np.ceil(7.0 / (2 * np.pi * rs / L))) + 2
    a_lr = oracle.ewald_force(xe, xs, [1.0], L, 1.0 / (2 * rs), 4, nk, kspace_only=True)
    split = np.linalg.norm(a_sr + a_lr - a_tot, axis=1) / np.linalg.norm(a_tot, axis=1)
    err = np.linalg.norm(a_pm + a_sr - a_tot, axis=1) / np.linalg.norm(a_tot, axis=1)
    return split, err


def test_treepm_split_and_pm_force_law():
    split, err = _point_mass_errors(64, 1.25)
    assert split.max() < 1e-10            # erfc short range + k-space long range = Ewald
    ref = GOLD["pm_force_error_at_matching_scale"]["max_rel_error_about"]
    assert ref / 4 < err.max() < 3 * ref, err.max()
    assert np.median(err) < 2e-3
    _, err4 = _point_mass_errors(64, 4.0)
    assert err4.max() < err.max() / 4     # larger A_smth, smaller PM error


def test_pm_momentum_and_lattice():
    L, N = 10.0, 32
    rng = np.random.default_rng(7)
    q, _ = _grid_points(rng, 3000, L)
    m = rng.uniform(0.5, 2.0, 3000)
    a, _ = pm.long_range(q, m, N, L, 1.25 * L / N)
    mom = np.linalg.norm((m[:, None] * a).sum(0)) / np.sum(m * np.linalg.norm(a, axis=1))
    assert mom < 1e-12, mom
    # particles on every mesh point: uniform density, no force
    i = np.arange(N, dtype=np.uint64) * (2 ** 32 // N)
    gx, gy, gz = np.meshgrid(i, i, i, indexing="ij")
    ql = np.stack([gx.ravel(), gy.ravel(), gz.ravel()]).astype(np.uint32)
    al, _ = pm.long_range(ql, np.ones(ql.shape[1]), N, L, 1.25 * L / N)
    assert np.max(np.abs(al)) < 1e-12


def test_pm_deconvolution_unbiased_at_matching_scale():
    """The sinc deconvolution compensates the CIC smoothing "in the mean" (Sec. 2.3): around
    the matching scale the PM force of a point mass has no radial bias beyond a few 1e-3 of the
    total force (without it, the bias is ~2e-2)."""
    L, N, A = 1.0, 64, 1.25
    rs = A * L / N
    rng = np.random.default_rng(1)
    qs, xs = _grid_points(rng, 1, L)
    u = rng.normal(size=(6000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    xe = (xs[0] + rng.uniform(0.5 * rs, 8 * rs, 6000)[:, None] * u) % L
    qe = np.floor(xe / L * 2 ** 32).astype(np.uint64).astype(np.uint32).T.copy()
    xe = qe.T.astype(np.float64) * L / 2 ** 32
    d = xe - xs[0]
    d -= L * np.round(d / L)
    r = np.linalg.norm(d, axis=1)
    nk = int(np.ceil(7.0 / (2 * np.pi * rs / L))) + 2
    a_lr = oracle.ewald_force(xe, xs, [1.0], L, 1 / (2 * rs), 4, nk, kspace_only=True)
    a_tot = oracle.ewald_force(xe, xs, [1.0], L, 2.0, 4, 10)
    a_pm, _ = pm.long_range(qs, np.array([1.0]), N, L, rs, sinks=qe)
    bias = ((a_pm - a_lr) * (d / r[:, None])).sum(1) / np.linalg.norm(a_tot, axis=1)
    for lo, hi in ((1, 2), (2, 3)):
        sel = (r >= lo * rs) & (r < hi * rs)
        assert abs(np.median(bias[sel])) < 5e-3, (lo, hi, np.median(bias[sel]))
