"""Pins of the Ewald-corrected pure periodic tree of the oracle (Sec. 2.2.4): the derivative
tensors of the correction potential psi (Eq. eqnewal) against the independently pinned Ewald
potential and force, Poisson's equation, finite differences and symmetry; the exact periodic
direct sum; and the tree walk with the correction against that direct sum."""
import json
import pathlib

import numpy as np
import pytest

import oracle
from paper_2010_03567_gb300 import synth

GOLD = json.loads((pathlib.Path(__file__).parent / "golden" / "paper_values.json").read_text())


def _relerr(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


POINTS = [np.array([0.3, -1.2, 2.1]), np.array([4.9, 0.1, -0.2]), np.array([0.01, 0.02, -0.005]),
          np.array([-4.99, 4.99, 4.99]), np.array([2.5, 2.5, -2.5])]


@pytest.mark.parametrize("x", POINTS)
def test_dpsi_matches_ewald_potential_and_force(x):
    """D_0 = psi(x) and D_1 = grad psi = -x/|x|^3 - a(x), with psi and the periodic
    acceleration a of a unit mass from the Ewald sums pinned in test_oracle_pm.py (another
    split parameter and more terms there)."""
    L = 10.0
    D = oracle.ewald_dpsi(x, L, 1)
    assert abs(D[0] - oracle.ewald_psi(x, L, 2.0 / L, nr=4, nk=10)) < 1e-12
    a = oracle.ewald_force(x[None, :], np.zeros((1, 3)), [1.0], L, 2.0 / L, 4, 10)[0]
    r = np.linalg.norm(x)
    assert np.max(np.abs(D[1] - (-x / r ** 3 - a))) < 1e-11


def test_dpsi_at_origin_is_the_printed_constant():
    for L in (1.0, 7.0):
        D = oracle.ewald_dpsi(np.zeros(3), L, 3)
        assert abs(D[0] * L - GOLD["ewald_correction_at_origin"]["psi0_times_L"]) < 1e-7
        assert np.max(np.abs(D[1])) < 1e-14 and np.max(np.abs(D[3])) < 1e-12   # odd orders vanish


@pytest.mark.parametrize("x", POINTS)
def test_dpsi_poisson_and_finite_differences(x):
    """psi = phi + 1/r with del^2 phi = 4 pi (delta - 1/V): the trace of D_2 is -4 pi/V and
    every trace of D_m, m >= 3, vanishes; D_(m+1) is the gradient of D_m (central
    differences); the tensors are symmetric."""
    L = 10.0
    D = oracle.ewald_dpsi(x, L, 5)
    assert abs(np.trace(D[2]) + 4 * np.pi / L ** 3) < 1e-13
    for m in range(3, 6):
        tr = np.trace(D[m], axis1=0, axis2=1)
        assert np.max(np.abs(tr)) < 1e-10 * max(1.0, np.max(np.abs(D[m]))), m
        assert np.allclose(D[m], np.swapaxes(D[m], 0, m - 1), atol=1e-14)
    h = 1e-4
    for m in range(5):
        fd = np.stack([(oracle.ewald_dpsi(x + h * e, L, m)[m] - oracle.ewald_dpsi(x - h * e, L, m)[m])
                       / (2 * h) for e in np.eye(3)], axis=-1)
        scale = max(np.max(np.abs(D[m + 1])), 1e-3 / L ** (m + 2))
        assert np.max(np.abs(fd - D[m + 1])) < 1e-6 * scale, m


def test_dpsi_parity_and_periodicity():
    """psi is even in each coordinate: D_m(-x) = (-1)^m D_m(x), and reflecting one axis flips
    the sign of every component with an odd number of that axis' indices; the full periodic
    potential psi - 1/|x| (not psi alone) and its gradient do not change under a shift by L."""
    L = 10.0
    x = np.array([0.7, -2.2, 3.1])
    D = oracle.ewald_dpsi(x, L, 4)
    Dm = oracle.ewald_dpsi(-x, L, 4)
    Dr = oracle.ewald_dpsi(x * np.array([-1.0, 1.0, 1.0]), L, 4)
    for m in range(5):
        assert np.allclose(Dm[m], (-1) ** m * D[m], rtol=1e-12, atol=1e-15)
        sign = np.ones((3,) * m)
        for idx in np.ndindex(*((3,) * m)):
            sign[idx] = (-1) ** sum(1 for i in idx if i == 0)
        assert np.allclose(Dr[m], sign * D[m], rtol=1e-12, atol=1e-15)
    # two images of one separation across the cell face (the sums are set up for
    # separations in the primary cell, |x_i| <= L/2, which the walk always passes)
    y = np.array([4.95, 1.0, -2.0])
    ys = y - np.array([L, 0.0, 0.0])
    Dy, Dys = oracle.ewald_dpsi(y, L, 1), oracle.ewald_dpsi(ys, L, 1)
    r, rs = np.linalg.norm(y), np.linalg.norm(ys)
    assert abs((Dy[0] - 1 / r) - (Dys[0] - 1 / rs)) < 1e-10
    assert np.max(np.abs((Dy[1] + y / r ** 3) - (Dys[1] + ys / rs ** 3))) < 1e-10


def _periodic_set(n, seed, L=10.0):
    g = np.random.default_rng(seed)
    # a clumpy periodic set: half uniform, half in three Gaussian blobs
    pos = np.concatenate([g.uniform(0, L, (n // 2, 3)),
                          (g.uniform(0, L, (3, 3))[g.integers(0, 3, n - n // 2)]
                           + g.normal(0, 0.6, (n - n // 2, 3)))]) % L
    ps = synth.ParticleSet(pos=pos, mass=g.uniform(0.5, 1.5, n), eps_class=np.zeros(n, np.uint8),
                           eps_table=np.array([0.01]), box_size=L, periodic=True)
    q = oracle.int_coords_periodic(ps.pos, L)
    return ps, q


def test_ewald_direct_two_bodies_and_momentum():
    """Two masses: the exact direct sum equals m times the pinned Ewald force of a unit mass;
    for a set, sum_i m_i a_i = 0 (pairwise antisymmetry of the periodic force)."""
    L = 10.0
    pos = np.array([[1.0, 2.0, 3.0], [4.5, 1.0, 8.5]])
    ps = synth.ParticleSet(pos=pos, mass=np.array([0.7, 1.3]), eps_class=np.zeros(2, np.uint8),
                           eps_table=np.array([1e-4]), box_size=L, periodic=True)
    q = oracle.int_coords_periodic(ps.pos, L)
    xq = q.T.astype(np.float64) * (L / 2 ** 32)
    OP = oracle.OracleParams(box=L, periodic=True, eps=ps.eps_table)
    a, _ = oracle.ewald_direct(q, ps.mass, None, np.arange(2), OP)
    ref = oracle.ewald_force(xq[:1], xq[1:], [1.3], L, 2.0 / L, 4, 10)[0]
    assert np.max(np.abs(a[0] - ref)) < 1e-12 * np.linalg.norm(ref)
    ps, q = _periodic_set(300, 7)
    a, _ = oracle.ewald_direct(q, ps.mass, None, np.arange(ps.n), OP)
    mom = np.sum(ps.mass[:, None] * a, axis=0)
    assert np.linalg.norm(mom) < 1e-12 * np.sum(ps.mass * np.linalg.norm(a, axis=1))


def test_ewald_tree_alpha0_is_the_exact_direct_sum():
    """With alpha = 0 every node is opened: the walk sums every pair with the correction, and
    equals the exact periodic direct sum (forces and potentials) to roundoff."""
    ps, q = _periodic_set(256, 11)
    OP = oracle.OracleParams(box=ps.box_size, periodic=True, eps=ps.eps_table, alpha=0.0,
                             order=3, ewald=True)
    run = oracle.prepare(q, ps.mass, None, np.ones(ps.n), OP, 4)
    at, pt, ct = oracle.tree_forces(run, np.arange(ps.n))
    ad, pd = oracle.ewald_direct(q, ps.mass, None, np.arange(ps.n), OP)
    assert np.all(ct[:, 1] == 0)
    assert np.max(_relerr(at, ad)) < 1e-10
    assert np.max(np.abs(pt - pd) / np.abs(pd)) < 1e-10


def test_ewald_tree_converges_with_order_and_needs_the_correction():
    """Geometric criterion theta = 0.6: the force error against the exact periodic sum falls
    from p = 2 to p = 3 to p = 4 (p = 1 equals p = 2: the dipole about the centre of mass
    vanishes); the walk without the correction (nearest images only) is off by far more."""
    ps, q = _periodic_set(400, 12)
    OPd = oracle.OracleParams(box=ps.box_size, periodic=True, eps=ps.eps_table)
    sinks = np.arange(0, ps.n, 2)
    ad, _ = oracle.ewald_direct(q, ps.mass, None, sinks, OPd)
    err = {}
    for p in (1, 2, 3, 4):
        OP = oracle.OracleParams(box=ps.box_size, periodic=True, eps=ps.eps_table, criterion=1,
                                 theta=0.6, order=p, ewald=True)
        run = oracle.prepare(q, ps.mass, None, None, OP, 4)
        at, _, _ = oracle.tree_forces(run, sinks)
        err[p] = np.percentile(_relerr(at, ad), 90)
    assert abs(err[1] - err[2]) < 1e-6 * err[2], err
    assert err[3] < 0.6 * err[2] and err[4] < 0.6 * err[3], err
    OPn = oracle.OracleParams(box=ps.box_size, periodic=True, eps=ps.eps_table, criterion=1,
                              theta=0.6, order=3, ewald=False)
    run = oracle.prepare(q, ps.mass, None, None, OPn, 4)
    an, _, _ = oracle.tree_forces(run, sinks)
    assert np.percentile(_relerr(an, ad), 90) > 10 * err[3]


def _fmm(ps, q, OP, leaf=4):
    run = oracle.prepare(q, ps.mass, None, None, OP, leaf)
    a_s, p_s, cnt = run.tree.fmm(OP)
    a = np.empty_like(a_s)
    a[run.perm] = a_s
    p = np.empty_like(p_s)
    p[run.perm] = p_s
    return a, p, cnt


def test_ewald_fmm_alpha0_is_the_exact_direct_sum():
    """The FMM with the correction (kernel 1/r - psi in every mutual expansion, psi for every
    pair, m_i psi(0) per particle): with alpha = 0 every pair is a particle pair, and the
    result is the exact periodic direct sum."""
    ps, q = _periodic_set(200, 13)
    OP = oracle.OracleParams(box=ps.box_size, periodic=True, eps=ps.eps_table, alpha=0.0,
                             order=3, ewald=True)
    run = oracle.prepare(q, ps.mass, None, np.ones(ps.n), OP, 4)
    a_s, p_s, cnt = run.tree.fmm(OP)
    a = np.empty_like(a_s)
    a[run.perm] = a_s
    p = np.empty_like(p_s)
    p[run.perm] = p_s
    ad, pd = oracle.ewald_direct(q, ps.mass, None, np.arange(ps.n), OP)
    assert cnt[0] == 0 and cnt[1] == 0
    assert np.max(_relerr(a, ad)) < 1e-10
    assert np.max(np.abs(p - pd) / np.abs(pd)) < 1e-10


def test_ewald_fmm_converges_and_conserves_momentum():
    """Geometric criterion theta = 0.6: the error against the exact periodic sum falls with the
    order, total momentum is conserved to roundoff (the periodic kernel is even), and without
    the correction the FMM is off by far more."""
    ps, q = _periodic_set(400, 14)
    OPd = oracle.OracleParams(box=ps.box_size, periodic=True, eps=ps.eps_table)
    ad, _ = oracle.ewald_direct(q, ps.mass, None, np.arange(ps.n), OPd)
    err = {}
    for p in (2, 3, 4):
        OP = oracle.OracleParams(box=ps.box_size, periodic=True, eps=ps.eps_table, criterion=1,
                                 theta=0.6, order=p, ewald=True)
        a, _, cnt = _fmm(ps, q, OP)
        assert cnt[0] > 0 and cnt[1] > 0
        err[p] = np.percentile(_relerr(a, ad), 90)
        mom = np.sum(ps.mass[:, None] * a, axis=0)
        assert np.linalg.norm(mom) < 1e-12 * np.sum(ps.mass * np.linalg.norm(a, axis=1))
    assert err[3] < 0.6 * err[2] and err[4] < 0.6 * err[3], err
    OPn = oracle.OracleParams(box=ps.box_size, periodic=True, eps=ps.eps_table, criterion=1,
                              theta=0.6, order=3, ewald=False)
    an, _, _ = _fmm(ps, q, OPn)
    assert np.percentile(_relerr(an, ad), 90) > 10 * err[3]
