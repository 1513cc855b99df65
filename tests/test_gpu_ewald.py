"""The pure periodic tree with the Ewald correction (Sec. 2.2.4) on the GPU against the oracle:
the correction tensors from the grid against the exact Ewald sums, the walk against the
oracle's walk with exact tensors (same interaction set), and against the exact periodic
direct sum."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2010_03567_gb300 import g4, synth  # noqa: E402

from _helpers import gpu_forces, gpu_params, oracle_params, relerr  # noqa: E402

pytestmark = pytest.mark.gpu

PARITY_P99 = 1e-5


def _periodic_set(n, seed, L=10.0):
    g = np.random.default_rng(seed)
    pos = np.concatenate([g.uniform(0, L, (n // 2, 3)),
                          (g.uniform(0, L, (3, 3))[g.integers(0, 3, n - n // 2)]
                           + g.normal(0, 0.6, (n - n // 2, 3)))]) % L
    ps = synth.ParticleSet(pos=pos, mass=g.uniform(0.5, 1.5, n), eps_class=np.zeros(n, np.uint8),
                           eps_table=np.array([0.01]), box_size=L, periodic=True)
    return ps, oracle.int_coords_periodic(ps.pos, L)


def _mono_of_full(D, nmax):
    """monomial components (g4_midx order) of the oracle's full tensors"""
    out = []
    for m in range(nmax + 1):
        for bc in range(m + 1):
            for c in range(bc + 1):
                a, b = m - bc, bc - c
                idx = (0,) * a + (1,) * b + (2,) * c
                out.append(D[m][idx] if m else float(D[0]))
    return np.array(out)


def test_ewald_grid_tensors_match_the_ewald_sums():
    """Third-order Taylor expansion about the nearest of 32^3 cell centres (one octant, signs
    by reflection) against the exact tensors, orders 0..4, over the primary cell."""
    L = 10.0
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(-L / 2, L / 2, (200, 3)), rng.uniform(-0.2, 0.2, (20, 3)),
                        np.array([[L / 2, L / 2, -L / 2], [0.0, 0.0, 0.0], [L / 2, 0.0, 1e-3]])])
    tg = g4.TreeGravity(64, g4.params(box_size=L, periodic=1, eps=[0.01]))
    got = g4.g4_ewald_eval(tg.tree, torch.from_numpy(x).cuda(), 4, L).cpu().numpy()
    ref = np.stack([_mono_of_full(oracle.ewald_dpsi(p, L, 4), 4) for p in x])
    off = 0
    for m in range(5):
        k = (m + 1) * (m + 2) // 2
        scale = np.max(np.abs(ref[:, off:off + k]))
        err = np.max(np.abs(got[:, off:off + k] - ref[:, off:off + k]))
        # orders 0..3 (those a p = 3 walk uses) to 1e-5 of their largest component, order 4 to
        # 3e-5 (the Taylor remainder grows with the order)
        assert err < (1e-5 if m <= 3 else 3e-5) * scale, (m, err, scale)
        off += k


def _walk_case(precision):
    ps, q = _periodic_set(1024, 21)
    kw = dict(criterion=1, theta=0.5, order_p=3, leaf_max=8, ewald=1, precision=precision)
    P = gpu_params(g4, ps, ps.box_size, **kw)
    ag, pg, cg, _ = gpu_forces(torch, g4, ps, q, P, None, cls=False)
    OP = oracle_params(ps, ps.box_size, **kw)
    run = oracle.prepare(q, ps.mass, None, None, OP, 8)
    ao, po, co = oracle.tree_forces(run, np.arange(ps.n))
    return ps, q, ag, pg, cg, ao, po, co


def test_ewald_walk_parity_fp32_and_exact_sum():
    ps, q, ag, pg, cg, ao, po, co = _walk_case(0)
    e = relerr(ag, ao)
    assert np.percentile(e, 99) < PARITY_P99, np.percentile(e, [50, 99, 100])
    assert np.percentile(np.abs(pg - po) / np.abs(po), 99) < PARITY_P99
    assert np.mean(np.all(cg == co, axis=1)) > 0.99 and co[:, 1].sum() > 0
    # the method's own error against the exact periodic sum (theta = 0.5, p = 3)
    sinks = np.arange(0, ps.n, 4)
    ad, _ = oracle.ewald_direct(q, ps.mass, None, sinks, oracle_params(ps, ps.box_size))
    assert np.percentile(relerr(ag[sinks], ad), 99) < 0.02
    assert np.percentile(relerr(ag[sinks], ad), 50) < 2e-3


def test_ewald_walk_parity_fp64():
    ps, q, ag, pg, cg, ao, po, co = _walk_case(1)
    assert np.percentile(relerr(ag, ao), 99) < 1e-6
    assert np.all(cg == co)


def test_ewald_walk_opened_everywhere_is_the_exact_sum():
    """Geometric criterion with theta -> 0: every node opened, every pair with the
    correction: the exact periodic direct sum up to the grid's and FP32's rounding."""
    ps, q = _periodic_set(512, 22)
    kw = dict(criterion=1, theta=1e-6, order_p=3, leaf_max=8, ewald=1)
    ag, pg, cg, _ = gpu_forces(torch, g4, ps, q, gpu_params(g4, ps, ps.box_size, **kw), None,
                               cls=False)
    ad, pd = oracle.ewald_direct(q, ps.mass, None, np.arange(ps.n), oracle_params(ps, ps.box_size))
    assert np.all(cg[:, 1] == 0)
    assert np.percentile(relerr(ag, ad), 99) < 2e-5
    assert np.percentile(np.abs(pg - pd) / np.abs(pd), 99) < 2e-5


def test_ewald_needs_a_periodic_tree_walk():
    with pytest.raises(g4.G4Error):
        tg = g4.TreeGravity(16, g4.params(box_size=1.0, periodic=0, ewald=1))
        tg.forces(torch.zeros((3, 16), dtype=torch.int32, device="cuda"),
                  torch.ones(16, device="cuda"), None, None,
                  g4.params(box_size=1.0, periodic=0, ewald=1, criterion=1))


def _gpu_fmm(ps, q, P):
    from _helpers import to_dev, u32_dev
    tg = g4.TreeGravity(ps.n, P)
    tg.prepare(u32_dev(torch, q), to_dev(torch, ps.mass, torch.float32), None, None, P)
    acc, pot, cnt, mom = tg.tree.gravity_fmm(tg.pos_s, tg.mass_s, None, None, P)
    torch.cuda.synchronize()
    tg.tree.status()
    perm = tg.perm.cpu().numpy()
    a = np.empty((ps.n, 3))
    a[perm] = acc.cpu().numpy().T
    p = np.empty(ps.n)
    p[perm] = pot.cpu().numpy()
    c = np.empty((ps.n, 3), np.int64)
    c[perm] = cnt.cpu().numpy().T
    return a, p, c, mom.cpu().numpy()


def test_ewald_fmm_parity_and_momentum():
    """The pure periodic FMM (kernel 1/r - psi in every expansion, psi for every particle
    pair) against the oracle's FMM with exact tensors, its momentum, and its error against the
    exact periodic sum."""
    ps, q = _periodic_set(1024, 23)
    kw = dict(criterion=1, theta=0.5, order_p=4, leaf_max=8, ewald=1)
    ag, pg, cg, mom = _gpu_fmm(ps, q, gpu_params(g4, ps, ps.box_size, **kw))
    OP = oracle_params(ps, ps.box_size, **kw)
    run = oracle.prepare(q, ps.mass, None, None, OP, 8)
    a_s, p_s, co, pc_s = run.tree.fmm(OP, per_particle=True)
    ao = np.empty_like(a_s)
    ao[run.perm] = a_s
    po = np.empty_like(p_s)
    po[run.perm] = p_s
    pc = np.empty_like(pc_s)
    pc[run.perm] = pc_s
    assert co[0] > 0 and co[1] > 0
    assert np.mean((cg[:, 0] == pc[:, 0]) & (cg[:, 1] == pc[:, 1])) >= 0.99
    e = relerr(ag, ao)
    assert np.percentile(e, 99) < PARITY_P99, np.percentile(e, [50, 99, 100])
    assert np.percentile(np.abs(pg - po) / np.abs(po), 99) < PARITY_P99
    assert np.linalg.norm(mom) < 1e-5 * np.sum(ps.mass * np.linalg.norm(ag, axis=1))
    sinks = np.arange(0, ps.n, 4)
    ad, _ = oracle.ewald_direct(q, ps.mass, None, sinks, oracle_params(ps, ps.box_size))
    assert np.percentile(relerr(ag[sinks], ad), 99) < 0.02


def test_ewald_fmm_opened_everywhere_is_the_exact_sum():
    ps, q = _periodic_set(512, 24)
    kw = dict(criterion=1, theta=1e-6, order_p=3, leaf_max=8, ewald=1)
    ag, pg, cg, _ = _gpu_fmm(ps, q, gpu_params(g4, ps, ps.box_size, **kw))
    ad, pd = oracle.ewald_direct(q, ps.mass, None, np.arange(ps.n), oracle_params(ps, ps.box_size))
    assert np.all(cg[:, 1] == 0)
    assert np.percentile(relerr(ag, ad), 99) < 2e-5
    assert np.percentile(np.abs(pg - pd) / np.abs(pd), 99) < 2e-5


@pytest.mark.parametrize("n", [1, 2])
def test_ewald_single_particle_and_pair(n):
    """One particle: no force, and the potential of its own images G m psi(0) with the
    printed psi(0) L = 2.8372975; two particles: the exact periodic sum, tree and FMM."""
    L = 10.0
    g = np.random.default_rng(31 + n)
    pos = g.uniform(0, L, (n, 3))
    ps = synth.ParticleSet(pos=pos, mass=g.uniform(0.5, 1.5, n), eps_class=np.zeros(n, np.uint8),
                           eps_table=np.array([0.01]), box_size=L, periodic=True)
    q = oracle.int_coords_periodic(ps.pos, L)
    kw = dict(criterion=1, theta=0.5, order_p=3, leaf_max=8, ewald=1)
    P = gpu_params(g4, ps, L, **kw)
    ag, pg, _, _ = gpu_forces(torch, g4, ps, q, P, None, cls=False)
    af, pf, _, _ = _gpu_fmm(ps, q, P)
    if n == 1:
        assert np.all(ag == 0) and np.all(af == 0)
        for p in (pg[0], pf[0]):
            assert abs(p * L / ps.mass[0] - 2.8372975) < 1e-5
    else:
        ad, pd = oracle.ewald_direct(q, ps.mass, None, np.arange(n), oracle_params(ps, L))
        for a, p in ((ag, pg), (af, pf)):
            assert np.max(relerr(a, ad)) < 1e-5 and np.max(np.abs(p - pd) / np.abs(pd)) < 1e-5
