"""Pins of the oracle's hierarchical time integration (Sec. 4.2; CPU only).

* the recursion equals the paper's operator sequence written out: for one level of fast
  particles, K_P^P(dt/2) K_F^F(-dt/2) E(H_F, dt/2) D_S(dt) E(H_F, dt/2) K_F^F(-dt/2) K_P^P(dt/2)
  with E(H_F, dt/2) a kick-drift-kick of F alone;
* with forces whose sources and sinks coincide (direct sum), the total momentum is conserved
  to roundoff however deep the hierarchy (Sec. 4.2: manifest momentum conservation);
* with a single level it is the leapfrog: energy errors of a two-body orbit fall as dt^2.
"""
import numpy as np

import oracle
from oracle import hierarchy as H
from paper_2010_03567_gb300 import synth


def _setup(n=256, seed=5):
    ps = synth.plummer(n, seed)
    q, frame = oracle.int_coords_isolated(ps.pos * 0.5)     # central quarter of the cube
    L = frame[3]
    rng = np.random.default_rng(seed)
    vel = rng.normal(scale=0.3, size=(n, 3))
    eps = np.full(n, 0.01)
    P = oracle.OracleParams(box=L, periodic=False, eps=np.array([0.01]))
    st = H.State(q, vel, ps.mass, L, eps)

    def force(idx):
        acc = np.zeros((n, 3))
        a, _ = oracle.direct(np.ascontiguousarray(st.pos[:, idx]), st.mass[idx], None,
                             np.arange(len(idx)), P)
        acc[idx] = a
        return acc
    return st, force


def test_recursion_is_the_operator_sequence():
    st, force = _setup()
    all_ = np.arange(st.pos.shape[1])
    acc = force(all_)
    a = np.linalg.norm(acc, axis=1)
    dt = 2.0 * np.sqrt(2 * 0.02 * 0.01 / np.median(a))    # about half of the particles fast
    st2 = H.State(st.pos, st.vel, st.mass, st.L, st.eps)
    H.step(st, all_, dt, acc, force, eta=0.02, max_level=1)
    # the same step written out (one level: F advanced by two kick-drift-kick half steps)
    f2 = lambda idx: _force_on(st2, idx)
    dti = np.sqrt(2 * 0.02 * st2.eps / a)
    F, S = all_[dti < dt], all_[dti >= dt]
    assert 0 < len(F) < len(all_)
    H.kick(st2, all_, acc, dt / 2)                       # K_P^P(dt/2)
    aF = f2(F)
    H.kick(st2, F, aF, -dt / 2)                          # K_F^F(-dt/2)
    for half in range(2):
        H.kick(st2, F, aF, dt / 4)                       # E(H_F, dt/2): K D K on F alone
        H.drift(st2, F, dt / 2)
        aF = f2(F)
        H.kick(st2, F, aF, dt / 4)
        if half == 0:
            H.drift(st2, S, dt)                          # D_S(dt)
    H.kick(st2, F, aF, -dt / 2)                          # K_F^F(-dt/2)
    aP = f2(all_)
    H.kick(st2, all_, aP, dt / 2)                        # K_P^P(dt/2)
    assert np.array_equal(st.pos, st2.pos)
    assert np.max(np.abs(st.vel - st2.vel)) <= 1e-14 * np.max(np.abs(st.vel))


def _force_on(st, idx):
    n = st.pos.shape[1]
    P = oracle.OracleParams(box=st.L, periodic=False, eps=np.array([0.01]))
    acc = np.zeros((n, 3))
    a, _ = oracle.direct(np.ascontiguousarray(st.pos[:, idx]), st.mass[idx], None,
                         np.arange(len(idx)), P)
    acc[idx] = a
    return acc


def test_momentum_conserved_through_the_hierarchy():
    st, force = _setup(300, 9)
    all_ = np.arange(300)
    acc = force(all_)
    a = np.linalg.norm(acc, axis=1)
    dt = 8.0 * np.sqrt(2 * 0.02 * 0.01 / np.median(a))    # several levels
    p0 = (st.mass[:, None] * st.vel).sum(0)
    scale = np.sum(st.mass * np.linalg.norm(st.vel, axis=1))
    n0 = 0
    for _ in range(3):
        acc = H.step(st, all_, dt, acc, force, eta=0.02, max_level=6)
        assert st.n_force > n0
        n0 = st.n_force
    p1 = (st.mass[:, None] * st.vel).sum(0)
    assert np.linalg.norm(p1 - p0) < 1e-13 * scale
    assert st.n_force > 3 * 2 * 300        # fast particles took extra force computations


def test_single_level_is_second_order():
    L = 4.0
    errs = []
    for nsteps in (100, 200):
        # two equal masses on an eccentric orbit (0.8 of the circular speed at separation 1;
        # G = 1, unsoftened range)
        x = np.array([[-0.5, 0, 0], [0.5, 0, 0]]) + 0.5 * L
        q = np.floor(x / L * 2 ** 32).astype(np.uint64).astype(np.uint32).T.copy()
        v = 0.8 * np.sqrt(1.0 / 2.0)             # circular: v^2 / r = m / d^2, r = 1/2, d = 1
        vel = np.array([[0, -v, 0], [0, v, 0]])
        st = H.State(q, vel, np.ones(2), L, np.full(2, 1e-4))
        P = oracle.OracleParams(box=L, periodic=False, eps=np.array([1e-4]))

        def force(idx, st=st, P=P):
            acc = np.zeros((2, 3))
            a, _ = oracle.direct(np.ascontiguousarray(st.pos[:, idx]), st.mass[idx], None,
                                 np.arange(len(idx)), P)
            acc[idx] = a
            return acc

        def energy():
            d = (st.pos[:, 1].astype(np.int64) - st.pos[:, 0].astype(np.int64)) * L / 2 ** 32
            return 0.5 * np.sum(st.vel ** 2) - 1.0 / np.linalg.norm(d)

        period = 2 * np.pi / np.sqrt(2.0)        # of the circular orbit: omega^2 = 2 m / d^3
        dt = period / nsteps
        e0 = energy()
        acc = force(np.arange(2))
        emax = 0.0
        for _ in range(nsteps):
            acc = H.step(st, np.arange(2), dt, acc, force, eta=1e9, max_level=0)
            emax = max(emax, abs(energy() - e0))
        errs.append(emax)
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.0, ratio
