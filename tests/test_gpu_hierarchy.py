"""Hierarchical time integration on the GPU (g4.HierarchicalKDK over g4_kick, g4_drift,
g4_timestep_bins and subset trees; Sec. 4.2) against the FP64 oracle integrator
(oracle/hierarchy.py) driven by the oracle's FMM with the same parameters, and the manifest
momentum conservation of the scheme with FMM forces (every force computation has equal source
and sink sets)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from oracle import hierarchy as H  # noqa: E402
from paper_2010_03567_gb300 import g4, synth  # noqa: E402

from _helpers import to_dev, u32_dev  # noqa: E402

pytestmark = pytest.mark.gpu


def _plummer_quarter(n, seed):
    """Plummer sphere in the central quarter of an isolated integer frame (room to drift)."""
    ps = synth.plummer(n, seed)
    ext = float(np.max(np.abs(ps.pos)))
    S = 2.0 ** np.ceil(np.log2(4.0 * ext))
    q = (np.floor(ps.pos / S * 2 ** 32) + 2 ** 31).astype(np.int64).astype(np.uint32).T.copy()
    rng = np.random.default_rng(seed)
    vel = rng.normal(scale=0.3, size=(n, 3))
    return ps, q, S, vel


def _dt_for_levels(q, ps, S, eps, eta, factor):
    OP = oracle.OracleParams(box=S, periodic=False, eps=np.array([eps]))
    a, _ = oracle.direct(q, ps.mass, None, np.arange(ps.n), OP)
    return factor * np.median(np.sqrt(2 * eta * eps / np.linalg.norm(a, axis=1)))


def test_gpu_hierarchy_matches_oracle_integrator():
    n, eps, eta = 1024, 0.01, 0.02
    ps, q, S, vel = _plummer_quarter(n, 12)
    dt = _dt_for_levels(q, ps, S, eps, eta, 4.0)
    kw = dict(box_size=S, periodic=0, eps=[eps], criterion=1, theta=0.5, order_p=4, leaf_max=8)
    P = g4.params(**kw)
    pos = u32_dev(torch, q)
    v = to_dev(torch, vel.T, torch.float32)
    m = to_dev(torch, ps.mass, torch.float32)
    hk = g4.HierarchicalKDK(pos, v, m, P, eta=eta, method="fmm", max_level=6)
    hk.step(dt)
    torch.cuda.synchronize()
    assert int(hk.flag.item()) == 0
    # the oracle: same scheme, FP64, the oracle FMM with the same parameters as the force
    OP = oracle.OracleParams(box=S, periodic=False, eps=np.array([eps]), criterion=1, theta=0.5, order=4)
    st = H.State(q, vel.astype(np.float32).astype(np.float64), ps.mass, S, np.full(n, eps))

    def force(idx):
        run = oracle.prepare(np.ascontiguousarray(st.pos[:, idx]), st.mass[idx], None, None, OP, 8)
        a_s, _, _ = run.tree.fmm(OP)
        acc = np.zeros((n, 3))
        sub = np.empty_like(a_s)
        sub[run.perm] = a_s
        acc[idx] = sub
        return acc

    all_ = np.arange(n)
    acc0 = force(all_)
    H.step(st, all_, dt, acc0, force, eta=eta, max_level=6)
    # force computations per particle inside the step (the GPU count also holds the initial
    # forces of all particles): the hierarchy had fast particles, and the same ones
    assert hk.n_force - n > 2 * n
    assert abs((hk.n_force - n) - st.n_force) <= 0.01 * st.n_force
    a_scale = np.linalg.norm(acc0, axis=1)
    dv = np.linalg.norm(hk.vel.cpu().numpy().T.astype(np.float64) - st.vel, axis=1) / (a_scale * dt)
    dx = (hk.pos.cpu().numpy().view(np.uint32).astype(np.int64) - st.pos.astype(np.int64)).T
    dx = np.linalg.norm(dx * (S / 2 ** 32), axis=1) / (a_scale * dt * dt)
    assert np.percentile(dv, 99) < 1e-3, np.percentile(dv, [50, 99, 100])
    assert np.percentile(dx, 99) < 1e-3, np.percentile(dx, [50, 99, 100])


def test_gpu_hierarchy_fmm_conserves_momentum():
    n, eps, eta = 2048, 0.01, 0.02
    ps, q, S, vel = _plummer_quarter(n, 21)
    vel -= np.average(vel, axis=0, weights=ps.mass)
    dt = _dt_for_levels(q, ps, S, eps, eta, 8.0)
    out = {}
    for method in ("fmm", "tree"):
        kw = dict(box_size=S, periodic=0, eps=[eps], criterion=1, theta=0.5, order_p=4, leaf_max=8)
        hk = g4.HierarchicalKDK(u32_dev(torch, q), to_dev(torch, vel.T, torch.float32),
                                to_dev(torch, ps.mass, torch.float32), g4.params(**kw), eta=eta,
                                method=method, max_level=8)
        hk.start()
        scale = float((hk.mass.double() * torch.linalg.vector_norm(hk.acc[0].double(), dim=0)).sum()) * dt
        p0 = hk.momentum()
        for _ in range(3):
            hk.step(dt)
        torch.cuda.synchronize()
        assert int(hk.flag.item()) == 0
        out[method] = float(torch.linalg.vector_norm(hk.momentum() - p0)) / scale
    # FMM: every kick is momentum-free up to FP32 rounding; the one-sided tree is not
    assert out["fmm"] < 1e-5, out
    assert out["fmm"] < out["tree"], out
