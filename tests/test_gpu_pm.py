"""GPU particle-mesh long-range force (g4_pm_long_range, Sec. 2.3) against the FP64 PM oracle
(oracle/pm.py: the same CIC -> FFT -> Green's function with sinc deconvolution -> FD4 -> CIC
steps) and, with the tree's short-range force added, against the periodic Ewald sum
(Sec. 2.1), the exact periodic force.

Tolerances.  The GPU mesh is FP32 (CIC sums by atomics, 2 x 3 FFT passes of log2 N radix-2
stages): the potential carries relative rounding ~1e-6 of its own scale; fourth-order
differences of neighbouring mesh values lose up to ~two more digits where the long-range field
is smooth, so the per-particle long-range force is compared at 1e-4 (99th percentile) of the
particle's long-range force.  Against Ewald, the total force's error is the PM method's own
(about 1% at most at the matching scale for A_smth = 1.25, Sec. 3.4): the GPU may exceed the
FP64 oracle's error there by the PM rounding only."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from oracle import pm  # noqa: E402
from paper_2010_03567_gb300 import g4  # noqa: E402

from _helpers import relerr, to_dev, u32_dev  # noqa: E402

pytestmark = pytest.mark.gpu


def _points(rng, n, L):
    x = rng.uniform(0, L, (n, 3))
    q = np.floor(x / L * 2 ** 32).astype(np.uint64).astype(np.uint32)
    return q.T.copy(), q.astype(np.float64) * L / 2 ** 32


@pytest.mark.parametrize("n_grid", [16, 64, 128])
def test_pm_parity_with_oracle(n_grid):
    L = 10.0
    rng = np.random.default_rng(11 + n_grid)
    q, _ = _points(rng, 20000, L)
    m = rng.uniform(0.5, 1.5, 20000)
    rs = 1.25 * L / n_grid
    ao, po = pm.long_range(q, m, n_grid, L, rs)
    P = g4.params(box_size=L, periodic=1, r_s=rs)
    ag, pg = g4.g4_pm_long_range(u32_dev(torch, q), to_dev(torch, m, torch.float32), P, n_grid)
    torch.cuda.synchronize()
    ag = ag.cpu().numpy().T.astype(np.float64)
    pg = pg.cpu().numpy().astype(np.float64)
    assert np.percentile(relerr(ag, ao), 99) < 1e-4, np.percentile(relerr(ag, ao), [50, 99, 100])
    assert np.percentile(np.abs(pg - po) / np.abs(po).max(), 99) < 1e-5
    # momentum: the same kernel for assignment and interpolation and an antisymmetric
    # difference operator conserve it (up to FP32 rounding here)
    mom = np.linalg.norm((m[:, None] * ag).sum(0)) / np.sum(m * np.linalg.norm(ag, axis=1))
    assert mom < 1e-5, mom


def test_pm_separate_sinks_and_accumulate():
    L, N = 1.0, 32
    rng = np.random.default_rng(5)
    q, _ = _points(rng, 3000, L)
    qs, _ = _points(rng, 500, L)
    m = np.full(3000, 1.0 / 3000)
    rs = 1.25 * L / N
    ao, _ = pm.long_range(q, m, N, L, rs, sinks=qs)
    P = g4.params(box_size=L, periodic=1, r_s=rs)
    base = torch.ones((3, 500), dtype=torch.float32, device="cuda")
    ag, _ = g4.g4_pm_long_range(u32_dev(torch, q), to_dev(torch, m, torch.float32), P, N,
                                sinks=u32_dev(torch, qs), acc=base, accumulate=True)
    torch.cuda.synchronize()
    a = ag.cpu().numpy().T.astype(np.float64) - 1.0
    assert np.percentile(relerr(a, ao), 99) < 1e-4


def test_pm_lattice_zero_force():
    L, N = 4.0, 32
    i = np.arange(N, dtype=np.uint64) * (2 ** 32 // N)
    gx, gy, gz = np.meshgrid(i, i, i, indexing="ij")
    q = np.stack([gx.ravel(), gy.ravel(), gz.ravel()]).astype(np.uint32)
    P = g4.params(box_size=L, periodic=1, r_s=1.25 * L / N)
    ag, _ = g4.g4_pm_long_range(u32_dev(torch, q), torch.ones(q.shape[1], device="cuda"), P, N)
    torch.cuda.synchronize()
    assert float(ag.abs().max()) < 1e-4


def test_treepm_total_force_against_ewald():
    """Short-range tree walk plus PM long range (g4.TreePMGravity) on a random periodic set:
    the total force against the Ewald sum, as accurate as the FP64 oracle's PM + direct short
    range; the relative criterion is fed the total |a| (Sec. 2.3 footnote)."""
    L, n, N = 1.0, 4096, 32
    rng = np.random.default_rng(3)
    q, x = _points(rng, n, L)
    m = np.full(n, 1.0 / n)
    rs = 1.25 * L / N
    eps = L / N / 300.0
    sinks = np.arange(0, n, 16)
    a_ew = oracle.ewald_force(x[sinks], x, m, L, 2.0 / L, 3, 5)
    OP = oracle.OracleParams(box=L, periodic=True, eps=np.array([eps]), r_s=rs, r_cut_factor=4.5)
    a_sr, _ = oracle.direct(q, m, None, sinks, OP, r_max=OP.r_cut)
    a_lr, _ = pm.long_range(q, m, N, L, rs, sinks=np.ascontiguousarray(q[:, sinks]))
    e_or = relerr(a_sr + a_lr, a_ew)
    kw = dict(box_size=L, periodic=1, r_s=rs, r_cut_factor=4.5, eps=[eps], leaf_max=8)
    tp = g4.TreePMGravity(n, g4.params(**kw, criterion=1, theta=0.5), N)
    pos, mass = u32_dev(torch, q), to_dev(torch, m, torch.float32)
    a0, _ = tp.forces(pos, mass)                          # bootstrap (geometric criterion)
    aold = torch.linalg.vector_norm(a0, dim=0).contiguous()
    ag, _ = tp.forces(pos, mass, None, aold, g4.params(**kw, alpha=0.0025))
    torch.cuda.synchronize()
    e_gpu = relerr(ag.cpu().numpy().T[sinks].astype(np.float64), a_ew)
    assert np.percentile(e_gpu, 99) < 1.1 * np.percentile(e_or, 99) + 1e-4
    assert np.median(e_gpu) < 1.1 * np.median(e_or) + 1e-4
    assert np.percentile(e_or, 99) < 0.05   # the PM method's own error at A_smth = 1.25
