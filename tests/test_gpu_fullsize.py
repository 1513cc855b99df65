"""Parity at the full sizes of the bench's workloads, in the configuration bench.py times
(TreeGravity.forces: keys, sort, gather, build, multipoles, walk, scatter; leaf 32, p = 3,
alpha = 0.0025, 5-block register cap), on outputs the oracle computes one by one.

* 256^3 clustered box (the headline workload): keys and permutation bit-exact, tree topology
  bit-exact, and the walk's forces of 1024 sampled sinks against the oracle's same-algorithm
  FP64 walk (99th percentile 1e-5, identical interaction counts for >= 99% of them) and
  against the FP64 direct sum over r < r_cut (99th percentile 1e-3).
* 512^3 box (drawn on the GPU by synth.zeldovich_gpu; too large for the oracle's tree): the
  walk's forces of 512 sampled sinks against the oracle's FP64 direct sum over r < r_cut.
* the FMM in the bench's configuration (256^3 box, leaf 32, p = 4): 1024 sampled sinks against
  the oracle's FP64 direct sum over r < r_cut, and total momentum (Sec. 2.4: conserved to
  the FP32 rounding of the sum); its same-algorithm parity is tested at 40^3 with the same
  spacing, split, leaf size and order (tests/test_gpu_fmm.py).

|a_old| is a caller input of the relative criterion; both sides get the same constant."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2010_03567_gb300 import g4, synth  # noqa: E402

from _helpers import relerr, u32_dev  # noqa: E402

pytestmark = pytest.mark.gpu

AOLD = 20.0   # |a_old| of every particle (the box's typical short-range |a| is O(10))


def _params(n_side, L):
    return dict(box_size=L, periodic=1, r_s=1.25 * L / (2 * n_side), r_cut_factor=4.5,
                eps=[L / n_side / 30.0], alpha=0.0025, order_p=3, leaf_max=32)


def test_fullsize_256cubed_keys_tree_and_sampled_forces():
    n_side, L = 256, 500.0
    ps = synth.zeldovich(n_side, L, 2.0, 1003)
    q = oracle.int_coords_periodic(ps.pos, L)
    kw = _params(n_side, L)
    P = g4.params(**kw)
    tg = g4.TreeGravity(ps.n, P)
    pos = u32_dev(torch, q)
    mass = torch.from_numpy(ps.mass.astype(np.float32)).cuda()
    aold = torch.full((ps.n,), AOLD, dtype=torch.float32, device="cuda")
    acc, pot = tg.forces(pos, mass, None, aold, P)
    torch.cuda.synchronize()
    tg.tree.status()
    OP = oracle.OracleParams(box=L, periodic=True, eps=np.array(kw["eps"]), r_s=kw["r_s"],
                             r_cut_factor=4.5, alpha=0.0025, order=3)
    run = oracle.prepare(q, ps.mass, None, np.full(ps.n, AOLD), OP, 32)
    # keys, permutation, tree: bit-exact
    assert np.array_equal(tg.keys.cpu().numpy().view(np.uint64), run.keys_sorted)
    assert np.array_equal(tg.perm.cpu().numpy(), run.perm)
    gn = tg.tree.nodes()
    on = run.tree.export()
    assert gn["level"].shape[0] == on["level"].shape[0]
    for k in ("level", "first", "count", "next"):
        assert np.array_equal(gn[k].cpu().numpy(), on[k].astype(np.int32)), k
    # sampled forces
    sinks = synth.subset(ps.n, 1024, 2002)
    ao, po, co = oracle.tree_forces(run, sinks)
    ag = acc.cpu().numpy().T[sinks].astype(np.float64)
    assert np.percentile(relerr(ag, ao), 99) < 1e-5
    cs = tg.counts.cpu().numpy().T
    cnt = np.empty_like(cs)
    cnt[tg.perm.cpu().numpy()] = cs
    assert np.mean(np.all(cnt[sinks] == co, axis=1)) >= 0.99
    ad, _ = oracle.direct(q, ps.mass, None, sinks, OP, r_max=OP.r_cut)
    assert np.percentile(relerr(ag, ad), 99) < 1e-3


def test_fullsize_512cubed_sampled_forces_vs_direct():
    n_side, L = 512, 1000.0
    pos_f = synth.zeldovich_gpu(n_side, L, 0.5, 1006)
    n = n_side ** 3
    kw = _params(n_side, L)
    P = g4.params(**kw)
    q_dev, _ = g4.g4_int_coords(pos_f, True, L)
    tg = g4.TreeGravity(n, P)
    mass = torch.ones(n, dtype=torch.float32, device="cuda")
    aold = torch.full((n,), AOLD, dtype=torch.float32, device="cuda")
    acc, _ = tg.forces(q_dev, mass, None, aold, P)
    torch.cuda.synchronize()
    tg.tree.status()
    sinks = synth.subset(n, 512, 2006)
    ag = acc[:, torch.from_numpy(sinks).cuda()].cpu().numpy().T.astype(np.float64)
    del tg, acc, q_dev, mass, aold
    torch.cuda.empty_cache()
    q = oracle.int_coords_periodic(pos_f.cpu().numpy(), L)   # the oracle converts on its own
    del pos_f
    OP = oracle.OracleParams(box=L, periodic=True, eps=np.array(kw["eps"]), r_s=kw["r_s"],
                             r_cut_factor=4.5)
    ad, _ = oracle.direct(q, np.ones(n), None, sinks, OP, r_max=OP.r_cut)
    e = relerr(ag, ad)
    assert np.percentile(e, 99) < 1e-3, np.percentile(e, [50, 99, 100])


def test_fullsize_256cubed_fmm_sampled_forces_and_momentum():
    n_side, L = 256, 500.0
    ps = synth.zeldovich(n_side, L, 2.0, 1003)
    q = oracle.int_coords_periodic(ps.pos, L)
    kw = dict(_params(n_side, L), order_p=4)
    P = g4.params(**kw)
    tg = g4.TreeGravity(ps.n, P)
    pos = u32_dev(torch, q)
    mass = torch.from_numpy(ps.mass.astype(np.float32)).cuda()
    # |a_old| from the geometric bootstrap walk (as the bench does): the FMM's relative
    # criterion compares node-node errors with the smallest |a| of the pair, so a constant
    # |a_old| would not bound the error of weakly pulled particles
    a0, _ = tg.forces(pos, mass, None, None, g4.params(**dict(kw, order_p=3), criterion=1, theta=0.5))
    aold = torch.linalg.vector_norm(a0, dim=0).contiguous()
    tg.prepare(pos, mass, None, aold, P)
    acc_s, _, cnt, mom = tg.tree.gravity_fmm(tg.pos_s, tg.mass_s, None, tg.aold_s, P)
    acc, _ = g4.g4_scatter(tg.perm, acc_s)
    torch.cuda.synchronize()
    tg.tree.status()
    amag = torch.linalg.vector_norm(acc_s.double(), dim=0)
    rel_mom = float(torch.linalg.vector_norm(mom).item() / (tg.mass_s.double() * amag).sum().item())
    assert rel_mom < 1e-5, rel_mom
    c = cnt.to(torch.int64).sum(dim=1).cpu().numpy()
    assert c[0] > 0 and c[1] >= 0
    sinks = synth.subset(ps.n, 1024, 2002)
    ag = acc.cpu().numpy().T[sinks].astype(np.float64)
    OP = oracle.OracleParams(box=L, periodic=True, eps=np.array(kw["eps"]), r_s=kw["r_s"],
                             r_cut_factor=4.5)
    ad, _ = oracle.direct(q, ps.mass, None, sinks, OP, r_max=OP.r_cut)
    e = relerr(ag, ad)
    # the bench measures 1.2e-6 here: at alpha = 0.0025 almost all of the FMM's work is particle
    # pairs; the gate is the headline's 1e-3
    assert np.percentile(e, 99) < 1e-3, np.percentile(e, [50, 99, 100])
