"""Active subsets of hierarchical time bins (g4.BinnedForces: each force call builds its tree
over the active particles only, Sec. 4.2) on a zoom box with two softening classes
(eps_ij = max(eps_i, eps_j), Sec. 2.7), compared bin by bin, sink by sink with the FP64 oracle's
tree walk over the same subset: 99th-percentile force error 1e-5 and identical interaction
counts for at least 99% of the sinks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2010_03567_gb300 import g4, synth  # noqa: E402

from _helpers import oracle_params, relerr, to_dev, u32_dev  # noqa: E402

pytestmark = pytest.mark.gpu

PARITY_P99 = 1e-5


def test_binned_subsets_two_softening_classes_match_oracle():
    L = 100.0
    ps = synth.zoom(32, L, 1004)
    n = ps.n
    assert set(np.unique(ps.eps_class)) == {0, 1}
    q = oracle.int_coords_periodic(ps.pos, L)
    base = dict(r_s=1.25 * L / 64, r_cut_factor=4.5)
    OPd = oracle_params(ps, L, **base)
    # |a_old| from the oracle's FP64 short-range direct sum, rounded to FP32 for both sides
    ad, _ = oracle.direct(q, ps.mass, ps.eps_class, np.arange(n), OPd, r_max=OPd.r_cut)
    aold = np.linalg.norm(ad, axis=1).astype(np.float32)
    order = np.argsort(-aold, kind="stable")
    lists = [np.sort(order[:max(32, int(f * n))]) for f in (0.03, 0.3, 1.0)]
    kw = dict(alpha=0.0025, order_p=3, **base)
    P = g4.params(box_size=L, periodic=1, eps=list(ps.eps_table), leaf_max=16, **kw)
    bf = g4.BinnedForces(n, lists, P, with_cls=True)
    bf.run(u32_dev(torch, q), to_dev(torch, ps.mass, torch.float32),
           to_dev(torch, ps.eps_class, torch.uint8), to_dev(torch, aold, torch.float32))
    torch.cuda.synchronize()
    OP = oracle_params(ps, L, **kw)
    for b, ix in enumerate(lists):
        tg = bf.bins[b][0]
        tg.tree.status()
        ag = bf.acc[b].cpu().numpy().T[ix].astype(np.float64)
        pg = bf.pot[b].cpu().numpy()[ix].astype(np.float64)
        perm = tg.perm.cpu().numpy()
        cg = np.empty((len(ix), 2), np.int64)
        cg[perm] = tg.counts.cpu().numpy().T
        run = oracle.prepare(np.ascontiguousarray(q[:, ix]), ps.mass[ix], ps.eps_class[ix],
                             aold[ix].astype(np.float64), OP, 16)
        ao, po, co = oracle.tree_forces(run, np.arange(len(ix)))
        e = relerr(ag, ao)
        assert np.percentile(e, 99) < PARITY_P99, (b, np.percentile(e, [50, 99, 100]))
        # sinks with no source inside r_cut (a sparse subset has some): exactly zero on both
        z = np.linalg.norm(ao, axis=1) == 0
        assert np.all(ag[z] == 0) and np.all(pg[z] == 0)
        assert np.percentile(np.abs(pg[~z] - po[~z]) / np.abs(po[~z]), 99) < PARITY_P99
        assert np.mean(np.all(cg == co, axis=1)) > 0.99
        # both softening classes are present among the bin's sinks
        assert len(np.unique(ps.eps_class[ix])) == 2 or len(ix) < 64
