"""GPU FMM (g4_gravity_fmm) against the FP64 oracle FMM: the same dual walk over pairs of nodes
or particles (node-node, particle-node and particle-particle interactions), fields both ways,
L2L/L2P downward pass (Sec. 2.4); plus momentum conservation and the alpha = 0 limit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2010_03567_gb300 import g4, synth  # noqa: E402

from _helpers import gpu_params, int_coords, oracle_params, relerr, to_dev, u32_dev  # noqa: E402

pytestmark = pytest.mark.gpu


def gpu_fmm(ps, q, P, aold, cls=False):
    """GPU FMM through the C ABI; caller order.  Counts (n, 3): particle pairs, particle-node
    terms, node-node fields of each particle.  cls: pass the softening classes."""
    tg = g4.TreeGravity(ps.n, P, with_cls=cls)
    tg.prepare(u32_dev(torch, q), to_dev(torch, ps.mass, torch.float32),
               to_dev(torch, ps.eps_class, torch.uint8) if cls else None,
               None if aold is None else to_dev(torch, aold, torch.float32), P)
    acc, pot, cnt, mom = tg.tree.gravity_fmm(tg.pos_s, tg.mass_s, tg.cls_s if cls else None,
                                             None if aold is None else tg.aold_s, P)
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


def oracle_fmm(ps, q, OP, aold, leaf=8, cls=False):
    """Oracle FMM; caller order.  Returns acc, pot, totals [NN, PN, PP], per-particle counts
    (n, 2): particle pairs, particle-node terms."""
    run = oracle.prepare(q, ps.mass, ps.eps_class if cls else None, aold, OP, leaf)
    acc_s, pot_s, cnt, pc_s = run.tree.fmm(OP, per_particle=True)
    a = np.empty_like(acc_s)
    a[run.perm] = acc_s
    p = np.empty_like(pot_s)
    p[run.perm] = pot_s
    pc = np.empty_like(pc_s)
    pc[run.perm] = pc_s
    return a, p, cnt, pc


def same_counts(cg, pc, frac=0.99):
    """At least `frac` of the particles see exactly the oracle's particle pairs and
    particle-node terms (FP32 decisions may fall on the other side of a threshold)."""
    same = (cg[:, 0] == pc[:, 0]) & (cg[:, 1] == pc[:, 1])
    return np.mean(same) >= frac


def _plummer(n=16384):
    ps = synth.plummer(n, 1001) if n != 16384 else synth.plummer_16k()
    q, box = int_coords(ps)
    ad, _ = oracle.direct(q, ps.mass, None, np.arange(ps.n), oracle_params(ps, box))
    return ps, q, box, np.linalg.norm(ad, axis=1).astype(np.float32), ad


def test_fmm_parity_plummer_p4():
    ps, q, box, aold, ad = _plummer()
    kw = dict(alpha=0.0025, order_p=4)
    ag, pg, cg, mom = gpu_fmm(ps, q, gpu_params(g4, ps, box, **kw), aold)
    ao, po, co, pc = oracle_fmm(ps, q, oracle_params(ps, box, **kw), aold.astype(np.float64))
    # the paper's three kinds of FMM interaction all occur (Sec. 3.2 counts them)
    assert co[0] > 0 and co[1] > 0 and co[2] > 0
    assert same_counts(cg, pc)
    assert abs(cg[:, 1].sum() - co[1]) <= 0.01 * co[1]
    assert abs(cg[:, 0].sum() - 2 * co[2]) <= 0.01 * 2 * co[2]
    e = relerr(ag, ao)
    assert np.percentile(e, 99) < 1e-5, np.percentile(e, [50, 99, 100])
    assert np.percentile(np.abs(pg - po) / np.abs(po), 99) < 1e-5
    # manifest momentum conservation (FP32 accumulation): sum m a ~ 0
    m = ps.mass
    rel = np.linalg.norm(mom) / np.sum(m * np.linalg.norm(ag, axis=1))
    assert rel < 1e-5, rel
    assert np.percentile(relerr(ag, ad), 99) < 2e-2


@pytest.mark.parametrize("order", [2, 3, 5])
def test_fmm_parity_orders_geometric(order):
    ps, q, box, aold, _ = _plummer(4000)
    kw = dict(criterion=1, theta=0.4, order_p=order)
    ag, pg, cg, _ = gpu_fmm(ps, q, gpu_params(g4, ps, box, **kw), None)
    ao, po, co, pc = oracle_fmm(ps, q, oracle_params(ps, box, **kw), None)
    assert co[1] > 0 and same_counts(cg, pc)
    assert np.percentile(relerr(ag, ao), 99) < 1e-5


def test_fmm_parity_treepm_box():
    L = 32 * 1.953125
    ps = synth.zeldovich(32, L, 2.0, 1003)
    q, box = int_coords(ps)
    kw = dict(alpha=0.0025, order_p=4, r_s=1.25 * L / 64, r_cut_factor=4.5)
    OP = oracle_params(ps, box, **kw)
    ad, _ = oracle.direct(q, ps.mass, None, np.arange(ps.n), OP, r_max=OP.r_cut)
    aold = np.linalg.norm(ad, axis=1).astype(np.float32)
    ag, pg, cg, mom = gpu_fmm(ps, q, gpu_params(g4, ps, box, **kw), aold)
    ao, po, co, pc = oracle_fmm(ps, q, OP, aold.astype(np.float64))
    assert same_counts(cg, pc)
    assert np.percentile(relerr(ag, ao), 99) < 1e-5
    # the FMM's own error against the hard-cutoff direct sum (shared by the oracle FMM):
    # node pairs straddling r_cut and the sink-side expansion (Sec. 3.1) at alpha = 0.0025
    eo = np.percentile(relerr(ao, ad), 99)
    assert np.percentile(relerr(ag, ad), 99) < 1.1 * eo + 1e-5 and eo < 1e-2


def test_fmm_parity_treepm_box_bench_leaf():
    """The bench's FMM configuration (leaf 32, p = 4, alpha = 0.0025, the same spacing and split
    as the 256^3 box) on a 40^3 box the oracle's FMM finishes in seconds."""
    L = 40 * 1.953125
    ps = synth.zeldovich(40, L, 2.0, 1013)
    q, box = int_coords(ps)
    kw = dict(alpha=0.0025, order_p=4, r_s=1.25 * L / 80, r_cut_factor=4.5, leaf_max=32)
    OP = oracle_params(ps, box, **kw)
    ad, _ = oracle.direct(q, ps.mass, None, np.arange(ps.n), OP, r_max=OP.r_cut)
    aold = np.linalg.norm(ad, axis=1).astype(np.float32)
    ag, pg, cg, mom = gpu_fmm(ps, q, gpu_params(g4, ps, box, **kw), aold)
    ao, po, co, pc = oracle_fmm(ps, q, OP, aold.astype(np.float64), leaf=32)
    assert same_counts(cg, pc)
    assert np.percentile(relerr(ag, ao), 99) < 1e-5
    rel = np.linalg.norm(mom) / np.sum(ps.mass * np.linalg.norm(ag, axis=1))
    assert rel < 1e-5, rel


@pytest.mark.parametrize("case", ["plummer", "treepm_box"])
def test_fmm_fp64_mode(case):
    """The FP64 reference mode (precision 1: FP64 node data, expansions, fields and particle
    pairs; decisions as in FP32): the same interactions as the oracle's FP64 FMM for >= 99% of
    the particles, and there agreement to the FP32 rounding of the outputs; closer to the
    oracle than the FP32 mode; momentum conserved to the outputs' rounding."""
    if case == "plummer":
        ps, q, box, aold, _ = _plummer(6000)
        kw = dict(alpha=0.0025, order_p=4)
        OP = oracle_params(ps, box, **kw)
        leaf = 8
    else:
        L = 24 * 1.953125
        ps = synth.zeldovich(24, L, 2.0, 1023)
        q, box = int_coords(ps)
        kw = dict(alpha=0.0025, order_p=4, r_s=1.25 * L / 48, r_cut_factor=4.5, leaf_max=32)
        OP = oracle_params(ps, box, **kw)
        ad, _ = oracle.direct(q, ps.mass, None, np.arange(ps.n), OP, r_max=OP.r_cut)
        aold = np.linalg.norm(ad, axis=1).astype(np.float32)
        leaf = 32
    ao, po, co, pc = oracle_fmm(ps, q, OP, aold.astype(np.float64), leaf=leaf)
    a32, _, c32, _ = gpu_fmm(ps, q, gpu_params(g4, ps, box, **kw), aold)
    a64, p64, c64, mom = gpu_fmm(ps, q, gpu_params(g4, ps, box, precision=1, **kw), aold)
    # FP32 decisions in both modes (on node records rounded from FP64 moments in this mode)
    assert np.mean(np.all(c64 == c32, axis=1)) >= 0.999
    assert same_counts(c64, pc)
    same = (c64[:, 0] == pc[:, 0]) & (c64[:, 1] == pc[:, 1])
    e64, e32 = relerr(a64, ao), relerr(a32, ao)
    assert np.percentile(e64[same], 99) < 5e-7, np.percentile(e64[same], [50, 99, 100])
    assert np.percentile(e64[same], 99) < 0.5 * np.percentile(e32[same], 99)
    assert np.percentile(np.abs(p64 - po)[same] / np.abs(po[same]), 99) < 5e-7
    rel = np.linalg.norm(mom) / np.sum(ps.mass * np.linalg.norm(a64, axis=1))
    assert rel < 1e-6, rel


def test_fmm_fp64_mode_needs_order4_and_fp64_moments():
    ps, q, box, aold, _ = _plummer(2000)
    tg = g4.TreeGravity(ps.n, gpu_params(g4, ps, box, alpha=0.0025, order_p=3))
    P3 = gpu_params(g4, ps, box, alpha=0.0025, order_p=3, precision=1)
    tg.prepare(u32_dev(torch, q), to_dev(torch, ps.mass, torch.float32), None,
               to_dev(torch, aold, torch.float32), P3)
    with pytest.raises(g4.G4Error, match="order_p 4"):
        tg.tree.gravity_fmm(tg.pos_s, tg.mass_s, None, tg.aold_s, P3)
    P4 = gpu_params(g4, ps, box, alpha=0.0025, order_p=4)
    tg.prepare(u32_dev(torch, q), to_dev(torch, ps.mass, torch.float32), None,
               to_dev(torch, aold, torch.float32), P4)           # FP32 multipoles only
    P4d = gpu_params(g4, ps, box, alpha=0.0025, order_p=4, precision=1)
    with pytest.raises(g4.G4Error, match="FP64 multipoles"):
        tg.tree.gravity_fmm(tg.pos_s, tg.mass_s, None, tg.aold_s, P4d)


def test_fmm_alpha0_is_direct_sum():
    ps, q, box, aold, ad = _plummer(3000)
    kw = dict(alpha=0.0, order_p=4)
    ag, pg, cg, _ = gpu_fmm(ps, q, gpu_params(g4, ps, box, **kw), aold)
    assert np.all(cg[:, 1] == 0) and np.all(cg[:, 2] == 0)
    assert np.all(cg[:, 0] == ps.n - 1)   # every pair, directly
    ad2, pd = oracle.direct(q, ps.mass, None, np.arange(ps.n), oracle_params(ps, box))
    assert np.percentile(relerr(ag, ad2), 99) < 1e-5


def test_fmm_inwalk_leaf_leaf_when_lists_are_full():
    """With the deferred particle-pair lists almost empty (one entry per particle) the dual walk
    evaluates the overflowing pairs itself: same interactions, same forces to rounding as the
    deferred pass."""
    L = 24 * 1.953125
    ps = synth.zeldovich(24, L, 2.0, 1003)
    q, box = int_coords(ps)
    kw = dict(criterion=1, theta=0.5, order_p=4, r_s=1.25 * L / 48, r_cut_factor=4.5, leaf_max=8)
    a0, p0, c0, _ = gpu_fmm(ps, q, gpu_params(g4, ps, box, **kw), None)
    a1, p1, c1, _ = gpu_fmm(ps, q, gpu_params(g4, ps, box, fmm_p2p_per_particle=1, **kw), None)
    assert np.array_equal(c0, c1)
    assert np.percentile(relerr(a1, a0), 99) < 2e-5


def test_fmm_sparse_leaves_keep_pairs_near_cutoff():
    """Sparse pairs 0.99 r_cut apart: sink leaves span many r_cut, beyond the range where the
    FP16 candidate test is exact; the particle-pair pass must still keep every pair."""
    L = 1.0
    rc = L / 1000
    ps = synth.sparse_pairs(2048, L, 0.99 * rc, 7001)
    q, box = int_coords(ps)
    kw = dict(alpha=0.0, order_p=4, r_s=rc / 4.5, r_cut_factor=4.5)
    aold = np.ones(ps.n, np.float32)   # alpha = 0: particle pairs only
    ag, pg, cg, _ = gpu_fmm(ps, q, gpu_params(g4, ps, box, **kw), aold)
    assert np.all(cg[:, 1] == 0) and np.all(cg[:, 2] == 0)
    OP = oracle_params(ps, box, **kw)
    ad, _ = oracle.direct(q, ps.mass, None, np.arange(ps.n), OP, r_max=OP.r_cut)
    # a dropped partner would leave its particle with no force at all
    assert np.percentile(relerr(ag, ad), 99) < 1e-5 and relerr(ag, ad).max() < 1e-3


def test_fmm_parity_two_softening_classes_leaf_above_32():
    """Leaves of up to 48 particles (two 32-sink chunks per leaf: the particle walk and the
    particle pairs per chunk) and two softening classes (eps_ij = max(eps_i, eps_j)); the
    same interactions as the oracle."""
    ps = synth.plummer(6000, 1101)
    ps.eps_class[::3] = 1
    ps.eps_table = np.array([0.01, 0.03])
    q, box = int_coords(ps)
    OPd = oracle_params(ps, box)
    cls = ps.eps_class
    ad, _ = oracle.direct(q, ps.mass, cls, np.arange(ps.n), OPd)
    aold = np.linalg.norm(ad, axis=1).astype(np.float32)
    kw = dict(alpha=0.001, order_p=3, leaf_max=48)
    P = gpu_params(g4, ps, box, **kw)
    tg = g4.TreeGravity(ps.n, P, with_cls=True)
    tg.prepare(u32_dev(torch, q), to_dev(torch, ps.mass, torch.float32),
               to_dev(torch, cls, torch.uint8), to_dev(torch, aold, torch.float32), P)
    acc, pot, cnt, _ = tg.tree.gravity_fmm(tg.pos_s, tg.mass_s, tg.cls_s, tg.aold_s, P)
    torch.cuda.synchronize()
    tg.tree.status()
    perm = tg.perm.cpu().numpy()
    ag = np.empty((ps.n, 3))
    ag[perm] = acc.cpu().numpy().T
    cg = np.empty((ps.n, 3), np.int64)
    cg[perm] = cnt.cpu().numpy().T
    OP = oracle_params(ps, box, **kw)
    run = oracle.prepare(q, ps.mass, cls, aold.astype(np.float64), OP, 48)
    acc_s, _, co, pc_s = run.tree.fmm(OP, per_particle=True)
    ao = np.empty_like(acc_s)
    ao[run.perm] = acc_s
    pc = np.empty_like(pc_s)
    pc[run.perm] = pc_s
    assert co[1] > 0
    assert same_counts(cg, pc)
    assert np.percentile(relerr(ag, ao), 99) < 1e-5


def test_fmm_parity_softened_node_rule():
    """The FMM under GADGET-4's softened-node rule (Sec. 2.7, soft_nodes = 1; node-node and
    particle-node pairs closer than 2.8 eps_ij use the softened kernel unless both sides are
    mixed) against the oracle's, with two softening classes mixed through every node; the
    GADGET-3 rule on the same set evaluates more particle pairs."""
    ps = synth.plummer(2000, 65)
    ps.eps_table = np.array([0.08, 0.3])
    ps.eps_class[::4] = 1
    q, box = int_coords(ps)
    ad, _ = oracle.direct(q, ps.mass, ps.eps_class, np.arange(ps.n), oracle_params(ps, box))
    aold = np.linalg.norm(ad, axis=1).astype(np.float32)
    pp = {}
    for soft in (0, 1):
        kw = dict(alpha=0.005, order_p=4, leaf_max=4, soft_nodes=soft)
        ag, pg, cg, mom = gpu_fmm(ps, q, gpu_params(g4, ps, box, **kw), aold, cls=True)
        ao, po, co, pc = oracle_fmm(ps, q, oracle_params(ps, box, **kw), aold.astype(np.float64),
                                    leaf=4, cls=True)
        assert same_counts(cg, pc), soft
        e = relerr(ag, ao)
        assert np.percentile(e, 99) < 1e-5, (soft, np.percentile(e, [50, 99, 100]))
        assert np.percentile(np.abs(pg - po) / np.abs(po), 99) < 1e-5
        assert np.percentile(relerr(ag, ad), 99) < 0.01
        amag = np.linalg.norm(ag, axis=1)
        assert np.linalg.norm(mom) < 1e-5 * np.sum(ps.mass * amag)
        pp[soft] = co[2]
    assert pp[1] < pp[0], pp


@pytest.mark.parametrize("n", [1, 2, 3, 33])
def test_fmm_small_and_degenerate_sets(n):
    """One particle (no force, no potential), two, three, and 33 particles of which 20 share
    one position (leaves at key resolution above leaf_max): the FMM against the oracle's."""
    ps = synth.plummer(max(n, 1), 91 + n)
    if n == 33:
        ps.pos[1:20] = ps.pos[0]
    q, box = int_coords(ps)
    kw = dict(criterion=1, theta=0.5, order_p=3)
    ag, pg, cg, mom = gpu_fmm(ps, q, gpu_params(g4, ps, box, **kw), None)
    ao, po, co, pc = oracle_fmm(ps, q, oracle_params(ps, box, **kw), None)
    if n == 1:
        assert np.all(ag == 0) and np.all(pg == 0)
    else:
        assert np.allclose(ag, ao, rtol=1e-5, atol=1e-6 * np.abs(ao).max())
        assert np.allclose(pg, po, rtol=1e-5)
