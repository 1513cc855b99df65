"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Integer work (coordinates, keys, sort permutation, tree topology, dyadic node masses)
must be bit-exact; forces must meet the 99th-percentile relative error 1e-5 against the
same-algorithm oracle (a few particles may differ where an FP32 opening decision lands on
the other side of the threshold than the FP64 one -- several results are then valid).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2010_03567_gb300 import g4, synth  # noqa: E402

from _helpers import (gpu_forces, gpu_params, int_coords, oracle_params, relerr, to_dev,  # noqa: E402
                      u32_dev, u32_host, u64_host)

pytestmark = pytest.mark.gpu

PARITY_P99 = 1e-5


def _treepm_box(n_side=32, rms=2.0, seed=1003):
    L = n_side * 1.953125          # same mean spacing as the 256^3, L = 500 workload
    ps = synth.zeldovich(n_side, L, rms, seed)
    return ps, dict(r_s=1.25 * L / (2 * n_side), r_cut_factor=4.5)


# ---- a1 / a2 / a3 ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["periodic", "isolated"])
def test_int_coords_bit_exact(kind):
    ps = synth.zeldovich(20, 7.0, 1.0, 3) if kind == "periodic" else synth.plummer(5000, 9)
    pos = torch.from_numpy(ps.pos).cuda()
    qg, frame = g4.g4_int_coords(pos, ps.periodic, ps.box_size)
    torch.cuda.synchronize()
    if ps.periodic:
        q = oracle.int_coords_periodic(ps.pos, ps.box_size)
        fr = np.array([0, 0, 0, ps.box_size])
    else:
        q, fr = oracle.int_coords_isolated(ps.pos)
    assert np.array_equal(u32_host(qg), q)
    assert np.array_equal(frame.cpu().numpy()[:4], fr)
    # a second call into the same frame buffer (its scratch part holds the first call's state)
    qg2, frame2 = g4.g4_int_coords(pos, ps.periodic, ps.box_size, frame=frame)
    assert np.array_equal(u32_host(qg2), q) and np.array_equal(frame2.cpu().numpy()[:4], fr)


@pytest.mark.parametrize("n", [1, 2, 7, 4095, 4096, 4097, 100003])
def test_keys_sort_bit_exact(n):
    g = np.random.default_rng(n)
    q = g.integers(0, 2 ** 32, size=(3, n), dtype=np.uint64).astype(np.uint32)
    if n > 10:
        q[:, n // 3: n // 3 + 50] = q[:, n // 3: n // 3 + 1]     # equal keys: stability
    keys, perm = g4.g4_keys_sort(u32_dev(torch, q))
    torch.cuda.synchronize()
    ko = oracle.keys(q)
    kso, permo = oracle.sort(ko)
    assert np.array_equal(u64_host(keys), kso)
    assert np.array_equal(perm.cpu().numpy().astype(np.int64), permo)


def test_keys_clustered_workload():
    ps, _ = _treepm_box(64)
    q, _ = int_coords(ps)
    keys, perm = g4.g4_keys_sort(u32_dev(torch, q))
    kso, permo = oracle.sort(oracle.keys(q))
    assert np.array_equal(u64_host(keys), kso)
    assert np.array_equal(perm.cpu().numpy().astype(np.int64), permo)


# ---- a4 / a5 ----------------------------------------------------------------------------------

def _tree_case(ps, leaf_max, order=3):
    q, box = int_coords(ps)
    P = gpu_params(g4, ps, box, leaf_max=leaf_max, order_p=order)
    tg = g4.TreeGravity(ps.n, P, with_cls=True)
    tg.prepare(u32_dev(torch, q), to_dev(torch, ps.mass, torch.float32),
               to_dev(torch, ps.eps_class, torch.uint8), None)
    torch.cuda.synchronize()
    OP = oracle_params(ps, box, order=order)
    run = oracle.prepare(q, ps.mass, ps.eps_class, None, OP, leaf_max)
    return tg, run, box


@pytest.mark.parametrize("case", ["plummer-8", "plummer-1", "box-4", "box-16", "tiny-3"])
def test_tree_topology_bit_exact(case):
    if case.startswith("plummer"):
        ps = synth.plummer_16k()
    elif case == "tiny-3":
        ps = synth.plummer(5, 2)
    else:
        ps, _ = _treepm_box(24)
    leaf = int(case.split("-")[1])
    tg, run, _ = _tree_case(ps, leaf)
    nd = {k: v.cpu().numpy() for k, v in tg.tree.nodes().items()}
    ot = run.tree.export()
    assert len(nd["level"]) == len(ot["level"])
    assert np.array_equal(nd["level"], ot["level"])
    assert np.array_equal(nd["first"], ot["first"])
    assert np.array_equal(nd["count"], ot["count"])
    assert np.array_equal(nd["next"], ot["next"])
    assert np.array_equal(nd["center"].view(np.uint32), ot["center"])


@pytest.mark.parametrize("order", [3, 4])
def test_moments_parity(order):
    ps = synth.plummer_16k()
    tg, run, box = _tree_case(ps, 8, order)
    gm = {k: v.cpu().numpy() for k, v in tg.tree.moments(order).items()}
    om = run.tree.export_moments()
    # node masses are dyadic sums: bit-exact
    assert np.array_equal(gm["mass"], om["mass"])
    lv = run.tree.export()["level"]
    side = box / 2.0 ** lv
    assert np.max(np.abs(gm["com"] - om["com"]) / side[:, None]) < 2e-6
    for n in range(2, order + 1):
        for a in range(n, -1, -1):
            for b in range(n - a, -1, -1):
                k = oracle.mono_index(a, b, n - a - b)
                scale = om["mass"] * side ** n
                err = np.abs(gm["mono"][:, k] - om["mono"][:, k]) / scale
                assert np.max(err) < 1e-5, (a, b, n - a - b, np.max(err))


# ---- a6 / a7: walk --------------------------------------------------------------------------

def _plummer_c1():
    ps = synth.plummer_16k()
    q, box = int_coords(ps)
    OP = oracle_params(ps, box)
    ad, _ = oracle.direct(q, ps.mass, None, np.arange(ps.n), OP)
    aold = np.linalg.norm(ad, axis=1).astype(np.float32)    # prior direct-sum pass, FP32
    return ps, q, box, aold, ad


def test_walk_parity_plummer_relative():
    ps, q, box, aold, ad = _plummer_c1()
    kw = dict(alpha=0.0025, order_p=3)
    P = gpu_params(g4, ps, box, **kw)
    ag, pg, cg, _ = gpu_forces(torch, g4, ps, q, P, aold)
    run = oracle.prepare(q, ps.mass, ps.eps_class, aold.astype(np.float64), oracle_params(ps, box, **kw), 8)
    ao, po, co = oracle.tree_forces(run, np.arange(ps.n))
    e = relerr(ag, ao)
    assert np.percentile(e, 99) < PARITY_P99, np.percentile(e, [50, 99, 100])
    ep = np.abs(pg - po) / np.abs(po)
    assert np.percentile(ep, 99) < PARITY_P99
    same = np.all(cg == co, axis=1)
    assert same.mean() > 0.99, same.mean()
    # accuracy against the FP64 direct sum (the method's own error at alpha = 0.0025): at the
    # leaf size the bench tunes (32) the 99th percentile meets the 1e-3 target; leaves of 8
    # accept more multipoles (measured 1.4e-3)
    assert np.percentile(relerr(ag, ad), 99) < 2e-3
    ag32, _, _, _ = gpu_forces(torch, g4, ps, q, gpu_params(g4, ps, box, leaf_max=32, **kw), aold)
    assert np.percentile(relerr(ag32, ad), 99) < 1e-3


@pytest.mark.parametrize("order", [1, 2, 4, 5])
def test_walk_parity_orders(order):
    ps, q, box, aold, _ = _plummer_c1()
    kw = dict(alpha=0.0025, order_p=order)
    P = gpu_params(g4, ps, box, **kw)
    ag, pg, cg, _ = gpu_forces(torch, g4, ps, q, P, aold)
    run = oracle.prepare(q, ps.mass, ps.eps_class, aold.astype(np.float64), oracle_params(ps, box, **kw), 8)
    sinks = np.arange(0, ps.n, 4)
    ao, po, co = oracle.tree_forces(run, sinks)
    assert np.percentile(relerr(ag[sinks], ao), 99) < PARITY_P99


def test_walk_parity_treepm_relative():
    ps, tp = _treepm_box(32)
    q, box = int_coords(ps)
    kw = dict(alpha=0.0025, **tp)
    OP = oracle_params(ps, box, **kw)
    ad, _ = oracle.direct(q, ps.mass, None, np.arange(ps.n), OP, r_max=OP.r_cut)
    aold = np.linalg.norm(ad, axis=1).astype(np.float32)
    P = gpu_params(g4, ps, box, **kw)
    ag, pg, cg, _ = gpu_forces(torch, g4, ps, q, P, aold)
    run = oracle.prepare(q, ps.mass, ps.eps_class, aold.astype(np.float64), OP, 8)
    ao, po, co = oracle.tree_forces(run, np.arange(ps.n))
    e = relerr(ag, ao)
    assert np.percentile(e, 99) < PARITY_P99, np.percentile(e, [50, 99, 100])
    assert np.mean(np.all(cg == co, axis=1)) > 0.99
    # against the hard-cutoff FP64 direct sum: the headline accuracy target
    assert np.percentile(relerr(ag, ad), 99) < 1e-3


def test_walk_parity_geometric_bootstrap():
    ps, tp = _treepm_box(24)
    q, box = int_coords(ps)
    kw = dict(criterion=1, theta=0.5, **tp)
    P = gpu_params(g4, ps, box, **kw)
    ag, pg, cg, _ = gpu_forces(torch, g4, ps, q, P, None)
    run = oracle.prepare(q, ps.mass, ps.eps_class, None, oracle_params(ps, box, **kw), 8)
    ao, po, co = oracle.tree_forces(run, np.arange(ps.n))
    assert np.percentile(relerr(ag, ao), 99) < PARITY_P99


def test_walk_alpha0_is_direct_sum():
    ps, tp = _treepm_box(16)
    q, box = int_coords(ps)
    kw = dict(alpha=0.0, **tp)
    P = gpu_params(g4, ps, box, **kw)
    ag, pg, cg, _ = gpu_forces(torch, g4, ps, q, P, np.ones(ps.n, np.float32))
    assert np.all(cg[:, 1] == 0)
    OP = oracle_params(ps, box, **kw)
    ad, pd = oracle.direct(q, ps.mass, None, np.arange(ps.n), OP, r_max=OP.r_cut)
    assert np.percentile(relerr(ag, ad), 99) < PARITY_P99
    # GPU direct-sum helper, same kernel
    acc, pot = g4.g4_direct(u32_dev(torch, q), to_dev(torch, ps.mass, torch.float32), None, P)
    assert np.percentile(relerr(acc.cpu().numpy().T, ad), 99) < PARITY_P99


def test_walk_fp64_mode():
    ps, q, box, aold, _ = _plummer_c1()
    kw = dict(alpha=0.0025, order_p=3)
    P = gpu_params(g4, ps, box, precision=1, **kw)
    ag, pg, cg, _ = gpu_forces(torch, g4, ps, q, P, aold)
    run = oracle.prepare(q, ps.mass, ps.eps_class, aold.astype(np.float64), oracle_params(ps, box, **kw), 8)
    ao, po, co = oracle.tree_forces(run, np.arange(ps.n))
    e = relerr(ag, ao)
    # FP64 arithmetic; the outputs are FP32, so the comparison floor is FP32 rounding
    assert np.percentile(e, 99) < 2e-7
    assert np.mean(np.all(cg == co, axis=1)) > 0.999


def test_active_subset_bitwise_equal_and_deterministic():
    ps, q, box, aold, _ = _plummer_c1()
    P = gpu_params(g4, ps, box, alpha=0.0025)
    tg = g4.TreeGravity(ps.n, P)
    pos = u32_dev(torch, q)
    mass = to_dev(torch, ps.mass, torch.float32)
    a = to_dev(torch, aold, torch.float32)
    tg.prepare(pos, mass, None, a)
    acc_s, pot_s, cnt = tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, P)
    acc2, pot2, _ = tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, P)
    assert torch.equal(acc_s, acc2) and torch.equal(pot_s, pot2)
    active = torch.arange(5, ps.n, 37, dtype=torch.int32, device="cuda")
    acc3, pot3, cnt3 = tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, P, active=active)
    idx = active.long()
    # same interactions for every sink whatever the group it shares; the FP32 sum order of the
    # particle pairs follows the group's batches, so values agree to rounding
    assert torch.equal(cnt3[:, idx], cnt[:, idx])
    a, b = acc3[:, idx].double(), acc_s[:, idx].double()
    assert torch.max(torch.abs(a - b)) <= 1e-6 * torch.max(torch.abs(b))


def test_walk_with_fused_scatter_equals_walk_then_scatter():
    """g4_gravity_tree_perm (the walk writing its results in input order) gives bitwise the
    results of g4_gravity_tree followed by g4_scatter, for all sinks and for an active subset,
    and is what TreeGravity.forces returns."""
    ps, q, box, aold, _ = _plummer_c1()
    P = gpu_params(g4, ps, box, alpha=0.0025)
    tg = g4.TreeGravity(ps.n, P)
    pos = u32_dev(torch, q)
    mass = to_dev(torch, ps.mass, torch.float32)
    a = to_dev(torch, aold, torch.float32)
    tg.prepare(pos, mass, None, a)
    acc_s, pot_s, cnt = tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, P)
    ref_acc, ref_pot = g4.g4_scatter(tg.perm, acc_s, pot_s)
    acc = torch.full((3, ps.n), float("nan"), device="cuda")
    pot = torch.full((ps.n,), float("nan"), device="cuda")
    _, _, cnt2 = tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, P, acc=acc, pot=pot,
                                      perm=tg.perm)
    assert torch.equal(acc, ref_acc) and torch.equal(pot, ref_pot) and torch.equal(cnt, cnt2)
    af, pf = tg.forces(pos, mass, None, a, P)
    assert torch.equal(af, ref_acc) and torch.equal(pf, ref_pot)
    # an active subset: only the listed sinks' input-order slots are written
    active = torch.arange(5, ps.n, 37, dtype=torch.int32, device="cuda")
    acc3, pot3, _ = tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, P, active=active)
    acc4 = torch.full((3, ps.n), float("nan"), device="cuda")
    pot4 = torch.full((ps.n,), float("nan"), device="cuda")
    tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, P, active=active, acc=acc4, pot=pot4,
                         perm=tg.perm)
    out = tg.perm[active.long()].long()
    assert torch.equal(acc4[:, out], acc3[:, active.long()]) and torch.equal(pot4[out], pot3[active.long()])
    written = torch.zeros(ps.n, dtype=torch.bool, device="cuda")
    written[out] = True
    assert bool(torch.isnan(pot4[~written]).all()) and not bool(torch.isnan(pot4[written]).any())


def _sparse_pairs():
    """2,048 pairs 0.99 r_cut apart in a box of 1,000 r_cut: every 32-sink group spans ~120
    r_cut, where FP16 positions relative to the group centre err by more than the candidate
    test's margin (an unguarded test drops ~4% of these pairs)."""
    L = 1.0
    rc = L / 1000
    ps = synth.sparse_pairs(2048, L, 0.99 * rc, 7001)
    return ps, dict(r_s=rc / 4.5, r_cut_factor=4.5, alpha=0.0)


def test_walk_sparse_groups_keep_pairs_near_cutoff():
    ps, kw = _sparse_pairs()
    q, box = int_coords(ps)
    OP = oracle_params(ps, box, **kw)
    aold = np.ones(ps.n, np.float32)   # alpha = 0: every node opened, a pure pair sum
    ag, pg, cg, _ = gpu_forces(torch, g4, ps, q, gpu_params(g4, ps, box, **kw), aold)
    run = oracle.prepare(q, ps.mass, ps.eps_class, aold.astype(np.float64), OP, 8)
    ao, po, co = oracle.tree_forces(run, np.arange(ps.n))
    # every particle sees its partner, 1% inside r_cut: the pair sets are identical
    assert np.array_equal(cg, co)
    assert np.all(cg[:, 0] >= 1) and np.all(cg[:, 1] == 0)
    assert np.percentile(relerr(ag, ao), 99) < PARITY_P99
    ad, _ = oracle.direct(q, ps.mass, None, np.arange(ps.n), OP, r_max=OP.r_cut)
    assert np.percentile(relerr(ag, ad), 99) < PARITY_P99


@pytest.mark.parametrize("n_pairs", [40, 64, 160])
def test_walk_groups_spanning_the_periodic_box_keep_pairs(n_pairs):
    """Sparse pairs 0.99 r_cut apart in a box of only 10 r_cut: groups of consecutive
    particles reach across half the box, where nearest-image offsets from the group centre wrap
    for sources on the far side of the periodic boundary; every pair must still be found (the
    tree walk and the FMM's particle pairs share this phase)."""
    L = 1.0
    rc = L / 10
    ps = synth.sparse_pairs(n_pairs, L, 0.99 * rc, 7100 + n_pairs)
    q, box = int_coords(ps)
    kw = dict(r_s=rc / 4.5, r_cut_factor=4.5, alpha=0.0)
    OP = oracle_params(ps, box, **kw)
    ad, _ = oracle.direct(q, ps.mass, None, np.arange(ps.n), OP, r_max=OP.r_cut)
    aold = np.ones(ps.n, np.float32)
    ag, pg, cg, _ = gpu_forces(torch, g4, ps, q, gpu_params(g4, ps, box, **kw), aold)
    e = relerr(ag, ad)
    assert np.percentile(e, 99) < PARITY_P99 and e.max() < 1e-3, np.percentile(e, [50, 99, 100])


def test_walk_without_pair_cutoff_keeps_more_pairs():
    """pp_cut = 0: particle pairs of every leaf the walk does not skip are kept, including
    those beyond r_cut; with the cutoff they are dropped.  Same nodes either way."""
    ps, tp = _treepm_box(16)
    q, box = int_coords(ps)
    kw = dict(criterion=1, theta=0.5, **tp)
    a1, _, c1, _ = gpu_forces(torch, g4, ps, q, gpu_params(g4, ps, box, **kw), None)
    a0, _, c0, _ = gpu_forces(torch, g4, ps, q, gpu_params(g4, ps, box, pp_cut=0, **kw), None)
    assert np.all(c0[:, 0] >= c1[:, 0]) and c0[:, 0].sum() > c1[:, 0].sum()
    assert np.array_equal(c0[:, 1], c1[:, 1])
    assert np.all(np.isfinite(a0))


@pytest.mark.parametrize("n", [1, 2, 3, 33])
def test_small_and_degenerate_sets(n):
    ps = synth.plummer(max(n, 1), 77 + n)
    if n == 33:   # many coincident particles: leaves at key resolution above leaf_max
        ps.pos[1:20] = ps.pos[0]
    q, box = int_coords(ps)
    P = gpu_params(g4, ps, box, criterion=1, theta=0.5)
    ag, pg, cg, _ = gpu_forces(torch, g4, ps, q, P, None)
    run = oracle.prepare(q, ps.mass, ps.eps_class, None, oracle_params(ps, box, criterion=1, theta=0.5), 8)
    ao, po, co = oracle.tree_forces(run, np.arange(ps.n))
    if n == 1:
        assert np.all(ag == 0) and np.all(pg == 0)
    else:
        assert np.allclose(ag, ao, rtol=1e-5, atol=1e-6 * np.abs(ao).max())
        assert np.allclose(pg, po, rtol=1e-5)


# ---- batched independent systems (forest): one sort, one build, one walk launch ---------------

def test_forest_many_plummer_spheres_parity():
    systems = synth.multi_plummer(24, 1005, n_min=256, n_max=4096)
    sizes = [ps.n for ps in systems]
    qs, boxes, aolds, refs = [], [], [], []
    for ps in systems:
        q, frame = oracle.int_coords_isolated(ps.pos)
        OP = oracle.OracleParams(box=frame[3], periodic=False, eps=ps.eps_table, alpha=0.0025)
        ad, _ = oracle.direct(q, ps.mass, None, np.arange(ps.n), OP)
        aold = np.linalg.norm(ad, axis=1).astype(np.float32)
        run = oracle.prepare(q, ps.mass, None, aold.astype(np.float64), OP, 8)
        ao, po, co = oracle.tree_forces(run, np.arange(ps.n))
        qs.append(q)
        boxes.append(frame[3])
        aolds.append(aold)
        refs.append((ao, po, co))
    P = g4.params(periodic=0, eps=[0.01], alpha=0.0025)
    fg = g4.ForestGravity(sizes, P)
    pos = u32_dev(torch, np.concatenate(qs, axis=1))
    mass = to_dev(torch, np.concatenate([ps.mass for ps in systems]), torch.float32)
    aold = to_dev(torch, np.concatenate(aolds), torch.float32)
    box = torch.tensor(boxes, dtype=torch.float64, device="cuda")
    acc, pot = fg.forces(pos, mass, box, aold)
    torch.cuda.synchronize()
    fg.tree.status()
    ag = acc.cpu().numpy().T.astype(np.float64)
    ao = np.concatenate([r[0] for r in refs])
    e = relerr(ag, ao)
    assert np.percentile(e, 99) < PARITY_P99, np.percentile(e, [50, 99, 100])
    # forest topology: every system's tree equals its own oracle tree
    nd = {k: v.cpu().numpy() for k, v in fg.tree.nodes().items()}
    off = 0
    for ps, q in zip(systems, qs):
        ks, perm = oracle.sort(oracle.keys(q))
        ot = oracle.Tree(ks, np.ascontiguousarray(q[:, perm]), 8).export()
        m = len(ot["level"])
        assert np.array_equal(nd["count"][off:off + m], ot["count"])
        assert np.array_equal(nd["next"][off:off + m] - off, ot["next"])
        off += m
    assert off == len(nd["level"])


def test_host_pipeline_equals_device_forces():
    """g4.HostPipeline (inputs from and results into pinned host memory, copies overlapped
    with the computation of neighbouring steps) returns exactly TreeGravity.forces' results,
    step by step, for changing inputs."""
    ps, tp = _treepm_box(24)
    q, box = int_coords(ps)
    P = gpu_params(g4, ps, box, alpha=0.0025, leaf_max=16, **tp)
    aold = torch.full((ps.n,), 5.0, dtype=torch.float32)
    h_pos = torch.from_numpy(np.ascontiguousarray(q).view(np.int32)).pin_memory()
    h_aold = aold.pin_memory()
    masses = [torch.from_numpy((ps.mass * s).astype(np.float32)).pin_memory() for s in (1.0, 0.5, 2.0)]
    h_acc = [torch.empty((3, ps.n), dtype=torch.float32).pin_memory() for _ in range(3)]
    h_pot = [torch.empty(ps.n, dtype=torch.float32).pin_memory() for _ in range(3)]
    pipe = g4.HostPipeline(ps.n, P)
    for k in range(3):
        pipe.submit(h_pos, masses[k], h_aold, h_acc[k], h_pot[k])
    torch.cuda.synchronize()
    tg = g4.TreeGravity(ps.n, P)
    for k in range(3):
        acc, pot = tg.forces(h_pos.cuda(), masses[k].cuda(), None, h_aold.cuda(), P)
        assert torch.equal(acc.cpu(), h_acc[k]) and torch.equal(pot.cpu(), h_pot[k])


@pytest.mark.parametrize("gs", [8, 16])
def test_walk_group_sizes_same_interactions(gs):
    """Smaller sink groups (group_size 8 or 16) walk the same per-sink interaction sets as
    32-sink groups; the sums differ only by rounding order."""
    ps, tp = _treepm_box(24)
    q, box = int_coords(ps)
    aold = np.full(ps.n, 5.0, np.float32)
    P32 = gpu_params(g4, ps, box, alpha=0.0025, leaf_max=16, **tp)
    Pgs = gpu_params(g4, ps, box, alpha=0.0025, leaf_max=16, group_size=gs, **tp)
    a32, p32, c32, _ = gpu_forces(torch, g4, ps, q, P32, aold)
    ags, pgs, cgs, _ = gpu_forces(torch, g4, ps, q, Pgs, aold)
    assert np.array_equal(c32, cgs)
    assert np.percentile(relerr(ags, a32), 99) < 2e-5


def test_walk_parity_softened_node_rule():
    """GADGET-4's softened node interactions (Sec. 2.7, soft_nodes = 1) against the oracle's:
    softenings comparable to the node sizes and two classes, so that both the softened
    multipoles and the forced opening of mixed nodes occur.  soft_nodes = 0 (the GADGET-3 rule,
    every node within 2.8 max(eps) opened) on the same set evaluates more particle pairs."""
    ps = synth.plummer(3000, 63)
    ps.eps_table = np.array([0.3, 0.08])
    ps.eps_class[::4] = 1
    q, box = int_coords(ps)
    ad, _ = oracle.direct(q, ps.mass, ps.eps_class, np.arange(ps.n), oracle_params(ps, box))
    aold = np.linalg.norm(ad, axis=1).astype(np.float32)
    pp = {}
    for soft in (0, 1):
        kw = dict(alpha=0.005, order_p=3, leaf_max=4, soft_nodes=soft)
        ag, pg, cg, _ = gpu_forces(torch, g4, ps, q, gpu_params(g4, ps, box, **kw), aold)
        run = oracle.prepare(q, ps.mass, ps.eps_class, aold.astype(np.float64),
                             oracle_params(ps, box, **kw), 4)
        ao, po, co = oracle.tree_forces(run, np.arange(ps.n))
        e = relerr(ag, ao)
        assert np.percentile(e, 99) < PARITY_P99, (soft, np.percentile(e, [50, 99, 100]))
        assert np.percentile(np.abs(pg - po) / np.abs(po), 99) < PARITY_P99
        assert np.mean(np.all(cg == co, axis=1)) > 0.99
        assert np.percentile(relerr(ag, ad), 99) < 0.01
        pp[soft] = cg[:, 0].sum()
    assert pp[1] < 0.95 * pp[0], pp


def test_union_walk_equals_per_group_walks():
    """The TreePM walk shares one walk among runs of four groups; with a group order set, every
    group walks on its own (the union walk is off).  Both give every sink the same
    interactions (identical counts) and the same forces up to the order of the sums."""
    ps, tp = _treepm_box(40)
    q, box = int_coords(ps)
    aold = np.full(ps.n, 5.0, np.float32)
    P = gpu_params(g4, ps, box, alpha=0.0025, leaf_max=32, **tp)
    tg = g4.TreeGravity(ps.n, P)
    pos, mass = u32_dev(torch, q), to_dev(torch, ps.mass, torch.float32)
    a = to_dev(torch, aold, torch.float32)
    tg.forces(pos, mass, None, a)
    acc_u, cnt_u = tg.acc.clone(), tg.counts.clone()
    ng = (ps.n + 31) // 32
    g4.set_group_order(tg.tree, torch.arange(ng, dtype=torch.int32, device="cuda"))
    tg.forces(pos, mass, None, a)
    acc_g, cnt_g = tg.acc.clone(), tg.counts.clone()
    g4.set_group_order(tg.tree, None)
    torch.cuda.synchronize()
    assert torch.equal(cnt_u, cnt_g)
    e = relerr(acc_u.cpu().numpy().T, acc_g.cpu().numpy().T)
    assert np.percentile(e, 99) < 1e-6 and e.max() < 1e-4, np.percentile(e, [50, 99, 100])
