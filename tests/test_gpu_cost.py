"""GPU cost model: BF16 MLP kernels against the FP64 oracle network (oracle/mlp.py, BF16
storage emulated), training on interaction counts logged by the walk, and the LPT schedule
(which must not change any force)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from oracle import mlp  # noqa: E402
from paper_2010_03567_gb300 import g4, synth  # noqa: E402

from _helpers import gpu_params, int_coords, oracle_params, to_dev, u32_dev  # noqa: E402

pytestmark = pytest.mark.gpu


def _rand_case(n=5000, seed=0):
    g = np.random.default_rng(seed)
    x = g.normal(0, 1, (n, 6)).astype(np.float32)
    t = g.normal(0, 1, n).astype(np.float32)
    return x, t


def test_mlp_forward_and_gradient_match_oracle():
    cm = g4.CostModel(seed=3)
    x, t = _rand_case()
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    p = cm.params.cpu().numpy().astype(np.float64)
    yo, _ = mlp.forward(p, x.astype(np.float64))
    yg = cm.predict(xd).cpu().numpy()
    assert np.max(np.abs(yg - yo)) < 1e-4 * max(1.0, np.max(np.abs(yo)))
    grad, loss = cm.gradient(xd, td)
    lo, go = mlp.loss_and_grad(p, x.astype(np.float64), t.astype(np.float64))
    gg = grad.cpu().numpy()
    assert abs(loss.item() - lo) < 1e-5 * max(1.0, lo)
    assert np.linalg.norm(gg - go) < 1e-4 * np.linalg.norm(go)


def test_training_deterministic_and_learns_walk_costs():
    ps = synth.zeldovich(32, 62.5, 2.0, 1003)
    q, box = int_coords(ps)
    kw = dict(alpha=0.0025, r_s=1.25 * 62.5 / 64, r_cut_factor=4.5)
    OP = oracle_params(ps, box, **kw)
    ad, _ = oracle.direct(q, ps.mass, None, np.arange(ps.n), OP, r_max=OP.r_cut)
    aold = np.linalg.norm(ad, axis=1).astype(np.float32)
    P = gpu_params(g4, ps, box, **kw)
    tg = g4.TreeGravity(ps.n, P)
    tg.prepare(u32_dev(torch, q), to_dev(torch, ps.mass, torch.float32), None,
               to_dev(torch, aold, torch.float32))
    tg.walk(P)
    feats = g4.cost_features(tg.tree, P, ps.n, tg.aold_s)
    labels = g4.cost_labels(tg.counts)
    runs = []
    for _ in range(2):
        cm = g4.CostModel(seed=1)
        losses = cm.train(feats, labels, steps=300, lr=3e-3).cpu().numpy()
        runs.append((cm.params.cpu().numpy(), losses))
    assert np.array_equal(runs[0][0], runs[1][0]), "training must be deterministic"
    losses = runs[0][1]
    assert losses[-1] < 0.5 * losses[0]
    pred = cm.predict(feats).cpu().numpy()
    lab = labels.cpu().numpy()
    rank = np.corrcoef(np.argsort(np.argsort(pred)), np.argsort(np.argsort(lab)))[0, 1]
    assert rank > 0.3, rank


def test_lpt_schedule_is_a_permutation_and_keeps_forces():
    ps = synth.plummer_16k()
    q, box = int_coords(ps)
    OP = oracle_params(ps, box)
    ad, _ = oracle.direct(q, ps.mass, None, np.arange(ps.n), OP)
    aold = np.linalg.norm(ad, axis=1).astype(np.float32)
    P = gpu_params(g4, ps, box, alpha=0.0025)
    tg = g4.TreeGravity(ps.n, P)
    tg.prepare(u32_dev(torch, q), to_dev(torch, ps.mass, torch.float32), None,
               to_dev(torch, aold, torch.float32))
    acc0, pot0, cnt0 = tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, P)
    acc0, pot0 = acc0.clone(), pot0.clone()
    feats = g4.cost_features(tg.tree, P, ps.n, tg.aold_s)
    cm = g4.CostModel(seed=2)
    cm.train(feats, g4.cost_labels(cnt0), steps=200)
    pred = cm.predict(feats)
    order = g4.schedule_lpt(pred)
    o = order.cpu().numpy()
    ng = (ps.n + 31) // 32
    assert np.array_equal(np.sort(o), np.arange(ng))
    pc = np.expm1(np.maximum(pred.cpu().numpy(), 0))
    gc = np.add.reduceat(pc, np.arange(0, ps.n, 32))
    assert np.all(np.diff(gc[o]) <= 1e-3 * gc.max())            # heaviest first
    g4.set_group_order(tg.tree, order)
    acc1, pot1, _ = tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, P)
    assert torch.equal(acc0, acc1) and torch.equal(pot0, pot1)
    g4.set_group_order(tg.tree, None)
