"""Random translation of the particle set (Sec. 3.8, g4_translate): loss-less and reversible on
integer coordinates; the tree walk on a translated set is the oracle's walk on the same
translated set; and translating between force computations decorrelates the directions of the
tree's force errors (the paper's motivation), while the errors keep their size."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2010_03567_gb300 import g4, synth  # noqa: E402

from _helpers import gpu_params, int_coords, oracle_params, relerr, to_dev, u32_dev  # noqa: E402

pytestmark = pytest.mark.gpu


def test_translate_is_lossless_and_reversible():
    rng = np.random.default_rng(1)
    q = rng.integers(0, 2 ** 32, size=(3, 10007), dtype=np.uint64).astype(np.uint32)
    s = [int(v) for v in rng.integers(0, 2 ** 32, size=3, dtype=np.uint64)]
    qd = u32_dev(torch, q)
    t = g4.g4_translate(qd, s)
    back = g4.g4_translate(t, [(1 << 32) - v for v in s])
    torch.cuda.synchronize()
    expect = ((q.astype(np.uint64) + np.array(s, np.uint64)[:, None]) % (1 << 32)).astype(np.uint32)
    assert np.array_equal(t.cpu().numpy().view(np.uint32), expect)
    assert np.array_equal(back.cpu().numpy().view(np.uint32), q)


def _box():
    L = 32.0
    ps = synth.zeldovich(32, L, 1.0, 3003)
    q, box = int_coords(ps)
    kw = dict(r_s=4.0 * L / 32, r_cut_factor=4.5, criterion=1, theta=0.7, order_p=3)
    return ps, q, box, kw


def test_translated_walk_matches_oracle_on_translated_set():
    ps, q, box, kw = _box()
    s = [123456789, 3000000000, 77]
    qs = ((q.astype(np.uint64) + np.array(s, np.uint64)[:, None]) % (1 << 32)).astype(np.uint32)
    P = gpu_params(g4, ps, box, **kw)
    tg = g4.TreeGravity(ps.n, P)
    acc, _ = tg.forces(u32_dev(torch, q), to_dev(torch, ps.mass, torch.float32), shift=s)
    torch.cuda.synchronize()
    run = oracle.prepare(qs, ps.mass, None, None, oracle_params(ps, box, **kw), 8)
    ao, _, _ = oracle.tree_forces(run, np.arange(ps.n))
    assert np.percentile(relerr(acc.cpu().numpy().T.astype(np.float64), ao), 99) < 1e-5


def test_translation_decorrelates_force_errors():
    ps, q, box, kw = _box()
    OP = oracle_params(ps, box, **kw)
    ad, _ = oracle.direct(q, ps.mass, None, np.arange(ps.n), OP, r_max=OP.r_cut)
    P = gpu_params(g4, ps, box, **kw)
    tg = g4.TreeGravity(ps.n, P)
    pos, mass = u32_dev(torch, q), to_dev(torch, ps.mass, torch.float32)
    rng = np.random.default_rng(9)
    errs = []
    for shift in (None, None, *[[int(v) for v in rng.integers(0, 2 ** 32, 3, dtype=np.uint64)]
                                for _ in range(2)]):
        a, _ = tg.forces(pos, mass, shift=shift)
        torch.cuda.synchronize()
        errs.append(a.cpu().numpy().T.astype(np.float64) - ad)
    cos = lambda u, v: np.sum(u * v, axis=1) / (np.linalg.norm(u, axis=1) * np.linalg.norm(v, axis=1))
    size = [np.median(np.linalg.norm(e, axis=1) / np.linalg.norm(ad, axis=1)) for e in errs]
    assert np.allclose(cos(errs[0], errs[1]), 1.0)          # no translation: the same errors
    c = cos(errs[2], errs[3])                                 # two random translations
    assert abs(np.median(c)) < 0.3, np.median(c)
    assert c.mean() < 0.5
    assert max(size) < 3 * min(size)                          # same size of error
