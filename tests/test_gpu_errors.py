"""Failure handling without faulting the GPU: argument errors, allocation failure, and a node
capacity overflow that the kernels detect, flag and survive (the device keeps working)."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2010_03567_gb300 import g4, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def test_allocation_failure_is_reported():
    h = C.c_void_p()
    # the first (largest) request is already impossible: nothing is allocated at all
    st = g4.lib().g4_tree_create(1 << 30, (1 << 31) - 2, C.byref(h))
    assert st == 2 and not h.value            # G4_ERR_OOM, no handle
    assert b"cudaMalloc" in g4.lib().g4_last_error()


def test_capacity_overflow_flagged_and_recoverable():
    ps = synth.plummer(20000, 5)
    pos = torch.from_numpy(ps.pos).cuda()
    q, frame = g4.g4_int_coords(pos, False)
    mass = torch.from_numpy(ps.mass.astype(np.float32)).cuda()
    P = g4.params(box_size=float(frame[3].item()), eps=[0.01], criterion=1, leaf_max=1)
    tg = g4.TreeGravity(ps.n, P, node_capacity=5000)       # far too small for leaf 1
    tg.forces(q, mass)
    with pytest.raises(g4.G4Error, match="status 7"):      # G4_ERR_CAPACITY
        tg.tree.status()
    # the context is intact: a correctly sized pipeline still works afterwards
    tg2 = g4.TreeGravity(ps.n, P)
    acc, _ = tg2.forces(q, mass)
    torch.cuda.synchronize()
    tg2.tree.status()
    assert torch.isfinite(acc).all()


def test_state_and_argument_errors():
    t = g4.Tree(100)
    pos = torch.zeros((3, 100), dtype=torch.int32, device="cuda")
    m = torch.ones(100, device="cuda")
    with pytest.raises(g4.G4Error, match="status 6"):      # walk before build
        t.gravity_tree(pos, m, None, m, g4.params())
    with pytest.raises(g4.G4Error, match="status 1"):      # order out of range
        t.gravity_tree(pos, m, None, m, g4.params(order_p=9))
