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


def test_walk_watchdog_times_out_cleanly():
    """The tree walk's work-queue watchdog (watchdog_cycles): with a budget of one SM clock cycle
    every warp stops taking groups, the call ends normally and g4_tree_status reports
    G4_ERR_TIMEOUT; the next build clears the flag and the same handle then walks every group
    (results equal to a walk on a fresh handle).  No spin, no trap: the device keeps working."""
    ps = synth.plummer(20000, 7)
    pos = torch.from_numpy(ps.pos).cuda()
    q, frame = g4.g4_int_coords(pos, False)
    mass = torch.from_numpy(ps.mass.astype(np.float32)).cuda()
    P = g4.params(box_size=float(frame[3].item()), eps=[0.01], criterion=1, theta=0.5)
    Pw = g4.params(box_size=float(frame[3].item()), eps=[0.01], criterion=1, theta=0.5,
                   watchdog_cycles=1)
    tg = g4.TreeGravity(ps.n, P)
    tg.prepare(q, mass, None, None, P)
    tg.walk(Pw, use_aold=False)
    with pytest.raises(g4.G4Error, match="status 4"):      # G4_ERR_TIMEOUT
        tg.tree.status()
    # not every sink was reached: the groups no warp took still carry no interactions
    cnt = tg.counts.to(torch.int64).sum(dim=0)
    assert int((cnt == 0).sum().item()) > 0
    acc, _ = tg.forces(q, mass, None, None, P)              # rebuild clears the flags
    torch.cuda.synchronize()
    tg.tree.status()
    ref = g4.TreeGravity(ps.n, P)
    acc_ref, _ = ref.forces(q, mass, None, None, P)
    torch.cuda.synchronize()
    assert torch.equal(acc, acc_ref)
    with pytest.raises(g4.G4Error, match="status 1"):      # a negative budget is refused
        tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, None,
                             g4.params(box_size=float(frame[3].item()), eps=[0.01], criterion=1,
                                       watchdog_cycles=-5))
