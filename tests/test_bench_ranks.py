"""Host logic of bench.py's multi-GPU mode (independent replicas, one per rank), run as two
gloo ranks on the CPU: the timed region's length is the maximum over ranks, the job's
throughput counts every rank's particles, and the reference arm's extra ranks exit without
work."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                     # rank 1 is the slow one
        m = bench.max_over_ranks(ms, "cpu", True)
        out.put((rank, m, bench.job_throughput(world, 1000, m)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_throughput_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == pytest.approx(2 * 1000 / 15e-3)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, "cpu", False) == 3.5
    assert bench.job_throughput(1, 16777216, 1000.0) == pytest.approx(16777216.0)


def test_reference_arm_extra_ranks_exit_without_work(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup = 1, 0
    assert bench.run_reference(A(), 1, 2) == 0
    assert capsys.readouterr().out == ""


def test_oracle_fmm_baseline_leg_on_a_small_sample():
    """The FMM's host baseline (the FP64 oracle FMM on a bounded sample of the headline's
    spacing and split) reports forces/s on one core and names its sample."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.oracle_fmm_throughput(n_side_cpu=12)
    assert r["value"] > 0 and r["cores"] == 1 and r["kind"] == "oracle" and r["unit"] == bench.UNIT
    assert "12^3" in r["sample"] and "p = 4" in r["sample"]


def test_params_defaults_include_the_watchdog_off():
    """The binding's ctypes mirror carries the walk's watchdog budget, off (0) by default."""
    sys.path.insert(0, ROOT)
    from paper_2010_03567_gb300 import g4
    p = g4.params()
    assert p.watchdog_cycles == 0
    assert g4.params(watchdog_cycles=1 << 40).watchdog_cycles == 1 << 40
