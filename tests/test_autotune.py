"""Host logic of the leaf-size autotuner (selection and cache), with a fake timer (CPU)."""
from paper_2010_03567_gb300 import autotune


class FakeParams:
    box_size = 100.0
    periodic = 1
    r_s = 0.5
    r_cut_factor = 4.5
    order_p = 3
    alpha = 0.0025
    criterion = 0


def test_pick_and_cache(tmp_path):
    path = str(tmp_path / "cache.json")
    calls = []

    def timer(leaf):
        calls.append(leaf)
        return {8: 5.0, 16: 3.0, 24: 2.5, 32: 2.5, 48: 2.7, 64: 4.0}[leaf]

    best, times = autotune.tune(timer, "GB300", 1 << 20, FakeParams(), path=path)
    assert best == 32            # tie between 24 and 32 goes to the larger leaf
    assert sorted(calls) == [8, 16, 24, 32, 48, 64]
    calls.clear()
    best2, times2 = autotune.tune(timer, "GB300", 1 << 20, FakeParams(), path=path)
    assert best2 == 32 and calls == [] and times2 == times
    # another workload class is tuned separately
    p = FakeParams()
    p.alpha = 0.01
    autotune.tune(timer, "GB300", 1 << 20, p, path=path)
    assert len(calls) == 6
    assert autotune.signature(1 << 20, p) != autotune.signature(1 << 20, FakeParams())


def test_partition_pick_and_cache(tmp_path):
    path = str(tmp_path / "cache.json")
    calls = []

    def timer(target):
        calls.append(target)
        return {0: 4.0, 1: 2.0, 2: 1.3, 4: 1.2, 8: 1.2, 16: 1.5}[target]

    best, times = autotune.tune_partition(timer, "GB300", 16384, FakeParams(), path=path)
    assert best == 4             # tie between 4 and 8 goes to the coarser partition
    assert sorted(calls) == [0, 1, 2, 4, 8, 16]
    calls.clear()
    assert autotune.tune_partition(timer, "GB300", 16384, FakeParams(), path=path)[0] == 4
    assert calls == []
    # the leaf threshold and the partition of the same workload are cached separately
    autotune.tune(lambda leaf: float(leaf), "GB300", 16384, FakeParams(), path=path)
    assert autotune.load_cache(path).keys() >= {
        "GB300|" + autotune.signature(16384, FakeParams()),
        "GB300|" + autotune.signature(16384, FakeParams()) + "|partition"}


def test_group_size_pick_and_cache(tmp_path):
    path = str(tmp_path / "cache.json")
    times = {8: 49.5, 16: 28.6, 32: 17.2}     # 256^3 walk, measured on a GB300
    best, got = autotune.tune_group_size(lambda g: times[g], "GB300", 1 << 24, FakeParams(), path=path)
    assert best == 32 and got == times
    best, _ = autotune.tune_group_size(lambda g: 1.0, "GB300", 1 << 24, FakeParams(), path=path)
    assert best == 32                            # cached
    best, _ = autotune.tune_group_size(lambda g: 1.0, "GB300", 1 << 10, FakeParams(), path=path)
    assert best == 32                            # tie goes to the larger group
