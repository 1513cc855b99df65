"""Autotuners for the tree walk: the leaf threshold, the sink-group size and the granularity
of the cost-model work partition.

The leaf threshold trades node visits against particle-pair candidates: small leaves mean a
deep tree whose frontier every 32-sink group must scan, large leaves mean coarser leaf
filtering.  The best value depends on the particle distribution, the cutoff and the GPU, so it
is measured: one complete force computation (sort, build, moments, walk) per candidate, timed
with CUDA events on the current stream, fastest wins.  Results are cached per GPU and workload
signature in a JSON file ($G4_AUTOTUNE_CACHE, default ~/.cache/g4_gb300/autotune.json).

Only host-side orchestration lives here; every timed step runs in the CUDA library.
"""
from __future__ import annotations

import json
import os

CANDIDATES = (8, 16, 24, 32, 48, 64)


def cache_path() -> str:
    return os.environ.get("G4_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "g4_gb300", "autotune.json"))


def signature(n: int, p) -> str:
    """Workload class: size, boundary, split scale relative to the mean spacing, order, alpha."""
    spacing = p.box_size / max(1.0, n ** (1.0 / 3.0))
    rs = p.r_s / spacing if p.r_s > 0 else 0.0
    return (f"n{n}-per{int(p.periodic)}-rs{rs:.3g}-rc{p.r_cut_factor:g}-p{p.order_p}"
            f"-a{p.alpha:g}-crit{p.criterion}")


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(key: str, entry: dict, path: str | None = None) -> None:
    path = path or cache_path()
    data = load_cache(path)
    data[key] = entry
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick(times: dict) -> int:
    """Fastest candidate; ties go to the larger leaf (smaller tree)."""
    return min(times, key=lambda k: (times[k], -k))


def tune(time_step, device_name: str, n: int, p, candidates=CANDIDATES, path: str | None = None,
         use_cache: bool = True) -> tuple[int, dict]:
    """time_step(leaf_max) -> milliseconds of one force computation.  Returns (best, times)."""
    key = f"{device_name}|{signature(n, p)}"
    if use_cache:
        hit = load_cache(path).get(key)
        if hit is not None:
            return int(hit["leaf_max"]), {int(k): v for k, v in hit["times_ms"].items()}
    times = {int(c): float(time_step(int(c))) for c in candidates}
    best = pick(times)
    store(key, {"leaf_max": best, "times_ms": times}, path)
    return best, times


def gpu_step_timer(pos_int, mass, aold, p, reps: int = 2):
    """A time_step for `tune`: builds a pipeline with the candidate leaf threshold and times
    `reps` complete force computations after one warm-up call."""
    import torch

    from . import g4

    def run(leaf_max: int) -> float:
        q = p.copy()
        q.leaf_max = leaf_max
        tg = g4.TreeGravity(pos_int.shape[1], q)
        tg.forces(pos_int, mass, None, aold, q)
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            tg.forces(pos_int, mass, None, aold, q)
        e1.record(s)
        torch.cuda.synchronize()
        tg.tree.close()
        return e0.elapsed_time(e1) / reps

    return run


# ---- work partition ------------------------------------------------------------------------

PARTITION_TARGETS = (0, 1, 2, 4, 8, 16)   # items per resident warp; 0 = plain 32-sink groups


def pick_partition(times: dict) -> int:
    """Fastest target; ties go to the coarser partition (fewer items)."""
    return min(times, key=lambda k: (times[k], k))


def tune_partition(time_walk, device_name: str, n: int, p, targets=PARTITION_TARGETS,
                   path: str | None = None, use_cache: bool = True) -> tuple[int, dict]:
    """time_walk(target) -> milliseconds of the walk with items at `target` items per resident
    warp (0: no partition).  Returns (best, times); cached like the leaf threshold."""
    key = f"{device_name}|{signature(n, p)}|partition"
    if use_cache:
        hit = load_cache(path).get(key)
        if hit is not None:
            return int(hit["target"]), {int(k): v for k, v in hit["times_ms"].items()}
    times = {int(t): float(time_walk(int(t))) for t in targets}
    best = pick_partition(times)
    store(key, {"target": best, "times_ms": times}, path)
    return best, times


def gpu_partition_timer(tg, p, pred_sorted, reps: int = 3):
    """A time_walk for `tune_partition` on a prepared TreeGravity: items from the per-sink
    predicted (or measured) costs at the candidate granularity, walk timed with CUDA events.
    Leaves the handle with plain groups."""
    import torch

    from . import g4

    n = tg.n
    walk = lambda: tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, p, acc=tg.acc_s,
                                        pot=tg.pot_s, counts=tg.counts)

    def run(target: int) -> float:
        if target > 0:
            items, ni = g4.schedule_items(pred_sorted, target * g4.resident_warps())
            g4.set_work_items(tg.tree, items, ni, n)
        else:
            g4.set_work_items(tg.tree, None)
        walk()
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            walk()
        e1.record(s)
        torch.cuda.synchronize()
        g4.set_work_items(tg.tree, None)
        return e0.elapsed_time(e1) / reps

    return run


# ---- sink-group size ---------------------------------------------------------------------------

GROUP_SIZES = (8, 16, 32)


def tune_group_size(time_walk, device_name: str, n: int, p, sizes=GROUP_SIZES,
                    path: str | None = None, use_cache: bool = True) -> tuple[int, dict]:
    """time_walk(group_size) -> milliseconds of the walk.  Fastest wins, ties to the larger
    group.  Cached per GPU and workload like the leaf threshold."""
    key = f"{device_name}|{signature(n, p)}|group"
    if use_cache:
        hit = load_cache(path).get(key)
        if hit is not None:
            return int(hit["group_size"]), {int(k): v for k, v in hit["times_ms"].items()}
    times = {int(g): float(time_walk(int(g))) for g in sizes}
    best = min(times, key=lambda k: (times[k], -k))
    store(key, {"group_size": best, "times_ms": times}, path)
    return best, times
