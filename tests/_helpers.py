"""Shared helpers for the GPU parity tests: run the same seeded particle set through the FP64
oracle and through the CUDA path (C ABI via the thin binding)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2010_03567_gb300 import synth


def relerr(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def int_coords(ps: synth.ParticleSet):
    if ps.periodic:
        return oracle.int_coords_periodic(ps.pos, ps.box_size), ps.box_size
    q, frame = oracle.int_coords_isolated(ps.pos)
    return q, float(frame[3])


def gpu_params(g4, ps, box, **kw):
    base = dict(box_size=box, periodic=int(ps.periodic), eps=list(ps.eps_table))
    base.update(kw)
    return g4.params(**base)


def oracle_params(ps, box, **kw):
    kw = dict(kw)
    kw.pop("leaf_max", None)
    kw.pop("fp64_count", None)
    kw.pop("precision", None)
    kw.pop("group_size", None)
    kw.pop("fmm_p2p_per_particle", None)
    if "order_p" in kw:
        kw["order"] = kw.pop("order_p")
    if "exclusion_zone" in kw:
        kw["exclusion"] = bool(kw.pop("exclusion_zone"))
    return oracle.OracleParams(box=box, periodic=ps.periodic, eps=ps.eps_table, **kw)


def to_dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def u32_dev(torch, q):
    return torch.from_numpy(np.ascontiguousarray(q).view(np.int32)).cuda()


def u32_host(t):
    return t.cpu().numpy().view(np.uint32)


def u64_host(t):
    return t.cpu().numpy().view(np.uint64)


def gpu_forces(torch, g4, ps, q, P, aold=None, cls=True):
    """Full pipeline through the C ABI.  Returns acc (n,3), pot (n,), counts (n,2) in caller
    order plus the TreeGravity object."""
    tg = g4.TreeGravity(ps.n, P, with_cls=cls)
    pos = u32_dev(torch, q)
    mass = to_dev(torch, ps.mass, torch.float32)
    c = to_dev(torch, ps.eps_class, torch.uint8) if cls else None
    a = to_dev(torch, aold, torch.float32) if aold is not None else None
    acc, pot = tg.forces(pos, mass, c, a)
    torch.cuda.synchronize()
    tg.tree.status()
    perm = tg.perm.cpu().numpy()
    cnt_s = tg.counts.cpu().numpy().T
    cnt = np.empty_like(cnt_s)
    cnt[perm] = cnt_s
    return acc.cpu().numpy().T.astype(np.float64), pot.cpu().numpy().astype(np.float64), cnt, tg
