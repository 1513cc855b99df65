"""Thin Python binding of libg4.so (include/g4.h): argument marshalling only.

Every function here forwards torch CUDA tensors (device pointers) and the current CUDA stream
to the C entry point of the same name; all arithmetic runs in the sm_103a kernels.  There is
no CPU fallback: if the library cannot be loaded, or no CUDA device is present, the calls
raise.

uint32 / uint64 device arrays are carried in int32 / int64 tensors (same bits).
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

_lib = None


class G4Error(RuntimeError):
    pass


MAX_EPS = 8


class G4Params(C.Structure):
    _fields_ = [("box_size", C.c_double), ("periodic", C.c_int), ("r_s", C.c_double),
                ("r_cut_factor", C.c_double), ("pp_cut", C.c_int), ("alpha", C.c_double),
                ("theta", C.c_double), ("criterion", C.c_int), ("order_p", C.c_int),
                ("leaf_max", C.c_int), ("exclusion_zone", C.c_int), ("precision", C.c_int),
                ("G", C.c_double), ("n_eps_classes", C.c_int),
                ("eps_table", C.c_double * MAX_EPS), ("group_size", C.c_int),
                ("fp64_count", C.c_int), ("keep_qp", C.c_int), ("fmm_p2p_per_particle", C.c_int),
                ("soft_nodes", C.c_int), ("ewald", C.c_int), ("watchdog_cycles", C.c_int64)]

    def copy(self) -> "G4Params":
        p = G4Params()
        C.memmove(C.byref(p), C.byref(self), C.sizeof(G4Params))
        return p


def lib():
    """Loads the in-tree libg4.so (building it with nvcc when it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if _build.needs_build():
            path = _build.build()
        if not os.path.exists(path):
            raise G4Error("libg4.so is missing and could not be built")
        L = C.CDLL(path)
        _declare(L)
        _lib = L
    return _lib


def _declare(L):
    vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int, C.c_double
    P = C.POINTER(G4Params)
    sig = {
        "g4_version": ([], C.c_char_p),
        "g4_last_error": ([], C.c_char_p),
        "g4_launch_count": ([], C.c_int64),
        "g4_params_default": ([P], i32),
        "g4_int_coords": ([vp, i64, i32, d, vp, vp, vp], i32),
        "g4_keys_sort_workspace": ([i64, C.POINTER(C.c_size_t)], i32),
        "g4_keys_sort": ([vp, i64, vp, vp, vp, C.c_size_t, vp], i32),
        "g4_keys_sort_noalloc": ([vp, i64, vp, vp, vp], i32),
        "g4_keys_sort_batched_workspace": ([i64, C.POINTER(C.c_size_t)], i32),
        "g4_keys_sort_batched": ([vp, i64, vp, vp, vp, vp, C.c_size_t, vp], i32),
        "g4_tree_build_forest": ([vp, vp, vp, i64, vp, vp, C.c_int32, P, vp], i32),
        "g4_gather": ([vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp], i32),
        "g4_scatter": ([vp, i64, vp, vp, vp, vp, vp], i32),
        "g4_gather_subset": ([vp, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp], i32),
        "g4_scatter_subset": ([vp, i64, i64, vp, vp, vp, vp, vp], i32),
        "g4_tree_create": ([i64, i64, C.POINTER(vp)], i32),
        "g4_tree_free": ([vp], None),
        "g4_tree_build": ([vp, vp, vp, i64, P, vp], i32),
        "g4_tree_status": ([vp, C.POINTER(i64), C.POINTER(C.c_int32), vp], i32),
        "g4_tree_nodes": ([vp, vp, vp, vp, vp, vp, vp], i32),
        "g4_multipoles": ([vp, vp, vp, vp, vp, P, vp], i32),
        "g4_tree_moments": ([vp, vp, vp, vp, vp], i32),
        "g4_gravity_tree": ([vp, vp, vp, vp, vp, vp, i64, P, vp, vp, vp, vp], i32),
        "g4_gravity_tree_perm": ([vp, vp, vp, vp, vp, vp, i64, P, vp, vp, vp, vp, vp], i32),
        "g4_fmm_workspace": ([vp, P, C.POINTER(C.c_size_t)], i32),
        "g4_gravity_fmm": ([vp, vp, vp, vp, vp, P, vp, vp, vp, vp, vp, C.c_size_t, vp], i32),
        "g4_direct": ([vp, vp, vp, i64, vp, i64, P, vp, vp, vp], i32),
        "g4_pm_workspace": ([C.c_int32, C.POINTER(C.c_size_t)], i32),
        "g4_kick": ([vp, vp, vp, i64, i64, d, vp], i32),
        "g4_translate": ([vp, vp, i64, C.POINTER(C.c_uint32), vp], i32),
        "g4_ewald_eval": ([vp, vp, i64, i32, d, vp, vp], i32),
        "g4_drift": ([vp, vp, vp, i64, i64, d, P, vp, vp], i32),
        "g4_timestep_bins": ([vp, vp, vp, i64, i64, P, d, d, C.c_int32, vp, vp], i32),
        "g4_pm_long_range": ([vp, vp, i64, vp, i64, P, C.c_int32, vp, vp, i32, vp, C.c_size_t, vp], i32),
        "g4_mlp_param_count": ([], C.c_int32),
        "g4_cost_features": ([vp, vp, vp, P, vp, vp, vp], i32),
        "g4_cost_labels": ([vp, i64, C.c_float, vp, vp], i32),
        "g4_mlp_forward": ([vp, vp, i64, vp, vp], i32),
        "g4_mlp_train_workspace": ([i64, C.POINTER(C.c_size_t)], i32),
        "g4_mlp_train_step": ([vp, vp, vp, C.c_int32, vp, vp, i64, C.c_float, vp, vp, vp,
                               C.c_size_t, vp], i32),
        "g4_schedule_workspace": ([i64, C.POINTER(C.c_size_t)], i32),
        "g4_schedule_lpt": ([vp, i64, C.c_int32, vp, vp, C.c_size_t, vp], i32),
        "g4_tree_set_group_order": ([vp, vp, i64], i32),
        "g4_schedule_items_workspace": ([i64, C.POINTER(C.c_size_t)], i32),
        "g4_schedule_items": ([vp, i64, C.c_int32, C.c_int32, vp, vp, vp, C.c_size_t, vp], i32),
        "g4_tree_set_work_items": ([vp, vp, vp, i64, i64, C.c_int32], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res


def _check(st: int, what: str):
    if st != 0:
        msg = lib().g4_last_error().decode(errors="replace")
        raise G4Error(f"{what} failed (status {st}): {msg}")


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise G4Error("expected a CUDA tensor")
    if not t.is_contiguous():
        raise G4Error("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def params(**kw) -> G4Params:
    """g4_params with the library defaults, overridden by keyword arguments.  ``eps`` may be
    a sequence of softening lengths (one per class)."""
    p = G4Params()
    _check(lib().g4_params_default(C.byref(p)), "g4_params_default")
    eps = kw.pop("eps", None)
    if eps is not None:
        eps = [float(e) for e in (eps if hasattr(eps, "__len__") else [eps])]
        if not 1 <= len(eps) <= MAX_EPS:
            raise G4Error("1..8 softening classes supported")
        p.n_eps_classes = len(eps)
        for k, e in enumerate(eps):
            p.eps_table[k] = e
    for k, v in kw.items():
        if not hasattr(p, k):
            raise G4Error(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def version() -> str:
    return lib().g4_version().decode()


def launch_count() -> int:
    """Kernel launches issued by libg4 since it was loaded."""
    return int(lib().g4_launch_count())


# ---- a1..a3 ----------------------------------------------------------------------------------

def g4_int_coords(pos: torch.Tensor, periodic: bool, box_size: float = 0.0, out=None, frame=None,
                  stream=None):
    """pos: (n,3) float64 CUDA -> (pos_int (3,n) int32 holding uint32 bits, frame (8,) f64
    whose first four entries are {origin_x, origin_y, origin_z, side})."""
    n = pos.shape[0]
    out = out if out is not None else torch.empty((3, n), dtype=torch.int32, device=pos.device)
    frame = frame if frame is not None else torch.empty(8, dtype=torch.float64, device=pos.device)
    if frame.numel() < 8:
        raise G4Error("frame needs 8 doubles")
    _check(lib().g4_int_coords(_ptr(pos), n, int(periodic), float(box_size), _ptr(out),
                               _ptr(frame), _stream(stream)), "g4_int_coords")
    return out, frame


def g4_keys_sort_workspace(n: int) -> int:
    b = C.c_size_t()
    _check(lib().g4_keys_sort_workspace(n, C.byref(b)), "g4_keys_sort_workspace")
    return int(b.value)


def g4_keys_sort(pos_int: torch.Tensor, keys=None, perm=None, workspace=None, stream=None):
    """pos_int (3,n) -> (keys (n,) int64 holding uint64 keys, perm (n,) int32)."""
    n = pos_int.shape[1]
    dev = pos_int.device
    keys = keys if keys is not None else torch.empty(n, dtype=torch.int64, device=dev)
    perm = perm if perm is not None else torch.empty(n, dtype=torch.int32, device=dev)
    if workspace is None:
        workspace = torch.empty(g4_keys_sort_workspace(n) + 256, dtype=torch.uint8, device=dev)
    wp = workspace.data_ptr()
    off = (-wp) % 256
    _check(lib().g4_keys_sort(_ptr(pos_int), n, _ptr(keys), _ptr(perm), C.c_void_p(wp + off),
                              workspace.numel() - off, _stream(stream)), "g4_keys_sort")
    return keys, perm


def g4_keys_sort_batched(pos_int: torch.Tensor, sys_id: torch.Tensor, keys=None, perm=None,
                         workspace=None, stream=None):
    """Sort by (system, key).  sys_id: (n,) int16 tensor holding uint16 system ids."""
    n = pos_int.shape[1]
    dev = pos_int.device
    keys = keys if keys is not None else torch.empty(n, dtype=torch.int64, device=dev)
    perm = perm if perm is not None else torch.empty(n, dtype=torch.int32, device=dev)
    if workspace is None:
        b = C.c_size_t()
        _check(lib().g4_keys_sort_batched_workspace(n, C.byref(b)), "g4_keys_sort_batched_workspace")
        workspace = torch.empty(int(b.value) + 256, dtype=torch.uint8, device=dev)
    wp = workspace.data_ptr()
    off = (-wp) % 256
    _check(lib().g4_keys_sort_batched(_ptr(pos_int), n, _ptr(sys_id), _ptr(keys), _ptr(perm),
                                      C.c_void_p(wp + off), workspace.numel() - off, _stream(stream)),
           "g4_keys_sort_batched")
    return keys, perm


def g4_gather(perm, pos, mass, cls=None, aold=None, out=None, stream=None):
    n = perm.shape[0]
    if out is None:
        out = (torch.empty_like(pos), torch.empty_like(mass),
               None if cls is None else torch.empty_like(cls),
               None if aold is None else torch.empty_like(aold))
    po, mo, co, ao = out
    _check(lib().g4_gather(_ptr(perm), n, _ptr(pos), _ptr(mass), _ptr(cls), _ptr(aold), _ptr(po),
                           _ptr(mo), _ptr(co), _ptr(ao), _stream(stream)), "g4_gather")
    return po, mo, co, ao


def g4_scatter(perm, acc_sorted, pot_sorted=None, out=None, stream=None):
    n = perm.shape[0]
    if out is None:
        out = (torch.empty_like(acc_sorted), None if pot_sorted is None else torch.empty_like(pot_sorted))
    ao, po = out
    _check(lib().g4_scatter(_ptr(perm), n, _ptr(acc_sorted), _ptr(pot_sorted), _ptr(ao), _ptr(po),
                            _stream(stream)), "g4_scatter")
    return ao, po


# ---- a4..a8 -----------------------------------------------------------------------------------

class Tree:
    """Library-owned tree handle (g4_tree): node arrays for up to n_max particles."""

    def __init__(self, n_max: int, node_capacity: int = 0):
        h = C.c_void_p()
        _check(lib().g4_tree_create(int(n_max), int(node_capacity), C.byref(h)), "g4_tree_create")
        self.h = h
        self.n_max = n_max

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().g4_tree_free(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build(self, keys_sorted, pos_sorted, p: G4Params, stream=None):
        _check(lib().g4_tree_build(self.h, _ptr(keys_sorted), _ptr(pos_sorted),
                                   int(pos_sorted.shape[1]), C.byref(p), _stream(stream)),
               "g4_tree_build")

    def build_forest(self, keys_sorted, pos_sorted, sys_first, sys_box, p: G4Params, stream=None):
        """sys_first: (n_sys+1,) int32 CUDA, sys_box: (n_sys,) float64 CUDA; both must outlive
        the handle's later calls (the library keeps the pointers)."""
        self._forest_refs = (sys_first, sys_box)
        _check(lib().g4_tree_build_forest(self.h, _ptr(keys_sorted), _ptr(pos_sorted),
                                          int(pos_sorted.shape[1]), _ptr(sys_first), _ptr(sys_box),
                                          int(sys_box.shape[0]), C.byref(p), _stream(stream)),
               "g4_tree_build_forest")

    def status(self, stream=None):
        nn = C.c_int64()
        ml = C.c_int32()
        _check(lib().g4_tree_status(self.h, C.byref(nn), C.byref(ml), _stream(stream)), "g4_tree_status")
        return int(nn.value), int(ml.value)

    def nodes(self, stream=None) -> dict:
        nn, _ = self.status(stream)
        dev = torch.device("cuda")
        out = {k: torch.empty(nn, dtype=torch.int32, device=dev) for k in ("level", "first", "count", "next")}
        out["center"] = torch.empty((nn, 3), dtype=torch.int32, device=dev)
        _check(lib().g4_tree_nodes(self.h, _ptr(out["level"]), _ptr(out["first"]), _ptr(out["count"]),
                                   _ptr(out["next"]), _ptr(out["center"]), _stream(stream)), "g4_tree_nodes")
        return out

    def multipoles(self, pos_sorted, mass_sorted, cls_sorted, aold_sorted, p: G4Params, stream=None):
        _check(lib().g4_multipoles(self.h, _ptr(pos_sorted), _ptr(mass_sorted), _ptr(cls_sorted),
                                   _ptr(aold_sorted), C.byref(p), _stream(stream)), "g4_multipoles")

    def moments(self, order: int, stream=None) -> dict:
        nn, _ = self.status(stream)
        nm = (order + 1) * (order + 2) * (order + 3) // 6
        dev = torch.device("cuda")
        out = {"mass": torch.empty(nn, dtype=torch.float64, device=dev),
               "com": torch.empty((nn, 3), dtype=torch.float64, device=dev),
               "mono": torch.empty((nn, nm), dtype=torch.float64, device=dev)}
        _check(lib().g4_tree_moments(self.h, _ptr(out["mass"]), _ptr(out["com"]), _ptr(out["mono"]),
                                     _stream(stream)), "g4_tree_moments")
        return out

    def gravity_tree(self, pos_sorted, mass_sorted, cls_sorted, aold_sorted, p: G4Params,
                     active=None, acc=None, pot=None, counts=None, stream=None, perm=None):
        """Tree walk; outputs in sorted order, or in input order through perm
        (g4_gravity_tree_perm: the scatter fused into the walk)."""
        n = pos_sorted.shape[1]
        dev = pos_sorted.device
        acc = acc if acc is not None else torch.zeros((3, n), dtype=torch.float32, device=dev)
        pot = pot if pot is not None else torch.zeros(n, dtype=torch.float32, device=dev)
        counts = counts if counts is not None else torch.zeros((2, n), dtype=torch.int32, device=dev)
        na = 0 if active is None else int(active.shape[0])
        if perm is None:
            _check(lib().g4_gravity_tree(self.h, _ptr(pos_sorted), _ptr(mass_sorted), _ptr(cls_sorted),
                                         _ptr(aold_sorted), _ptr(active), na, C.byref(p), _ptr(acc),
                                         _ptr(pot), _ptr(counts), _stream(stream)), "g4_gravity_tree")
        else:
            _check(lib().g4_gravity_tree_perm(self.h, _ptr(pos_sorted), _ptr(mass_sorted),
                                              _ptr(cls_sorted), _ptr(aold_sorted), _ptr(active), na,
                                              C.byref(p), _ptr(perm), _ptr(acc), _ptr(pot),
                                              _ptr(counts), _stream(stream)), "g4_gravity_tree_perm")
        return acc, pot, counts

    def fmm_workspace(self, p: G4Params) -> int:
        b = C.c_size_t()
        _check(lib().g4_fmm_workspace(self.h, C.byref(p), C.byref(b)), "g4_fmm_workspace")
        return int(b.value)

    def gravity_fmm(self, pos_sorted, mass_sorted, cls_sorted, aold_sorted, p: G4Params,
                    workspace=None, acc=None, pot=None, counts=None, momentum=None, stream=None):
        """FMM forces (g4_gravity_fmm).  counts: (3, n) particle pairs, particle-node terms,
        node-node fields of each particle."""
        n = pos_sorted.shape[1]
        dev = pos_sorted.device
        acc = acc if acc is not None else torch.zeros((3, n), dtype=torch.float32, device=dev)
        pot = pot if pot is not None else torch.zeros(n, dtype=torch.float32, device=dev)
        counts = counts if counts is not None else torch.zeros((3, n), dtype=torch.int32, device=dev)
        momentum = momentum if momentum is not None else torch.zeros(3, dtype=torch.float64, device=dev)
        if workspace is None:
            workspace = torch.empty(self.fmm_workspace(p) + 256, dtype=torch.uint8, device=dev)
        wp = workspace.data_ptr()
        off = (-wp) % 256
        _check(lib().g4_gravity_fmm(self.h, _ptr(pos_sorted), _ptr(mass_sorted), _ptr(cls_sorted),
                                    _ptr(aold_sorted), C.byref(p), _ptr(acc), _ptr(pot),
                                    _ptr(counts), _ptr(momentum),
                                    C.c_void_p(wp + off), workspace.numel() - off, _stream(stream)),
               "g4_gravity_fmm")
        return acc, pot, counts, momentum


def g4_direct(pos, mass, cls, p: G4Params, sinks=None, acc=None, pot=None, stream=None):
    n = pos.shape[1]
    dev = pos.device
    acc = acc if acc is not None else torch.zeros((3, n), dtype=torch.float32, device=dev)
    pot = pot if pot is not None else torch.zeros(n, dtype=torch.float32, device=dev)
    ns = 0 if sinks is None else int(sinks.shape[0])
    _check(lib().g4_direct(_ptr(pos), _ptr(mass), _ptr(cls), n, _ptr(sinks), ns, C.byref(p),
                           _ptr(acc), _ptr(pot), _stream(stream)), "g4_direct")
    return acc, pot


# ---- long-range particle-mesh force (TreePM) -------------------------------------------------------

def g4_pm_workspace(n_grid: int) -> int:
    b = C.c_size_t()
    _check(lib().g4_pm_workspace(int(n_grid), C.byref(b)), "g4_pm_workspace")
    return int(b.value)


def g4_pm_long_range(pos, mass, p: G4Params, n_grid: int, sinks=None, acc=None, pot=None,
                     accumulate: bool = False, workspace=None, stream=None):
    """Long-range PM accelerations (3, ns) and potentials (ns,) at the sinks' integer positions
    (3, ns) (default: the sources pos (3, n)); accumulate adds into the given acc/pot."""
    sinks = pos if sinks is None else sinks
    ns = sinks.shape[1]
    dev = pos.device
    acc = acc if acc is not None else torch.zeros((3, ns), dtype=torch.float32, device=dev)
    pot = pot if pot is not None else torch.zeros(ns, dtype=torch.float32, device=dev)
    if workspace is None:
        workspace = torch.empty(g4_pm_workspace(n_grid) + 256, dtype=torch.uint8, device=dev)
    wp = workspace.data_ptr()
    off = (-wp) % 256
    _check(lib().g4_pm_long_range(_ptr(pos), _ptr(mass), int(pos.shape[1]), _ptr(sinks), ns,
                                  C.byref(p), int(n_grid), _ptr(acc), _ptr(pot), int(bool(accumulate)),
                                  C.c_void_p(wp + off), workspace.numel() - off, _stream(stream)),
           "g4_pm_long_range")
    return acc, pot


# ---- whole pipeline ------------------------------------------------------------------------------

class TreeGravity:
    """Preallocated pipeline: keys + sort -> gather -> tree -> moments -> walk (writing its
    results in input order: the scatter is fused into the walk).

    All buffers are allocated once (torch, on the current device), so ``forces`` performs no
    allocation and no host synchronisation and can be captured in a CUDA graph.
    """

    def __init__(self, n: int, p: G4Params, node_capacity: int = 0, with_cls: bool = False):
        dev = torch.device("cuda")
        self.n = n
        self.p = p
        if node_capacity == 0:
            node_capacity = 4096 + int(n * max(1.5, 3.5 / max(1, int(p.leaf_max))))
        self.tree = Tree(n, node_capacity)
        self.keys = torch.empty(n, dtype=torch.int64, device=dev)
        self.perm = torch.empty(n, dtype=torch.int32, device=dev)
        self.ws = torch.empty(g4_keys_sort_workspace(n) + 256, dtype=torch.uint8, device=dev)
        self.pos_s = torch.empty((3, n), dtype=torch.int32, device=dev)
        self.mass_s = torch.empty(n, dtype=torch.float32, device=dev)
        self.cls_s = torch.empty(n, dtype=torch.uint8, device=dev) if with_cls else None
        self.aold_s = torch.empty(n, dtype=torch.float32, device=dev)
        self.acc_s = torch.zeros((3, n), dtype=torch.float32, device=dev)
        self.pot_s = torch.zeros(n, dtype=torch.float32, device=dev)
        self.counts = torch.zeros((2, n), dtype=torch.int32, device=dev)
        self.acc = torch.zeros((3, n), dtype=torch.float32, device=dev)
        self.pot = torch.zeros(n, dtype=torch.float32, device=dev)

    def prepare(self, pos_int, mass, cls=None, aold=None, p: G4Params | None = None, stream=None,
                shift=None):
        """Keys, sort, gather, tree and multipoles.  shift: optional integer vector added to all
        positions first (the random translation of Sec. 3.8; periodic boxes), on a copy."""
        p = p or self.p
        if shift is not None:
            if getattr(self, "pos_shift", None) is None:
                self.pos_shift = torch.empty_like(pos_int)
            pos_int = g4_translate(pos_int, shift, out=self.pos_shift, stream=stream)
        g4_keys_sort(pos_int, self.keys, self.perm, self.ws, stream)
        g4_gather(self.perm, pos_int, mass, cls if self.cls_s is not None else None, aold,
                  out=(self.pos_s, self.mass_s, self.cls_s if cls is not None else None,
                       self.aold_s if aold is not None else None), stream=stream)
        self.tree.build(self.keys, self.pos_s, p, stream)
        self.tree.multipoles(self.pos_s, self.mass_s, self.cls_s if cls is not None else None,
                             self.aold_s if aold is not None else None, p, stream)

    def walk(self, p: G4Params | None = None, use_aold: bool = True, stream=None):
        """The walk, writing accelerations and potentials straight to input order."""
        p = p or self.p
        self.tree.gravity_tree(self.pos_s, self.mass_s, self.cls_s,
                               self.aold_s if use_aold else None, p, acc=self.acc, pot=self.pot,
                               counts=self.counts, stream=stream, perm=self.perm)
        return self.acc, self.pot

    def forces(self, pos_int, mass, cls=None, aold=None, p: G4Params | None = None, stream=None,
               shift=None):
        self.prepare(pos_int, mass, cls, aold, p, stream, shift)
        return self.walk(p, use_aold=aold is not None, stream=stream)


class TreePMGravity:
    """Total TreePM forces (Sec. 2.3): the tree walk's short-range forces plus the PM long-range
    forces, both on the PH-sorted particles, then one scatter to input order.  The relative
    opening criterion takes |a_old| of the total force (the paper compares the node error
    with the total acceleration, PM included)."""

    def __init__(self, n: int, p: G4Params, n_grid: int, node_capacity: int = 0, with_cls: bool = False):
        self.tg = TreeGravity(n, p, node_capacity, with_cls)
        self.p = p
        self.n_grid = n_grid
        self.ws = torch.empty(g4_pm_workspace(n_grid) + 256, dtype=torch.uint8, device="cuda")

    def forces(self, pos_int, mass, cls=None, aold=None, p: G4Params | None = None, stream=None):
        p = p or self.p
        tg = self.tg
        tg.prepare(pos_int, mass, cls, aold, p, stream)
        tg.tree.gravity_tree(tg.pos_s, tg.mass_s, tg.cls_s if cls is not None else None,
                             tg.aold_s if aold is not None else None, p, acc=tg.acc_s, pot=tg.pot_s,
                             counts=tg.counts, stream=stream)
        g4_pm_long_range(tg.pos_s, tg.mass_s, p, self.n_grid, acc=tg.acc_s, pot=tg.pot_s,
                         accumulate=True, workspace=self.ws, stream=stream)
        g4_scatter(tg.perm, tg.acc_s, tg.pot_s, out=(tg.acc, tg.pot), stream=stream)
        return tg.acc, tg.pot


class HostPipeline:
    """Forces for a stream of host input sets (pinned host tensors), double-buffered: the copy
    of the next step's inputs to the device and the copy of the previous step's results back to
    the host run on two copy streams while the current step computes.  Every step still moves its
    whole input (positions, masses, |a_old|) and output (accelerations, potentials) across the
    link; the results are those of TreeGravity.forces."""

    def __init__(self, n: int, p: G4Params, node_capacity: int = 0):
        dev = torch.device("cuda")
        self.n, self.p = n, p
        self.tg = TreeGravity(n, p, node_capacity)
        self.h2d = torch.cuda.Stream()
        self.d2h = torch.cuda.Stream()
        self.inp = [(torch.empty((3, n), dtype=torch.int32, device=dev),
                     torch.empty(n, dtype=torch.float32, device=dev),
                     torch.empty(n, dtype=torch.float32, device=dev)) for _ in range(2)]
        self.out = [(torch.empty((3, n), dtype=torch.float32, device=dev),
                     torch.empty(n, dtype=torch.float32, device=dev)) for _ in range(2)]
        ev = lambda: [torch.cuda.Event() for _ in range(2)]
        self.in_ready, self.in_free, self.out_ready, self.out_free = ev(), ev(), ev(), ev()
        self.k = 0

    def submit(self, h_pos, h_mass, h_aold, h_acc, h_pot, p: G4Params | None = None):
        """Enqueue one step: inputs from, results into pinned host tensors (h_acc (3, n),
        h_pot (n,)).  Returns an event (on the result-copy stream) that completes when h_acc and h_pot
        hold this step's results."""
        p = p or self.p
        b = self.k & 1
        cs, ds, ms = self.h2d, self.d2h, torch.cuda.current_stream()
        d_pos, d_mass, d_aold = self.inp[b]
        d_acc, d_pot = self.out[b]
        cs.wait_event(self.in_free[b])          # step k-2 has finished reading this input set
        with torch.cuda.stream(cs):
            d_pos.copy_(h_pos, non_blocking=True)
            d_mass.copy_(h_mass, non_blocking=True)
            d_aold.copy_(h_aold, non_blocking=True)
            self.in_ready[b].record(cs)
        ms.wait_event(self.in_ready[b])
        ms.wait_event(self.out_free[b])         # step k-2's results have left this buffer
        tg = self.tg
        tg.prepare(d_pos, d_mass, None, d_aold, p)
        self.in_free[b].record(ms)
        tg.tree.gravity_tree(tg.pos_s, tg.mass_s, None, tg.aold_s, p, acc=d_acc, pot=d_pot,
                             counts=tg.counts, perm=tg.perm)
        self.out_ready[b].record(ms)
        ds.wait_event(self.out_ready[b])
        done = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(ds):
            h_acc.copy_(d_acc, non_blocking=True)
            h_pot.copy_(d_pot, non_blocking=True)
            self.out_free[b].record(ds)
            done.record(ds)
        self.k += 1
        return done


class ForestGravity:
    """Many independent systems solved together: one batched sort, one forest build, one
    moments pass and one persistent walk launch for all systems (no per-system launches).

    sizes: particle count per system; particles are passed system-major (system 0 first).
    """

    def __init__(self, sizes, p: G4Params, node_capacity: int = 0):
        dev = torch.device("cuda")
        sizes = [int(k) for k in sizes]
        if min(sizes) < 1:
            raise G4Error("every system needs at least one particle")
        self.n = n = sum(sizes)
        self.p = p
        first = [0]
        for k in sizes:
            first.append(first[-1] + k)
        self.sys_first = torch.tensor(first, dtype=torch.int32, device=dev)
        self.sys_id = torch.repeat_interleave(torch.arange(len(sizes), dtype=torch.int32),
                                              torch.tensor(sizes)).to(torch.int16).to(dev)
        if node_capacity == 0:
            node_capacity = 4096 + len(sizes) + int(n * max(1.5, 3.5 / max(1, int(p.leaf_max))))
        self.tree = Tree(n, node_capacity)
        b = C.c_size_t()
        _check(lib().g4_keys_sort_batched_workspace(n, C.byref(b)), "g4_keys_sort_batched_workspace")
        self.ws = torch.empty(int(b.value) + 256, dtype=torch.uint8, device=dev)
        self.keys = torch.empty(n, dtype=torch.int64, device=dev)
        self.perm = torch.empty(n, dtype=torch.int32, device=dev)
        self.pos_s = torch.empty((3, n), dtype=torch.int32, device=dev)
        self.mass_s = torch.empty(n, dtype=torch.float32, device=dev)
        self.aold_s = torch.empty(n, dtype=torch.float32, device=dev)
        self.acc_s = torch.zeros((3, n), dtype=torch.float32, device=dev)
        self.pot_s = torch.zeros(n, dtype=torch.float32, device=dev)
        self.counts = torch.zeros((2, n), dtype=torch.int32, device=dev)
        self.acc = torch.zeros((3, n), dtype=torch.float32, device=dev)
        self.pot = torch.zeros(n, dtype=torch.float32, device=dev)

    def forces(self, pos_int, mass, sys_box, aold=None, p: G4Params | None = None, stream=None):
        """pos_int (3,n) int32 (each system in its own integer frame), mass (n,) float32,
        sys_box (n_sys,) float64 CUDA (kept alive by this object until the next call)."""
        p = p or self.p
        self.sys_box = sys_box
        g4_keys_sort_batched(pos_int, self.sys_id, self.keys, self.perm, self.ws, stream)
        g4_gather(self.perm, pos_int, mass, None, aold,
                  out=(self.pos_s, self.mass_s, None, self.aold_s if aold is not None else None),
                  stream=stream)
        self.tree.build_forest(self.keys, self.pos_s, self.sys_first, sys_box, p, stream)
        self.tree.multipoles(self.pos_s, self.mass_s, None, self.aold_s if aold is not None else None,
                             p, stream)
        self.tree.gravity_tree(self.pos_s, self.mass_s, None, self.aold_s if aold is not None else None,
                               p, acc=self.acc, pot=self.pot, counts=self.counts, stream=stream,
                               perm=self.perm)
        return self.acc, self.pot


# ---- learned cost model ---------------------------------------------------------------------------

class CostModel:
    """6 -> 32 -> 32 -> 1 MLP (BF16 weights/activations, FP32 sums) predicting log(1 + cost)
    of each sink's walk from tree features; trained on the GPU by g4_mlp_train_step."""

    def __init__(self, seed: int = 0):
        dev = torch.device("cuda")
        self.np = int(lib().g4_mlp_param_count())
        g = torch.Generator().manual_seed(seed)
        p = torch.empty(self.np)
        # He-style initialisation, biases zero (layout W1,b1,W2,b2,W3,b3)
        o = 0
        for shape in ((32, 6), (32,), (32, 32), (32,), (32,), (1,)):
            k = 1
            for d in shape:
                k *= d
            if len(shape) == 2:
                p[o:o + k] = torch.randn(k, generator=g) * (2.0 / shape[1]) ** 0.5
            else:
                p[o:o + k] = 0.0
            o += k
        p[self.np - 33:self.np - 1] = torch.randn(32, generator=g) * (1.0 / 32) ** 0.5
        self.params = p.to(dev)
        self.m = torch.zeros(self.np, device=dev)
        self.v = torch.zeros(self.np, device=dev)
        self.step = 0
        self.loss = torch.zeros(1, device=dev)

    def train(self, features, labels, steps: int = 200, lr: float = 3e-3, stream=None):
        n = labels.shape[0]
        b = C.c_size_t()
        _check(lib().g4_mlp_train_workspace(n, C.byref(b)), "g4_mlp_train_workspace")
        ws = torch.empty(int(b.value) // 4 + 64, dtype=torch.float32, device=labels.device)
        losses = []
        for _ in range(steps):
            self.step += 1
            _check(lib().g4_mlp_train_step(_ptr(self.params), _ptr(self.m), _ptr(self.v), self.step,
                                           _ptr(features), _ptr(labels), n, float(lr), _ptr(self.loss),
                                           None, _ptr(ws), ws.numel() * 4, _stream(stream)),
                   "g4_mlp_train_step")
            losses.append(self.loss.clone())
        return torch.cat(losses)

    def gradient(self, features, labels, stream=None):
        n = labels.shape[0]
        b = C.c_size_t()
        _check(lib().g4_mlp_train_workspace(n, C.byref(b)), "g4_mlp_train_workspace")
        ws = torch.empty(int(b.value) // 4 + 64, dtype=torch.float32, device=labels.device)
        grad = torch.empty(self.np, device=labels.device)
        m = torch.zeros_like(self.m)
        v = torch.zeros_like(self.v)
        _check(lib().g4_mlp_train_step(_ptr(self.params), _ptr(m), _ptr(v), 1, _ptr(features),
                                       _ptr(labels), n, 0.0, _ptr(self.loss), _ptr(grad), _ptr(ws),
                                       ws.numel() * 4, _stream(stream)), "g4_mlp_train_step")
        return grad, self.loss.clone()

    def predict(self, features, out=None, stream=None):
        n = features.shape[0]
        out = out if out is not None else torch.empty(n, device=features.device)
        _check(lib().g4_mlp_forward(_ptr(self.params), _ptr(features), n, _ptr(out), _stream(stream)),
               "g4_mlp_forward")
        return out


def cost_features(tree: Tree, p: G4Params, n: int, aold_sorted=None, bins_sorted=None, out=None,
                  scratch=None, stream=None):
    """(n, 6) float32 features of the tree's PH-sorted particles (g4_cost_features)."""
    dev = torch.device("cuda")
    out = out if out is not None else torch.empty((n, 6), dtype=torch.float32, device=dev)
    scratch = scratch if scratch is not None else torch.empty(n, dtype=torch.int32, device=dev)
    _check(lib().g4_cost_features(tree.h, _ptr(aold_sorted), _ptr(bins_sorted), C.byref(p), _ptr(out),
                                  _ptr(scratch), _stream(stream)), "g4_cost_features")
    return out


def cost_labels(counts, c_pn: float = 5.0, out=None, stream=None):
    n = counts.shape[1]
    out = out if out is not None else torch.empty(n, device=counts.device)
    _check(lib().g4_cost_labels(_ptr(counts), n, float(c_pn), _ptr(out), _stream(stream)), "g4_cost_labels")
    return out


def schedule_lpt(pred_sorted, chunk: int = 1, group_order=None, stream=None):
    n = pred_sorted.shape[0]
    ng = (n + 31) // 32
    group_order = group_order if group_order is not None else torch.empty(ng, dtype=torch.int32,
                                                                         device=pred_sorted.device)
    b = C.c_size_t()
    _check(lib().g4_schedule_workspace(n, C.byref(b)), "g4_schedule_workspace")
    ws = torch.empty(int(b.value) + 256, dtype=torch.uint8, device=pred_sorted.device)
    wp = ws.data_ptr()
    off = (-wp) % 256
    _check(lib().g4_schedule_lpt(_ptr(pred_sorted), n, int(chunk), _ptr(group_order), C.c_void_p(wp + off),
                                 ws.numel() - off, _stream(stream)), "g4_schedule_lpt")
    return group_order


ITEM_SPLIT_MAX = 8


def resident_warps() -> int:
    """Warps the persistent walk keeps resident on the current GPU (5 four-warp blocks per SM)."""
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count * 5 * 4


MAX_SPLIT = 16384     # split groups per handle (6 KB of partial sums each)


def schedule_items(pred_sorted, target: int = 0, max_split: int = MAX_SPLIT, stream=None):
    """Cost-partitioned work items of the walk (g4_schedule_items): returns (items, n_items),
    items a (capacity, 4) int32 tensor of (first sink, count, part | parts << 8, split slot),
    n_items a 1-element device tensor.  target = 0: four items per resident warp."""
    n = pred_sorted.shape[0]
    dev = pred_sorted.device
    cap = ITEM_SPLIT_MAX * ((n + 31) // 32)
    items = torch.zeros((max(cap, 1), 4), dtype=torch.int32, device=dev)
    n_items = torch.zeros(1, dtype=torch.int32, device=dev)
    b = C.c_size_t()
    _check(lib().g4_schedule_items_workspace(n, C.byref(b)), "g4_schedule_items_workspace")
    ws = torch.empty(int(b.value) + 256, dtype=torch.uint8, device=dev)
    wp = ws.data_ptr()
    off = (-wp) % 256
    tgt = int(target) if target else 4 * resident_warps()
    _check(lib().g4_schedule_items(_ptr(pred_sorted), n, tgt, int(max_split), _ptr(items), _ptr(n_items),
                                   C.c_void_p(wp + off), ws.numel() - off, _stream(stream)),
           "g4_schedule_items")
    return items, n_items


def set_work_items(tree: Tree, items=None, n_items=None, n_sinks: int = 0, max_split: int = MAX_SPLIT):
    """Make later walks on this handle take their work from `items` (None: plain groups)."""
    tree._items_ref = (items, n_items)
    cap = 0 if items is None else int(items.shape[0])
    _check(lib().g4_tree_set_work_items(tree.h, _ptr(items), _ptr(n_items), cap,
                                        int(n_sinks) if items is not None else 0, int(max_split)),
           "g4_tree_set_work_items")


def set_group_order(tree: Tree, group_order=None):
    ng = 0 if group_order is None else int(group_order.shape[0])
    tree._order_ref = group_order
    _check(lib().g4_tree_set_group_order(tree.h, _ptr(group_order), ng), "g4_tree_set_group_order")


# ---- hierarchical time bins: one force call per bin over its active subset -------------------------

class BinnedForces:
    """Force calls over nested active subsets (the hierarchical time integration of the paper
    builds each force call's tree over the active particles only).  Every bin has its own
    preallocated pipeline, so the whole sequence allocates nothing and can be captured in one
    CUDA graph (``capture``) and replayed."""

    def __init__(self, n_all: int, active_lists, p: G4Params, with_cls: bool = False):
        dev = torch.device("cuda")
        self.n_all = n_all
        self.p = p
        self.idx = [torch.as_tensor(a, dtype=torch.int32).to(dev) for a in active_lists]
        self.bins = []
        for ix in self.idx:
            k = int(ix.shape[0])
            tg = TreeGravity(k, p, with_cls=with_cls)
            sub = (torch.empty((3, k), dtype=torch.int32, device=dev),
                   torch.empty(k, dtype=torch.float32, device=dev),
                   torch.empty(k, dtype=torch.uint8, device=dev) if with_cls else None,
                   torch.empty(k, dtype=torch.float32, device=dev))
            self.bins.append((tg, sub))
        self.acc = [torch.zeros((3, n_all), dtype=torch.float32, device=dev) for _ in self.idx]
        self.pot = [torch.zeros(n_all, dtype=torch.float32, device=dev) for _ in self.idx]
        self.graph = None

    def run_bin(self, b, pos_int, mass, cls, aold, stream=None):
        """One force call: gather bin b's active subset, its own tree and walk, scatter."""
        ix, (tg, sub) = self.idx[b], self.bins[b]
        k = int(ix.shape[0])
        _check(lib().g4_gather_subset(_ptr(ix), k, self.n_all, _ptr(pos_int), _ptr(mass), _ptr(cls),
                                      _ptr(aold), _ptr(sub[0]), _ptr(sub[1]), _ptr(sub[2]),
                                      _ptr(sub[3]), _stream(stream)), "g4_gather_subset")
        acc, pot = tg.forces(sub[0], sub[1], sub[2], sub[3], self.p, stream)
        _check(lib().g4_scatter_subset(_ptr(ix), k, self.n_all, _ptr(acc), _ptr(pot), _ptr(self.acc[b]),
                                       _ptr(self.pot[b]), _stream(stream)), "g4_scatter_subset")

    def run(self, pos_int, mass, cls, aold, stream=None):
        for b in range(len(self.idx)):
            self.run_bin(b, pos_int, mass, cls, aold, stream)
        return self.acc, self.pot

    def set_cost_model(self, model, stream=None):
        """Partition every bin's walk by the model's predicted costs (g4_schedule_items), from
        the features of the bin's current tree; None restores the plain groups."""
        if model is None:
            self.set_partition(None)
            return
        self.set_partition([model.predict(cost_features(tg.tree, self.p, int(ix.shape[0]), tg.aold_s,
                                                        stream=stream), stream=stream)
                            for ix, (tg, sub) in zip(self.idx, self.bins)], stream)

    def measured_costs(self):
        """log(1 + cost) per sorted sink of every bin from the interaction counts of its last
        walk: the paper's q_i, the interactions of the last force computation (Sec. 6.1)."""
        return [cost_labels(tg.counts) for tg, _ in self.bins]

    def set_partition(self, preds, stream=None):
        """Partition bin b's walk by preds[b] (log(1 + cost) per sorted sink); None: plain."""
        for b, (ix, (tg, sub)) in enumerate(zip(self.idx, self.bins)):
            if preds is None:
                set_work_items(tg.tree, None)
                continue
            items, ni = schedule_items(preds[b], stream=stream)
            set_work_items(tg.tree, items, ni, int(ix.shape[0]))
        self.graph = None

    def capture(self, pos_int, mass, cls, aold):
        """Capture the whole bin sequence in one CUDA graph (inputs are bound by address)."""
        self.run(pos_int, mass, cls, aold)          # first call outside capture (lazy init)
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.run(pos_int, mass, cls, aold)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()
        return self.acc, self.pot


# ---- hierarchical time integration (Sec. 4.2) -------------------------------------------------------

def g4_translate(pos_in, shift, out=None, stream=None):
    """pos_in + shift modulo 2^32 (Sec. 3.8); shift: three integers (taken modulo 2^32)."""
    n = pos_in.shape[1]
    out = out if out is not None else torch.empty_like(pos_in)
    sh = (C.c_uint32 * 3)(*[int(v) % (1 << 32) for v in shift])
    _check(lib().g4_translate(_ptr(pos_in), _ptr(out), n, sh, _stream(stream)), "g4_translate")
    return out


def g4_kick(vel, acc, dt: float, idx=None, stream=None):
    n = vel.shape[1]
    m = n if idx is None else int(idx.shape[0])
    _check(lib().g4_kick(_ptr(vel), _ptr(acc), _ptr(idx), m, n, float(dt), _stream(stream)), "g4_kick")


def g4_drift(pos_int, vel, dt: float, p: G4Params, idx=None, flag=None, stream=None):
    n = vel.shape[1]
    m = n if idx is None else int(idx.shape[0])
    _check(lib().g4_drift(_ptr(pos_int), _ptr(vel), _ptr(idx), m, n, float(dt), C.byref(p), _ptr(flag),
                          _stream(stream)), "g4_drift")


def g4_timestep_bins(acc, p: G4Params, eta: float, dt_max: float, max_bin: int, bins, cls=None, idx=None,
                     stream=None):
    n = acc.shape[1]
    m = n if idx is None else int(idx.shape[0])
    _check(lib().g4_timestep_bins(_ptr(acc), _ptr(cls), _ptr(idx), m, n, C.byref(p), float(eta),
                                  float(dt_max), int(max_bin), _ptr(bins), _stream(stream)),
           "g4_timestep_bins")


class SubsetForces:
    """Forces of a particle subset on itself: the subset is gathered, sorted, gets its own tree
    (the hierarchical scheme builds the tree over the particles of the current force
    computation only) and its tree walk or FMM; the results are written into full-size arrays
    at the subset's indices.  One handle and one set of buffers sized for all n particles."""

    def __init__(self, n: int, p: G4Params, method: str = "fmm", with_cls: bool = False):
        if method not in ("fmm", "tree"):
            raise G4Error("method must be 'fmm' or 'tree'")
        dev = torch.device("cuda")
        self.n, self.p, self.method = n, p, method
        self.tree = Tree(n, 4096 + int(n * max(1.5, 3.5 / max(1, int(p.leaf_max)))))
        self.keys = torch.empty(n, dtype=torch.int64, device=dev)
        self.perm = torch.empty(n, dtype=torch.int32, device=dev)
        self.ws = torch.empty(g4_keys_sort_workspace(n) + 256, dtype=torch.uint8, device=dev)
        f = lambda dt, k=1: torch.empty(k * n, dtype=dt, device=dev)
        self.pos_sub, self.pos_s = f(torch.int32, 3), f(torch.int32, 3)
        self.mass_sub, self.mass_s = f(torch.float32), f(torch.float32)
        self.aold_sub, self.aold_s = f(torch.float32), f(torch.float32)
        self.cls_sub = f(torch.uint8) if with_cls else None
        self.cls_s = f(torch.uint8) if with_cls else None
        self.acc_s, self.acc_sub = f(torch.float32, 3), f(torch.float32, 3)
        self.pot_s, self.pot_sub = f(torch.float32), f(torch.float32)
        self.counts = torch.zeros(3 * n, dtype=torch.int32, device=dev)
        self.fmm_ws = (torch.empty(self.tree.fmm_workspace(p) + 256, dtype=torch.uint8, device=dev)
                       if method == "fmm" else None)

    def __call__(self, pos_all, mass_all, cls_all, aold_all, idx, acc_out, pot_out, p=None, stream=None):
        p = p or self.p
        k = int(idx.shape[0])
        n_all = int(pos_all.shape[1])
        v3 = lambda t: t[:3 * k].view(3, k)
        cls_sub = self.cls_sub[:k] if cls_all is not None else None
        aold_sub = self.aold_sub[:k] if aold_all is not None else None
        _check(lib().g4_gather_subset(_ptr(idx), k, n_all, _ptr(pos_all), _ptr(mass_all), _ptr(cls_all),
                                      _ptr(aold_all), _ptr(v3(self.pos_sub)), _ptr(self.mass_sub[:k]),
                                      _ptr(cls_sub), _ptr(aold_sub), _stream(stream)), "g4_gather_subset")
        g4_keys_sort(v3(self.pos_sub), self.keys[:k], self.perm[:k], self.ws, stream)
        cls_s = self.cls_s[:k] if cls_all is not None else None
        aold_s = self.aold_s[:k] if aold_all is not None else None
        g4_gather(self.perm[:k], v3(self.pos_sub), self.mass_sub[:k], cls_sub, aold_sub,
                  out=(v3(self.pos_s), self.mass_s[:k], cls_s, aold_s), stream=stream)
        self.tree.build(self.keys[:k], v3(self.pos_s), p, stream)
        self.tree.multipoles(v3(self.pos_s), self.mass_s[:k], cls_s, aold_s, p, stream)
        if self.method == "fmm":
            self.tree.gravity_fmm(v3(self.pos_s), self.mass_s[:k], cls_s, aold_s, p, workspace=self.fmm_ws,
                                  acc=v3(self.acc_s), pot=self.pot_s[:k], counts=v3(self.counts),
                                  stream=stream)
            g4_scatter(self.perm[:k], v3(self.acc_s), self.pot_s[:k], out=(v3(self.acc_sub), self.pot_sub[:k]),
                       stream=stream)
        else:
            self.tree.gravity_tree(v3(self.pos_s), self.mass_s[:k], cls_s, aold_s, p, acc=v3(self.acc_sub),
                                   pot=self.pot_sub[:k], counts=self.counts[:2 * k].view(2, k), stream=stream,
                                   perm=self.perm[:k])
        _check(lib().g4_scatter_subset(_ptr(idx), k, n_all, _ptr(v3(self.acc_sub)), _ptr(self.pot_sub[:k]),
                                       _ptr(acc_out), _ptr(pot_out), _stream(stream)), "g4_scatter_subset")


class HierarchicalKDK:
    """Hierarchical time integration (Sec. 4.2) on the GPU.  A step dt of a set P with known
    forces a_P (sourced by P): kick P by a_P dt/2; split P into fast particles F (timestep
    criterion sqrt(2 eta eps_i / |a_i|) < dt, g4_timestep_bins) and slow S; no F: drift P by dt,
    forces of P, kick by dt/2; otherwise forces of F on F, kick F by -dt/2, two recursive steps
    of F over dt/2 with the drift of S by dt between them, kick F by -dt/2 with F's final
    forces, forces of P, kick P by dt/2.  Every force computation has equal source and sink sets
    (SubsetForces: a tree over that set only), so with the FMM the total momentum is conserved
    to the rounding of the kicks.  pos_int (3, n) int32 (uint32 bits) and vel (3, n) float32 are
    updated in place.  criterion 0 (relative) takes |a_old| from each particle's latest force."""

    def __init__(self, pos_int, vel, mass, p: G4Params, eta: float = 0.025, method: str = "fmm",
                 cls=None, max_level: int = 10):
        dev = torch.device("cuda")
        self.pos, self.vel, self.mass, self.cls = pos_int, vel, mass, cls
        self.n = n = int(pos_int.shape[1])
        self.p, self.eta, self.max_level = p, eta, max_level
        self.forces = SubsetForces(n, p, method, cls is not None)
        self.acc = [torch.zeros((3, n), dtype=torch.float32, device=dev) for _ in range(max_level + 2)]
        self.pot = torch.zeros(n, dtype=torch.float32, device=dev)
        self.aold = torch.zeros(n, dtype=torch.float32, device=dev)
        self.bins = torch.zeros(n, dtype=torch.uint8, device=dev)
        self.flag = torch.zeros(1, dtype=torch.int32, device=dev)
        self.all = torch.arange(n, dtype=torch.int32, device=dev)
        self.n_force = 0
        self.started = False

    def _force(self, idx, level):
        use_aold = self.p.criterion == 0
        self.forces(self.pos, self.mass, self.cls, self.aold if use_aold else None, idx,
                    self.acc[level], self.pot)
        if use_aold:
            a = torch.linalg.vector_norm(self.acc[level][:, idx.long()], dim=0)
            self.aold[idx.long()] = a
        self.n_force += int(idx.shape[0])

    def start(self, p_bootstrap: G4Params | None = None):
        """Forces of all particles (with p_bootstrap, e.g. the geometric criterion, when the
        relative criterion has no |a_old| yet)."""
        if p_bootstrap is not None:
            self.forces(self.pos, self.mass, self.cls, None, self.all, self.acc[0], self.pot, p_bootstrap)
            self.aold = torch.linalg.vector_norm(self.acc[0], dim=0).contiguous()
        self._force(self.all, 0)
        self.started = True

    def step(self, dt: float):
        if not self.started:
            self.start()
        self._step(self.all, dt, 0)

    def _step(self, P, dt, level):
        acc = self.acc[level]
        g4_kick(self.vel, acc, 0.5 * dt, P)
        F = None
        if level < self.max_level:
            g4_timestep_bins(acc, self.p, self.eta, dt, 1, self.bins, self.cls, P)
            fast = self.bins[P.long()] > 0
            if bool(fast.any()):
                F, S = P[fast].contiguous(), P[~fast].contiguous()
        if F is None:
            g4_drift(self.pos, self.vel, dt, self.p, P, self.flag)
            self._force(P, level)
            g4_kick(self.vel, acc, 0.5 * dt, P)
            return
        self._force(F, level + 1)
        g4_kick(self.vel, self.acc[level + 1], -0.5 * dt, F)
        self._step(F, 0.5 * dt, level + 1)
        if S.numel():
            g4_drift(self.pos, self.vel, dt, self.p, S, self.flag)
        self._step(F, 0.5 * dt, level + 1)
        g4_kick(self.vel, self.acc[level + 1], -0.5 * dt, F)
        self._force(P, level)
        g4_kick(self.vel, acc, 0.5 * dt, P)

    def momentum(self):
        """Total momentum sum m v (FP64)."""
        return (self.mass.double()[None, :] * self.vel.double()).sum(dim=1)


# ---- pure periodic tree: the Ewald correction grid (Sec. 2.2.4) ------------------------------

def g4_ewald_eval(tree: "Tree", x, nmax: int, box: float, stream=None):
    """D_abc[psi] (a + b + c <= nmax) of the Ewald correction potential at separations x (n, 3)
    FP64 (nearest-image range), from the handle's grid by Taylor expansion: (n, nmono) FP64."""
    x = x.contiguous().to(torch.float64)
    n = x.shape[0]
    nm = (nmax + 1) * (nmax + 2) * (nmax + 3) // 6
    out = torch.empty((n, nm), dtype=torch.float64, device=x.device)
    _check(lib().g4_ewald_eval(tree.h, x.data_ptr(), n, int(nmax), float(box), out.data_ptr(),
                               _stream(stream)), "g4_ewald_eval")
    return out
