"""FP64 CPU oracle for the short-range tree/FMM gravity path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package.  The product path (the CUDA library and its binding)
never calls it; the two share no code.  The arithmetic lives in ``g4_oracle.c``, built with
plain gcc (``-O2 -fopenmp -ffp-contract=off``, no fast-math) into ``oracle/_build``.

Parity pins for every function are in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "g4_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libg4oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, OpenMP, no FMA contraction, no fast-math)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-std=gnu11",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_OUT)
        _declare(_lib)
    return _lib


class _Params(C.Structure):
    _fields_ = [("box", C.c_double), ("periodic", C.c_int), ("r_s", C.c_double),
                ("r_cut", C.c_double), ("pp_cut", C.c_int), ("alpha", C.c_double),
                ("theta", C.c_double), ("criterion", C.c_int), ("order", C.c_int),
                ("exclusion", C.c_int), ("G", C.c_double), ("n_eps", C.c_int),
                ("eps", C.POINTER(C.c_double)), ("keep_qp", C.c_int), ("soft_nodes", C.c_int),
                ("ewald", C.c_int)]


@dataclass
class OracleParams:
    box: float
    periodic: bool
    eps: np.ndarray
    r_s: float = 0.0
    r_cut_factor: float = 4.5
    pp_cut: bool = True
    alpha: float = 0.0025
    theta: float = 0.5
    criterion: int = 0          # 0 relative, 1 geometric
    order: int = 3
    exclusion: bool = True
    G: float = 1.0
    keep_qp: bool = False
    soft_nodes: bool = False
    ewald: bool = False         # periodic, r_s = 0: Ewald-corrected pure tree (Sec. 2.2.4)
    _eps_buf: np.ndarray = field(default=None, repr=False)

    @property
    def r_cut(self) -> float:
        """r_cut = max(R_cut r_s, 2.8 eps_max) (Sec. 2.3)."""
        if self.r_s <= 0:
            return 0.0
        return max(self.r_cut_factor * self.r_s, 2.8 * float(np.max(self.eps)))

    def c(self) -> _Params:
        self._eps_buf = np.ascontiguousarray(self.eps, dtype=np.float64)
        return _Params(float(self.box), int(self.periodic), float(self.r_s), float(self.r_cut),
                       int(self.pp_cut), float(self.alpha), float(self.theta),
                       int(self.criterion), int(self.order), int(self.exclusion),
                       float(self.G), int(len(self._eps_buf)),
                       self._eps_buf.ctypes.data_as(C.POINTER(C.c_double)),
                       int(self.keep_qp), int(self.soft_nodes), int(self.ewald))


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None else C.c_void_p(0)


def _declare(L):
    i64, vp, d, i32 = C.c_int64, C.c_void_p, C.c_double, C.c_int
    L.or_int_coords_periodic.argtypes = [vp, i64, d, vp]
    L.or_int_coords_isolated.argtypes = [vp, i64, vp, vp]
    L.or_hilbert_key.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, i32]
    L.or_hilbert_key.restype = C.c_uint64
    L.or_keys.argtypes = [vp, i64, vp]
    L.or_sort.argtypes = [vp, i64, vp, vp]
    L.or_tree_build.argtypes = [vp, vp, i64, i32]
    L.or_tree_build.restype = vp
    L.or_tree_nnodes.argtypes = [vp]
    L.or_tree_nnodes.restype = i64
    L.or_tree_export.argtypes = [vp, vp, vp, vp, vp, vp]
    L.or_tree_free.argtypes = [vp]
    L.or_multipoles.argtypes = [vp, vp, i64, vp, vp, vp, C.POINTER(_Params)]
    L.or_tree_export_moments.argtypes = [vp, vp, vp, vp, vp, vp]
    L.or_soft_kernel.argtypes = [d, d, C.POINTER(d), C.POINTER(d)]
    L.or_pair_kernel.argtypes = [d, d, d, C.POINTER(d), C.POINTER(d)]
    L.or_gn.argtypes = [d, d, i32, vp]
    L.or_gn_soft.argtypes = [d, d, d, i32, vp]
    L.or_pn_soft_eval.argtypes = [vp, vp, i32, d, d, d, vp, vp]
    L.or_D_full.argtypes = [i32, vp, vp, vp]
    L.or_tree_walk.argtypes = [vp, vp, i64, vp, vp, vp, vp, i64, C.POINTER(_Params), vp, vp, vp]
    L.or_direct.argtypes = [vp, i64, vp, vp, vp, i64, C.POINTER(_Params), d, vp, vp]
    L.or_ewald_direct.argtypes = [vp, i64, vp, vp, vp, i64, C.POINTER(_Params), vp, vp]
    L.or_ewald_dpsi_flat.argtypes = [vp, d, i32, vp]
    L.or_fmm.argtypes = [vp, vp, i64, vp, vp, vp, C.POINTER(_Params), vp, vp, vp, vp]
    L.or_moments_points.argtypes = [vp, vp, i64, i32, vp, vp]
    L.or_ewald_psi.argtypes = [vp, d, d, i32, i32]
    L.or_ewald_psi.restype = d
    L.or_ewald_force.argtypes = [vp, d, d, i32, i32, i32, vp]
    L.or_ewald_force_many.argtypes = [vp, i64, vp, vp, i64, d, d, i32, i32, i32, vp]
    L.or_two_node_tree.argtypes = [vp, i64, vp, vp, i64, i32, d, d, vp, vp]
    L.or_two_node_fmm.argtypes = [vp, vp, i64, vp, vp, i64, i32, d, d, i32, vp, vp, vp, vp]


# ---- a1 / a2 / a3 ------------------------------------------------------------------------

def int_coords_periodic(pos: np.ndarray, L: float) -> np.ndarray:
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    out = np.empty((3, pos.shape[0]), np.uint32)
    lib().or_int_coords_periodic(_p(pos), pos.shape[0], float(L), _p(out))
    return out


def int_coords_isolated(pos: np.ndarray):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    out = np.empty((3, pos.shape[0]), np.uint32)
    frame = np.empty(4, np.float64)
    lib().or_int_coords_isolated(_p(pos), pos.shape[0], _p(out), _p(frame))
    return out, frame


def hilbert_key(x: int, y: int, z: int, bits: int) -> int:
    return int(lib().or_hilbert_key(x, y, z, bits))


def keys(pos_int: np.ndarray) -> np.ndarray:
    pos_int = np.ascontiguousarray(pos_int, dtype=np.uint32)
    out = np.empty(pos_int.shape[1], np.uint64)
    lib().or_keys(_p(pos_int), pos_int.shape[1], _p(out))
    return out


def sort(k: np.ndarray):
    k = np.ascontiguousarray(k, dtype=np.uint64)
    ks = np.empty_like(k)
    perm = np.empty(k.shape[0], np.int64)
    lib().or_sort(_p(k), k.shape[0], _p(ks), _p(perm))
    return ks, perm


# ---- kernels ------------------------------------------------------------------------------

def soft_kernel(r: float, h: float):
    g0, g1 = C.c_double(), C.c_double()
    lib().or_soft_kernel(float(r), float(h), C.byref(g0), C.byref(g1))
    return g0.value, g1.value


def pair_kernel(r: float, h: float, r_s: float):
    g0, g1 = C.c_double(), C.c_double()
    lib().or_pair_kernel(float(r), float(h), float(r_s), C.byref(g0), C.byref(g1))
    return g0.value, g1.value


def gn(r: float, r_s: float, nmax: int) -> np.ndarray:
    g = np.zeros(8, np.float64)
    lib().or_gn(float(r), float(r_s), int(nmax), _p(g))
    return g[: nmax + 1].copy()


def gn_soft(r: float, h: float, r_s: float, nmax: int) -> np.ndarray:
    """g_n of the softened kernel (spline inside h, TreePM part when r_s > 0)."""
    g = np.zeros(8, np.float64)
    lib().or_gn_soft(float(r), float(h), float(r_s), int(nmax), _p(g))
    return g[: nmax + 1].copy()


def pn_soft(mono, rvec, order: int, r_s: float, h: float, G: float = 1.0):
    """Particle-node term of the softened kernel: (acc (3,), pot)."""
    mono = np.ascontiguousarray(mono, np.float64)
    rv = np.ascontiguousarray(rvec, np.float64)
    acc = np.zeros(3)
    pot = C.c_double()
    lib().or_pn_soft_eval(_p(mono), _p(rv), int(order), float(r_s), float(h), float(G), _p(acc),
                          C.byref(pot))
    return acc, pot.value


def D_full(m: int, rvec, g) -> np.ndarray:
    rv = np.ascontiguousarray(rvec, dtype=np.float64)
    gg = np.zeros(8, np.float64)
    gg[: len(g)] = g
    out = np.empty(3 ** m, np.float64)
    lib().or_D_full(int(m), _p(rv), _p(gg), _p(out))
    return out


def nmono(order: int) -> int:
    return (order + 1) * (order + 2) * (order + 3) // 6


def mono_index(a: int, b: int, c: int) -> int:
    n = a + b + c
    return n * (n + 1) * (n + 2) // 6 + (n - a) * (n - a + 1) // 2 + (n - a - b)


# ---- tree ---------------------------------------------------------------------------------

class Tree:
    """Oracle oct-tree over PH-sorted particles (depth-first pre-order, children in PH order)."""

    def __init__(self, keys_sorted: np.ndarray, pos_sorted: np.ndarray, leaf_max: int):
        self.keys = np.ascontiguousarray(keys_sorted, dtype=np.uint64)
        self.pos = np.ascontiguousarray(pos_sorted, dtype=np.uint32)
        self.n = int(self.pos.shape[1])
        self.h = lib().or_tree_build(_p(self.keys), _p(self.pos), self.n, int(leaf_max))
        self.order = None

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_tree_free(self.h)
            self.h = None

    @property
    def nnodes(self) -> int:
        return int(lib().or_tree_nnodes(self.h))

    def export(self) -> dict:
        nn = self.nnodes
        level = np.empty(nn, np.int32)
        first = np.empty(nn, np.int64)
        count = np.empty(nn, np.int64)
        nxt = np.empty(nn, np.int64)
        center = np.empty((nn, 3), np.uint32)
        lib().or_tree_export(self.h, _p(level), _p(first), _p(count), _p(nxt), _p(center))
        return {"level": level, "first": first, "count": count, "next": nxt, "center": center}

    def multipoles(self, mass, cls, aold, params: OracleParams):
        self.mass = np.ascontiguousarray(mass, dtype=np.float64)
        self.cls = None if cls is None else np.ascontiguousarray(cls, dtype=np.uint8)
        self.aold = None if aold is None else np.ascontiguousarray(aold, dtype=np.float64)
        cp = params.c()
        lib().or_multipoles(self.h, _p(self.pos), self.n, _p(self.mass), _p(self.cls),
                            _p(self.aold), C.byref(cp))
        self.order = params.order

    def export_moments(self) -> dict:
        nn = self.nnodes
        nm = nmono(self.order)
        mass = np.empty(nn)
        com = np.empty((nn, 3))
        mono = np.empty((nn, nm))
        em = np.empty(nn)
        am = np.empty(nn)
        lib().or_tree_export_moments(self.h, _p(mass), _p(com), _p(mono), _p(em), _p(am))
        return {"mass": mass, "com": com, "mono": mono, "eps_max": em, "amin": am}

    def walk(self, sinks: np.ndarray, params: OracleParams, aold=None):
        """Per-particle one-sided walk for the given sorted-order sinks.
        Returns acc (ns,3), pot (ns,), counts (ns,2) [PP, PN]."""
        sinks = np.ascontiguousarray(sinks, dtype=np.int64)
        ns = sinks.shape[0]
        acc = np.empty((ns, 3))
        pot = np.empty(ns)
        cnt = np.empty((ns, 2), np.int64)
        a = self.aold if aold is None else np.ascontiguousarray(aold, dtype=np.float64)
        cp = params.c()
        lib().or_tree_walk(self.h, _p(self.pos), self.n, _p(self.mass), _p(self.cls), _p(a),
                           _p(sinks), ns, C.byref(cp), _p(acc), _p(pot), _p(cnt))
        return acc, pot, cnt

    def fmm(self, params: OracleParams, per_particle: bool = False):
        """Full FP64 FMM for all particles (sorted order): acc (n,3), pot (n,), counts
        [node-node, particle-node, particle-particle] (each unordered pair once); with
        ``per_particle`` also (n,2) [particle pairs, particle-node terms] of each particle."""
        acc = np.empty((self.n, 3))
        pot = np.empty(self.n)
        cnt = np.empty(3, np.int64)
        pc = np.empty((self.n, 2), np.int64) if per_particle else None
        cp = params.c()
        lib().or_fmm(self.h, _p(self.pos), self.n, _p(self.mass), _p(self.cls), _p(self.aold),
                     C.byref(cp), _p(acc), _p(pot), _p(cnt), _p(pc))
        return (acc, pot, cnt, pc) if per_particle else (acc, pot, cnt)


def moments_points(x, m, order: int):
    """Centre of mass and monomial moments (orders 0..order) of points x (n,3), masses m."""
    x = np.ascontiguousarray(x, np.float64)
    m = np.ascontiguousarray(m, np.float64)
    com = np.empty(3)
    mono = np.empty(nmono(order))
    lib().or_moments_points(_p(x), _p(m), x.shape[0], int(order), _p(com), _p(mono))
    return com, mono


def two_node_tree(xa, xb, mb, order: int, r_s: float = 0.0, G: float = 1.0):
    """One-sided expansion of group B (positions xb (nb,3), masses mb) at the points xa."""
    xa = np.ascontiguousarray(xa, np.float64)
    xb = np.ascontiguousarray(xb, np.float64)
    mb = np.ascontiguousarray(mb, np.float64)
    acc = np.empty((xa.shape[0], 3))
    pot = np.empty(xa.shape[0])
    lib().or_two_node_tree(_p(xa), xa.shape[0], _p(xb), _p(mb), xb.shape[0], int(order),
                           float(r_s), float(G), _p(acc), _p(pot))
    return acc, pot


def two_node_fmm(xa, ma, xb, mb, order: int, r_s: float = 0.0, G: float = 1.0,
                 keep_qp: bool = False):
    """Mutual FMM expansion of groups A and B: (acc_a, pot_a, acc_b, pot_b)."""
    xa = np.ascontiguousarray(xa, np.float64)
    ma = np.ascontiguousarray(ma, np.float64)
    xb = np.ascontiguousarray(xb, np.float64)
    mb = np.ascontiguousarray(mb, np.float64)
    aa, pa = np.empty((xa.shape[0], 3)), np.empty(xa.shape[0])
    ab, pb = np.empty((xb.shape[0], 3)), np.empty(xb.shape[0])
    lib().or_two_node_fmm(_p(xa), _p(ma), xa.shape[0], _p(xb), _p(mb), xb.shape[0], int(order),
                          float(r_s), float(G), int(keep_qp), _p(aa), _p(pa), _p(ab), _p(pb))
    return aa, pa, ab, pb


# ---- periodic Ewald reference (Sec. 2.1) ------------------------------------------------------

def ewald_psi(x, L: float, alpha: float | None = None, nr: int = 4, nk: int = 8) -> float:
    """Correction potential psi(x) of Eq. (eqnewal) for a cubic box of side L."""
    a = 2.0 / L if alpha is None else alpha
    xx = np.ascontiguousarray(x, np.float64)
    return float(lib().or_ewald_psi(_p(xx), float(L), float(a), int(nr), int(nk)))


def ewald_force(xe, ys, m, L: float, alpha: float | None = None, nr: int = 4, nk: int = 8,
                kspace_only: bool = False):
    """Periodic accelerations (G = 1) at the points xe (ne,3) due to masses m at ys (ns,3), by
    Ewald summation; kspace_only with alpha = 1/(2 r_s): the exact long-range TreePM force."""
    a = 2.0 / L if alpha is None else alpha
    xe = np.ascontiguousarray(np.atleast_2d(xe), np.float64)
    ys = np.ascontiguousarray(np.atleast_2d(ys), np.float64)
    m = np.ascontiguousarray(np.atleast_1d(m), np.float64)
    out = np.empty_like(xe)
    lib().or_ewald_force_many(_p(xe), xe.shape[0], _p(ys), _p(m), ys.shape[0], float(L), float(a),
                              int(nr), int(nk), int(kspace_only), _p(out))
    return out


def ewald_dpsi(x, L: float, mmax: int):
    """Derivative tensors D_m[psi](x), m = 0..mmax (<= 6), of the Ewald correction potential
    (full tensors: D[m] has shape (3,)*m)."""
    xx = np.ascontiguousarray(x, np.float64)
    n = sum(3 ** m for m in range(mmax + 1))
    out = np.empty(n)
    lib().or_ewald_dpsi_flat(_p(xx), float(L), int(mmax), _p(out))
    res, o = [], 0
    for m in range(mmax + 1):
        res.append(out[o:o + 3 ** m].reshape((3,) * m) if m else out[o:o + 1].reshape(()))
        o += 3 ** m
    return res


def ewald_direct(pos_int: np.ndarray, mass, cls, sinks, params: OracleParams):
    """Exact periodic forces and potentials (Eq. eqnpo1): softened nearest-image pairs plus the
    Ewald correction psi of every pair, and m_i psi(0) of each sink's own images."""
    pos_int = np.ascontiguousarray(pos_int, dtype=np.uint32)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    cls = None if cls is None else np.ascontiguousarray(cls, dtype=np.uint8)
    sinks = np.ascontiguousarray(sinks, dtype=np.int64)
    ns = sinks.shape[0]
    acc = np.empty((ns, 3))
    pot = np.empty(ns)
    cp = params.c()
    lib().or_ewald_direct(_p(pos_int), pos_int.shape[1], _p(mass), _p(cls), _p(sinks), ns,
                          C.byref(cp), _p(acc), _p(pot))
    return acc, pot


def direct(pos_int: np.ndarray, mass, cls, sinks, params: OracleParams, r_max: float = 0.0):
    """FP64 direct summation for the given sinks over all particles (nearest image when
    periodic); r_max > 0 keeps only pairs with r < r_max."""
    pos_int = np.ascontiguousarray(pos_int, dtype=np.uint32)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    cls = None if cls is None else np.ascontiguousarray(cls, dtype=np.uint8)
    sinks = np.ascontiguousarray(sinks, dtype=np.int64)
    ns = sinks.shape[0]
    acc = np.empty((ns, 3))
    pot = np.empty(ns)
    cp = params.c()
    lib().or_direct(_p(pos_int), pos_int.shape[1], _p(mass), _p(cls), _p(sinks), ns,
                    C.byref(cp), float(r_max), _p(acc), _p(pot))
    return acc, pot


# ---- whole pipeline in caller order ----------------------------------------------------------

@dataclass
class OracleRun:
    pos_int: np.ndarray      # (3, N) caller order
    keys_sorted: np.ndarray
    perm: np.ndarray         # sorted -> original
    tree: Tree
    params: OracleParams


def prepare(pos_int: np.ndarray, mass, cls, aold, params: OracleParams, leaf_max: int) -> OracleRun:
    """Keys, stable sort, gather, tree and multipoles (all in FP64, by definition)."""
    k = keys(pos_int)
    ks, perm = sort(k)
    pos_s = np.ascontiguousarray(pos_int[:, perm])
    t = Tree(ks, pos_s, leaf_max)
    m = np.asarray(mass, np.float64)[perm]
    c = None if cls is None else np.asarray(cls, np.uint8)[perm]
    a = None if aold is None else np.asarray(aold, np.float64)[perm]
    t.multipoles(m, c, a, params)
    return OracleRun(pos_int=pos_int, keys_sorted=ks, perm=perm, tree=t, params=params)


def tree_forces(run: OracleRun, sinks_orig: np.ndarray, params: OracleParams | None = None):
    """Tree walk for the given caller-order sink indices; returns acc (ns,3), pot, counts."""
    params = params or run.params
    inv = np.empty_like(run.perm)
    inv[run.perm] = np.arange(run.perm.shape[0])
    return run.tree.walk(inv[np.asarray(sinks_orig, np.int64)], params)
