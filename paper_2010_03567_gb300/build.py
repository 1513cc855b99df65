"""Builds libg4.so (the sm_103a CUDA library behind include/g4.h) in-tree with nvcc.

Every .cu file under csrc/ is compiled in parallel for sm_103a only (the FMM variant file once
per variant, see VARIANTS), then linked into
paper_2010_03567_gb300/_build/libg4.so.  Rebuilds only when a source or header is newer
than the library.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUTDIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUTDIR, "libg4.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the sm_103a library cannot be built")


# sources compiled once per variant (extra macros, object suffix): the FMM dual walk's eight
# (order, TreePM) variants compile in parallel instead of in one long translation unit
VARIANTS = {
    "g4_fmm_variant.cu": [([f"-DG4_FMM_P={p}", f"-DG4_FMM_TREEPM={t}"], f"_p{p}t{t}")
                          for p in (2, 3, 4, 5) for t in (0, 1)] +
                         [([f"-DG4_FMM_P=4", f"-DG4_FMM_TREEPM={t}", "-DG4_FMM_FP64=1"], f"_p4t{t}d")
                          for t in (0, 1)],
}


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _units():
    """(source, object, extra flags) of every translation unit."""
    out = []
    for s in _sources():
        stem = os.path.basename(s)[:-3]
        for flags, suffix in VARIANTS.get(os.path.basename(s), [([], "")]):
            out.append((s, os.path.join(OUTDIR, stem + suffix + ".o"), flags))
    # the longest units first, so that they start early
    out.sort(key=lambda u: 0 if os.path.basename(u[0]) in VARIANTS else 1)
    return out


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + [os.path.join(INCLUDE, "g4.h"), os.path.abspath(__file__)])


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(OUTDIR, exist_ok=True)
    cc = nvcc()
    units = _units()
    objs = [o for _, o, _ in units]

    def one(unit):
        s, o, vflags = unit
        cmd = [cc, *ARCH, *FLAGS, *vflags, *(extra or []), "-c", s, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(s)}:\n{r.stderr}")
        return r.stderr

    workers = max(1, min(len(units), os.cpu_count() or 8))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        logs = list(ex.map(one, units))
    if verbose:
        for l in logs:
            if l.strip():
                print(l)
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
