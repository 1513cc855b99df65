"""The C-ABI library builds for sm_103a, loads on a CPU-only host and exports every entry
point that include/g4.h declares.  Only host-side calls are made (no kernels)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "g4.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(g4_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2010_03567_gb300 import build
    path = build.build()
    lib = C.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_calls():
    from paper_2010_03567_gb300 import g4
    assert "sm_103a" in g4.version()
    p = g4.params(alpha=0.01, eps=[0.1, 0.2])
    assert p.alpha == 0.01 and p.n_eps_classes == 2 and p.eps_table[1] == 0.2
    assert p.leaf_max == 8 and p.order_p == 3 and p.r_cut_factor == 4.5
    # argument errors are reported synchronously with a message, without touching a GPU
    b = C.c_size_t()
    st = g4.lib().g4_keys_sort_workspace(-1, C.byref(b))
    assert st == 1 and b"bad args" in g4.lib().g4_last_error()
    assert g4.g4_keys_sort_workspace(1 << 20) > 12 * (1 << 20)
    with pytest.raises(g4.G4Error):
        g4.params(no_such_field=1)


def test_binding_argument_counts_match_header():
    """Every entry point the binding declares takes as many arguments as its prototype in
    include/g4.h (a missing argument would shift every later pointer)."""
    from paper_2010_03567_gb300 import g4
    src = open(os.path.join(ROOT, "include", "g4.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    protos = dict(re.findall(r"\b(g4_[a-z0-9_]+)\s*\(([^()]*)\)\s*;", src))
    L = g4.lib()
    checked = 0
    for name, args in protos.items():
        at = getattr(L, name).argtypes
        if at is None:
            continue
        a = args.strip()
        n = 0 if a in ("", "void") else a.count(",") + 1
        assert len(at) == n, (name, len(at), n)
        checked += 1
    assert checked >= 30 and "g4_gravity_tree_perm" in protos
    # the fused-scatter walk rejects a NULL permutation before touching a GPU
    p = g4.params()
    st = L.g4_gravity_tree_perm(None, None, None, None, None, None, 0, C.byref(p), None, None,
                                None, None, None)
    assert st == 1 and b"NULL perm" in L.g4_last_error()


def test_oracle_and_library_share_no_code():
    # the oracle is plain C under oracle/, the library CUDA under the package: no includes across
    import glob
    for f in glob.glob(os.path.join(ROOT, "paper_2010_03567_gb300", "csrc", "*")):
        assert "oracle" not in open(f).read().lower().replace("oracle-free", "")
    txt = open(os.path.join(ROOT, "oracle", "g4_oracle.c")).read()
    assert "g4.h" not in txt and "g4_internal" not in txt


def test_params_struct_layout_matches_header(tmp_path):
    """The binding's ctypes mirror of g4_params has the header's size and field offsets (a
    field missing on the Python side would let the library write past the caller's struct)."""
    import shutil
    import subprocess
    from paper_2010_03567_gb300 import g4
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f[0] for f in g4.G4Params._fields_]
    prog = ["#include <stdio.h>", "#include <stddef.h>", '#include "g4.h"', "int main(void) {",
            '  printf("%zu\\n", sizeof(g4_params));']
    prog += [f'  printf("%zu\\n", offsetof(g4_params, {f}));' for f in fields]
    prog += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(prog) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    hdr = open(os.path.join(ROOT, "include", "g4.h")).read()
    body = re.search(r"typedef struct g4_params \{(.*?)\} g4_params;", hdr, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    declared = re.findall(r"(\w+)\s*(?:\[[^\]]*\])?\s*;", body)
    assert declared == fields, (declared, fields)
    assert out[0] == C.sizeof(g4.G4Params)
    assert out[1:] == [getattr(g4.G4Params, f).offset for f in fields]
