"""The allocation-free key sort (g4_keys_sort_noalloc) against the workspace version.

Some callers cannot allocate device memory when they sort (for example an application whose
device memory belongs to another allocator).
The allocation-free entry point keeps its scratch in a fixed array inside the library.  This
test calls it through the C ABI twice in a row -- the second call reuses the scratch left by
the first -- and checks that keys and permutation are bit-identical to g4_keys_sort (the
tolerance for integer work).  It lives in its own file, collected last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2010_03567_gb300 import g4  # noqa: E402

pytestmark = pytest.mark.gpu

LIMIT = 1 << 20


def _noalloc(pos_int):
    n = pos_int.shape[1]
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    st = g4.lib().g4_keys_sort_noalloc(C.c_void_p(pos_int.data_ptr()), n, C.c_void_p(keys.data_ptr()),
                                       C.c_void_p(perm.data_ptr()),
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, g4.lib().g4_last_error()
    return keys, perm


def _case(n, seed):
    g = np.random.default_rng(seed)
    q = g.integers(0, 2 ** 32, size=(3, n), dtype=np.uint64).astype(np.uint32)
    q[:, : n // 10] = q[:, :1]        # a run of equal keys: the sort must stay stable
    return torch.from_numpy(q.view(np.int32)).cuda()


def test_noalloc_matches_workspace_sort_on_two_calls():
    for n, seed in [(LIMIT, 1), (300001, 2)]:          # second call smaller: stale scratch
        pos = _case(n, seed)
        k_ref, p_ref = g4.g4_keys_sort(pos)
        k, p = _noalloc(pos)
        torch.cuda.synchronize()
        assert torch.equal(k, k_ref) and torch.equal(p, p_ref)


def test_noalloc_rejects_oversize():
    n = LIMIT + 1
    st = g4.lib().g4_keys_sort_noalloc(C.c_void_p(16), n, C.c_void_p(16), C.c_void_p(16), None)
    assert st == 1
    assert b"static scratch limit" in g4.lib().g4_last_error()
