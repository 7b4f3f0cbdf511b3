"""The allocation-free entry point nnsemd_solve_small_noalloc.

It serves callers that cannot call cudaMalloc (for example a plugin running
inside another framework's launch callback, or a process whose device memory
a caching allocator already holds): its scratch is a fixed __device__ array
inside the library.  Here it is called through the C ABI and its R is
compared, bit for bit, with nnsemd_solve's on the same inputs, for two calls
in a row (the second call must not see the first one's leftovers).  The file
is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2401_07378_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _call_noalloc(lib, x, a, y, b, metric):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    P = ctypes.c_void_p
    f = lib.nnsemd_solve_small_noalloc
    f.argtypes = [P, P, ctypes.c_int64, P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, P, P]
    f.restype = ctypes.c_int
    rc = f(x.data_ptr(), a.data_ptr(), x.shape[0], y.data_ptr(), b.data_ptr(), y.shape[0], x.shape[1],
           {"l2": 0, "sql2": 1, "l1": 2}[metric], out.data_ptr(), stream)
    return rc, float(out.item())


def test_noalloc_matches_solve_on_two_calls_in_a_row():
    from paper_2401_07378_gb300 import nnsemd
    ctx = nnsemd.Context(0)
    cases = [(wl.uniform_pair(1024, 777, 2, 11, "dirichlet"), "l2"),
             (wl.uniform_pair(300, 1000, 3, 12, "uniform"), "sql2")]
    for pair, metric in cases:
        t = [torch.as_tensor(v).cuda() for v in (pair.x, pair.a, pair.y, pair.b)]
        want = ctx.solve(*t, metric=metric).cost
        rc, got = _call_noalloc(nnsemd._lib, *t, metric)
        assert rc == 0
        assert got == want
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    from paper_2401_07378_gb300 import nnsemd
    p = wl.uniform_pair(1025, 10, 2, 13)
    t = [torch.as_tensor(v).cuda() for v in (p.x, p.a, p.y, p.b)]
    rc, _ = _call_noalloc(nnsemd._lib, *t, "l2")
    assert rc == 8  # NNSEMD_ERR_UNSUPPORTED
