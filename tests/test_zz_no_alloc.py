"""The allocation-free entry point nnsemd_solve_small_noalloc.

It serves callers that cannot call cudaMalloc (for example a plugin running
inside another framework's launch callback, or a process whose device memory
a caching allocator already holds): its scratch is a fixed __device__ array
inside the library.  Here it is called through the C ABI and its R is
compared, bit for bit, with nnsemd_solve's and with the CPU oracle's on the
same inputs, for calls in a row: a failing call (a NaN coordinate) that
leaves its error word in the shared array must not leak into the valid call
after it.  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2401_07378_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NNSEMD_ERR_NONFINITE = 2
NNSEMD_ERR_UNSUPPORTED = 8


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


def _dev(pair):
    return [torch.as_tensor(v).cuda() for v in (pair.x, pair.a, pair.y, pair.b)]


def test_noalloc_matches_solve_on_two_calls_in_a_row():
    from paper_2401_07378_gb300 import nnsemd
    ctx = nnsemd.Context(0)
    cases = [(wl.uniform_pair(1024, 777, 2, 11, "dirichlet"), "l2"),
             (wl.uniform_pair(300, 1000, 3, 12, "uniform"), "sql2")]
    for pair, metric in cases:
        t = _dev(pair)
        want = ctx.solve(*t, metric=metric).cost
        rc, got = _call_noalloc(nnsemd._lib, *t, metric)
        assert rc == 0
        assert got == want
    ctx.close()


@pytest.mark.parametrize("metric", ["l2", "sql2", "l1"])
def test_noalloc_matches_the_oracle_for_every_dimension(metric):
    from paper_2401_07378_gb300 import nnsemd
    for d in range(1, 9):
        pair = wl.uniform_pair(200 + 37 * d, 150 + 53 * d, d, 100 + d, "dirichlet")
        rc, got = _call_noalloc(nnsemd._lib, *_dev(pair), metric)
        assert rc == 0, (d, metric)
        assert got == oracle.solve_pair(pair, metric).cost, (d, metric)


def test_a_failed_call_does_not_leak_into_the_next():
    from paper_2401_07378_gb300 import nnsemd
    bad = wl.uniform_pair(64, 80, 3, 21)
    bad.x[5, 1] = np.nan
    rc, _ = _call_noalloc(nnsemd._lib, *_dev(bad), "l2")
    assert rc == NNSEMD_ERR_NONFINITE
    good = wl.uniform_pair(500, 420, 3, 22, "dirichlet")
    ctx = nnsemd.Context(0)
    want = ctx.solve(*_dev(good), metric="l2").cost
    ctx.close()
    rc, got = _call_noalloc(nnsemd._lib, *_dev(good), "l2")
    assert rc == 0
    assert got == want == oracle.solve_pair(good, "l2").cost


def test_noalloc_rejects_sizes_beyond_its_limit():
    from paper_2401_07378_gb300 import nnsemd
    p = wl.uniform_pair(1025, 10, 2, 13)
    rc, _ = _call_noalloc(nnsemd._lib, *_dev(p), "l2")
    assert rc == NNSEMD_ERR_UNSUPPORTED
    p = wl.uniform_pair(10, 10, 9, 14)
    rc, _ = _call_noalloc(nnsemd._lib, *_dev(p), "l2")
    assert rc == NNSEMD_ERR_UNSUPPORTED
