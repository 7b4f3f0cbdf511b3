"""Thin ctypes binding of the C ABI in include/nnsemd.h.

Argument marshalling only: every step of a solve runs in the CUDA library.
PyTorch supplies device memory and the current stream.  If the library has
not been built this module raises at import -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libnnsemd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"the NNS-EMD CUDA library is not built ({LIB_PATH} missing); "
                      "run paper_2401_07378_gb300.build.build() first")

_lib = ctypes.CDLL(LIB_PATH)

NNSEMD_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "NONFINITE", 3: "ZERO_MASS", 4: "CUDA", 5: "OOM",
          6: "TIMEOUT", 7: "ITER_LIMIT", 8: "UNSUPPORTED", 9: "CAPACITY"}
METRIC = {"l2": 0, "sql2": 1, "l1": 2}
PRECISION = {"fp32": 0, "bf16": 1, "fp16": 2, "fp8": 3, "bf16x3": 4}
FLAG_TIME_KERNELS = 1
FLAG_AUTOTUNE = 2
FLAG_GRAPH = 4


class nnsemd_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("stream", ctypes.c_void_p), ("workspace_bytes_hint", ctypes.c_size_t)]


class nnsemd_options(ctypes.Structure):
    _fields_ = [("metric", ctypes.c_int32), ("precision", ctypes.c_int32), ("rerank_k", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("proposal", ctypes.c_void_p), ("protocol", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class nnsemd_plan(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("nnz", ctypes.c_int64), ("i", ctypes.c_void_p),
                ("j", ctypes.c_void_p), ("f", ctypes.c_void_p)]


class nnsemd_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("pair_evals", ctypes.c_int64), ("leftover_mass", ctypes.c_double),
                ("certified", ctypes.c_int64), ("fallbacks", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("nns_kernel_ms", ctypes.c_double), ("nns_kernel_launches", ctypes.c_int64),
                ("nns_kernel_pairs", ctypes.c_int64), ("tail_kernel_ms", ctypes.c_double),
                ("near_ties", ctypes.c_int64), ("widened", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_lib.nnsemd_create.argtypes = [ctypes.POINTER(_P), ctypes.POINTER(nnsemd_config)]
_lib.nnsemd_destroy.argtypes = [_P]
_lib.nnsemd_set_stream.argtypes = [_P, _P]
_lib.nnsemd_solve.argtypes = [_P, _P, _P, _I64, _P, _P, _I64, ctypes.c_int32, ctypes.POINTER(nnsemd_options),
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(nnsemd_plan),
                              ctypes.POINTER(nnsemd_stats)]
_lib.nnsemd_solve_host.argtypes = _lib.nnsemd_solve.argtypes
_lib.nnsemd_solve_batched.argtypes = [_P, ctypes.c_int32, _P, _P, _P, _P, _P, _P, ctypes.c_int32,
                                      ctypes.POINTER(nnsemd_options), _P, ctypes.POINTER(nnsemd_stats)]
_lib.nnsemd_last_error.argtypes = [_P]
_lib.nnsemd_last_error.restype = ctypes.c_char_p
_lib.nnsemd_status_string.argtypes = [ctypes.c_int]
_lib.nnsemd_status_string.restype = ctypes.c_char_p
_lib.nnsemd_abi_version.restype = ctypes.c_int
_lib.nnsemd_nearest.argtypes = [_P, _P, _I64, _P, _I64, ctypes.c_int32, ctypes.c_int32, _P]
_lib.nnsemd_proposal_create.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                        ctypes.POINTER(_P)]
_lib.nnsemd_proposal_destroy.argtypes = [_P]
_lib.nnsemd_proposal_fit.argtypes = [_P, _P, _P, _I64, ctypes.c_int32, ctypes.c_uint64]
_lib.nnsemd_proposal_train.argtypes = [_P, _P, _P, _P, _I64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                       ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
_lib.nnsemd_proposal_loss_grad.argtypes = [_P, _P, _P, _P, _I64, ctypes.POINTER(ctypes.c_double), _P]
_lib.nnsemd_proposal_info.argtypes = [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]
_lib.nnsemd_proposal_params.argtypes = [_P, _P, _P, ctypes.c_int32]
_lib.nnsemd_proposal_save.argtypes = [_P, _P, ctypes.c_char_p]
_lib.nnsemd_proposal_load.argtypes = [_P, ctypes.c_char_p, ctypes.POINTER(_P)]
for _f in ("nnsemd_nearest", "nnsemd_proposal_create", "nnsemd_proposal_destroy", "nnsemd_proposal_fit",
           "nnsemd_proposal_train", "nnsemd_proposal_loss_grad", "nnsemd_proposal_info", "nnsemd_proposal_params",
           "nnsemd_proposal_save", "nnsemd_proposal_load"):
    getattr(_lib, _f).restype = ctypes.c_int
_lib.nnsemd_solve_one_to_many.argtypes = [_P, ctypes.c_int32, _P, _P, _P, _P, _P, _I64, ctypes.c_int32,
                                          ctypes.POINTER(nnsemd_options), _P, ctypes.POINTER(nnsemd_stats)]
_lib.nnsemd_kmeans.argtypes = [_P, _P, _I64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P, _P]
_lib.nnsemd_barycentric.argtypes = [_P, ctypes.POINTER(nnsemd_plan), _P, _I64, _P, _I64, ctypes.c_int32, _P]
_lib.nnsemd_recolour.argtypes = [_P, _P, _I64, _P, ctypes.c_int32, ctypes.c_int32, _P]
for _f in ("nnsemd_create", "nnsemd_destroy", "nnsemd_set_stream", "nnsemd_solve", "nnsemd_solve_host",
           "nnsemd_solve_batched", "nnsemd_solve_one_to_many", "nnsemd_kmeans", "nnsemd_barycentric",
           "nnsemd_recolour"):
    getattr(_lib, _f).restype = ctypes.c_int


class NNSEMDError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


@dataclass
class SolveResult:
    cost: float
    plan_i: Optional[object] = None   # int32 [nnz] supplier index (device tensor or numpy)
    plan_j: Optional[object] = None   # int32 [nnz] consumer index
    plan_f: Optional[object] = None   # float64 [nnz] flow
    stats: Optional[dict] = None


def abi_version() -> int:
    return _lib.nnsemd_abi_version()


ABI_VERSION = 4  # the nnsemd.h this binding mirrors
if abi_version() != ABI_VERSION:
    raise ImportError(f"libnnsemd.so has ABI {abi_version()}, this binding expects {ABI_VERSION}: rebuild")


PROTOCOL = {"greedy": 0, "random": 1}


def _options(metric: str, precision: str, rerank_k: int, flags: int = 0, proposal=None, protocol: str = "greedy",
             seed: int = 0) -> nnsemd_options:
    return nnsemd_options(METRIC[metric], PRECISION[precision], rerank_k, flags,
                          proposal._h.value if proposal is not None else None, PROTOCOL[protocol], 0, seed)


def _ptr(t) -> int:
    return t.data_ptr()


class Context:
    """One nnsemd_ctx: a device, a stream binding and a workspace."""

    def __init__(self, device: int = 0, workspace_bytes_hint: int = 0):
        self._h = _P()
        cfg = nnsemd_config(device, None, workspace_bytes_hint)
        rc = _lib.nnsemd_create(ctypes.byref(self._h), ctypes.byref(cfg))
        if rc != NNSEMD_OK:
            raise NNSEMDError(rc, _lib.nnsemd_last_error(None).decode())
        self.device = device

    def close(self):
        if self._h:
            _lib.nnsemd_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != NNSEMD_OK:
            raise NNSEMDError(rc, _lib.nnsemd_last_error(self._h).decode())

    def set_stream(self, stream_handle: int):
        self._check(_lib.nnsemd_set_stream(self._h, stream_handle))

    def _bind_current_stream(self):
        import torch
        self.set_stream(torch.cuda.current_stream(self.device).cuda_stream)

    # -- nnsemd_solve --------------------------------------------------------
    def solve(self, x, a, y, b, metric: str = "l2", precision: str = "fp32", rerank_k: int = 0,
              plan: bool = False, flags: int = 0, proposal=None, protocol: str = "greedy",
              seed: int = 0) -> SolveResult:
        """Device tensors: x [m,d] float32, a [m] float64, y [n,d] float32, b [n] float64.
        ``proposal``: a trained Proposal (d > 8) replacing the full NNS scan."""
        import torch
        for t, dt in ((x, torch.float32), (a, torch.float64), (y, torch.float32), (b, torch.float64)):
            if not t.is_cuda or t.dtype != dt or not t.is_contiguous():
                raise ValueError("solve wants contiguous CUDA tensors: x, y float32; a, b float64")
        m, d = x.shape
        n = y.shape[0]
        self._bind_current_stream()
        opt = _options(metric, precision, rerank_k, flags, proposal, protocol, seed)
        cost = ctypes.c_double()
        st = nnsemd_stats()
        pl = None
        if plan:
            cap = max(m + n - 1, 1)
            pi = torch.empty(cap, dtype=torch.int32, device=x.device)
            pj = torch.empty(cap, dtype=torch.int32, device=x.device)
            pf = torch.empty(cap, dtype=torch.float64, device=x.device)
            pl = nnsemd_plan(cap, 0, _ptr(pi), _ptr(pj), _ptr(pf))
        rc = _lib.nnsemd_solve(self._h, _ptr(x), _ptr(a), m, _ptr(y), _ptr(b), n, d, ctypes.byref(opt),
                               ctypes.byref(cost), ctypes.byref(pl) if pl else None, ctypes.byref(st))
        self._check(rc)
        res = SolveResult(cost.value, stats=st.as_dict())
        if plan:
            k = pl.nnz
            res.plan_i, res.plan_j, res.plan_f = pi[:k], pj[:k], pf[:k]
        return res

    # -- nnsemd_solve_host ---------------------------------------------------
    def solve_host(self, x, a, y, b, metric: str = "l2", precision: str = "fp32", rerank_k: int = 0,
                   plan: bool = False, plan_out=None, flags: int = 0, proposal=None, protocol: str = "greedy",
                   seed: int = 0) -> SolveResult:
        """Host arrays (numpy, or pinned CPU torch tensors): the copies to and
        from the device happen inside the call.  ``plan_out`` may pass
        preallocated (i, j, f) host arrays of capacity >= m + n - 1."""
        def host_ptr(t, dt):
            if isinstance(t, np.ndarray):
                if t.dtype != dt or not t.flags["C_CONTIGUOUS"]:
                    raise ValueError("host arrays must be C-contiguous with the right dtype")
                return t.ctypes.data
            return t.data_ptr()
        m, d = x.shape
        n = y.shape[0]
        self._bind_current_stream()
        opt = _options(metric, precision, rerank_k, flags, proposal, protocol, seed)
        cost = ctypes.c_double()
        st = nnsemd_stats()
        pl = None
        if plan:
            if plan_out is None:
                cap = max(m + n - 1, 1)
                plan_out = (np.empty(cap, np.int32), np.empty(cap, np.int32), np.empty(cap, np.float64))
            pi, pj, pf = plan_out
            pl = nnsemd_plan(len(pi), 0, host_ptr(pi, np.int32), host_ptr(pj, np.int32), host_ptr(pf, np.float64))
        rc = _lib.nnsemd_solve_host(self._h, host_ptr(x, np.float32), host_ptr(a, np.float64), m,
                                    host_ptr(y, np.float32), host_ptr(b, np.float64), n, d, ctypes.byref(opt),
                                    ctypes.byref(cost), ctypes.byref(pl) if pl else None, ctypes.byref(st))
        self._check(rc)
        res = SolveResult(cost.value, stats=st.as_dict())
        if plan:
            k = pl.nnz
            res.plan_i, res.plan_j, res.plan_f = pi[:k], pj[:k], pf[:k]
        return res

    # -- nnsemd_solve_batched ------------------------------------------------
    def solve_batched(self, x, a, x_off, y, b, y_off, metric: str = "l2", precision: str = "fp32",
                      rerank_k: int = 0, costs=None, stats: bool = True, flags: int = 0, protocol: str = "greedy",
                      seed: int = 0):
        """Packed device tensors plus host offset arrays (np.int64, P+1).
        Returns the device tensor of P costs (and the stats dict)."""
        import torch
        x_off = np.ascontiguousarray(x_off, np.int64)
        y_off = np.ascontiguousarray(y_off, np.int64)
        P = len(x_off) - 1
        d = x.shape[1]
        if costs is None:
            costs = torch.empty(P, dtype=torch.float64, device=x.device)
        self._bind_current_stream()
        opt = _options(metric, precision, rerank_k, flags, None, protocol, seed)
        st = nnsemd_stats()
        rc = _lib.nnsemd_solve_batched(self._h, P, _ptr(x), _ptr(a), x_off.ctypes.data, _ptr(y), _ptr(b),
                                       y_off.ctypes.data, d, ctypes.byref(opt), _ptr(costs),
                                       ctypes.byref(st) if stats else None)
        self._check(rc)
        return costs, (st.as_dict() if stats else None)


    # -- nnsemd_solve_one_to_many ---------------------------------------------
    def solve_one_to_many(self, x, a, x_off, y, b, metric: str = "l2", precision: str = "fp32",
                          rerank_k: int = 0, costs=None, stats: bool = True, flags: int = 0,
                          protocol: str = "greedy", seed: int = 0):
        """Packed supplier histograms (device x, a; host x_off, P+1 entries)
        against one consumer histogram (device y [n, d], b [n]).  Returns the
        device tensor of P costs (and the stats dict)."""
        import torch
        x_off = np.ascontiguousarray(x_off, np.int64)
        P = len(x_off) - 1
        d = x.shape[1]
        if costs is None:
            costs = torch.empty(P, dtype=torch.float64, device=x.device)
        self._bind_current_stream()
        opt = _options(metric, precision, rerank_k, flags, None, protocol, seed)
        st = nnsemd_stats()
        rc = _lib.nnsemd_solve_one_to_many(self._h, P, _ptr(x), _ptr(a), x_off.ctypes.data, _ptr(y), _ptr(b),
                                           y.shape[0], d, ctypes.byref(opt), _ptr(costs),
                                           ctypes.byref(st) if stats else None)
        self._check(rc)
        return costs, (st.as_dict() if stats else None)

    # -- colour transfer -----------------------------------------------------
    def kmeans(self, pts, k: int, iters: int):
        """Device pts [N, d] float32 -> (centroids [k, d], labels [N] int32, counts [k] int64), device."""
        import torch
        N, d = pts.shape
        cent = torch.empty(k, d, dtype=torch.float32, device=pts.device)
        lab = torch.empty(N, dtype=torch.int32, device=pts.device)
        cnt = torch.empty(k, dtype=torch.int64, device=pts.device)
        self._bind_current_stream()
        self._check(_lib.nnsemd_kmeans(self._h, _ptr(pts), N, d, k, iters, _ptr(cent), _ptr(lab), _ptr(cnt)))
        return cent, lab, cnt

    def barycentric(self, plan_i, plan_j, plan_f, x, y):
        """Device plan arrays (int32, int32, float64), x [m, d], y [n, d] -> y' [n, d]."""
        import torch
        out = torch.empty_like(y)
        pl = nnsemd_plan(plan_f.numel(), plan_f.numel(), _ptr(plan_i), _ptr(plan_j), _ptr(plan_f))
        self._bind_current_stream()
        self._check(_lib.nnsemd_barycentric(self._h, ctypes.byref(pl), _ptr(x), x.shape[0], _ptr(y), y.shape[0],
                                            y.shape[1], _ptr(out)))
        return out

    def recolour(self, labels, palette):
        import torch
        out = torch.empty(labels.shape[0], palette.shape[1], dtype=torch.float32, device=labels.device)
        self._bind_current_stream()
        self._check(_lib.nnsemd_recolour(self._h, _ptr(labels), labels.shape[0], _ptr(palette), palette.shape[0],
                                         palette.shape[1], _ptr(out)))
        return out

    # -- nnsemd_nearest ------------------------------------------------------
    def nearest(self, x, y, metric: str = "l2"):
        """Round one of Alg. 1: the nearest supplier of every consumer (device int32 tensor)."""
        import torch
        out = torch.empty(y.shape[0], dtype=torch.int32, device=y.device)
        self._bind_current_stream()
        self._check(_lib.nnsemd_nearest(self._h, _ptr(x), x.shape[0], _ptr(y), y.shape[0], x.shape[1],
                                        METRIC[metric], _ptr(out)))
        return out


class Proposal:
    """Learned candidate proposal (nnsemd_proposal_*): a k-means codebook and
    an MLP scoring its cells.  Not in the paper."""

    def __init__(self, ctx: Context, d: int, cells: int = 4096, hidden: int = 256, seed: int = 0, _handle=None):
        self.ctx = ctx
        self._h = _P()
        if _handle is not None:
            self._h = _handle
        else:
            ctx._check(_lib.nnsemd_proposal_create(ctx._h, d, cells, hidden, seed, ctypes.byref(self._h)))
        dd, cc, hh, npar = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _lib.nnsemd_proposal_info(self._h, ctypes.byref(dd), ctypes.byref(cc), ctypes.byref(hh), ctypes.byref(npar))
        self.d, self.cells, self.hidden, self.nparams = dd.value, cc.value, hh.value, npar.value

    def close(self):
        if self._h:
            _lib.nnsemd_proposal_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fit(self, pts, iters: int = 10, seed: int = 0):
        self.ctx._bind_current_stream()
        self.ctx._check(_lib.nnsemd_proposal_fit(self.ctx._h, self._h, _ptr(pts), pts.shape[0], iters, seed))

    def train(self, y, x_nn, epochs: int = 3, batch: int = 4096, lr: float = 1e-3, seed: int = 0) -> float:
        loss = ctypes.c_double()
        self.ctx._bind_current_stream()
        self.ctx._check(_lib.nnsemd_proposal_train(self.ctx._h, self._h, _ptr(y), _ptr(x_nn), y.shape[0], epochs,
                                                   batch, lr, seed, ctypes.byref(loss)))
        return loss.value

    def loss_grad(self, y, labels):
        import torch
        grad = torch.empty(self.nparams, dtype=torch.float32, device=y.device)
        loss = ctypes.c_double()
        self.ctx._bind_current_stream()
        self.ctx._check(_lib.nnsemd_proposal_loss_grad(self.ctx._h, self._h, _ptr(y), _ptr(labels), y.shape[0],
                                                       ctypes.byref(loss), _ptr(grad)))
        return loss.value, grad

    def params(self) -> np.ndarray:
        out = np.empty(self.nparams, np.float32)
        self.ctx._check(_lib.nnsemd_proposal_params(self.ctx._h, self._h, out.ctypes.data, 0))
        return out

    def set_params(self, values: np.ndarray):
        v = np.ascontiguousarray(values, np.float32)
        assert v.size == self.nparams
        self.ctx._check(_lib.nnsemd_proposal_params(self.ctx._h, self._h, v.ctypes.data, 1))

    def save(self, path: str):
        self.ctx._check(_lib.nnsemd_proposal_save(self.ctx._h, self._h, path.encode()))

    @classmethod
    def load(cls, ctx: Context, path: str) -> "Proposal":
        h = _P()
        ctx._check(_lib.nnsemd_proposal_load(ctx._h, path.encode(), ctypes.byref(h)))
        return cls(ctx, 0, _handle=h)
