"""TEST INFRASTRUCTURE -- the CPU oracle of NNS-EMD.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does: it shares
no code with the CUDA library and must not fall back to it.

``solve`` restates the paper's Algorithm 1 (Sec. III-A, greedy protocol):

1. Normalise the weights (Sec. II-A assumes sum_i s_i = sum_j c_j = 1).  The
   total is the correctly rounded sum of the weights (``math.fsum``, a library
   primitive), then each weight is divided by it (IEEE division), so the
   normalised weights do not depend on a summation order.
2. Run the rounds of Algorithm 1 in plain C (``nnsemd_oracle.c``).
3. The cost R is the correctly rounded sum of the per-flow costs f*D_ij
   (again ``math.fsum``); Algorithm 1's own left-to-right accumulation is
   returned beside it as ``cost_seq``.

``solve(..., threads=k)`` with k != 1 runs the multi-core twin of the C
oracle (``oracle_nnsemd_omp``: the NNS operation and the group sorts in
parallel, the flows serial); the tests check that it returns exactly what
the serial oracle returns.  ``solve_many`` runs the serial oracle on many
pairs at once, one pair per host process.

Zero weights are allowed and the corresponding points never take part
(Sec. II-A: histograms are over the bins with positive weight).
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nnsemd_oracle.c")
_SRC_OMP = os.path.join(_HERE, "nnsemd_oracle_omp.c")  # includes _SRC, adds the multi-core twin
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libnnsemd_oracle.so")
_lock = threading.Lock()
_lib = None

METRICS = {"l2": 0, "sql2": 1, "l1": 2}


class _Stats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_int64),
        ("pair_evals", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("near_ties", ctypes.c_int64),
        ("violations", ctypes.c_int64),
        ("max_rel_gap", ctypes.c_double),
        ("cost_seq", ctypes.c_double),
        ("leftover_s", ctypes.c_double),
        ("leftover_c", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-adds, -O2), with OpenMP
    for the multi-core twin where the compiler has it (else the twin runs on
    one core)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_OMP))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp,
                _SRC_OMP]
        if subprocess.run(base + ["-fopenmp", "-lm"], capture_output=True).returncode != 0:
            subprocess.run(base + ["-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            f = lib.oracle_nnsemd
            P = ctypes.c_void_p
            f.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, P, P, P, P,
                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                          ctypes.c_int64, P, P, P, P,
                          ctypes.c_int64, P, P,
                          ctypes.c_int64, P, P,
                          ctypes.POINTER(_Stats)]
            f.restype = ctypes.c_int
            g = lib.oracle_nnsemd_omp
            g.argtypes = f.argtypes[:-1] + [ctypes.c_int32, ctypes.POINTER(_Stats)]
            g.restype = ctypes.c_int
            lib.oracle_omp_max_threads.restype = ctypes.c_int
            lib.oracle_splitmix64_output.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.oracle_splitmix64_output.restype = ctypes.c_uint64
            if lib.oracle_stats_size() != ctypes.sizeof(_Stats):
                raise RuntimeError("oracle stats layout mismatch")
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


@dataclass
class OracleResult:
    cost: float                  # correctly rounded sum of f*D over the plan
    cost_seq: float              # Alg. 1's sequential accumulation of R
    plan_i: np.ndarray           # int32 [nnz] supplier index
    plan_j: np.ndarray           # int32 [nnz] consumer index
    plan_f: np.ndarray           # float64 [nnz] flow
    plan_term: np.ndarray        # float64 [nnz] f * D_ij
    s: np.ndarray                # normalised supplier weights (before the solve)
    c: np.ndarray                # normalised consumer weights
    s_left: np.ndarray           # residual supplier weights after the solve
    c_left: np.ndarray           # residual consumer weights after the solve
    rounds: int
    pair_evals: int
    near_ties: int
    violations: int
    max_rel_gap: float
    m_t: np.ndarray = field(default=None)
    n_t: np.ndarray = field(default=None)
    trace_j: np.ndarray = field(default=None)
    trace_nn: np.ndarray = field(default=None)

    @property
    def leftover(self) -> float:
        return float(self.s_left.sum() + self.c_left.sum())


def normalise(w: np.ndarray) -> np.ndarray:
    """Sec. II-A normalisation: w / sum(w), the sum correctly rounded."""
    w = np.asarray(w, np.float64)
    if w.size and not np.all(np.isfinite(w)):
        raise OracleError("non-finite weight")
    if np.any(w < 0):
        raise OracleError("negative weight")
    total = math.fsum(w.tolist())
    if not total > 0.0:
        raise OracleError("zero total mass")
    return w / total


PROTOCOLS = {"greedy": 0, "random": 1}


def max_threads() -> int:
    """Host threads the multi-core twin uses with threads=0 (1 without OpenMP)."""
    return int(_load().oracle_omp_max_threads())


def splitmix64_output(seed: int, k: int) -> int:
    """Output number k (k >= 1) of SplitMix64 seeded with `seed` (the
    generator of the random protocol's order; see nnsemd_oracle.c)."""
    return int(_load().oracle_splitmix64_output(seed, k))


def solve(x, a, y, b, metric: str = "l2", decide: str = "fp32", trace: bool = False,
          protocol: str = "greedy", seed: int = 0, threads: int = 1) -> OracleResult:
    """Run NNS-EMD (Alg. 1) on one pair.

    x: [m, d] float32 suppliers S with weights a; y: [n, d] float32 consumers
    C with weights b.  ``decide`` is the precision of the argmin and greedy
    order decisions ("fp32" or "fp64"); mass and cost are FP64 either way.
    ``protocol``: "greedy" (the paper's default) or "random" (a supplier
    serves its consumers in a seeded random order, Sec. III-A).
    ``threads``: 1 runs the serial oracle; any other value the multi-core
    twin on that many host threads (0 = all).
    """
    lib = _load()
    x = np.ascontiguousarray(x, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    if x.ndim != 2 or y.ndim != 2 or x.shape[1] != y.shape[1]:
        raise OracleError("coordinate shapes")
    if not (np.all(np.isfinite(x)) and np.all(np.isfinite(y))):
        raise OracleError("non-finite coordinate")
    m, d = x.shape
    n = y.shape[0]
    s0 = normalise(a)
    c0 = normalise(b)
    if s0.shape[0] != m or c0.shape[0] != n:
        raise OracleError("weight shapes")
    s = s0.copy()
    c = c0.copy()
    cap = max(m + n, 1)
    pi = np.zeros(cap, np.int32)
    pj = np.zeros(cap, np.int32)
    pf = np.zeros(cap, np.float64)
    pt = np.zeros(cap, np.float64)
    rcap = m + n + 1
    m_t = np.zeros(rcap, np.int64)
    n_t = np.zeros(rcap, np.int64)
    tcap = 0
    if trace:
        tcap = max(4 * n, 16)
    while True:
        tj = np.zeros(max(tcap, 1), np.int32)
        tn = np.zeros(max(tcap, 1), np.int32)
        st = _Stats()
        s[:] = s0
        c[:] = c0
        args = (m, n, d, x.ctypes.data, s.ctypes.data, y.ctypes.data, c.ctypes.data,
                METRICS[metric], 1 if decide == "fp32" else 0, PROTOCOLS[protocol], seed,
                cap, pi.ctypes.data, pj.ctypes.data, pf.ctypes.data, pt.ctypes.data,
                rcap, m_t.ctypes.data, n_t.ctypes.data,
                tcap if trace else 0, tj.ctypes.data if trace else None,
                tn.ctypes.data if trace else None)
        if threads == 1:
            rc = lib.oracle_nnsemd(*args, ctypes.byref(st))
        else:
            rc = lib.oracle_nnsemd_omp(*args, threads, ctypes.byref(st))
        if rc != 0:
            raise OracleError(f"oracle failed with status {rc}")
        if trace and int(np.sum(n_t[: st.rounds])) > tcap:
            tcap = int(np.sum(n_t[: st.rounds]))
            continue
        break
    nnz = int(st.nnz)
    terms = pt[:nnz].copy()
    return OracleResult(
        cost=math.fsum(terms.tolist()), cost_seq=float(st.cost_seq),
        plan_i=pi[:nnz].copy(), plan_j=pj[:nnz].copy(), plan_f=pf[:nnz].copy(), plan_term=terms,
        s=s0, c=c0, s_left=s, c_left=c,
        rounds=int(st.rounds), pair_evals=int(st.pair_evals), near_ties=int(st.near_ties),
        violations=int(st.violations), max_rel_gap=float(st.max_rel_gap),
        m_t=m_t[: st.rounds].copy(), n_t=n_t[: st.rounds].copy(),
        trace_j=tj[: int(np.sum(n_t[: st.rounds]))].copy() if trace else None,
        trace_nn=tn[: int(np.sum(n_t[: st.rounds]))].copy() if trace else None)


def solve_pair(pair, metric: str = "l2", decide: str = "fp32", trace: bool = False, protocol: str = "greedy",
               seed: int = 0, threads: int = 1) -> OracleResult:
    return solve(pair.x, pair.a, pair.y, pair.b, metric, decide, trace, protocol, seed, threads)


def _solve_packed(job):
    """Worker of solve_many: one pair given as (x, a, y, b, metric, decide, protocol, seed)."""
    x, a, y, b, metric, decide, protocol, seed = job
    return solve(x, a, y, b, metric, decide, False, protocol, seed)


def process_pool(workers: int = 0):
    """A pool of ``workers`` (0 = every core) host processes for solve_many,
    started with ``spawn`` (safe after CUDA has been initialised in the
    caller); each worker builds nothing and loads the oracle library once."""
    import multiprocessing as mp
    workers = workers or os.cpu_count() or 1
    return cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"), initializer=_load)


def solve_many(pairs, metric: str = "l2", decide: str = "fp32", protocol: str = "greedy", seed: int = 0,
               workers: int = 0, pool=None) -> list[OracleResult]:
    """The serial oracle on every pair of ``pairs``, several pairs at a time,
    one pair per host process (``pool``, from process_pool; else a pool of
    ``workers`` processes made for this call, 0 = every core; 1 runs in this
    process).  Results in the order of ``pairs``."""
    pairs = list(pairs)
    jobs = [(p.x, p.a, p.y, p.b, metric, decide, protocol, seed) for p in pairs]
    if pool is not None:
        return list(pool.map(_solve_packed, jobs, chunksize=max(1, len(jobs) // (8 * pool._max_workers))))
    workers = workers or os.cpu_count() or 1
    if workers == 1 or len(pairs) <= 1:
        return [_solve_packed(j) for j in jobs]
    build()
    with process_pool(workers) as ex:
        return list(ex.map(_solve_packed, jobs, chunksize=max(1, len(jobs) // (8 * workers))))
