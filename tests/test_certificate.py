"""The certificate of the reduced-precision NNS step (csrc/tc_common.cuh), on
the CPU.

The library's certify_floor / certify are compiled for the host
(tests/native/certify_host.cu) and checked against the same bound restated
here in exact rational arithmetic:

    E     = gamma (ny + rx^2) + 2 (dot_eta + dot_acc) + 2 u32 (rx^2 + 2 xt yt + c rx)
    floor = (ny + tau - E) (1 - gamma)   where ny + tau - E > 0, else ny + tau - E

(the library multiplies a positive floor by a further (1 - 2^-30) to cover
its own double-precision rounding).  A best exact key is certified only strictly
below the floor, so the tests (1) check that the double evaluation never
exceeds the exact floor and sits within 2^-28 of it, (2) drive best_key to
the float32 values around the floor (the near-ties of the certificate) and
require a refusal at and above it, and (3) emulate the whole step for BF16
operands -- quantised rows, tensor-core dot products perturbed anywhere
within the accumulation bound d 2^-22 |x~||y~| the bound assumes (the
reading of the tensor cores' FP32 accumulation that the design states),
FP32 epilogue, top-K, tau, exact FP32 keys -- on point sets with planted
near-ties and duplicates, and require that whatever is certified is the
strict nearest supplier.
"""
import ctypes
import math
import os
import shutil
import subprocess
from fractions import Fraction as Fr

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "certify_host.cu")
BUILD = os.path.join(ROOT, "tests", "_build")
FMT_F16, FMT_BF16, FMT_E4M3, FMT_BF16X3 = 0, 1, 2, 3
U32 = Fr(1, 2 ** 24)


@pytest.fixture(scope="module")
def lib():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    os.makedirs(BUILD, exist_ok=True)
    so = os.path.join(BUILD, f"libcertify_host.{os.getpid()}.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-shared", "-I", os.path.join(ROOT, "include"), "-I",
                    os.path.join(ROOT, "paper_2401_07378_gb300", "csrc"), SRC, "-o", so], check=True)
    L = ctypes.CDLL(so)
    D = ctypes.c_double
    L.certify_floor_host.argtypes = [ctypes.c_int, ctypes.c_int, D, D, D, D, D, D, D, ctypes.c_float]
    L.certify_floor_host.restype = D
    L.certify_host.argtypes = L.certify_floor_host.argtypes + [ctypes.c_float]
    L.certify_host.restype = ctypes.c_int
    P = ctypes.POINTER
    L.tag_list_host.argtypes = [P(ctypes.c_float), ctypes.c_int, ctypes.c_int, ctypes.c_int, P(ctypes.c_float),
                                P(ctypes.c_int)]
    L.tag_list_host.restype = ctypes.c_int
    yield L
    os.unlink(so)


def quant_unit(fmt):
    return {FMT_BF16: Fr(1, 2 ** 8), FMT_BF16X3: Fr(1, 2 ** 8), FMT_F16: Fr(1, 2 ** 11),
            FMT_E4M3: Fr(1, 2 ** 4)}[fmt]


def quant_err(fmt):
    """Q with |<x~, y~> - <x, y>| <= Q sum |x_k y_k| (derived in the module
    docstring of the emulation below for BF16X3)."""
    u = quant_unit(fmt)
    return u * u * (3 + 2 * u + 2 * u * u) if fmt == FMT_BF16X3 else 2 * u + u * u


def exact_floor(fmt, d, ny, yl2, yl1, sy, rx, rx1, sxm, tau):
    """The certificate's bound in exact arithmetic (sqrt(d) rounded up, which
    only lowers the bound)."""
    ny, yl2, yl1, sy, rx, rx1, sxm, tau = (Fr(v) for v in (ny, yl2, yl1, sy, rx, rx1, sxm, tau))
    uq = quant_unit(fmt)
    bf = fmt in (FMT_BF16, FMT_BF16X3)
    gam = d * U32 / (1 - d * U32)
    kdim = 3 * d if fmt == FMT_BF16X3 else d
    eta_unit = {FMT_BF16: Fr(1, 2 ** 134), FMT_BF16X3: Fr(1, 2 ** 132), FMT_F16: Fr(1, 2 ** 25),
                FMT_E4M3: Fr(1, 2 ** 10)}[fmt]
    eta_x = eta_unit * (1 if bf else sxm)
    eta_y = eta_unit * (1 if bf else sy)
    sqd = Fr(math.sqrt(kdim)) * (1 + Fr(1, 2 ** 50))
    if fmt == FMT_BF16X3:
        dot_eta = 3 * (eta_x * (2 * yl1 + eta_y * d) + 2 * eta_y * rx1)
        nf = Fr(1.4142135623731) * (1 + uq) + uq + uq * uq   # >= sqrt(2) (1 + u) + u + u^2
    else:
        dot_eta = eta_x * (yl1 + eta_y * d) + eta_y * rx1 + eta_x * uq * yl1 + eta_y * uq * rx1
        nf = 1 + uq
    xt = nf * rx + eta_x * sqd
    yt = nf * yl2 + eta_y * sqd
    dot_acc = kdim * Fr(1, 2 ** 22) * xt * yt
    c = 2 * quant_err(fmt) * yl2 * (1 + Fr(1, 10 ** 5))
    E = gam * (ny + rx * rx) + 2 * (dot_eta + dot_acc) + 2 * U32 * (rx * rx + 2 * xt * yt + c * rx) + Fr(1e-30)
    base = ny + tau - E
    return base * (1 - gam) if base > 0 else base


def random_inputs(rng, fmt, d):
    ny = float(np.float32(rng.uniform(0.1, 4e4)))
    yl2 = math.sqrt(ny) * (1 + 1e-12)
    yl1 = yl2 * math.sqrt(d) * rng.uniform(0.3, 1.0)
    rx = float(np.float32(rng.uniform(0.1, 300.0)))
    rx1 = rx * math.sqrt(d) * rng.uniform(0.3, 1.0)
    sy = 2.0 ** int(rng.integers(-8, 4)) if fmt in (FMT_F16, FMT_E4M3) else 1.0
    sxm = 2.0 ** int(rng.integers(-8, 4)) if fmt in (FMT_F16, FMT_E4M3) else 1.0
    tau = float(np.float32(rng.uniform(-2 * rx * yl2, rx * rx)))
    return ny, yl2, yl1, sy, rx, rx1, sxm, tau


@pytest.mark.parametrize("fmt", [FMT_BF16, FMT_F16, FMT_E4M3, FMT_BF16X3])
@pytest.mark.parametrize("d", [9, 64, 128, 300])
def test_double_evaluation_stays_below_the_exact_bound(lib, fmt, d):
    rng = np.random.default_rng(fmt * 1000 + d)
    for _ in range(300):
        args = random_inputs(rng, fmt, d)
        got = lib.certify_floor_host(fmt, d, *args)
        want = exact_floor(fmt, d, *args)
        if want <= 0:       # nothing can be certified: no key (>= 0) lies below the floor
            assert got <= 0, (args, got, float(want))
            continue
        assert Fr(got) <= want, (args, got, float(want))
        assert abs(Fr(got) - want) <= abs(want) * Fr(1, 2 ** 28), (args, got, float(want))


@pytest.mark.parametrize("fmt", [FMT_BF16, FMT_F16, FMT_E4M3, FMT_BF16X3])
def test_keys_at_the_floor_are_refused(lib, fmt):
    """Near-ties of the certificate itself: best keys at, just above and just
    below the floor."""
    rng = np.random.default_rng(7 + fmt)
    refused = accepted = 0
    for _ in range(400):
        d = int(rng.choice([9, 64, 300]))
        args = random_inputs(rng, fmt, d)
        fl = exact_floor(fmt, d, *args)
        if fl <= 0:
            continue
        k = np.float32(float(fl))
        for key in (np.nextafter(k, np.float32(np.inf)), k, np.nextafter(k, np.float32(0)),
                    np.nextafter(np.nextafter(k, np.float32(0)), np.float32(0))):
            ok = lib.certify_host(fmt, d, *args, float(key))
            if Fr(float(key)) >= fl:
                assert ok == 0, (args, float(key), float(fl))
                refused += 1
            elif ok:
                accepted += 1
    assert refused > 100 and accepted > 100


def test_infinite_tau_means_every_supplier_was_a_candidate(lib):
    assert lib.certify_host(FMT_BF16, 64, 1.0, 1.0, 8.0, 1.0, 1.0, 8.0, 1.0, float("inf"), 3.0) == 1


# ---------------------------------------------------------------------------
# the whole step emulated for BF16 operands
# ---------------------------------------------------------------------------

def f32(v: Fr) -> Fr:
    """Round an exact value to the nearest float32 (ties to even)."""
    c = np.float32(float(v))
    best = None
    for cand in (np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))):
        e = abs(Fr(float(cand)) - v)
        if best is None or e < best[0] or (e == best[0] and (int(np.float32(cand).view(np.uint32)) & 1) == 0):
            best = (e, cand)
    return Fr(float(best[1]))


def bf16(v: float) -> Fr:
    """Round a float32 value to bfloat16 (nearest, ties to even)."""
    b = int(np.float32(v).view(np.uint32))
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return Fr(float(np.uint32(b).view(np.float32)))


def key32(x, y):
    """The FP32 decision key of the library (sequential fma of the squared
    differences), exactly."""
    acc = None
    for xk, yk in zip(x, y):
        t = f32(Fr(float(xk)) - Fr(float(yk)))
        acc = f32(t * t) if acc is None else f32(t * t + acc)
    return acc


def norm2_32(v):
    acc = Fr(0)
    for vk in v:
        acc = f32(Fr(float(vk)) * Fr(float(vk)) + acc)
    return acc


def packed_rows(x, y, split):
    """The operand rows the tensor cores see: one BF16 copy of each side, or
    for the BF16X3 split (h = bf16(v), l = bf16(v - h), v - h exact in FP32)
    the supplier row [h, l, h] against the consumer row [h, h, l].  With
    v = h + l + e, |v - h| <= u|v|, |e| <= u^2 |v| and |l| <= (u + u^2)|v|
    (u = 2^-8), their product <h,h> + <l,h> + <h,l> = <x - e_x, y - e_y> -
    <l_x, l_y> is within u^2 (3 + 2u + 2u^2) sum |x_k y_k| of <x, y>."""
    if not split:
        return [bf16(v) for v in x], [bf16(v) for v in y]
    hx = [bf16(v) for v in x]
    lx = [bf16(float(np.float32(Fr(float(v)) - h))) for v, h in zip(x, hx)]
    hy = [bf16(v) for v in y]
    ly = [bf16(float(np.float32(Fr(float(v)) - h))) for v, h in zip(y, hy)]
    return hx + lx + hx, hy + hy + ly


def emulated_step(rng, X, y, K, split=False):
    """One consumer's reduced-precision NNS over suppliers X: returns the
    certified supplier or None, and the exact keys."""
    d = X.shape[1]
    fmt = FMT_BF16X3 if split else FMT_BF16
    ny = norm2_32(y)
    cy = f32(Fr(float(np.float32(2 * float(quant_err(fmt)) * math.sqrt(float(ny)) * (1 + 1e-4)))))
    vals = []
    for i in range(X.shape[0]):
        xq, yq = packed_rows(X[i], y, split)
        dot = sum(a * b for a, b in zip(xq, yq))
        nxq = math.sqrt(float(sum(a * a for a in xq)))
        nyq = math.sqrt(float(sum(b * b for b in yq)))
        err = Fr(len(xq)) * Fr(1, 2 ** 22) * Fr(nxq) * Fr(nyq)
        acc = f32(dot + err * Fr(float(rng.uniform(-1, 1))))          # somewhere inside the assumed bound
        nx = norm2_32(X[i])
        ns = f32(Fr(float(np.float32(math.sqrt(float(nx)) * (1 + 1e-4)))))
        v = f32(-cy * ns + f32(Fr(-2) * acc + nx))
        vals.append(v)
    order = sorted(range(len(vals)), key=lambda i: (vals[i], i))
    cand = order[:K]
    tau = vals[order[K - 1]] if len(order) > K else None  # None: every supplier is a candidate
    keys = [key32(X[i], y) for i in range(X.shape[0])]
    best = min(cand, key=lambda i: (keys[i], i))
    if tau is None:
        return best, keys, cand
    yl2 = math.sqrt(sum(float(v) ** 2 for v in y)) * (1 + 1e-12)
    yl1 = sum(abs(float(v)) for v in y)
    rx = max(float(np.float32(math.sqrt(float(norm2_32(X[i]))) * (1 + 1e-4))) for i in range(X.shape[0]))
    rx1 = max(float(np.float32(sum(abs(float(v)) for v in X[i]) * (1 + 1e-4))) for i in range(X.shape[0]))
    fl = exact_floor(fmt, d, float(ny), yl2, yl1, 1.0, rx, rx1, 1.0, float(tau))
    return (best if keys[best] < fl else None), keys, cand


def test_split_bf16_dot_product_error_bound():
    """The BF16X3 bound on the dot product itself, on random and adversarial
    rows (values at BF16 rounding boundaries)."""
    rng = np.random.default_rng(3)
    u = Fr(1, 2 ** 8)
    for trial in range(200):
        d = int(rng.integers(1, 40))
        x = rng.normal(0, 1, d).astype(np.float32)
        y = rng.normal(0, 1, d).astype(np.float32)
        if trial % 2:   # values just off a BF16 tie
            x = (np.round(x * 256) / 256 + np.float32(2 ** -9 + 2 ** -20)).astype(np.float32)
        a, b = packed_rows(x, y, True)
        got = sum(p * q for p, q in zip(a, b))
        exact = sum(Fr(float(p)) * Fr(float(q)) for p, q in zip(x, y))
        bound = quant_err(FMT_BF16X3) * sum(abs(Fr(float(p)) * Fr(float(q))) for p, q in zip(x, y))
        assert abs(got - exact) <= bound, trial
        assert quant_err(FMT_BF16X3) < 4 * u * u


@pytest.mark.parametrize("split", [False, True], ids=["bf16", "bf16x3"])
def test_emulated_bf16_step_certifies_only_the_strict_nearest(split):
    rng = np.random.default_rng(11)
    certified = 0
    for trial in range(30):
        d = int(rng.choice([9, 16, 24]))
        m = int(rng.integers(12, 28))
        X = rng.normal(0, 1, (m, d)).astype(np.float32)
        y = rng.normal(0, 1, d).astype(np.float32)
        # planted near-ties: a supplier at y plus a tiny offset, a copy of it,
        # and one at a distance equal to it up to the last bits
        base = (y + np.float32(0.05) * rng.normal(0, 1, d).astype(np.float32)).astype(np.float32)
        X[0] = base
        X[1] = base
        X[2] = (base + np.float32(1e-6)).astype(np.float32)
        X = X[rng.permutation(m)]
        got, keys, cand = emulated_step(rng, X, y, K=4, split=split)
        if got is None:
            continue
        certified += 1
        for i in range(m):
            if i != got:
                assert keys[i] > keys[got] or (keys[i] == keys[got] and i > got), (trial, i, got)
    assert certified > 5


# ---------------------------------------------------------------------------
# the K2 epilogue's tagged lists
# ---------------------------------------------------------------------------

def tag_list(lib, vals, kl, floor=True):
    vals = np.ascontiguousarray(vals, dtype=np.float32)
    out_v = np.empty(kl, np.float32)
    out_p = np.empty(kl, np.int32)
    F, I = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)
    assert lib.tag_list_host(vals.ctypes.data_as(F), len(vals), kl, int(floor), out_v.ctypes.data_as(F),
                             out_p.ctypes.data_as(I)) == 0
    return out_v, out_p


def tag_streams():
    rng = np.random.default_rng(11)
    yield rng.normal(-240.0, 6.0, 5000)                     # GMM-like: negative values near one another
    yield rng.normal(0.0, 1.0, 3000)                        # both signs, values near zero
    yield np.repeat(rng.normal(5.0, 1.0, 300), 7)           # many exact ties
    yield np.sort(rng.normal(0.0, 1.0, 1000))[::-1]         # descending: every value enters the list
    yield np.concatenate([[0.0, -0.0] * 20, rng.normal(0.0, 1e-30, 200)])  # zeros and subnormal-sized
    base = np.float32(-123.4567)                            # one high-bit pattern, every tag order
    bits = base.view(np.uint32) & np.uint32(~31 & 0xFFFFFFFF)
    yield np.array([np.uint32(bits | k).view(np.float32) for k in rng.permutation(32)], np.float32)
    yield rng.normal(0.0, 1.0, 5)                           # shorter than the list


@pytest.mark.parametrize("kl", [8, 16])
def test_tagged_list_bounds_every_excluded_value(lib, kl):
    """The floored K-th entry is a lower bound of every value left out (the
    certificate's tau), each entry's floored value is at most its own value,
    positions are distinct, and the list holds the kl smallest values up to
    the tag's perturbation (2^5 units in the last place at most)."""
    for vals in tag_streams():
        vals = np.asarray(vals, np.float32)
        v, p = tag_list(lib, vals, kl)
        n = len(vals)
        real = p >= 0
        assert real.sum() == min(n, kl)
        assert len(set(p[real].tolist())) == real.sum()
        assert np.all(v[real] <= vals[p[real]])
        assert np.all(np.diff(v[real]) >= 0)
        if n <= kl:
            assert sorted(p[real].tolist()) == list(range(n))
            continue
        tau = v[kl - 1]
        out = np.setdiff1d(np.arange(n), p)
        assert np.all(vals[out] >= tau)
        kth = np.sort(vals)[kl - 1]
        slack = 64 * np.spacing(np.abs(kth).astype(np.float32)) + np.float32(1e-44)
        assert np.all(vals[p] <= kth + slack)


def test_tagged_list_needs_its_floor(lib):
    """Without the floor a tagged entry can stand above a value it pushed
    out (same high bits, the larger tag on the smaller value): the unfloored
    K-th entry then fails as a bound, the floored one holds."""
    kl = 8
    base = np.float32(1000.0).view(np.uint32) & np.uint32(~15 & 0xFFFFFFFF)
    # 8 values take tags 0..7 in arrival order; a ninth, smaller in exact
    # terms than the eighth, gets tag 8 and so compares above it
    vals = [np.uint32(base | k).view(np.float32) for k in (15, 14, 13, 12, 11, 10, 9, 8)]
    vals.append(np.uint32(base | 0).view(np.float32))
    vals = np.array(vals, np.float32)
    raw_v, raw_p = tag_list(lib, vals, kl, floor=False)
    flo_v, flo_p = tag_list(lib, vals, kl, floor=True)
    out_raw = np.setdiff1d(np.arange(len(vals)), raw_p)
    assert len(out_raw) == 1
    assert vals[out_raw].min() < raw_v[kl - 1]
    out = np.setdiff1d(np.arange(len(vals)), flo_p)
    assert np.all(vals[out] >= flo_v[kl - 1])
