"""The kernels' DD/QD arithmetic (csrc/ddqd.cuh, compiled for the host -- same bits as on
the GPU) against exact rationals: dot products with partial-sum combination, the MGS
update y - c x, division by a real, product with a real, square root."""

import ctypes
import math
from fractions import Fraction as F

import numpy as np
import pytest

import pins
from paper_1210_0800_gb300 import build, inputs

dp = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def hl():
    lib = ctypes.CDLL(build.build_host())
    i = ctypes.c_int
    lib.h_dot.argtypes = [i, i, i, dp, dp, dp]
    lib.h_norm2.argtypes = [i, i, i, dp, dp]
    lib.h_update.argtypes = [i, dp, dp, dp, dp]
    lib.h_div_real.argtypes = [i, dp, dp, dp]
    lib.h_mul_real.argtypes = [i, dp, dp, dp]
    lib.h_sqrt.argtypes = [i, dp, dp]
    lib.h_two_sum.argtypes = [ctypes.c_double, ctypes.c_double, dp, dp]
    lib.h_two_prod.argtypes = [ctypes.c_double, ctypes.c_double, dp, dp]
    lib.h_dot_parts.argtypes = [i, i, i, dp, dp, dp]
    lib.h_axpy_parts.argtypes = [i, i, dp, dp, dp, dp]
    lib.h_update_split_qd.argtypes = [dp, dp, dp, dp]
    return lib


def P(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(dp)


def cplx(L, seed, count, spread=(-20, 20)):
    return pins.rand_limbs(L, seed, 2 * count, spread).reshape(count, 2, L)


U = {2: 2.0 ** -104, 4: 2.0 ** -208}  # a few ulps of the format, the bound unit used below
UNIT = {2: 2.0 ** -106, 4: 2.0 ** -212}


def test_two_sum_two_prod_exact(hl):
    vals = np.ldexp(inputs.uniform_pm1(31, 600), inputs.uniform_int(32, 600, -80, 80))
    s, e = ctypes.c_double(), ctypes.c_double()
    for a, b in zip(vals[::2], vals[1::2]):
        hl.h_two_sum(a, b, ctypes.byref(s), ctypes.byref(e))
        assert F(s.value) + F(e.value) == F(a) + F(b) and s.value == a + b
        hl.h_two_prod(a, b, ctypes.byref(s), ctypes.byref(e))
        assert F(s.value) + F(e.value) == F(a) * F(b) and s.value == a * b


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("n,split", [(1, 1), (7, 3), (40, 40), (64, 17), (300, 150)])
def test_dot(hl, L, n, split):
    x, y = cplx(L, 100 + n, n), cplx(L, 200 + n, n)
    out = np.zeros((2, L))
    xa, xp = P(x)
    ya, yp = P(y)
    oa, op = P(out)
    hl.h_dot(L, n, split, xp, yp, op)
    ex = (F(0), F(0))
    scale = 0.0
    for i in range(n):
        a, b = pins.cval(x[i]), pins.cval(y[i])
        ex = pins.cadd(ex, pins.cmul(pins.cconj(a), b))
        scale += math.sqrt(float(pins.cabs2(a)) * float(pins.cabs2(b)))
    err = pins.cnorm_inf(pins.csub(pins.cval(oa), ex))
    # a length-n sum in the format grows its error like n units of the last limb
    assert err <= 4 * (n + 2) * UNIT[L] * scale, (err / scale, L, n)


@pytest.mark.parametrize("L", [2, 4])
def test_dot_cancellation(hl, L):
    """x^H y with heavy cancellation: the error stays relative to sum |x||y|."""
    n = 64
    x = cplx(L, 301, n)
    y = x.copy()
    y[n // 2:] = -x[: n // 2]  # second half cancels the first
    y[: n // 2] = x[: n // 2]
    x2 = x.copy()
    x2[n // 2:] = x[: n // 2]
    out = np.zeros((2, L))
    _, xp = P(x2)
    _, yp = P(y)
    oa, op = P(out)
    hl.h_dot(L, n, 5, xp, yp, op)
    scale = sum(float(pins.cabs2(pins.cval(x2[i]))) for i in range(n))
    assert pins.cnorm_inf(pins.cval(oa)) <= 4 * (n + 2) * UNIT[L] * scale


@pytest.mark.parametrize("L", [2, 4])
def test_norm2(hl, L):
    n = 50
    x = cplx(L, 401, n)
    out = np.zeros((2, L))
    _, xp = P(x)
    oa, op = P(out)
    hl.h_norm2(L, n, 20, xp, op)
    ex = sum((pins.cabs2(pins.cval(x[i])) for i in range(n)), F(0))
    r = pins.cval(oa)
    assert r[1] == 0
    assert abs(r[0] - ex) <= 4 * U[L] * ex


@pytest.mark.parametrize("L", [2, 4])
def test_update(hl, L):
    ys, cs, xs = cplx(L, 501, 200), cplx(L, 502, 200), cplx(L, 503, 200)
    # include near-cancellation: y close to c x
    for k in range(0, 200, 10):
        p = pins.cmul(pins.cval(cs[k]), pins.cval(xs[k]))
        ys[k, 0, 0], ys[k, 1, 0] = float(p[0]), float(p[1])
        ys[k, :, 1:] = 0.0
    out = np.zeros((2, L))
    for y, c, x in zip(ys, cs, xs):
        _, yp = P(y)
        _, cp = P(c)
        _, xp = P(x)
        oa, op = P(out)
        hl.h_update(L, yp, cp, xp, op)
        cy, cc, cxv = pins.cval(y), pins.cval(c), pins.cval(x)
        ex = pins.csub(cy, pins.cmul(cc, cxv))
        scale = math.sqrt(float(pins.cabs2(cy))) + math.sqrt(float(pins.cabs2(cc)) * float(pins.cabs2(cxv)))
        assert pins.cnorm_inf(pins.csub(pins.cval(oa), ex)) <= 4 * U[L] * scale


def test_update_split_qd(hl):
    """y - c x with each part's two products on two accumulators that are then merged (the
    back-substitution chain's form), including near-cancellation."""
    L = 4
    ys, cs, xs = cplx(L, 511, 200), cplx(L, 512, 200), cplx(L, 513, 200)
    for k in range(0, 200, 10):
        p = pins.cmul(pins.cval(cs[k]), pins.cval(xs[k]))
        ys[k, 0, 0], ys[k, 1, 0] = float(p[0]), float(p[1])
        ys[k, :, 1:] = 0.0
    out = np.zeros((2, L))
    for y, c, x in zip(ys, cs, xs):
        _, yp = P(y)
        _, cp = P(c)
        _, xp = P(x)
        oa, op = P(out)
        hl.h_update_split_qd(yp, cp, xp, op)
        cy, cc, cxv = pins.cval(y), pins.cval(c), pins.cval(x)
        ex = pins.csub(cy, pins.cmul(cc, cxv))
        scale = math.sqrt(float(pins.cabs2(cy))) + math.sqrt(float(pins.cabs2(cc)) * float(pins.cabs2(cxv)))
        assert pins.cnorm_inf(pins.csub(pins.cval(oa), ex)) <= 4 * U[L] * scale


@pytest.mark.parametrize("L", [2, 4])
def test_div_mul_real(hl, L):
    As = cplx(L, 601, 150)
    Rs = pins.rand_limbs(L, 602, 150, (-30, 30))
    Rs[:, 0] = np.abs(Rs[:, 0])
    Rs[:, 1:] = np.where(Rs[:, :1] < 0, -Rs[:, 1:], Rs[:, 1:])
    out = np.zeros((2, L))
    for a, r in zip(As, Rs):
        _, ap = P(a)
        _, rp = P(r)
        oa, op = P(out)
        hl.h_div_real(L, ap, rp, op)
        fa, fr = pins.cval(a), pins.fval(r)
        ex = (fa[0] / fr, fa[1] / fr)
        assert pins.cnorm_inf(pins.csub(pins.cval(oa), ex)) <= 4 * U[L] * pins.cnorm_inf(ex)
        hl.h_mul_real(L, ap, rp, op)
        ex = (fa[0] * fr, fa[1] * fr)
        assert pins.cnorm_inf(pins.csub(pins.cval(oa), ex)) <= 4 * U[L] * pins.cnorm_inf(ex)


@pytest.mark.parametrize("L", [2, 4])
def test_sqrt(hl, L):
    Ss = np.abs(pins.rand_limbs(L, 701, 150, (-60, 60)))
    Ss[:, 1:] = pins.rand_limbs(L, 701, 150, (-60, 60))[:, 1:]
    Ss = np.concatenate([Ss, [[4.0] + [0.0] * (L - 1), [2.0] + [0.0] * (L - 1)]])
    out = np.zeros(L)
    for s in Ss:
        _, sp = P(s)
        oa, op = P(out)
        hl.h_sqrt(L, sp, op)
        fs, r = pins.fval(s), pins.fval(oa)
        assert r > 0 and abs(r * r - fs) <= 8 * U[L] * fs, float((r * r - fs) / fs)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("n,split", [(1, 0), (9, 4), (64, 31)])
def test_dot_parts(hl, L, n, split):
    """Real and imaginary parts of x^H y accumulated separately (as the kernels' lanes do)."""
    x, y = cplx(L, 800 + n, n), cplx(L, 900 + n, n)
    out = np.zeros((2, L))
    _, xp = P(x)
    _, yp = P(y)
    oa, op = P(out)
    hl.h_dot_parts(L, n, split, xp, yp, op)
    ex = (F(0), F(0))
    scale = 0.0
    for i in range(n):
        a, b = pins.cval(x[i]), pins.cval(y[i])
        ex = pins.cadd(ex, pins.cmul(pins.cconj(a), b))
        scale += math.sqrt(float(pins.cabs2(a)) * float(pins.cabs2(b)))
    assert pins.cnorm_inf(pins.csub(pins.cval(oa), ex)) <= 4 * (n + 2) * UNIT[L] * scale


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("n", [1, 5, 32])
def test_axpy_parts(hl, L, n):
    """y - sum_i r_i x_i with part accumulators (the back-substitution update)."""
    y, r, x = cplx(L, 1000 + n, 1), cplx(L, 1100 + n, n), cplx(L, 1200 + n, n)
    out = np.zeros((2, L))
    _, yp = P(y[0])
    _, rp = P(r)
    _, xp = P(x)
    oa, op = P(out)
    hl.h_axpy_parts(L, n, yp, rp, xp, op)
    ex = pins.cval(y[0])
    scale = math.sqrt(float(pins.cabs2(ex)))
    for i in range(n):
        a, b = pins.cval(r[i]), pins.cval(x[i])
        ex = pins.csub(ex, pins.cmul(a, b))
        scale += math.sqrt(float(pins.cabs2(a)) * float(pins.cabs2(b)))
    assert pins.cnorm_inf(pins.csub(pins.cval(oa), ex)) <= 4 * (n + 2) * UNIT[L] * scale
