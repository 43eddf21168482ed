"""CPU oracle for complex DD/QD modified Gram-Schmidt least squares.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of the
benchmark may use it; the product path never does.  The arithmetic lives in
``mdx_oracle.c`` (plain C, compiled with gcc -O2 -ffp-contract=off); this module only
builds it and marshals numpy arrays through ctypes.

Array conventions are those of ``paper_1210_0800_gb300.inputs``: matrices (n, m, 2, L)
column-major by element, vectors (m, 2, L), L limbs per real number.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "mdx_oracle.c")
LIBRARY = os.path.join(_HERE, "libmdx_oracle.so")

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared"]


def build(plant: int = 0, out: str | None = None) -> str:
    """Compile the oracle (with an optional planted mistake, for the pin tests)."""
    if out is None:
        if plant:
            raise ValueError("a planted build needs an explicit output path")
        out = LIBRARY
    cmd = ["gcc", *CFLAGS, f"-DORACLE_PLANT={int(plant)}", "-o", out, SOURCE, "-lm"]
    subprocess.check_call(cmd)
    return out


_dp = ctypes.POINTER(ctypes.c_double)


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


class Oracle:
    """A loaded oracle library."""

    def __init__(self, path: str | None = None):
        path = path or LIBRARY
        if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(SOURCE):
            if path != LIBRARY:
                raise FileNotFoundError(path)
            build()
        self.lib = lib = ctypes.CDLL(path)
        i, d, vp = ctypes.c_int, ctypes.c_double, _dp
        sig = {
            "oracle_selfcheck": (i, []),
            "oracle_plant": (i, []),
            "oracle_overflowed": (i, []),
            "oracle_two_sum": (None, [d, d, vp, vp]),
            "oracle_two_prod": (None, [d, d, vp, vp]),
            "oracle_add": (None, [i, vp, vp, vp]),
            "oracle_sub": (None, [i, vp, vp, vp]),
            "oracle_mul": (None, [i, vp, vp, vp]),
            "oracle_div": (None, [i, vp, vp, vp]),
            "oracle_sqrt": (None, [i, vp, vp]),
            "oracle_cmul": (None, [i, vp, vp, vp]),
            "oracle_cconjmul": (None, [i, vp, vp, vp]),
            "oracle_mgs": (i, [i, vp, i, i, i, vp, i, i]),
            "oracle_backsub": (i, [i, vp, i, i, vp, vp]),
            "oracle_ls_solve": (i, [i, vp, vp, vp, vp, vp, i, i, i, i]),
            "oracle_qr": (i, [i, vp, vp, i, i, i, i]),
            "oracle_matvec": (None, [i, vp, i, i, i, vp, i, vp]),
            "oracle_matvec_conjT": (None, [i, vp, i, i, i, vp, i, vp]),
            "oracle_qr_error": (d, [i, vp, i, vp, i, vp, i, i, i, vp]),
            "oracle_orth_error": (d, [i, vp, i, i, i]),
            "oracle_residual": (d, [i, vp, i, vp, vp, i, i, i, vp]),
            "oracle_rinv_fro": (d, [i, vp, i, i]),
            "oracle_max_abs_diff": (d, [i, vp, i, vp, ctypes.c_long, vp]),
            "oracle_fwdsub_conjT": (i, [i, vp, i, i, vp, vp]),
            "oracle_ls_adjoint": (i, [i, vp, vp, vp, i, i, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args

    # ------------------------------------------------------------ primitives
    def selfcheck(self) -> bool:
        return bool(self.lib.oracle_selfcheck())

    def plant(self) -> int:
        return int(self.lib.oracle_plant())

    def _binop(self, fn, L, a, b):
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        out = np.zeros(L, dtype=np.float64)
        fn(L, _ptr(a), _ptr(b), _ptr(out))
        return out

    def add(self, L, a, b):
        return self._binop(self.lib.oracle_add, L, a, b)

    def sub(self, L, a, b):
        return self._binop(self.lib.oracle_sub, L, a, b)

    def mul(self, L, a, b):
        return self._binop(self.lib.oracle_mul, L, a, b)

    def div(self, L, a, b):
        return self._binop(self.lib.oracle_div, L, a, b)

    def sqrt(self, L, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        out = np.zeros(L, dtype=np.float64)
        self.lib.oracle_sqrt(L, _ptr(a), _ptr(out))
        return out

    def cmul(self, L, a, b):
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(2 * L)
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(2 * L)
        out = np.zeros(2 * L, dtype=np.float64)
        self.lib.oracle_cmul(L, _ptr(a), _ptr(b), _ptr(out))
        return out.reshape(2, L)

    def cconjmul(self, L, a, b):
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(2 * L)
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(2 * L)
        out = np.zeros(2 * L, dtype=np.float64)
        self.lib.oracle_cconjmul(L, _ptr(a), _ptr(b), _ptr(out))
        return out.reshape(2, L)

    # ------------------------------------------------------------ method
    def ls_solve(self, A: np.ndarray, b: np.ndarray):
        """MGS on [A b] then back substitution.  Returns dict(Q, R, x, z, resid, status).

        A: (n, m, 2, L); b: (m, 2, L).  R is returned as (n, n, 2, L) column-major (R[j, k]
        is element (k, j)); z as (L,); resid (m, 2, L) is what MGS leaves of b."""
        n, m, _, L = A.shape
        Q = np.ascontiguousarray(A, dtype=np.float64).copy()
        r = np.ascontiguousarray(b, dtype=np.float64).copy()
        x = np.zeros((n, 2, L))
        R = np.zeros((n, n, 2, L))
        z = np.zeros(L)
        st = self.lib.oracle_ls_solve(L, _ptr(Q), _ptr(r), _ptr(x), _ptr(R), _ptr(z), m, n, m, n)
        return dict(Q=Q, R=R, x=x, z=z, resid=r, status=int(st))

    def qr(self, A: np.ndarray):
        n, m, _, L = A.shape
        Q = np.ascontiguousarray(A, dtype=np.float64).copy()
        R = np.zeros((n, n, 2, L))
        st = self.lib.oracle_qr(L, _ptr(Q), _ptr(R), m, n, m, n)
        return Q, R, int(st)

    def backsub(self, R: np.ndarray, y: np.ndarray):
        n = R.shape[0]
        L = R.shape[-1]
        R = np.ascontiguousarray(R, dtype=np.float64)
        yy = np.ascontiguousarray(y, dtype=np.float64).copy()
        x = np.zeros((n, 2, L))
        st = self.lib.oracle_backsub(L, _ptr(R), n, n, _ptr(yy), _ptr(x))
        return x, int(st)

    # ------------------------------------------------------------ exact helpers
    def matvec(self, A: np.ndarray, x: np.ndarray, Lout: int | None = None):
        """b = A x, each entry exact then rounded to Lout limbs."""
        n, m, _, L = A.shape
        Lout = Lout or L
        A = np.ascontiguousarray(A, dtype=np.float64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        b = np.zeros((m, 2, Lout))
        self.lib.oracle_matvec(L, _ptr(A), m, n, m, _ptr(x), Lout, _ptr(b))
        return b

    def matvec_conjT(self, A: np.ndarray, v: np.ndarray, Lout: int | None = None):
        """A^H v, each entry exact then rounded to Lout limbs (v: (m, 2, L))."""
        n, m, _, L = A.shape
        Lout = Lout or L
        A = np.ascontiguousarray(A, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros((n, 2, Lout))
        self.lib.oracle_matvec_conjT(L, _ptr(A), m, n, m, _ptr(v), Lout, _ptr(out))
        return out

    def qr_error(self, A, Q, R):
        """Eq. (2): max_ij |a_ij - (QR)_ij| (exact residual, modulus in double)."""
        n, m, _, L = A.shape
        part = ctypes.c_double(0.0)
        e = self.lib.oracle_qr_error(L, _ptr(np.ascontiguousarray(A)), m, _ptr(np.ascontiguousarray(Q)), m,
                                     _ptr(np.ascontiguousarray(R)), n, m, n, ctypes.byref(part))
        return float(e), float(part.value)

    def orth_error(self, Q):
        n, m, _, L = Q.shape
        return float(self.lib.oracle_orth_error(L, _ptr(np.ascontiguousarray(Q)), m, m, n))

    def residual(self, A, b, x, Lout: int = 4):
        """r = b - A x (exact, rounded to Lout limbs) and ||r||^2."""
        n, m, _, L = A.shape
        r = np.zeros((m, 2, Lout))
        nrm2 = self.lib.oracle_residual(L, _ptr(np.ascontiguousarray(A)), m, _ptr(np.ascontiguousarray(b)),
                                        _ptr(np.ascontiguousarray(x)), m, n, Lout, _ptr(r))
        return r, float(nrm2)

    def rinv_fro(self, R):
        n = R.shape[0]
        L = R.shape[-1]
        return float(self.lib.oracle_rinv_fro(L, _ptr(np.ascontiguousarray(R)), n, n))

    def max_abs_diff(self, a, b):
        """max_i |a_i - b_i| (exact difference) and max_i |b_i| over complex elements; a and
        b may carry different limb counts."""
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        La, Lb = a.shape[-1], b.shape[-1]
        ca, cb = a.size // (2 * La), b.size // (2 * Lb)
        assert ca == cb
        bmax = ctypes.c_double(0.0)
        d = self.lib.oracle_max_abs_diff(La, _ptr(a), Lb, _ptr(b), ca, ctypes.byref(bmax))
        return float(d), float(bmax.value)


    def newton_step(self, J, F, x):
        """One Newton corrector step (Section 7) on the caller's Jacobian J and residual F:
        s = argmin ||F - J s|| by ls_solve, then x - s per real part.  Returns
        (x_new, s, z, status)."""
        r = self.ls_solve(J, F)
        L = x.shape[-1]
        xn = np.empty_like(x)
        for j in range(x.shape[0]):
            for p in range(2):
                xn[j, p] = self.sub(L, x[j, p], r["x"][j, p])
        return xn, r["x"], r["z"], r["status"]

    def ls_adjoint(self, A, b, G):
        """Gradients (grad_A, grad_b) of a real loss with dL/dx = G (PyTorch's complex
        convention) through x = argmin ||b - A x||; also returns x and the status."""
        n, m, _, L = A.shape
        gA = np.zeros_like(A)
        gb = np.zeros((m, 2, L))
        x = np.zeros((n, 2, L))
        st = self.lib.oracle_ls_adjoint(L, _ptr(np.ascontiguousarray(A)), _ptr(np.ascontiguousarray(b)),
                                        _ptr(np.ascontiguousarray(G)), m, n, _ptr(gA), _ptr(gb), _ptr(x))
        return gA, gb, x, int(st)


_default: Oracle | None = None


def get() -> Oracle:
    """The default oracle build (compiled on first use if missing or stale)."""
    global _default
    if _default is None:
        _default = Oracle()
    return _default
