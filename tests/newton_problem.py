"""A nonlinear test system for the Newton corrector, evaluated by the oracle (the caller's
side of the interface: the library itself evaluates no functions).

    F_i(x) = (A x)_i + c_i x_{p(i)}^2 - b_i,  p(i) = i mod n,  i = 0..m-1
    J_ij   = a_ij + 2 c_i x_j [j = p(i)]

with b = A x* + c x*_p^2 formed by the oracle, so that x* is a root."""

import numpy as np

from paper_1210_0800_gb300 import inputs


def problem(orc, m, n, L, seed, cscale=0.25):
    A, xs, _ = inputs.system(m, n, L, seed)
    c = inputs.vector_uniform(m, L, inputs.substream(seed, 7)) * cscale
    b = _quad(orc, A, c, xs, L)
    return A, c, b, xs


def _quad(orc, A, c, x, L):
    """A x + c x_p^2 (rounded to L limbs)."""
    n, m = A.shape[0], A.shape[1]
    ax = orc.matvec(A, x, Lout=L)
    out = np.empty_like(ax)
    for i in range(m):
        xp = x[i % n]
        q = orc.cmul(L, c[i], orc.cmul(L, xp, xp))
        for p in range(2):
            out[i, p] = orc.add(L, ax[i, p], q[p])
    return out


def evaluate(orc, A, c, b, x):
    """(J, F) at x."""
    n, m, _, L = A.shape
    q = _quad(orc, A, c, x, L)
    F = np.empty_like(q)
    for i in range(m):
        for p in range(2):
            F[i, p] = orc.sub(L, q[i, p], b[i, p])
    J = A.copy()
    two = np.zeros((2, L))
    two[0, 0] = 2.0
    for i in range(m):
        j = i % n
        d = orc.cmul(L, orc.cmul(L, two, c[i]), x[j])
        for p in range(2):
            J[j, i, p] = orc.add(L, A[j, i, p], d[p])
    return J, F
