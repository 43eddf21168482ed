"""Seeded synthetic inputs for the complex DD/QD least-squares workloads.

This module only draws random numbers and places them into limb arrays; it contains
none of the method's arithmetic (no Gram-Schmidt, no back substitution, no DD/QD
operations).  Both the CUDA path and the CPU oracle are fed from here.

Array conventions (shared with the C-ABI and the oracle):
  * a real number carries L float64 limbs (L = 1 double, 2 double-double, 4 quad-double),
    its value being the exact sum of the limbs, largest first;
  * a complex element is 2L consecutive float64 values {re_0..re_{L-1}, im_0..im_{L-1}};
  * an m x n matrix is stored column-major by element: numpy shape (n, m, 2, L), element
    (i, j) at [j, i]; a vector of length m has shape (m, 2, L).

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", 2014): state_k = seed + k * 0x9E3779B97F4A7C15, output = the
published 64-bit finaliser of state_k.  A uniform double in [0, 1) is (z >> 11) * 2^-53.

Lower limbs.  The workloads ask for a leading limb drawn from the value distribution and
a lower limb of size about 2^-53 times the leading one.  Here limb k+1 is drawn uniformly
from [-ulp(limb_k)/2, +ulp(limb_k)/2] (ulp = numpy.spacing), so every generated number is a
normalised expansion without any renormalisation step.
"""

from __future__ import annotations

import math

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1

# Seeds of the five workloads (seed of workload i = BASE_SEED + i).
BASE_SEED = 20130113


def splitmix64(seed: int, count: int) -> np.ndarray:
    """``count`` consecutive SplitMix64 outputs for ``seed`` (uint64 array)."""
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + k * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [-1, 1) (2u - 1 is exact for u = k 2^-53)."""
    return 2.0 * uniform01(seed, count) - 1.0


def uniform_int(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Uniform integers in [lo, hi] inclusive."""
    u = uniform01(seed, count)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


def substream(seed: int, tag: int) -> int:
    """Independent seed for one use (tag) of a workload seed."""
    return (seed ^ ((tag + 1) * GOLDEN)) & MASK64


def system_seed(seed: int, index: int) -> int:
    """Seed of system ``index`` of a batch."""
    return (seed ^ ((index * GOLDEN) & MASK64)) & MASK64


def with_lower_limbs(lead: np.ndarray, L: int, seed: int) -> np.ndarray:
    """Append L-1 lower limbs to the leading limbs ``lead`` (any shape); returns shape + (L,).

    Limb k+1 is uniform in [-ulp(limb_k)/2, ulp(limb_k)/2]; products of a double with a
    power of two (numpy.spacing) are exact.
    """
    lead = np.asarray(lead, dtype=np.float64)
    out = np.zeros(lead.shape + (L,), dtype=np.float64)
    out[..., 0] = lead
    prev = lead
    for k in range(1, L):
        u = uniform01(substream(seed, 100 + k), lead.size).reshape(lead.shape) - 0.5
        limb = np.where(prev == 0.0, 0.0, u * np.spacing(np.abs(prev)))
        out[..., k] = limb
        prev = limb
    return out


def complex_uniform(shape, L: int, seed: int) -> np.ndarray:
    """Complex numbers with leading limbs of re and im uniform in [-1, 1)."""
    count = int(np.prod(shape))
    re = uniform_pm1(substream(seed, 1), count).reshape(shape)
    im = uniform_pm1(substream(seed, 2), count).reshape(shape)
    out = np.empty(tuple(shape) + (2, L), dtype=np.float64)
    out[..., 0, :] = with_lower_limbs(re, L, substream(seed, 3))
    out[..., 1, :] = with_lower_limbs(im, L, substream(seed, 4))
    return out


def complex_polar(shape, L: int, seed: int, g: float, log_uniform: bool = False) -> np.ndarray:
    """r exp(i theta) with theta uniform in [0, 2 pi) and r uniform in [10^-g, 10^g]
    (linear scale; or log-uniform when ``log_uniform``): the generator of the paper's
    accuracy experiment (Section 4, Table 2)."""
    count = int(np.prod(shape))
    u = uniform01(substream(seed, 5), count).reshape(shape)
    if log_uniform:
        r = 10.0 ** (g * (2.0 * u - 1.0))
    else:
        lo, hi = 10.0 ** (-g), 10.0 ** g
        r = lo + (hi - lo) * u
    theta = 2.0 * math.pi * uniform01(substream(seed, 6), count).reshape(shape)
    out = np.empty(tuple(shape) + (2, L), dtype=np.float64)
    out[..., 0, :] = with_lower_limbs(r * np.cos(theta), L, substream(seed, 7))
    out[..., 1, :] = with_lower_limbs(r * np.sin(theta), L, substream(seed, 8))
    return out


def scale_leading(M: np.ndarray, factors: np.ndarray, L: int, seed: int) -> np.ndarray:
    """Return a copy of M whose leading limbs are multiplied by ``factors`` (broadcast over
    the element shape) and whose lower limbs are redrawn for the new leading limbs.  The
    stored, scaled numbers are the truth both sides compute with."""
    lead = M[..., 0] * factors[..., None]
    out = np.empty_like(M)
    out[..., 0, :] = with_lower_limbs(lead[..., 0], L, substream(seed, 9))
    out[..., 1, :] = with_lower_limbs(lead[..., 1], L, substream(seed, 10))
    return out


# --------------------------------------------------------------------------- workloads


def matrix_uniform(m: int, n: int, L: int, seed: int) -> np.ndarray:
    """m x n complex matrix (shape (n, m, 2, L)), leading limbs uniform in [-1, 1)."""
    return complex_uniform((n, m), L, substream(seed, 11))


def vector_uniform(m: int, L: int, seed: int) -> np.ndarray:
    """Complex vector (shape (m, 2, L)), leading limbs uniform in [-1, 1)."""
    return complex_uniform((m,), L, substream(seed, 12))


def matrix_extreme(m: int, n: int, L: int, seed: int, row_exp=(-12, 12), col_exp=(-4, 4)) -> np.ndarray:
    """Jacobian-like extreme-value matrix: a uniform matrix whose row i is scaled by
    10^{e_i}, e_i uniform in row_exp, and column j by 10^{f_j}, f_j uniform in col_exp
    (the factors are the doubles nearest to the powers of ten)."""
    A = matrix_uniform(m, n, L, seed)
    e = uniform_int(substream(seed, 13), m, row_exp[0], row_exp[1])
    f = uniform_int(substream(seed, 14), n, col_exp[0], col_exp[1])
    factors = (10.0 ** f.astype(np.float64))[:, None] * (10.0 ** e.astype(np.float64))[None, :]
    return scale_leading(A, factors, L, substream(seed, 15))


def ragged_shapes(batch: int, seed: int, n_lo=16, n_hi=192, extra_lo=0, extra_hi=16):
    """Batch of (m, n): n uniform in [n_lo, n_hi], m = n + uniform{extra_lo..extra_hi}."""
    n = uniform_int(substream(seed, 16), batch, n_lo, n_hi)
    m = n + uniform_int(substream(seed, 17), batch, extra_lo, extra_hi)
    return m.astype(np.int64), n.astype(np.int64)


WORKLOADS = {
    "c0": dict(desc="complex DD MGS least squares, m=n=32, one system", m=32, n=32, L=2, seed=BASE_SEED + 0),
    "c1": dict(desc="complex QD MGS least squares, m=320, n=256, dependent sequence of solves",
               m=320, n=256, L=4, seed=BASE_SEED + 1),
    "c2": dict(desc="extreme-value complex DD, m=n=256, rows x10^U{-12..12}, cols x10^U{-4..4}",
               m=256, n=256, L=2, seed=BASE_SEED + 2),
    "c3": dict(desc="batched ragged complex DD, 512 systems, n~U{16..192}, m=n+U{0..16}",
               batch=512, L=2, seed=BASE_SEED + 3),
    "c4": dict(desc="differentiated complex DD least squares, m=160, n=128, batch 64",
               m=160, n=128, batch=64, L=2, seed=BASE_SEED + 4),
}


def workload_seed(name: str) -> int:
    """Base seed of a named workload (its c0..c4 prefix); other names use c1's."""
    key = name.split("_")[0]
    return WORKLOADS[key]["seed"] if key in WORKLOADS else WORKLOADS["c1"]["seed"]


def ragged_batch(L: int, batch: int, n_rng, e_rng, seed: int):
    """A ragged batch of independent systems [(A, b_generic)], shapes from ragged_shapes."""
    ms, ns = ragged_shapes(batch, seed, n_rng[0], n_rng[1], e_rng[0], e_rng[1])
    return [(lambda s: (s[0], s[2]))(system(int(m), int(n), L, system_seed(seed, i))) for i, (m, n) in
            enumerate(zip(ms, ns))]


def system(m: int, n: int, L: int, seed: int, extreme: bool = False):
    """One least-squares system: (A, x_true, b_generic).

    A has shape (n, m, 2, L); x_true shape (n, 2, L) with the same value distribution;
    b_generic shape (m, 2, L) is an independent right-hand side of the same distribution
    as A's entries (a generic Newton residual).  A right-hand side with a planted solution,
    b = A x_true, is formed by the callers that need it (it takes extended-precision
    arithmetic, which this module does not do).
    """
    A = matrix_extreme(m, n, L, seed) if extreme else matrix_uniform(m, n, L, seed)
    x = vector_uniform(n, L, substream(seed, 20))
    b = vector_uniform(m, L, substream(seed, 21))
    if extreme:
        # the generic right-hand side follows the row scaling of A
        e = uniform_int(substream(seed, 13), m, -12, 12)
        b = scale_leading(b, 10.0 ** e.astype(np.float64), L, substream(seed, 22))
    return A, x, b
