"""Seeded synthetic right-hand sides in factored form F = U V^T.

This module only generates inputs; it holds none of the solver's arithmetic
(no sine transform, no symbol, no cross, no rounding of the solution).  Both the
CUDA path and the CPU oracle receive the same factor bits from here.

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): a counter-based generator, so a
stream is a pure function of (seed, index).  Normals use the Box-Muller
transform.

Workloads (shapes follow the paper's model problem, Section 2 and Section 6:
unit square, homogeneous Dirichlet, RHS sampled at interior grid nodes
x_i = i/(n+1)):

* ``separable_random``  -- column k of U is cos(b_k x + c_k), column k of V is
  a_k exp(d_k y), with b_k, c_k, d_k ~ U[0,4) and a_k ~ N(0,1) drawn per column
  in that order.
* ``smooth_sum``        -- f(x,y) = 1/(1+x+y) + 0.5 sin(3 pi x) exp(-2y), given in
  factored form and compressed to a relative Frobenius tolerance.
* ``batch_problems``    -- a list of (n, r) drawn with n log-uniform in
  [n_lo, n_hi] and r uniform in {1..r_hi}, each with separable_random factors.
"""
from __future__ import annotations

import math
import numpy as np

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(seed: int, count: int) -> np.ndarray:
    """First ``count`` outputs of splitmix64 started at state ``seed`` (uint64)."""
    idx = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + idx * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on pairs of splitmix64 uniforms."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]                       # (0, 1], safe for log
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:count]


def grid(n: int) -> np.ndarray:
    """Interior nodes i/(n+1), i = 1..n."""
    return np.arange(1, n + 1, dtype=np.float64) / (n + 1)


def separable_random(n: int, r: int, seed: int = 0):
    """U (n x r), V (n x r) Fortran-ordered float64 with the random-coefficient
    separable columns described in the module docstring."""
    u = uniform01(seed, 3 * r).reshape(r, 3) * 4.0   # per column: b, c, d
    a = normal(seed ^ 0x5DEECE66D, r)
    x = grid(n)
    U = np.cos(np.outer(x, u[:, 0]) + u[:, 1])
    V = a * np.exp(np.outer(x, u[:, 2]))
    return np.asfortranarray(U), np.asfortranarray(V)


def _compress(P: np.ndarray, Q: np.ndarray, tol: float):
    """Re-express P Q^T with the fewest columns that keep a relative Frobenius
    error <= tol (numpy QR + SVD; input preparation only)."""
    qp, rp = np.linalg.qr(P)
    qq, rq = np.linalg.qr(Q)
    w, s, zt = np.linalg.svd(rp @ rq.T)
    total = float(np.sqrt(np.sum(s * s)))
    keep = len(s)
    tail = 0.0
    for k in range(len(s) - 1, 0, -1):       # drop from the smallest upward
        tail_new = math.sqrt(tail * tail + s[k] * s[k])
        if tail_new > tol * total:
            break
        tail = tail_new
        keep = k
    root = np.sqrt(s[:keep])
    U = (qp @ w[:, :keep]) * root
    V = (qq @ zt[:keep].T) * root
    return np.asfortranarray(U), np.asfortranarray(V)


def smooth_sum(n: int, tol: float):
    """f(x,y) = 1/(1+x+y) + 0.5 sin(3 pi x) exp(-2y) on the n x n interior grid,
    in factored form compressed to relative Frobenius tolerance ``tol``.

    1/s for s = 1+x+y in [1, 3] is written as the integral of exp(t - s e^t)
    over t in R and discretised by the trapezoidal rule with step 0.3 on
    [-40, 4] (147 nodes, relative error below 2e-13 on [1, 3]); every node is a
    separable term e^{t_k} e^{-e^{t_k}(1+x)} e^{-e^{t_k} y}.  The second term of
    f is already separable.  The stacked factors are then compressed.
    """
    x = grid(n)
    t = np.arange(-40.0, 4.0, 0.3)
    et = np.exp(t)
    P = np.exp(np.outer(-(1.0 + x), et)) * (0.3 * et)
    Q = np.exp(np.outer(-x, et))
    P = np.hstack([P, (0.5 * np.sin(3.0 * np.pi * x))[:, None]])
    Q = np.hstack([Q, np.exp(-2.0 * x)[:, None]])
    return _compress(P, Q, tol)


def smooth_sum_dense(n: int) -> np.ndarray:
    """The same f sampled directly on the grid (for small-n checks only)."""
    x = grid(n)
    return (1.0 / (1.0 + x[:, None] + x[None, :])
            + 0.5 * np.sin(3.0 * np.pi * x)[:, None] * np.exp(-2.0 * x)[None, :])


def batch_problems(count: int, n_lo: int, n_hi: int, r_hi: int, seed: int):
    """(n_p, r_p, seed_p) for ``count`` problems: n log-uniform in [n_lo, n_hi]
    (rounded), r uniform in {1..r_hi}."""
    u = uniform01(seed, 2 * count)
    lo, hi = math.log(n_lo), math.log(n_hi)
    out = []
    for p in range(count):
        n = int(round(math.exp(lo + (hi - lo) * u[2 * p])))
        n = min(max(n, n_lo), n_hi)
        r = 1 + min(int(u[2 * p + 1] * r_hi), r_hi - 1)
        out.append((n, r, (seed * 1000003 + p) & _MASK))
    return out
