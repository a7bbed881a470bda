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
* ``smooth3d``          -- f(x,y,z) = exp(-(x+2y+3z)) + 1/sqrt(x^2+y^2+z^2+0.01) on
  the n^3 interior grid, in Tucker format compressed to a relative tolerance.
* ``block_diagonal_freq`` -- frequency-space factors with disjoint supports
  (a block-diagonal frequency-space solution; residual-probe cases).
* ``tucker_random``     -- random Tucker tensors with separable factor columns
  and normal core entries (3D parity cases).
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



def block_diagonal_freq(n: int, split: int, seed: int = 5):
    """Two frequency-space factor columns (n x 2, Fortran order) with disjoint
    supports: column 0 is standard normal on indices < split and zero after,
    column 1 standard normal on indices >= split and zero before, in both Uh
    and Vh.  Uh Vh^T (and any entrywise rescaling of it) is block diagonal.
    The caller maps them to space with the sine transform."""
    z = normal(seed, 4 * n).reshape(4, n)
    Uh, Vh = np.zeros((n, 2), order="F"), np.zeros((n, 2), order="F")
    Uh[:split, 0], Vh[:split, 0] = z[0, :split], z[1, :split]
    Uh[split:, 1], Vh[split:, 1] = z[2, split:], z[3, split:]
    return Uh, Vh

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


# ---------------------------------------------------------------- 3D (Tucker)
# Tensors in Tucker format (Section 3, Eq. flr:tucker): a core G of shape
# (r1, r2, r3), C-ordered (G[a, b, c] at (a r2 + b) r3 + c), and factors U_k,
# n_k x r_k, Fortran-ordered; A = G x_1 U1 x_2 U2 x_3 U3.

def _orth_trunc(A: np.ndarray, tol: float):
    """Orthonormal basis of the columns of A up to relative size tol (numpy SVD;
    input preparation only)."""
    w, s, _ = np.linalg.svd(A, full_matrices=False)
    keep = max(1, int(np.sum(s > tol * s[0])))
    return w[:, :keep]


def _cp_to_tucker(A1: np.ndarray, A2: np.ndarray, A3: np.ndarray, lam: np.ndarray, tol: float):
    """The CP tensor sum_q lam_q A1[:, q] o A2[:, q] o A3[:, q] re-expressed in
    Tucker format with relative Frobenius error <= tol: a basis of each factor
    matrix's columns (to 1e-15), the core in those bases, then the core's
    higher-order SVD truncated with tol / sqrt(3) per mode (De Lathauwer, De
    Moor, Vandewalle 2000).  Input preparation only."""
    W = [_orth_trunc(A, 1e-15) for A in (A1, A2, A3)]
    B = [w.T @ A for w, A in zip(W, (A1, A2, A3))]
    core = np.einsum("q,aq,bq,cq->abc", lam, B[0], B[1], B[2], optimize=True)
    total = np.linalg.norm(core)
    Z = []
    for mode in range(3):
        unf = np.moveaxis(core, mode, 0).reshape(core.shape[mode], -1)
        z, s, _ = np.linalg.svd(unf, full_matrices=False)
        keep = len(s)
        tail = 0.0
        for k in range(len(s) - 1, 0, -1):
            tail_new = math.sqrt(tail * tail + s[k] * s[k])
            if tail_new > tol / math.sqrt(3.0) * total:
                break
            tail = tail_new
            keep = k
        Z.append(z[:, :keep])
    G = np.einsum("abc,ai,bj,ck->ijk", core, Z[0], Z[1], Z[2], optimize=True)
    Us = [np.asfortranarray(w @ z) for w, z in zip(W, Z)]
    return np.ascontiguousarray(G), Us[0], Us[1], Us[2]


def smooth3d(n: int, tol: float):
    """f(x,y,z) = exp(-(x+2y+3z)) + 1/sqrt(x^2+y^2+z^2+0.01) on the n^3 interior
    grid in Tucker format, relative Frobenius tolerance ``tol``.

    1/sqrt(s) = (2/sqrt(pi)) int_R exp(-s e^{2t}) e^t dt (s = x^2+y^2+z^2+0.01 in
    [0.01, 3.01]), discretised by the trapezoidal rule with step 0.15 on
    [-34, 5] (261 nodes; relative error below 1e-13 on that interval): each
    node is the separable term e^{-0.01 e^{2t}} e^{-x^2 e^{2t}} e^{-y^2 e^{2t}}
    e^{-z^2 e^{2t}}.  With the separable first term this is a CP tensor of 262
    terms, compressed to Tucker format.
    Returns (G, U1, U2, U3)."""
    x = grid(n)
    t = np.arange(-34.0, 5.0 + 1e-9, 0.15)
    e2 = np.exp(2.0 * t)
    lam = (2.0 / math.sqrt(math.pi)) * 0.15 * np.exp(t) * np.exp(-0.01 * e2)
    E = np.exp(-np.outer(x * x, e2))
    A1 = np.hstack([E, np.exp(-x)[:, None]])
    A2 = np.hstack([E, np.exp(-2.0 * x)[:, None]])
    A3 = np.hstack([E, np.exp(-3.0 * x)[:, None]])
    return _cp_to_tucker(A1, A2, A3, np.append(lam, 1.0), tol)


def smooth3d_dense(n: int) -> np.ndarray:
    """The same f sampled directly on the grid (small n only), C-ordered
    [i, j, k] with i along x."""
    x = grid(n)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    return np.exp(-(X + 2.0 * Y + 3.0 * Z)) + 1.0 / np.sqrt(X * X + Y * Y + Z * Z + 0.01)


def tucker_random(n, r, seed: int = 0):
    """Random Tucker tensor with separable factor columns like separable_random:
    mode 1 cos(b x + c), mode 2 exp(d y), mode 3 cos(b' z + c'), coefficients in
    [0, 4); core entries N(0, 1).  n and r are ints or 3-tuples.
    Returns (G, U1, U2, U3)."""
    ns = (n, n, n) if np.isscalar(n) else tuple(n)
    rs = (r, r, r) if np.isscalar(r) else tuple(r)
    u = uniform01(seed, 5 * max(rs)).reshape(max(rs), 5) * 4.0
    U1 = np.cos(np.outer(grid(ns[0]), u[:rs[0], 0]) + u[:rs[0], 1])
    U2 = np.exp(np.outer(grid(ns[1]), u[:rs[1], 2]) * 0.5)
    U3 = np.cos(np.outer(grid(ns[2]), u[:rs[2], 3]) + u[:rs[2], 4])
    G = normal(seed ^ 0x3C6EF372, rs[0] * rs[1] * rs[2]).reshape(rs)
    return (np.ascontiguousarray(G), np.asfortranarray(U1), np.asfortranarray(U2), np.asfortranarray(U3))
