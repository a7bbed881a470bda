"""Plain FP64 CPU oracle for the 2D Stokes problem on semi-staggered grids
and its Uzawa reduction (Section 2, Eq. flr:stprob, Eq. flr:schur).

TEST INFRASTRUCTURE ONLY: imported by tests/ and the CPU legs of bench.py,
never by the CUDA library.  Dense, full-format and slow on purpose.

Unknowns (n cells per direction, h = 1/n): the velocity components u, v on
the (n-1) x (n-1) interior vertices, the pressure P on the n x n cell
centres; the first matrix index runs along x.  With the (n-1) x n matrices
G = E - Z, H = E + Z of Section 2 the discrete gradient is

    B_x P = G P H^T / (4h),   B_y P = H P G^T / (4h),

its transpose (the discrete divergence up to sign) is

    B^T (u, v) = (G^T u H + H^T v G) / (4h),

and the Laplacian is Delta = B_x B_x^T + B_y B_y^T, i.e.

    Delta U = (G G^T U H H^T + H H^T U G G^T) / (16 h^2),

the ``"semi"`` kind of ``poisson_lowrank`` on m = n - 1 unknowns.  The system
[[A, B], [B^T, 0]] [u; p] = [f; 0] with A = I_2 (x) Delta is reduced to the
Schur equation (B^T A^-1 B) p = B^T A^-1 f (Eq. flr:schur; g = 0 in the
workloads), solved by conjugate gradients (Section 2).

Readings of the paper taken here:

* "G (x) H" is read with G acting on the x index (the paper does not fix the
  Kronecker convention; the other reading swaps the roles of u and v).
* Uzawa is conjugate gradients on the Schur equation (Section 2); the
  pressure's two kernel modes (constant and checkerboard) are projected out
  and the iteration stops on the relative Schur residual
  ||B^T u|| / ||B^T A^-1 f||, where u = A^-1 (f - B p) is the velocity.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import poisson_lowrank as P


def gh(n: int):
    """(G, H), both (n-1) x n (Section 2)."""
    return P.g_matrix(n), P.h_matrix(n)


def bx(Pm: np.ndarray, n: int) -> np.ndarray:
    G, H = gh(n)
    return G @ Pm @ H.T * (n / 4.0)


def by(Pm: np.ndarray, n: int) -> np.ndarray:
    G, H = gh(n)
    return H @ Pm @ G.T * (n / 4.0)


def bt(u: np.ndarray, v: np.ndarray, n: int) -> np.ndarray:
    G, H = gh(n)
    return (G.T @ u @ H + H.T @ v @ G) * (n / 4.0)


def laplace(U: np.ndarray, n: int) -> np.ndarray:
    """Delta U from the B operators (Delta = B_x B_x^T + B_y B_y^T)."""
    G, H = gh(n)
    return (G @ G.T @ U @ H @ H.T + H @ H.T @ U @ G @ G.T) * (n * n / 16.0)


def laplace_solve(F: np.ndarray, n: int) -> np.ndarray:
    """Delta^-1 F by the DST diagonalisation (Eq. flr:diag), m = n - 1."""
    return P.solve_full(F, "semi")


def schur_apply(Pm: np.ndarray, n: int) -> np.ndarray:
    """(B^T A^-1 B) P (Eq. flr:schur)."""
    return bt(laplace_solve(bx(Pm, n), n), laplace_solve(by(Pm, n), n), n)


def kernel_modes(n: int):
    """Orthonormal basis of the Schur kernel: the constant and the
    checkerboard pressure (B annihilates both)."""
    one = np.ones((n, n))
    c = (-1.0) ** np.arange(n)
    chk = np.outer(c, c)
    return one / n, chk / n


def project_kernel(Pm: np.ndarray, n: int) -> np.ndarray:
    for K in kernel_modes(n):
        Pm = Pm - np.sum(Pm * K) * K
    return Pm


def body_force(n: int):
    """The benchmark body force at the interior vertices, as rank-1 factors:
    f1 = sin(pi x) cos(pi y), f2 = -cos(pi x) sin(pi y) (1 + y)."""
    x = np.arange(1, n) / n
    f1 = (np.sin(np.pi * x)[:, None], np.cos(np.pi * x)[:, None])
    f2 = (-np.cos(np.pi * x)[:, None], (np.sin(np.pi * x) * (1.0 + x))[:, None])
    return f1, f2


@dataclass
class UzawaResult:
    u: np.ndarray
    v: np.ndarray
    p: np.ndarray
    iters: int
    resid: float        # ||B^T u|| / ||B^T A^-1 f|| at exit
    history: list


def uzawa_cg(f1: np.ndarray, f2: np.ndarray, n: int, tol: float = 1e-10, maxit: int = 500,
             g: np.ndarray | None = None) -> UzawaResult:
    """Conjugate gradients on (B^T A^-1 B) p = B^T A^-1 f - g, p0 = 0, full
    format.  g (n x n, default 0) is the right-hand side of the divergence
    equation B^T u = g; the Schur equation of Eq. flr:schur is printed
    without it, and elimination of u = A^-1 (f - B p) gives the -g (reading
    G5).  Only the part of g orthogonal to the kernel modes can be met."""
    rhs = bt(laplace_solve(f1, n), laplace_solve(f2, n), n)
    if g is not None:
        rhs = rhs - g
    rhs = project_kernel(rhs, n)
    nr0 = np.linalg.norm(rhs)
    p = np.zeros((n, n))
    r = rhs.copy()
    d = r.copy()
    rr = np.sum(r * r)
    hist = [1.0]
    it = 0
    while it < maxit and np.sqrt(rr) > tol * nr0:
        q = schur_apply(d, n)
        alpha = rr / np.sum(d * q)
        p = p + alpha * d
        r = project_kernel(r - alpha * q, n)
        rr_new = np.sum(r * r)
        d = r + (rr_new / rr) * d
        rr = rr_new
        it += 1
        hist.append(np.sqrt(rr) / nr0)
    p = project_kernel(p, n)
    u = laplace_solve(f1 - bx(p, n), n)
    v = laplace_solve(f2 - by(p, n), n)
    div = bt(u, v, n) if g is None else bt(u, v, n) - project_kernel(g, n)
    res = np.linalg.norm(div) / nr0 if nr0 > 0.0 else 0.0  # zero force: u = p = 0
    return UzawaResult(u, v, p, it, res, hist)


def saddle_dense(f1: np.ndarray, f2: np.ndarray, n: int, g: np.ndarray | None = None):
    """The assembled saddle system of Eq. flr:stprob (small n), divergence
    equation B^T u = g (default 0), solved by least squares with the
    minimum-norm pressure (independent of the DST and of the Uzawa
    reduction)."""
    m = n - 1
    G, H = gh(n)
    # vec with the first index fastest: vec(G P H^T) = (H (x) G) vec(P)
    Bx = np.kron(H, G) * (n / 4.0)
    By = np.kron(G, H) * (n / 4.0)
    D = Bx @ Bx.T + By @ By.T
    nv = m * m
    K = np.zeros((2 * nv + n * n, 2 * nv + n * n))
    K[:nv, :nv] = D
    K[nv:2 * nv, nv:2 * nv] = D
    K[:nv, 2 * nv:] = Bx
    K[nv:2 * nv, 2 * nv:] = By
    K[2 * nv:, :nv] = Bx.T
    K[2 * nv:, nv:2 * nv] = By.T
    gv = np.zeros(n * n) if g is None else g.reshape(-1, order="F")
    rhs = np.concatenate([f1.reshape(-1, order="F"), f2.reshape(-1, order="F"), gv])
    sol = np.linalg.lstsq(K, rhs, rcond=None)[0]
    u = sol[:nv].reshape(m, m, order="F")
    v = sol[nv:2 * nv].reshape(m, m, order="F")
    p = project_kernel(sol[2 * nv:].reshape(n, n, order="F"), n)
    return u, v, p


def schur_dense(n: int) -> np.ndarray:
    """The n^2 x n^2 Schur complement B^T A^-1 B assembled densely (small n)."""
    m = n - 1
    G, H = gh(n)
    Bx = np.kron(H, G) * (n / 4.0)
    By = np.kron(G, H) * (n / 4.0)
    D = Bx @ Bx.T + By @ By.T
    Di = np.linalg.inv(D)
    return Bx.T @ Di @ Bx + By.T @ Di @ By
