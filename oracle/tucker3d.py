"""Plain FP64 CPU oracle for the 3D low-rank Poisson solve in Tucker format
(Section 3, Eq. flr:tucker; Section 4.1 and 4.2 in three dimensions).

TEST INFRASTRUCTURE ONLY: imported by tests/ and the CPU legs of bench.py,
never by the CUDA library.  Plain numpy, slow on purpose.

Problem: the 7-point Laplacian of the unit cube with homogeneous Dirichlet
conditions, n_k interior points in direction k, h_k = 1/(n_k + 1):

    A = T_1/h_1^2 (x) I (x) I + I (x) T_2/h_2^2 (x) I + I (x) I (x) T_3/h_3^2,

T = tridiag(-1, 2, -1), the 3D Kronecker sum of the 5-point operator.  The
DST-I matrices S_k diagonalise T_k (Section 4.1), so

    X = Xh x_1 S_1 x_2 S_2 x_3 S_3,   Xh(i, j, k) = Fh(i, j, k) / (mu_i + mu_j + mu_k),

mu the 1D eigenvalues (4/h^2) sin^2(i pi h / 2).  With the right-hand side in
Tucker format F = G x_1 U_1 x_2 U_2 x_3 U_3 (Eq. flr:tucker), Fh = G x_k (S_k
U_k) and any entry of Xh costs O(r^3) operations: Section 4.2 approximates Xh
directly by a cross method for tensors (the Tucker cross it cites) and rounds
the result (Section 3: QR of the factors and an SVD of the core, the
higher-order SVD of De Lathauwer, De Moor and Vandewalle 2000).

Tensor layout: C-ordered numpy arrays [i, j, k], i along x; a core G of
shape (r1, r2, r3); factors n_k x r_k.

The paper prints no 3D cross algorithm.  Reading taken here ("Tucker fibre
cross", the cross of Oseledets, Savostyanov and Tyrtyshnikov 2008 in an
incremental form):

* state: orthonormal bases Q_k (n_k x p_k), interpolation indices I_k (p_k of
  them) and the core C = Xh(I_1, I_2, I_3) x_1 Q_1(I_1)^-1 x_2 Q_2(I_2)^-1 x_3
  Q_3(I_3)^-1, so that Y = C x_k Q_k interpolates Xh on I_1 x I_2 x I_3 and
  ||Y||_F = ||C||_F;
* a step searches a pivot by alternating maximisation of the residual
  R = Xh - Y along fibres: from (i, j, k) = (i_s, j_s, k_s), two rounds of:
  the mode-2 fibre R(i, :, k) gives j, the mode-3 fibre R(i, j, :) gives k,
  the mode-1 fibre R(:, j, k) gives i (lowest index on ties); the three
  residual fibres through the pivot (i, j, k) are added to the bases (two
  passes of classical Gram-Schmidt; a fibre whose orthogonal part is below
  1e-13 of it is not added), each new basis vector bringing the DEIM index
  (Chaturantabut and Sorensen 2010) of its interpolation residual; then C is
  recomputed;
* the first step starts at (0, 0, 0) (the lowest frequencies, where 1/Lambda
  is largest); each later one at i_s = the largest |R(:, j, k)| of the last
  mode-1 fibre outside I_1, (j_s, k_s) = the last (j, k);
* the step test: the rank-one size ||e_1|| ||e_2|| ||e_3|| / rho^2 of the
  step (e_k its residual fibres, rho = R(i, j, k)) is <= tol ||C||_F on two
  consecutive steps, or |rho| <= 1e-14 of the first pivot.  It sees only the
  fibres through the pivot, so a probe round confirms it (the 3D form of
  the 2D cross's residual probes), with two estimates of the residual:
  - random fibres: for each mode, `probes` residual fibres at the other two
    indices drawn by splitmix64 (Steele, Lea and Flood 2014; state seed +
    round, outputs in mode order, output z gives the lower other index
    (z >> 32) mod n and the higher one (z & 0xffffffff) mod n); their mean
    square norm times the number of such fibres estimates ||R||_F^2 without
    bias;
  - cross fibres: for each mode, all p_a p_b residual fibres at the other two
    modes' interpolation indices I_a x I_b.  There R measures exactly what
    the mode's basis misses of the cross's own fibres, where the residual of
    an interpolation concentrates (it vanishes on the index grid itself);
    the root of the sum of their square norms is the estimate;
  the cross stops if every estimate is <= tol ||C||_F; otherwise the search
  restarts from the probed fibre of largest norm (at most 4 probe rounds);
* the cross also stops on a tensor that is exactly zero or after rmax steps;
  tol = tol_factor eps with tol_factor = 0.1 by default (the rounding after
  it is at eps).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import poisson_lowrank as P


# ------------------------------------------------------------ operator, symbol
def mu(n: int) -> np.ndarray:
    """1D eigenvalues of T / h^2 (h = 1/(n+1)), the 5-point symbol's a."""
    return P.symbol(n, "5pt")[0]


def dense_operator3(n1: int, n2: int, n3: int) -> np.ndarray:
    """The assembled 7-point operator on vec(X) with the LAST index fastest
    (C order of X[i, j, k]); small sizes only."""
    T = [P.second_difference(n) * (n + 1) ** 2 for n in (n1, n2, n3)]
    I = [np.eye(n) for n in (n1, n2, n3)]
    return (np.kron(np.kron(T[0], I[1]), I[2]) + np.kron(np.kron(I[0], T[1]), I[2])
            + np.kron(np.kron(I[0], I[1]), T[2]))


def apply_operator3(X: np.ndarray) -> np.ndarray:
    """A X on a full grid function (stencil form)."""
    Y = np.zeros_like(X)
    for ax in range(3):
        n = X.shape[ax]
        Xm = np.moveaxis(X, ax, 0)
        Ym = 2.0 * Xm.copy()
        Ym[1:] -= Xm[:-1]
        Ym[:-1] -= Xm[1:]
        Y += np.moveaxis(Ym, 0, ax) * (n + 1) ** 2
    return Y


def mode_product(T: np.ndarray, M: np.ndarray, mode: int) -> np.ndarray:
    """T x_mode M: contracts T's index `mode` with M's columns (M is rows x
    T.shape[mode])."""
    return np.moveaxis(np.tensordot(M, T, axes=(1, mode)), 0, mode)


def tucker_full(G: np.ndarray, U1, U2, U3) -> np.ndarray:
    """The full tensor of Eq. flr:tucker (small sizes only)."""
    return mode_product(mode_product(mode_product(G, U1, 0), U2, 1), U3, 2)


def dst3(X: np.ndarray) -> np.ndarray:
    """X x_1 S_1 x_2 S_2 x_3 S_3 (full tensor)."""
    for ax in range(3):
        X = np.moveaxis(P.dst1(np.moveaxis(X, ax, 0).reshape(X.shape[ax], -1)).reshape(
            np.moveaxis(X, ax, 0).shape), 0, ax)
    return X


def solve_full3(F: np.ndarray) -> np.ndarray:
    """X* = S((S F S) / Lambda)S in three modes: the full-format solve."""
    n1, n2, n3 = F.shape
    lam = mu(n1)[:, None, None] + mu(n2)[None, :, None] + mu(n3)[None, None, :]
    return dst3(dst3(F) / lam)


# ---------------------------------------------------------- the tensor Xh
class FreqTensor:
    """Xh(i, j, k) = Fh(i, j, k) / (mu1_i + mu2_j + mu3_k) with Fh = G x_k Uh_k:
    fibres and sub-blocks evaluated from the Tucker factors (Section 4.2: any
    entry in O(r) operations per mode)."""

    def __init__(self, G, Uh1, Uh2, Uh3):
        self.G = G
        self.Uh = (Uh1, Uh2, Uh3)
        self.mu = tuple(mu(U.shape[0]) for U in self.Uh)
        self.n = tuple(U.shape[0] for U in self.Uh)

    def block(self, I1, I2, I3) -> np.ndarray:
        Fh = tucker_full(self.G, self.Uh[0][I1], self.Uh[1][I2], self.Uh[2][I3])
        lam = (self.mu[0][I1][:, None, None] + self.mu[1][I2][None, :, None]
               + self.mu[2][I3][None, None, :])
        return Fh / lam

    def fibre(self, mode: int, a: int, b: int) -> np.ndarray:
        """The mode-`mode` fibre at the other two indices (a, b), in mode order."""
        idx = [None, None, None]
        others = [m for m in range(3) if m != mode]
        idx[others[0]] = [a]
        idx[others[1]] = [b]
        idx[mode] = np.arange(self.n[mode])
        return self.block(*idx).reshape(-1)


class DenseTensor:
    """An explicit tensor behind the same interface (pins)."""

    def __init__(self, T):
        self.T = T
        self.n = T.shape

    def block(self, I1, I2, I3):
        return self.T[np.ix_(I1, I2, I3)]

    def fibre(self, mode, a, b):
        idx = [a, b]
        idx.insert(mode, slice(None))
        return self.T[tuple(idx)].copy()


# ------------------------------------------------------------------ the cross
@dataclass
class TuckerCross:
    Q: list                     # orthonormal bases n_k x p_k
    I: list                     # interpolation indices, p_k each
    C: np.ndarray               # core p1 x p2 x p3
    pivots: list = field(default_factory=list)   # (i, j, k) per step
    steps: int = 0
    probe_rounds: int = 0
    converged: bool = False


def _argmax_abs(v: np.ndarray, exclude=()) -> int:
    """Lowest index of the largest |v| outside `exclude`."""
    a = np.abs(v).copy()
    if len(exclude):
        a[list(exclude)] = -1.0
    return int(np.argmax(a))


def _interp_core(X, Q, I):
    """C = X(I1, I2, I3) x_k Q_k(I_k)^-1 (square solves)."""
    C = X.block(I[0], I[1], I[2])
    for mode in range(3):
        C = mode_product(C, np.linalg.inv(Q[mode][I[mode]]), mode)
    return C


def _resid_fibre(X, Q, C, mode, a, b):
    """R = Xh - C x_k Q_k along the mode-`mode` fibre at the other indices (a, b)."""
    others = [m for m in range(3) if m != mode]
    v = C
    # contract the two other modes with the basis rows a, b (higher mode first)
    v = np.tensordot(v, Q[others[1]][b], axes=(others[1], 0))
    v = np.tensordot(v, Q[others[0]][a], axes=(others[0], 0))
    return X.fibre(mode, a, b) - Q[mode] @ v


def _add_basis(Q, I, mode, e):
    """Append the part of e orthogonal to Q[mode] (two CGS passes) and its DEIM
    index; nothing if that part is below 1e-13 of e."""
    q = Q[mode]
    ne = np.linalg.norm(e)
    if ne == 0.0:
        return False
    v = e - q @ (q.T @ e)
    v = v - q @ (q.T @ v)
    nv = np.linalg.norm(v)
    if nv <= 1e-13 * ne:
        return False
    v = v / nv
    if q.shape[1]:
        res = v - q @ np.linalg.solve(q[I[mode]], v[I[mode]])
    else:
        res = v
    idx = _argmax_abs(res, I[mode])
    Q[mode] = np.hstack([q, v[:, None]])
    I[mode] = I[mode] + [idx]
    return True


def _probe_round(X, Q, I, C, probes: int, seed: int):
    """(largest estimate of ||R||_F over the probe sets, restart position at
    the probed fibre of largest norm)."""
    est, worst, wpos = 0.0, -1.0, (0, 0, 0)
    zs = P.splitmix64_stream(seed, 3 * probes)

    def visit(mode, a, b):
        nonlocal worst, wpos
        ep = _resid_fibre(X, Q, C, mode, a, b)
        nn = float(np.dot(ep, ep))
        if nn > worst:
            pos = [0, 0, 0]
            others = [m for m in range(3) if m != mode]
            pos[others[0]], pos[others[1]], pos[mode] = a, b, _argmax_abs(ep)
            worst, wpos = nn, tuple(pos)
        return nn

    for mode in range(3):
        oa, ob = [m for m in range(3) if m != mode]
        ss = 0.0
        for z in zs[mode * probes:(mode + 1) * probes]:
            ss += visit(mode, (z >> 32) % X.n[oa], (z & 0xFFFFFFFF) % X.n[ob])
        est = max(est, math.sqrt(ss * X.n[oa] * X.n[ob] / probes))
        ss = 0.0
        for a in I[oa]:
            for b in I[ob]:
                ss += visit(mode, a, b)
        est = max(est, math.sqrt(ss))
    return est, wpos


def tucker_cross(X, eps: float, rmax: int = 64, tol_factor: float = 0.1, probes: int = 16, seed: int = 0,
                 max_probe_rounds: int = 4) -> TuckerCross:
    """The Tucker fibre cross of the module docstring on the tensor X (an
    object with .n, .fibre(mode, a, b) and .block(I1, I2, I3))."""
    tol = tol_factor * eps
    Q = [np.zeros((n, 0)) for n in X.n]
    I = [[], [], []]
    C = np.zeros((0, 0, 0))
    start = (0, 0, 0)
    small = 0
    rho0 = None
    out = TuckerCross(Q, I, C)
    for step in range(rmax):
        i, j, k = start
        for _ in range(2):
            j = _argmax_abs(_resid_fibre(X, Q, C, 1, i, k))
            k = _argmax_abs(_resid_fibre(X, Q, C, 2, i, j))
            e1 = _resid_fibre(X, Q, C, 0, j, k)
            i = _argmax_abs(e1)
        rho = e1[i]
        out.steps = step + 1
        if rho0 is None:
            rho0 = abs(rho)
            if rho0 == 0.0:
                out.converged = True
                break
        if abs(rho) <= 1e-14 * rho0:
            small = 2
        else:
            e2 = _resid_fibre(X, Q, C, 1, i, k)
            e3 = _resid_fibre(X, Q, C, 2, i, j)
            out.pivots.append((i, j, k))
            for mode, ev in ((0, e1), (1, e2), (2, e3)):
                _add_basis(Q, I, mode, ev)
            C = _interp_core(X, Q, I)
            upd = np.linalg.norm(e1) * np.linalg.norm(e2) * np.linalg.norm(e3) / (rho * rho)
            small = small + 1 if upd <= tol * np.linalg.norm(C) else 0
            start = (_argmax_abs(e1, I[0]), j, k)
        if small >= 2:
            if probes <= 0 or out.probe_rounds >= max_probe_rounds:
                out.converged = True
                break
            est, wpos = _probe_round(X, Q, I, C, probes, seed + out.probe_rounds)
            out.probe_rounds += 1
            if est <= tol * np.linalg.norm(C):
                out.converged = True
                break
            small = 0
            start = wpos
    out.Q, out.I, out.C = Q, I, C
    return out


# --------------------------------------------------------------- the rounding
def truncation_rank(s: np.ndarray, tol_abs: float) -> int:
    """Smallest R with sqrt(sum_{i >= R} s_i^2) <= tol_abs (s descending), R >= 1
    unless s is all zero."""
    R = len(s)
    tail = 0.0
    while R > 0:
        t = math.sqrt(tail * tail + s[R - 1] * s[R - 1])
        if t > tol_abs:
            break
        tail = t
        R -= 1
    return R


def hosvd_round(C: np.ndarray, Qs, eps: float):
    """Rounding of the Tucker tensor C x_k Q_k (Q_k orthonormal): the SVD of
    each unfolding of the core, each mode truncated with a tail <= eps ||C|| /
    sqrt(3) (so the error is <= eps ||C||), core projected on the kept
    singular vectors.  Returns (G, [U_k], [sigma_k])."""
    if C.size == 0 or not np.any(C):
        # the zero tensor: its rounding keeps nothing (ranks 0)
        return np.zeros((0, 0, 0)), [q[:, :0] for q in Qs], [np.zeros(0)] * 3
    total = np.linalg.norm(C)
    W, sig = [], []
    for mode in range(3):
        unf = np.moveaxis(C, mode, 0).reshape(C.shape[mode], -1)
        w, s, _ = np.linalg.svd(unf, full_matrices=False)
        R = truncation_rank(s, eps * total / math.sqrt(3.0))
        W.append(w[:, :R])
        sig.append(s)
    G = C
    for mode in range(3):
        G = mode_product(G, W[mode].T, mode)
    return G, [q @ w for q, w in zip(Qs, W)], sig


# ---------------------------------------------------------------- the solve
@dataclass
class Tucker3Result:
    G: np.ndarray
    U: list
    cross: TuckerCross


def lr_poisson3d(G: np.ndarray, U1, U2, U3, eps: float, rmax: int = 64, tol_factor: float = 0.1,
                 probes: int = 16, seed: int = 0) -> Tucker3Result:
    """Low-rank 3D solve: DST of the factors, Tucker cross of Xh, rounding,
    inverse DST of the factors."""
    X = FreqTensor(G, P.dst1(U1), P.dst1(U2), P.dst1(U3))
    cr = tucker_cross(X, eps, rmax, tol_factor, probes, seed)
    Gs, Us, _ = hosvd_round(cr.C, cr.Q, eps)
    return Tucker3Result(Gs, [P.dst1(U) for U in Us], cr)


def rel_error_full(res: Tucker3Result, F: np.ndarray) -> float:
    """||X - X*||_F / ||X*||_F against the full-format solve (small n)."""
    Xs = solve_full3(F)
    X = tucker_full(res.G, *res.U)
    return float(np.linalg.norm(X - Xs) / np.linalg.norm(Xs))


def rel_error_freq_sampled(G_out, U_out, G, U1, U2, U3, slices) -> float:
    """Relative Frobenius error of a Tucker solution (G_out, [U_out]) on the
    frequency-space slices Xh(:, :, k), k in `slices`, against the exact
    Fh / Lambda there (large n: the DST is orthogonal, so the error of the
    whole tensor is its error in frequency space, of which these slices are
    a sample)."""
    Xf = FreqTensor(G, P.dst1(U1), P.dst1(U2), P.dst1(U3))
    Uh = [P.dst1(U) for U in U_out]
    num = den = 0.0
    for k in slices:
        ref = Xf.block(np.arange(Xf.n[0]), np.arange(Xf.n[1]), [k])[:, :, 0]
        got = np.einsum("abc,ia,jb,c->ij", G_out, Uh[0], Uh[1], Uh[2][k], optimize=True)
        num += np.sum((got - ref) ** 2)
        den += np.sum(ref ** 2)
    return math.sqrt(num / den)
