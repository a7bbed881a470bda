"""Plain FP64 CPU oracle for the low-rank Poisson solve (arXiv:1306.2150).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py, never by the CUDA library.  Slow and literal on purpose.

Problem (Section 2, Section 4.1): on the unit square with homogeneous Dirichlet
conditions and m interior grid points per direction (h = 1/(m+1)), solve the
SPD system  A X = F  where X[i, j] is the unknown at (x_i, y_j) and

    A X = scale * (P X Q + Q X P)                                   (*)

with symmetric m x m matrices P, Q:

* kind ``"5pt"``  : the 5-point Laplacian, P = T = tridiag(-1, 2, -1), Q = I,
  scale = 1/h^2.  Its frequency-space symbol is mu_i + mu_j (Eq. flr:div).
* kind ``"semi"`` : the semi-staggered Laplacian of Section 2,
  Delta = B_x B_x^T + B_y B_y^T with B_x = G (x) H / (4h), B_y = H (x) G / (4h),
  i.e. P = A1 = G G^T, Q = A2 = H H^T, scale = 1/(16 h^2) (Section 4.1), with
  m = n - 1 velocity unknowns per direction on a grid of n cells (h = 1/n).

The DST-I matrix S (orthonormal, symmetric, S = S^-1) diagonalises P and Q
(Section 4.1, Eq. flr:diag), so with Uh = S U, Vh = S V the frequency-space
solution of F = U V^T is  Xh[i, j] = (Uh V h^T)[i, j] / Lambda[i, j]  (Eq. flr:div)
and X = S Xh S.  Lambda[i, j] = a_i b_j + b_i a_j covers both kinds:
5pt a = mu, b = 1;  semi a = lambda/(16 h^2), b = 4 - lambda.

Readings of the paper taken here (the paper is silent or inconsistent):

* The printed symbol (4 - l_i) l_i + (4 - l_j) l_j of Section 4.2 does not match
  its own Delta = A1 (x) A2 + A2 (x) A1; the semi kind uses the symbol of that
  Delta, l_i (4 - l_j) + (4 - l_i) l_j, and the 5pt kind the sum mu_i + mu_j.
* The cross of Section 4.2 is read as adaptive cross approximation with partial
  pivoting (the cited Bebendorf / Tyrtyshnikov cross): see ``aca_cross``.
* Rounding (Section 3): QR of both factors, SVD of the small core, drop the
  smallest singular values while sqrt(sum of dropped s^2) <= eps * ||s||_2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

try:  # scipy is a library FFT used as one step for large m
    import scipy.fft as _sfft
except Exception:  # pragma: no cover
    _sfft = None

KINDS = ("5pt", "semi")
DENSE_DST_MAX = 4096


# --------------------------------------------------------------------------
# Section 2: the grid operators
# --------------------------------------------------------------------------
def shift_matrices(n: int):
    """E and Z, both (n-1) x n (Section 2): E drops the first entry of a vector
    (moving the rest up), Z drops the last entry."""
    E = np.zeros((n - 1, n))
    Z = np.zeros((n - 1, n))
    for i in range(n - 1):
        E[i, i + 1] = 1.0
        Z[i, i] = 1.0
    return E, Z


def g_matrix(n: int) -> np.ndarray:
    """G = E - Z (Section 2): discrete difference, (n-1) x n."""
    E, Z = shift_matrices(n)
    return E - Z


def h_matrix(n: int) -> np.ndarray:
    """H = E + Z (Section 2): discrete average (times 2), (n-1) x n."""
    E, Z = shift_matrices(n)
    return E + Z


def second_difference(m: int) -> np.ndarray:
    """T = tridiag(-1, 2, -1) of order m (the 1D Dirichlet second difference)."""
    T = 2.0 * np.eye(m)
    for i in range(m - 1):
        T[i, i + 1] = T[i + 1, i] = -1.0
    return T


def operator_parts(m: int, kind: str):
    """(P, Q, scale) of form (*) for m unknowns per direction."""
    h = 1.0 / (m + 1)
    if kind == "5pt":
        return second_difference(m), np.eye(m), 1.0 / (h * h)
    if kind == "semi":
        n = m + 1                       # cells per direction, h = 1/n
        G, H = g_matrix(n), h_matrix(n)
        return G @ G.T, H @ H.T, 1.0 / (16.0 * h * h)
    raise ValueError(kind)


def dense_operator(m: int, kind: str) -> np.ndarray:
    """The m^2 x m^2 matrix of (*) acting on vec(X) (column-major, i fastest).
    vec(P X Q) = (Q (x) P) vec(X) for symmetric Q.  Small m only."""
    P, Q, s = operator_parts(m, kind)
    return s * (np.kron(Q, P) + np.kron(P, Q))


def _tridiag_apply(X: np.ndarray, diag: float, off: float) -> np.ndarray:
    """(tridiag(off, diag, off) X) along axis 0, any size."""
    Y = diag * X
    Y[1:] += off * X[:-1]
    Y[:-1] += off * X[1:]
    return Y


def apply_parts(X: np.ndarray, kind: str):
    """(P X, Q X) along axis 0 without forming P, Q (tridiagonal)."""
    if kind == "5pt":
        return _tridiag_apply(X, 2.0, -1.0), X.copy()
    if kind == "semi":
        return _tridiag_apply(X, 2.0, -1.0), _tridiag_apply(X, 2.0, 1.0)
    raise ValueError(kind)


def op_scale(m: int, kind: str) -> float:
    h = 1.0 / (m + 1)
    return 1.0 / (h * h) if kind == "5pt" else 1.0 / (16.0 * h * h)


def apply_operator(X: np.ndarray, kind: str) -> np.ndarray:
    """A X of form (*) on a full m x m grid function."""
    m = X.shape[0]
    PX, QX = apply_parts(X, kind)
    PXQ = apply_parts(PX.T, kind)[1].T
    QXP = apply_parts(QX.T, kind)[0].T
    return op_scale(m, kind) * (PXQ + QXP)


# --------------------------------------------------------------------------
# Section 4.1: the DST diagonalisation
# --------------------------------------------------------------------------
def dst1_matrix(m: int) -> np.ndarray:
    """S[i, k] = sqrt(2/(m+1)) sin(pi i k/(m+1)), i, k = 1..m (Section 4.1).
    The product i*k is reduced modulo 2(m+1) in integers first (sine has period
    2 pi), so every argument lies in [0, 2 pi)."""
    N = m + 1
    k = np.arange(1, m + 1, dtype=np.int64)
    q = np.outer(k, k) % (2 * N)
    return math.sqrt(2.0 / N) * np.sin(np.pi * q.astype(np.float64) / N)


def dst1(X: np.ndarray) -> np.ndarray:
    """S X (columns transformed).  Dense definition for m <= DENSE_DST_MAX,
    otherwise scipy's orthonormal DST-I (a library FFT)."""
    X = np.asarray(X, dtype=np.float64)
    m = X.shape[0]
    if m <= DENSE_DST_MAX or _sfft is None:
        return dst1_matrix(m) @ X
    return _sfft.dst(X, type=1, norm="ortho", axis=0)


def dst1_entry(x: np.ndarray, k: int) -> float:
    """(S x)[k] for one 0-based frequency index k, by a direct sum."""
    m = x.shape[0]
    N = m + 1
    i = np.arange(1, m + 1, dtype=np.int64)
    q = (i * (k + 1)) % (2 * N)
    return float(math.sqrt(2.0 / N) * np.dot(np.sin(np.pi * q / N), x))


def eig_second_difference(m: int) -> np.ndarray:
    """lambda_k = 4 sin^2(k pi / (2(m+1))), k = 1..m: eigenvalues of T for the
    eigenvectors that are the columns of S."""
    k = np.arange(1, m + 1, dtype=np.float64)
    return 4.0 * np.sin(k * np.pi / (2.0 * (m + 1))) ** 2


def symbol(m: int, kind: str):
    """(a, b) with Lambda[i, j] = a_i b_j + b_i a_j, the diagonal of S A S in the
    Kronecker sense (Eq. flr:diagmat, Eq. flr:div)."""
    lam = eig_second_difference(m)
    h = 1.0 / (m + 1)
    if kind == "5pt":
        return lam / (h * h), np.ones(m)
    if kind == "semi":          # S (G G^T) S = diag(lam), S (H H^T) S = diag(4 - lam)
        # 4 - lam_k = 4 cos^2(k pi / (2(m+1))), the eigenvalues of H H^T =
        # tridiag(1, 2, 1), evaluated directly: the subtraction cancels for k
        # near m (relative error up to ~1e-10 at m = 2049)
        k = np.arange(1, m + 1, dtype=np.float64)
        return lam / (16.0 * h * h), 4.0 * np.cos(k * np.pi / (2.0 * (m + 1))) ** 2
    raise ValueError(kind)


def symbol_matrix(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return np.outer(a, b) + np.outer(b, a)


# --------------------------------------------------------------------------
# Full-format solves (the exact discrete solution)
# --------------------------------------------------------------------------
def solve_full(F: np.ndarray, kind: str) -> np.ndarray:
    """X* = S [ (S F S) / Lambda ] S, the textbook full-format solve of
    Eq. flr:diag (apply the DST, invert the diagonal, apply the DST back)."""
    m = F.shape[0]
    a, b = symbol(m, kind)
    Fh = dst1(dst1(F).T).T
    return dst1(dst1(Fh / symbol_matrix(a, b)).T).T


def solve_dense(F: np.ndarray, kind: str) -> np.ndarray:
    """Dense LU solve of (*) (numpy.linalg.solve on the assembled m^2 x m^2
    matrix).  Independent of the DST; m <= 32."""
    m = F.shape[0]
    A = dense_operator(m, kind)
    x = np.linalg.solve(A, F.reshape(-1, order="F"))
    return x.reshape((m, m), order="F")


# --------------------------------------------------------------------------
# Section 4.2: exact frequency-space entries and the cross
# --------------------------------------------------------------------------
def freq_row(Uh, Vh, a, b, i: int) -> np.ndarray:
    """Row i of Xh: (Uh[i] . Vh[j]) / (a_i b_j + b_i a_j) for all j.  O(m r)."""
    return (Vh @ Uh[i]) / (a[i] * b + b[i] * a)


def freq_col(Uh, Vh, a, b, j: int) -> np.ndarray:
    """Column j of Xh.  O(m r)."""
    return (Uh @ Vh[j]) / (a * b[j] + b * a[j])


def freq_entry(Uh, Vh, a, b, i: int, j: int) -> float:
    return float(np.dot(Uh[i], Vh[j]) / (a[i] * b[j] + b[i] * a[j]))


def splitmix64_stream(seed: int, count: int):
    """splitmix64 (Steele, Lea & Flood 2014), outputs 1..count from state seed."""
    mask = (1 << 64) - 1
    out = []
    z0 = seed & mask
    for t in range(1, count + 1):
        z = (z0 + t * 0x9E3779B97F4A7C15) & mask
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append(z ^ (z >> 31))
    return out


@dataclass
class CrossResult:
    C: np.ndarray            # m x k, column l = residual column / delta_l (C[I_l, l] = 1)
    R: np.ndarray            # m x k, column l = residual row / delta_l   (|R| <= 1)
    d: np.ndarray            # k pivot values delta_l
    I: list = field(default_factory=list)
    J: list = field(default_factory=list)
    norm2: float = 0.0       # ||S_k||_F^2 of the skeleton
    probe_rounds: int = 0
    zero_rows: int = 0
    converged: bool = True

    @property
    def k(self) -> int:
        return len(self.d)


def start_scores(Uh, a, b) -> np.ndarray:
    """Row score ||Uh[i]||^2 / Lambda[i, 0]^2 used to pick the first pivot row
    (and any row after an exactly-zero residual row): an upper-bound proxy for
    the size of row i of Xh."""
    lam0 = a * b[0] + b * a[0]
    return np.sum(Uh * Uh, axis=1) / (lam0 * lam0)


def _argmax_abs(v: np.ndarray, mask: np.ndarray) -> int:
    """Lowest index of the largest |v| among mask == True; -1 if none."""
    if not mask.any():
        return -1
    w = np.where(mask, np.abs(v), -1.0)
    return int(np.argmax(w))          # numpy returns the first maximum


def aca_cross(Uh, Vh, a, b, tol: float, rmax: int, probes: int = 16,
              seed: int = 0, max_probe_rounds: int = 4,
              max_zero_rows: int = 16) -> CrossResult:
    """Cross approximation of Xh (Section 4.2) by ACA with partial pivoting.

    Xh ~= sum_l delta_l C[:, l] R[:, l]^T, built one rank-1 term per step from
    one residual row and one residual column, each O(m (r + k)):

      1. row i* (first: largest start score), residual row
         rho_j = Xh[i*, j] - sum_l C[i*, l] delta_l R[j, l];
      2. j* = argmax over unused columns |rho_j| (lowest index on ties),
         delta = rho_{j*}.  If delta == 0 the row is already exact: mark it
         used, move to the best-scored unused row (at most max_zero_rows times);
      3. residual column c_i = (Xh[i, j*] - sum_l C[i, l] delta_l R[j*, l]) / delta,
         R[:, k] = rho / delta, C[:, k] = c;
      4. ||S_k||_F^2 += 2 sum_{l<k} delta_l delta_k (C_l.C_k)(R_l.R_k)
                        + delta_k^2 |C_k|^2 |R_k|^2;
      5. the term is small if |delta_k| |C_k| |R_k| <= tol ||S_k||_F; stop after
         two consecutive small terms, then probe ``probes`` entries drawn by
         splitmix64(seed); an entry whose residual exceeds tol ||S_k||_F restarts
         the loop at its row (at most max_probe_rounds times);
      6. otherwise the next row is argmax over unused rows |c_i|.
    The loop also ends at k = rmax (converged = False).
    """
    m = Uh.shape[0]
    Cs, Rs, ds, I, J = [], [], [], [], []
    used_r = np.zeros(m, bool)
    used_c = np.zeros(m, bool)
    score = start_scores(Uh, a, b)
    istar = _argmax_abs(score, ~used_r)
    norm2 = 0.0
    small = 0
    probe_rounds = 0
    zero_rows = 0
    converged = False
    gc_cols, gr_cols = [], []
    while len(ds) < rmax:
        k = len(ds)
        rho = freq_row(Uh, Vh, a, b, istar)
        for l in range(k):
            rho = rho - (Cs[l][istar] * ds[l]) * Rs[l]
        used_r[istar] = True
        jstar = _argmax_abs(rho, ~used_c)
        delta = rho[jstar] if jstar >= 0 else 0.0
        if delta == 0.0:
            zero_rows += 1
            nxt = _argmax_abs(score, ~used_r)
            if zero_rows > max_zero_rows or nxt < 0:
                converged = True
                break
            istar = nxt
            continue
        used_c[jstar] = True
        col = freq_col(Uh, Vh, a, b, jstar)
        for l in range(k):
            col = col - Cs[l] * (ds[l] * Rs[l][jstar])
        c = col / delta
        r = rho / delta
        gc = [float(np.dot(Cs[l], c)) for l in range(k)]
        gr = [float(np.dot(Rs[l], r)) for l in range(k)]
        cc, rr = float(np.dot(c, c)), float(np.dot(r, r))
        norm2 += 2.0 * sum(ds[l] * delta * gc[l] * gr[l] for l in range(k))
        norm2 += delta * delta * cc * rr
        Cs.append(c); Rs.append(r); ds.append(delta); I.append(istar); J.append(jstar)
        gc_cols.append(gc); gr_cols.append(gr)
        term = abs(delta) * math.sqrt(cc * rr)
        small = small + 1 if term <= tol * math.sqrt(max(norm2, 0.0)) else 0
        if small >= 2:
            if probe_rounds >= max_probe_rounds or probes <= 0:
                converged = True
                break
            zs = splitmix64_stream(seed + probe_rounds, probes)
            worst, worst_i = -1.0, -1
            for z in zs:
                pi, pj = (z >> 32) % m, (z & 0xFFFFFFFF) % m
                res = freq_entry(Uh, Vh, a, b, pi, pj)
                for l in range(len(ds)):
                    res -= Cs[l][pi] * ds[l] * Rs[l][pj]
                if abs(res) > worst:
                    worst, worst_i = abs(res), pi
            probe_rounds += 1
            if worst <= tol * math.sqrt(max(norm2, 0.0)):
                converged = True
                break
            small = 0
            istar = worst_i if not used_r[worst_i] else _argmax_abs(score, ~used_r)
            if istar < 0:
                converged = True
                break
            continue
        nxt = _argmax_abs(c, ~used_r)
        if nxt < 0:
            converged = True
            break
        istar = nxt
    k = len(ds)
    C = np.array(Cs).T if k else np.zeros((m, 0))
    R = np.array(Rs).T if k else np.zeros((m, 0))
    return CrossResult(C=C, R=R, d=np.array(ds), I=I, J=J, norm2=norm2,
                       probe_rounds=probe_rounds, zero_rows=zero_rows,
                       converged=converged)


# --------------------------------------------------------------------------
# Section 3: rounding (recompression) of a low-rank matrix
# --------------------------------------------------------------------------
def truncation_rank(s: np.ndarray, eps: float) -> int:
    """Smallest K with sqrt(sum_{i >= K} s_i^2) <= eps * ||s||_2 (s sorted
    descending); at least 1 when s has a nonzero entry."""
    s = np.asarray(s, dtype=np.float64)
    if s.size == 0 or s[0] == 0.0:
        return 0
    total = math.sqrt(float(np.sum(s * s)))
    tail2 = 0.0
    K = len(s)
    for i in range(len(s) - 1, 0, -1):
        t2 = tail2 + s[i] * s[i]
        if math.sqrt(t2) > eps * total:
            break
        tail2 = t2
        K = i
    return K


def lr_round(L: np.ndarray, d: np.ndarray, R: np.ndarray, eps: float, rmax: int):
    """Rounding of L diag(d) R^T (Section 3): QR of both factors, SVD of the
    k x k core, truncation at eps.  Returns (U, s, V, ok) with orthonormal U, V;
    ok is False if more than rmax singular values were needed (result cut)."""
    if L.shape[1] == 0:
        m1, m2 = L.shape[0], R.shape[0]
        return np.zeros((m1, 0)), np.zeros(0), np.zeros((m2, 0)), True
    ql, rl = np.linalg.qr(L)
    qr, rr = np.linalg.qr(R)
    w, s, zt = np.linalg.svd((rl * d) @ rr.T)
    K = truncation_rank(s, eps)
    ok = K <= rmax
    K = min(K, rmax)
    return ql @ w[:, :K], s[:K], qr @ zt[:K].T, ok


def svd_truncate(X: np.ndarray, eps: float):
    """Optimal (Eckart-Young) truncation of a full matrix at eps."""
    u, s, vt = np.linalg.svd(X, full_matrices=False)
    K = truncation_rank(s, eps)
    return u[:, :K], s[:K], vt[:K].T


@dataclass
class SolveInfo:
    cross: CrossResult
    rank: int
    ok: bool


def lr_poisson2d(U: np.ndarray, V: np.ndarray, kind: str, eps: float,
                 rmax: int = 128, aca_tol_factor: float = 1.0, probes: int = 16,
                 seed: int = 0):
    """Low-rank solve of A X = U V^T (Sections 4.1-4.2 then Section 3):
    Uh = S U, Vh = S V; cross approximation of Xh at tol = aca_tol_factor*eps;
    rounding at eps (orthogonal S commutes with the truncation, so it is done in
    frequency space); X = (S Uo) diag(s) (S Vo)^T.  Returns (Uo, s, Vo, info)."""
    m = U.shape[0]
    a, b = symbol(m, kind)
    Uh, Vh = dst1(U), dst1(V)
    cr = aca_cross(Uh, Vh, a, b, aca_tol_factor * eps, rmax, probes, seed)
    uo, s, vo, ok = lr_round(cr.C, cr.d, cr.R, eps, rmax)
    info = SolveInfo(cross=cr, rank=len(s), ok=ok and cr.converged)
    return dst1(uo), s, dst1(vo), info


def lr_truncate(U: np.ndarray, s, V: np.ndarray, eps: float, rmax: int):
    """Rounding of U diag(s) V^T (s None means all ones), Section 3."""
    d = np.ones(U.shape[1]) if s is None else np.asarray(s, dtype=np.float64)
    uo, so, vo, ok = lr_round(U, d, V, eps, rmax)
    return uo, so, vo, ok


# --------------------------------------------------------------------------
# Exact error and residual evaluation at any m
# --------------------------------------------------------------------------
def rel_error_freq(Uo, s, Vo, U, V, kind: str, rows=None, block: int = 512):
    """Relative Frobenius error ||X - X*|| / ||X*|| of X = Uo diag(s) Vo^T
    against the exact discrete solution X* of A X* = U V^T.  S is orthogonal,
    so the error is evaluated in frequency space entry by entry (Parseval) and
    no m x m spatial grid is formed.  ``rows`` restricts to a row sample."""
    m = U.shape[0]
    a, b = symbol(m, kind)
    Uh, Vh = dst1(U), dst1(V)
    Uoh, Voh = dst1(Uo) * np.asarray(s)[None, :], dst1(Vo)
    idx = np.arange(m) if rows is None else np.asarray(rows)
    e2 = x2 = 0.0
    for p in range(0, len(idx), block):
        ii = idx[p:p + block]
        lam = np.outer(a[ii], b) + np.outer(b[ii], a)
        xs = (Uh[ii] @ Vh.T) / lam
        xa = Uoh[ii] @ Voh.T
        e2 += float(np.sum((xs - xa) ** 2))
        x2 += float(np.sum(xs * xs))
    return math.sqrt(e2 / x2) if x2 > 0 else math.sqrt(e2)


def lowrank_residual(Uo, s, Vo, U, V, kind: str) -> float:
    """||A X - F||_F / ||F||_F for X = Uo diag(s) Vo^T, F = U V^T, exact at any
    m: A X - F = [c P Uo s, c Q Uo s, -U] [Q Vo, P Vo, V]^T is low rank, and its
    Frobenius norm is that of the product of the two QR triangles."""
    m = U.shape[0]
    c = op_scale(m, kind)
    Us = Uo * np.asarray(s)[None, :]
    PU, QU = apply_parts(Us, kind)
    PV, QV = apply_parts(Vo, kind)
    L = np.hstack([c * PU, c * QU, -U])
    R = np.hstack([QV, PV, V])
    _, rl = np.linalg.qr(L)
    _, rr = np.linalg.qr(R)
    _, ru = np.linalg.qr(U)
    _, rv = np.linalg.qr(V)
    return float(np.linalg.norm(rl @ rr.T) / np.linalg.norm(ru @ rv.T))
