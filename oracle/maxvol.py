"""Plain FP64 CPU oracle for the maxvol row selection that Section 4.2 names as
the quasi-optimal way to choose the rows and columns of the cross (the
maxvol algorithm of Goreinov, Oseledets, Savostyanov, Tyrtyshnikov and
Zamarashkin, "How to find a good submatrix", 2010, which the paper cites).

TEST INFRASTRUCTURE ONLY: imported by tests/ and never by the CUDA library.

Given a tall matrix C (m x k, full column rank) and k distinct rows I with
C[I, :] nonsingular, the coefficients of every row of C in the basis of the
rows I are

    B = C C[I, :]^{-1}          (m x k, B[I, :] = identity).

B[I, :] is the identity by this definition and is stored as the exact
identity (a solve would give it only up to rounding, and a rounded 1 + 2^-52
would look like a coefficient above 1 at delta = 0).

If some |B[i, j]| > 1 + delta, putting row i in place of I[j] multiplies
|det C[I, :]| by |B[i, j]| (Cramer: row i = sum_l B[i, l] C[I[l], :]), and
the coefficients of the new basis follow from the old by a rank-1 update
(Sherman-Morrison on C[I', :] = (identity + e_j (B[i, :] - e_j^T)) C[I, :]):

    B' = B - B[:, j] (B[i, :] - e_j^T) / B[i, j].

The algorithm takes the largest |B[i, j]| each time (lowest column-major
index j m + i on ties) and stops once it is <= 1 + delta: then C[I, :] is a
(1 + delta)-dominant submatrix, whose volume is within ((1 + delta) sqrt(k))^k
of the largest (Hadamard's inequality on B[I_max, :]).
"""
from __future__ import annotations

import numpy as np


def coefficients(C: np.ndarray, rows) -> np.ndarray:
    """B = C C[rows, :]^{-1}, by one dense solve of C[rows, :]^T B^T = C^T."""
    A = C[np.asarray(rows, dtype=np.int64), :]
    return np.linalg.solve(A.T, C.T).T


def _largest(B: np.ndarray):
    """(i, j, |B[i, j]|) of the largest |B| entry, lowest j m + i on ties."""
    flat = np.abs(B).ravel(order="F")
    q = int(np.argmax(flat))
    m = B.shape[0]
    return q % m, q // m, float(flat[q])


def maxvol(C: np.ndarray, rows, delta: float, maxswaps: int, trace: bool = False):
    """Maxvol refinement of the rows ``rows`` of C (m x k, float64).

    Returns (rows, nswaps, bmax): the refined rows (position j holds the row
    whose coefficient vector is e_j), the swaps made and the final largest
    |B| (<= 1 + delta unless maxswaps ran out).  With ``trace`` also a list
    with one (i, j, largest, second largest, largest outside the selected
    rows) per decision, the last one the decision to stop, so a test can see
    how far each decision was from a tie.
    """
    C = np.asarray(C, dtype=np.float64)
    m, k = C.shape
    rows = [int(r) for r in rows]
    if len(rows) != k or len(set(rows)) != k or min(rows) < 0 or max(rows) >= m:
        raise ValueError("rows must be k distinct indices in [0, m)")
    B = coefficients(C, rows)
    B[rows, :] = np.eye(k)
    nswaps = 0
    log = []
    while True:
        i, j, big = _largest(B)
        if trace:
            absb = np.abs(B)
            top2 = np.partition(absb.ravel(), -2)[-2:] if B.size > 1 else np.zeros(2)
            out = np.delete(absb, rows, axis=0)
            log.append((i, j, big, float(top2[0]),
                        float(out.max()) if out.size else 0.0))
        if not big > 1.0 + delta or nswaps >= maxswaps:
            break
        piv = B[i, j]
        r = B[i, :].copy()
        r[j] -= 1.0
        f = B[:, j] / piv
        B = B - np.outer(f, r)
        B[i, :] = 0.0
        B[i, j] = 1.0
        rows[j] = i
        nswaps += 1
    if trace:
        return rows, nswaps, big, log
    return rows, nswaps, big


# --------------------------------------------------------------------------
# Maxvol-refined pivots for the cross of Section 4.2 (the optional refinement
# of the ACA's pivots): alternate maxvol on the columns Xh[:, J] (rows I) and
# on the rows Xh[I, :] (columns J), then rebuild the skeleton on the refined
# index sets and round it as the plain solve does.
# --------------------------------------------------------------------------
def restricted_cross(Uh, Vh, a, b, I, J):
    """Cross of Xh on the rows I and columns J only (|I| = |J| = k): ACA with
    partial pivoting whose candidates are restricted to I and J, run for k
    steps, i.e. Gaussian elimination with partial pivoting on Xh[I, J].  Start
    row: the row of I with the largest start score (as the plain cross); each
    column: argmax over the unused columns of J of the residual row; each next
    row: argmax over the unused rows of I of the residual column (lowest index
    on ties).  After k steps the skeleton interpolates Xh on the rows I and the
    columns J:  sum_l d_l C_l R_l^T = Xh[:, J] Xh[I, J]^{-1} Xh[I, :].
    Raises ValueError if Xh[I, J] is singular (a zero residual pivot)."""
    from . import poisson_lowrank as P
    m = Uh.shape[0]
    I, J = [int(i) for i in I], [int(j) for j in J]
    k = len(I)
    if len(J) != k or len(set(I)) != k or len(set(J)) != k:
        raise ValueError("I and J must hold k distinct indices each")
    allow_r = np.zeros(m, bool)
    allow_r[I] = True
    allow_c = np.zeros(m, bool)
    allow_c[J] = True
    Cs, Rs, ds, Io, Jo = [], [], [], [], []
    istar = P._argmax_abs(P.start_scores(Uh, a, b), allow_r)
    for step in range(k):
        rho = P.freq_row(Uh, Vh, a, b, istar)
        for l in range(step):
            rho = rho - (Cs[l][istar] * ds[l]) * Rs[l]
        allow_r[istar] = False
        jstar = P._argmax_abs(rho, allow_c)
        delta = rho[jstar]
        if delta == 0.0:
            raise ValueError("Xh[I, J] is singular")
        allow_c[jstar] = False
        col = P.freq_col(Uh, Vh, a, b, jstar)
        for l in range(step):
            col = col - Cs[l] * (ds[l] * Rs[l][jstar])
        Cs.append(col / delta)
        Rs.append(rho / delta)
        ds.append(delta)
        Io.append(istar)
        Jo.append(jstar)
        if step < k - 1:
            istar = P._argmax_abs(Cs[-1], allow_r)
    C = np.array(Cs).T if k else np.zeros((m, 0))
    R = np.array(Rs).T if k else np.zeros((m, 0))
    return P.CrossResult(C=C, R=R, d=np.array(ds), I=Io, J=Jo, converged=True)


def refine_pivots(Uh, Vh, a, b, I, J, delta: float, maxswaps: int, rounds: int = 4):
    """Alternating maxvol: the rows I on the columns Xh[:, J], then the
    columns J on the rows Xh[I, :] (as columns of Xh[I, :]^T), until a round
    makes no swap or ``rounds`` rounds ran.  Returns (I, J, swaps, rounds run);
    after a round without swaps Xh[I, J] is (1 + delta)-dominant in both
    Xh[:, J] and Xh[I, :]^T."""
    from . import poisson_lowrank as P
    I, J = [int(i) for i in I], [int(j) for j in J]
    total = 0
    q = 0
    while q < rounds:
        q += 1
        CJ = np.stack([P.freq_col(Uh, Vh, a, b, j) for j in J], axis=1)
        I, s1, _ = maxvol(CJ, I, delta, maxswaps)
        RI = np.stack([P.freq_row(Uh, Vh, a, b, i) for i in I], axis=1)
        J, s2, _ = maxvol(RI, J, delta, maxswaps)
        total += s1 + s2
        if s1 + s2 == 0:
            break
    return I, J, total, q


def lr_poisson2d_maxvol(U, V, kind: str, eps: float, delta: float = 1e-2, rmax: int = 128,
                        rounds: int = 4, probes: int = 16, seed: int = 0):
    """The low-rank solve of ``poisson_lowrank.lr_poisson2d`` with maxvol-refined
    pivots: the ACA picks the rank k and the first pivots, ``refine_pivots``
    improves them, ``restricted_cross`` rebuilds the skeleton on the refined
    pivots, and the rounding at eps follows as before.  Returns
    (Uo, s, Vo, info) with info = (aca cross, refined cross, swaps, rounds)."""
    from . import poisson_lowrank as P
    m = U.shape[0]
    a, b = P.symbol(m, kind)
    Uh, Vh = P.dst1(U), P.dst1(V)
    cr = P.aca_cross(Uh, Vh, a, b, eps, rmax, probes, seed)
    if cr.k == 0:
        uo, s, vo, _ = P.lr_round(cr.C, cr.d, cr.R, eps, rmax)
        return P.dst1(uo), s, P.dst1(vo), (cr, cr, 0, 0)
    I, J, swaps, q = refine_pivots(Uh, Vh, a, b, cr.I, cr.J, delta, 16 * cr.k, rounds)
    cr2 = restricted_cross(Uh, Vh, a, b, I, J)
    uo, s, vo, _ = P.lr_round(cr2.C, cr2.d, cr2.R, eps, rmax)
    return P.dst1(uo), s, P.dst1(vo), (cr, cr2, swaps, q)
