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
