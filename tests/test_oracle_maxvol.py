"""Pins of the maxvol oracle (the row selection Section 4.2 cites for the
cross) against facts it does not compute itself: the closed form at k = 1,
the definition of a dominant submatrix checked by a fresh solve, Cramer's
rule for the volume gained by each swap, Hadamard's bound against brute force
over every k-subset of a tiny matrix, and invariance under a change of basis
of the columns.  CPU only.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import maxvol as M


def _gauss(m, k, seed):
    return np.random.default_rng(seed).standard_normal((m, k))


def test_k1_picks_the_largest_entry():
    # k = 1: B = c / c[start], so maxvol with delta = 0 moves to argmax |c|.
    c = np.array([[0.5], [-3.0], [2.0], [2.9], [-0.1]])
    for start in range(5):
        rows, nswaps, bmax = M.maxvol(c, [start], 0.0, 10)
        assert rows == [1]
        assert nswaps == (0 if start == 1 else 1)
        assert bmax == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("m,k,delta,seed", [(50, 4, 0.0, 1), (300, 10, 1e-2, 2), (1000, 32, 5e-2, 3)])
def test_result_is_dominant_by_a_fresh_solve(m, k, delta, seed):
    C = _gauss(m, k, seed)
    rows, nswaps, bmax = M.maxvol(C, list(range(k)), delta, 10 * k)
    B = M.coefficients(C, rows)  # fresh solve, not the rank-1 updates
    assert np.abs(B).max() <= 1.0 + delta + 1e-10
    assert np.abs(B).max() == pytest.approx(bmax, rel=1e-9)
    assert np.allclose(B[rows, :], np.eye(k), atol=1e-12)
    assert nswaps > 0


def test_each_swap_multiplies_the_volume_by_the_removed_coefficient():
    # Cramer: replacing row I[j] by row i scales det C[I, :] by B[i, j].
    C = _gauss(200, 6, 7)
    rows0 = [3, 17, 40, 41, 99, 150]
    rows, nswaps, _, log = M.maxvol(C, rows0, 0.0, 50, trace=True)
    assert len(log) == nswaps + 1
    cur = list(rows0)
    for i, j, big, _, _ in log[:-1]:
        before = abs(np.linalg.det(C[cur, :]))
        cur[j] = i
        after = abs(np.linalg.det(C[cur, :]))
        assert after / before == pytest.approx(big, rel=1e-9)
        assert big > 1.0
    assert cur == rows


@pytest.mark.parametrize("delta", [0.0, 0.05, 0.5])
@pytest.mark.parametrize("seed", [11, 12, 13, 14])
def test_volume_within_hadamard_bound_of_brute_force(delta, seed):
    m, k = 9, 3
    C = _gauss(m, k, seed)
    vmax = max(abs(np.linalg.det(C[list(s), :])) for s in itertools.combinations(range(m), k))
    start = [0, 1, 2]
    rows, _, _ = M.maxvol(C, start, delta, 100)
    v = abs(np.linalg.det(C[rows, :]))
    assert v >= abs(np.linalg.det(C[start, :])) * (1 - 1e-12)
    assert vmax <= ((1.0 + delta) * math.sqrt(k)) ** k * v * (1 + 1e-12)


def test_identity_block_special_cases():
    k = 4
    G = np.random.default_rng(5).uniform(-0.2, 0.2, (20, k))
    C = np.vstack([np.eye(k), G])
    rows, nswaps, bmax = M.maxvol(C, list(range(k)), 0.0, 10)
    assert rows == list(range(k)) and nswaps == 0 and bmax == 1.0
    # one coefficient of 3 in row k + 2, column 1: one swap puts that row at
    # position 1, after which every coefficient is below 1 (|G| <= 0.2, so the
    # update changes none by more than 0.2 * 1.2 / 3).
    C[k + 2, 1] = 3.0
    rows, nswaps, _, log = M.maxvol(C, list(range(k)), 0.0, 10, trace=True)
    assert log[0][:3] == (k + 2, 1, 3.0)
    assert rows == [0, k + 2, 2, 3] and nswaps == 1


def test_change_of_column_basis_keeps_the_rows():
    # B = C C[I]^{-1} depends on the column space of C only.
    C = _gauss(500, 8, 21)
    T = np.random.default_rng(22).standard_normal((8, 8)) + 4 * np.eye(8)
    r1, n1, b1 = M.maxvol(C, list(range(8)), 1e-2, 100)
    r2, n2, b2 = M.maxvol(C @ T, list(range(8)), 1e-2, 100)
    assert r1 == r2 and n1 == n2
    assert b1 == pytest.approx(b2, rel=1e-9)


def test_swap_cap_and_argument_checks():
    C = _gauss(100, 5, 31)
    rows, nswaps, bmax = M.maxvol(C, list(range(5)), 0.0, 0)
    assert rows == list(range(5)) and nswaps == 0
    assert bmax == pytest.approx(np.abs(M.coefficients(C, range(5))).max(), rel=1e-12)
    assert bmax > 1.0
    with pytest.raises(ValueError):
        M.maxvol(C, [0, 1, 2, 3, 3], 0.0, 10)
    with pytest.raises(ValueError):
        M.maxvol(C, [0, 1, 2, 3, 100], 0.0, 10)


# ---- maxvol-refined pivots of the cross (restricted cross, alternating maxvol)
from oracle import poisson_lowrank as O  # noqa: E402
from paper_1306_2150_gb300 import inputs  # noqa: E402


def _freq_problem(m, r, seed):
    U, V = inputs.separable_random(m, r, seed)
    a, b = O.symbol(m, "5pt")
    Uh, Vh = O.dst1(U), O.dst1(V)
    Xh = np.stack([O.freq_row(Uh, Vh, a, b, i) for i in range(m)])
    return Uh, Vh, a, b, Xh


def _skeleton(cr):
    return (cr.C * cr.d) @ cr.R.T


def test_restricted_cross_is_the_cur_interpolant():
    Uh, Vh, a, b, Xh = _freq_problem(40, 5, 3)
    rng = np.random.default_rng(4)
    I = list(rng.choice(40, 6, replace=False))
    J = list(rng.choice(40, 6, replace=False))
    cr = M.restricted_cross(Uh, Vh, a, b, I, J)
    S = _skeleton(cr)
    cur = Xh[:, J] @ np.linalg.solve(Xh[np.ix_(I, J)], Xh[I, :])
    assert np.linalg.norm(S - cur) <= 1e-9 * np.linalg.norm(cur)
    assert np.allclose(S[I, :], Xh[I, :], rtol=0, atol=1e-12 * np.abs(Xh).max())
    assert np.allclose(S[:, J], Xh[:, J], rtol=0, atol=1e-12 * np.abs(Xh).max())
    assert sorted(cr.I) == sorted(I) and sorted(cr.J) == sorted(J)


def test_restricted_cross_on_the_aca_pivots_gives_the_aca_skeleton():
    Uh, Vh, a, b, Xh = _freq_problem(64, 6, 5)
    aca = O.aca_cross(Uh, Vh, a, b, 1e-8, 64)
    cr = M.restricted_cross(Uh, Vh, a, b, aca.I, aca.J)
    S0, S1 = _skeleton(aca), _skeleton(cr)
    assert np.linalg.norm(S1 - S0) <= 1e-9 * np.linalg.norm(S0)


def test_restricted_cross_rejects_a_singular_block():
    Uh, Vh, a, b, _ = _freq_problem(30, 4, 6)
    Uh = Uh.copy()
    Uh[7] = 0.0  # row 7 of Xh is zero
    with pytest.raises(ValueError):
        M.restricted_cross(Uh, Vh, a, b, [7, 1, 2], [0, 1, 2])


def test_refined_pivots_are_dominant_both_ways():
    Uh, Vh, a, b, Xh = _freq_problem(200, 6, 7)
    aca = O.aca_cross(Uh, Vh, a, b, 1e-10, 64)
    I, J, swaps, q = M.refine_pivots(Uh, Vh, a, b, aca.I, aca.J, 1e-2, 400, rounds=8)
    assert q < 8  # the last round made no swap
    assert np.abs(M.coefficients(Xh[:, J], I)).max() <= 1.01 + 1e-9
    assert np.abs(M.coefficients(Xh[I, :].T, J)).max() <= 1.01 + 1e-9
    v0 = abs(np.linalg.det(Xh[np.ix_(aca.I, aca.J)]))
    assert abs(np.linalg.det(Xh[np.ix_(I, J)])) >= v0 * (1 - 1e-12)


@pytest.mark.parametrize("case", ["config0", "smooth1024"])
def test_solve_with_refined_pivots(case):
    if case == "config0":
        U, V = inputs.separable_random(256, 8, 0)
        eps = 1e-10
    else:
        U, V = inputs.smooth_sum(1024, 1e-6)
        eps = 1e-6
    Uo, so, Vo, _ = O.lr_poisson2d(U, V, "5pt", eps)
    Um, sm, Vm, (cr, cr2, swaps, q) = M.lr_poisson2d_maxvol(U, V, "5pt", eps)
    assert swaps > 0 and cr2.k == cr.k
    assert len(sm) <= len(so)
    assert O.rel_error_freq(Um, sm, Vm, U, V, "5pt") <= 10 * eps
