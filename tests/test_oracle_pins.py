"""Pins of the CPU oracle against facts it does not compute itself.

Each test ties one oracle function to something fixed outside it: a hand
solution (tests/golden), a closed form, a library routine, an invariant of the
method, or brute force on a tiny case.  CPU only.
"""
import math
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

from oracle import poisson_lowrank as O
from paper_1306_2150_gb300 import inputs

GOLDEN = Path(__file__).parent / "golden"


def _read_golden_solves():
    out = []
    lines = [l for l in (GOLDEN / "small_solves.txt").read_text().splitlines()
             if l.strip() and not l.startswith("#")]
    p = 0
    while p < len(lines):
        kind, m = lines[p].split()
        m = int(m)
        rows = [[float(Fraction(t)) for t in lines[p + 1 + i].split()] for i in range(m)]
        out.append((kind, m, np.array(rows)))
        p += 1 + m
    return out


# ---------------------------------------------------------------- generator
def test_splitmix64_published_first_output():
    # splitmix64 from state 0: first output 0xE220A8397B1DCDAF (Steele et al.)
    assert int(inputs.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF
    assert O.splitmix64_stream(0, 1)[0] == 0xE220A8397B1DCDAF
    a = [int(z) for z in inputs.splitmix64(12345, 5)]
    assert a == O.splitmix64_stream(12345, 5)


def test_separable_random_is_the_stated_recipe():
    U, V = inputs.separable_random(16, 3, seed=7)
    assert U.flags.f_contiguous and V.flags.f_contiguous
    u = inputs.uniform01(7, 9).reshape(3, 3) * 4
    x = np.arange(1, 17) / 17
    assert np.allclose(U[:, 1], np.cos(u[1, 0] * x + u[1, 1]), rtol=0, atol=1e-15)
    assert np.all(u >= 0) and np.all(u < 4)


def test_smooth_sum_compression_tolerance():
    for tol in (1e-6, 1e-10):
        U, V = inputs.smooth_sum(200, tol)
        F = inputs.smooth_sum_dense(200)
        err = np.linalg.norm(U @ V.T - F) / np.linalg.norm(F)
        assert err <= 1.01 * tol + 1e-12


# ---------------------------------------------------------------- Section 4.1
@pytest.mark.parametrize("m", [1, 2, 7, 64])
def test_dst_orthonormal_symmetric(m):
    S = O.dst1_matrix(m)
    assert np.allclose(S, S.T, atol=0)
    assert np.abs(S @ S - np.eye(m)).max() < 1e-14


@pytest.mark.parametrize("kind", O.KINDS)
@pytest.mark.parametrize("m", [3, 10, 33])
def test_dst_diagonalises_operator_parts(kind, m):
    # P, Q built from G, H (Section 2) / T; S P S and S Q S must be diagonal with
    # the oracle's symbol, whose sorted values must equal LAPACK's eigenvalues.
    P, Q, scale = O.operator_parts(m, kind)
    S = O.dst1_matrix(m)
    DP, DQ = S @ P @ S, S @ Q @ S
    assert np.abs(DP - np.diag(np.diag(DP))).max() < 1e-12
    assert np.abs(DQ - np.diag(np.diag(DQ))).max() < 1e-12
    a, b = O.symbol(m, kind)
    lam = np.diag(DP) * scale
    lam_q = np.diag(DQ)
    if kind == "5pt":
        assert np.allclose(a, lam, rtol=1e-13, atol=0)
        assert np.allclose(b, lam_q, rtol=0, atol=1e-13)
    else:
        assert np.allclose(a, lam, rtol=1e-12, atol=0)
        assert np.allclose(b, lam_q, rtol=1e-12, atol=1e-13)
    assert np.allclose(np.sort(np.diag(DP)), np.linalg.eigvalsh(P), atol=1e-12)


def test_symbol_closed_form_golden():
    env = {"sqrt": math.sqrt}
    lam_expected = []
    for line in (GOLDEN / "symbol_m4.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            k, expr = line.split(maxsplit=1)
            lam_expected.append(eval(expr, {"__builtins__": {}}, env))
    lam = O.eig_second_difference(4)
    assert np.allclose(lam, lam_expected, rtol=0, atol=2e-15)
    a, b = O.symbol(4, "semi")
    assert np.allclose(b, 4 - np.array(lam_expected), atol=1e-15)
    a5, b5 = O.symbol(4, "5pt")
    assert np.allclose(a5, 25 * np.array(lam_expected), rtol=1e-15)


@pytest.mark.parametrize("m", [5, 100, 1000])
def test_dense_dst_matches_library_fft(m):
    scipy_fft = pytest.importorskip("scipy.fft")
    X = np.random.default_rng(m).standard_normal((m, 3))
    ref = scipy_fft.dst(X, type=1, norm="ortho", axis=0)
    assert np.abs(O.dst1_matrix(m) @ X - ref).max() < 1e-13 * np.abs(ref).max() * math.sqrt(m)


def test_large_dst_path_matches_direct_sums():
    pytest.importorskip("scipy.fft")
    m = O.DENSE_DST_MAX + 905
    x = np.random.default_rng(1).standard_normal(m)
    y = O.dst1(x[:, None])[:, 0]
    for k in (0, 1, 17, m // 2, m - 1):
        assert abs(y[k] - O.dst1_entry(x, k)) < 1e-12 * np.linalg.norm(x)


# ---------------------------------------------------------------- solves
@pytest.mark.parametrize("kind,m,X", _read_golden_solves())
def test_hand_solved_golden(kind, m, X):
    F = np.ones((m, m))
    assert np.allclose(O.solve_full(F, kind), X, rtol=1e-14, atol=0)
    assert np.allclose(O.solve_dense(F, kind), X, rtol=1e-14, atol=0)


@pytest.mark.parametrize("kind", O.KINDS)
@pytest.mark.parametrize("m", [4, 9, 16, 32])
def test_full_solve_matches_dense_lu(kind, m):
    F = np.random.default_rng(m).standard_normal((m, m))
    Xd = O.solve_dense(F, kind)
    Xf = O.solve_full(F, kind)
    assert np.linalg.norm(Xf - Xd) <= 1e-12 * np.linalg.norm(Xd)


@pytest.mark.parametrize("kind", O.KINDS)
def test_stencil_matches_assembled_operator(kind):
    m = 8
    X = np.random.default_rng(3).standard_normal((m, m))
    A = O.dense_operator(m, kind)
    assert np.allclose(O.apply_operator(X, kind).reshape(-1, order="F"),
                       A @ X.reshape(-1, order="F"), rtol=1e-13, atol=1e-10)


@pytest.mark.parametrize("kind", O.KINDS)
def test_full_solve_residual(kind):
    m = 96
    F = np.random.default_rng(5).standard_normal((m, m))
    X = O.solve_full(F, kind)
    assert np.linalg.norm(O.apply_operator(X, kind) - F) <= 1e-11 * np.linalg.norm(F)


@pytest.mark.parametrize("kind", O.KINDS)
@pytest.mark.parametrize("kl", [(1, 1), (2, 5), (7, 3)])
def test_eigenfunction_solution(kind, kl):
    # F = sin(k pi x) sin(l pi y) is an eigenfunction of the discrete operator;
    # its eigenvalue is read off the stencil (A F / F), not from the symbol code.
    m = 40
    k, l = kl
    x = np.arange(1, m + 1) / (m + 1)
    u, v = np.sin(k * np.pi * x), np.sin(l * np.pi * x)
    F = np.outer(u, v)
    AF = O.apply_operator(F, kind)
    ev = (AF[m // 3, m // 4] / F[m // 3, m // 4])
    assert np.allclose(AF, ev * F, rtol=1e-10, atol=1e-10 * abs(ev))
    X = O.solve_full(F, kind)
    assert np.allclose(X, F / ev, rtol=1e-12, atol=1e-14 / abs(ev))
    # the low-rank solve recovers the rank-1 solution
    Uo, s, Vo, info = O.lr_poisson2d(u[:, None], v[:, None], kind, 1e-10)
    assert info.rank == 1
    Xl = (Uo * s) @ Vo.T
    assert np.linalg.norm(Xl - F / ev) <= 1e-12 * np.linalg.norm(F / ev)


# ---------------------------------------------------------------- cross
def test_cross_recovers_exact_rank_matrix():
    # a = 1/2, b = 1 makes Lambda == 1, so Xh = Uh Vh^T has rank exactly r.
    m, r = 300, 6
    rng = np.random.default_rng(11)
    Uh, Vh = rng.standard_normal((m, r)), rng.standard_normal((m, r))
    a, b = np.full(m, 0.5), np.ones(m)
    cr = O.aca_cross(Uh, Vh, a, b, 1e-12, 64)
    X = Uh @ Vh.T
    Xa = (cr.C * cr.d) @ cr.R.T
    assert cr.converged
    assert cr.k <= r + 2
    assert np.linalg.norm(X - Xa) <= 1e-12 * np.linalg.norm(X)


def test_cross_interpolates_on_its_crosses():
    # ACA skeleton equals Xh on every chosen row I and column J, C[I_l, l] = 1,
    # R[J_l, l] = 1 and |R| <= 1 (partial pivoting on rows).
    m = 48
    U, V = inputs.separable_random(m, 4, seed=2)
    a, b = O.symbol(m, "5pt")
    Uh, Vh = O.dst1(U), O.dst1(V)
    Xh = (Uh @ Vh.T) / O.symbol_matrix(a, b)
    cr = O.aca_cross(Uh, Vh, a, b, 1e-9, 64)
    Xa = (cr.C * cr.d) @ cr.R.T
    sc = np.abs(Xh).max()
    assert np.abs(Xa[cr.I, :] - Xh[cr.I, :]).max() <= 1e-13 * sc
    assert np.abs(Xa[:, cr.J] - Xh[:, cr.J]).max() <= 1e-13 * sc
    for l, (i, j) in enumerate(zip(cr.I, cr.J)):
        # c_{i_l} = 1 up to rounding of entries of size sc, seen through delta_l
        assert abs(cr.C[i, l] - 1) * abs(cr.d[l]) <= 1e-13 * sc
        assert abs(cr.R[j, l] - 1) < 1e-14
    assert np.abs(cr.R).max() <= 1 + 1e-14
    assert len(set(cr.I)) == cr.k and len(set(cr.J)) == cr.k


def test_cross_brute_force_small():
    # At m = 14 the whole Xh is formed by brute force; the cross must reach the
    # requested relative Frobenius tolerance, and its norm estimate must be the
    # skeleton's true Frobenius norm.
    m = 14
    U, V = inputs.separable_random(m, 5, seed=4)
    for kind in O.KINDS:
        a, b = O.symbol(m, kind)
        Uh, Vh = O.dst1(U), O.dst1(V)
        Xh = (Uh @ Vh.T) / O.symbol_matrix(a, b)
        cr = O.aca_cross(Uh, Vh, a, b, 1e-8, 64)
        Xa = (cr.C * cr.d) @ cr.R.T
        assert np.linalg.norm(Xh - Xa) <= 1e-7 * np.linalg.norm(Xh)
        assert math.isclose(math.sqrt(cr.norm2), np.linalg.norm(Xa), rel_tol=1e-10)


def test_cross_zero_first_row_moves_on():
    # An eigenfunction with frequency 3 in x: only row 2 of Uh is nonzero, so
    # rows with zero residual must be skipped, not stop the cross.
    m = 30
    x = np.arange(1, m + 1) / (m + 1)
    u = np.sin(3 * np.pi * x)[:, None]
    v = (np.sin(np.pi * x) + 0.3 * np.sin(2 * np.pi * x))[:, None]
    Uo, s, Vo, info = O.lr_poisson2d(u, v, "5pt", 1e-12)
    assert info.cross.I[0] == 2
    assert O.rel_error_freq(Uo, s, Vo, u, v, "5pt") < 1e-13



@pytest.mark.parametrize("kind", O.KINDS)
@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_cross_probe_restart_finds_untouched_block(kind, tol):
    # Section 4.2's cross with the residual probes of the stop rule (reading
    # G7) on a block-diagonal Xh: block A (rows and columns < split, the low
    # frequencies where the cross starts) and block B.  Partial pivoting in A
    # never sees B (its residual rows and columns are exactly zero there), so
    # the first converged skeleton covers block A only; a probe lands in
    # block B, whose residual is the full entry, and the loop restarts at that
    # probe's row.  Pinned by brute force on the whole Xh: the result reaches
    # the tolerance only because of the restart, and the restart row is the
    # row of the largest probed residual of the first round.
    m, split = 128, 32
    a, b = O.symbol(m, kind)
    Uh, Vh = inputs.block_diagonal_freq(m, split)
    Xh = (Uh @ Vh.T) / O.symbol_matrix(a, b)
    cr = O.aca_cross(Uh, Vh, a, b, tol, 64, probes=16, seed=0)
    Xa = (cr.C * cr.d) @ cr.R.T
    assert cr.converged and cr.probe_rounds == 2
    assert np.linalg.norm(Xh - Xa) <= tol * np.linalg.norm(Xh)
    # the steps before the restart stay in block A, the restart row is in B
    k1 = next(l for l, i in enumerate(cr.I) if i >= split)
    assert k1 >= 2 and all(i < split and j < split for i, j in zip(cr.I[:k1], cr.J[:k1]))
    # brute force: residual of the first skeleton at the 16 probed entries
    X1 = (cr.C[:, :k1] * cr.d[:k1]) @ cr.R[:, :k1].T
    n1 = np.linalg.norm(X1)
    best, best_row = -1.0, -1
    for z in O.splitmix64_stream(0, 16):
        pi, pj = (z >> 32) % m, (z & 0xFFFFFFFF) % m
        res = abs(Xh[pi, pj] - X1[pi, pj])
        if res > best:
            best, best_row = res, pi
    assert best > tol * n1            # the first round fails ...
    assert cr.I[k1] == best_row       # ... and restarts at the worst probe's row
    # without probes the cross stops after block A: the error is block B's size
    cr0 = O.aca_cross(Uh, Vh, a, b, tol, 64, probes=0)
    X0 = (cr0.C * cr0.d) @ cr0.R.T
    eB = np.linalg.norm(Xh[split:, split:]) / np.linalg.norm(Xh)
    assert max(cr0.I) < split and cr0.probe_rounds == 0
    assert np.linalg.norm(Xh - X0) / np.linalg.norm(Xh) == pytest.approx(eB, rel=1e-6)
    assert eB > 1e3 * tol



@pytest.mark.parametrize("factor,restarts", [(2.0, True), (0.5, False)])
def test_cross_probe_threshold_is_tol_times_skeleton_norm(factor, restarts):
    # The probe test compares |residual| with tol ||S_k||_F (reading G7).
    # Block A is scaled so that ||S_k||_F is far from 1 (a threshold on
    # ||S_k||^2 or without the norm would move by orders of magnitude); block
    # B is scaled so that its largest probed entry (restart expected) or its
    # largest entry anywhere (no restart) is `factor` times the threshold.
    m, split, tol = 128, 32, 1e-6
    a, b = O.symbol(m, "5pt")
    Uh, Vh = inputs.block_diagonal_freq(m, split)
    Uh[:, 0] *= 1e4
    lam = O.symbol_matrix(a, b)
    XA = np.outer(Uh[:, 0], Vh[:, 0]) / lam
    XB = np.outer(Uh[:, 1], Vh[:, 1]) / lam
    nA = np.linalg.norm(XA)
    assert nA > 1e2
    probed = [((z >> 32) % m, (z & 0xFFFFFFFF) % m) for z in O.splitmix64_stream(0, 16)]
    size = max(abs(XB[i, j]) for i, j in probed) if restarts else np.abs(XB).max()
    Uh[:, 1] *= factor * tol * nA / size
    cr = O.aca_cross(Uh, Vh, a, b, tol, 64, probes=16, seed=0)
    assert cr.converged
    if restarts:
        assert cr.probe_rounds == 2 and max(cr.I) >= split
    else:
        assert cr.probe_rounds == 1 and max(cr.I) < split


# ---------------------------------------------------------------- rounding
def test_truncation_rank_hand_cases():
    assert O.truncation_rank(np.array([1.0, 0.0, 0.0]), 1e-12) == 1
    assert O.truncation_rank(np.array([3.0, 4.0 * 1e-7]), 1e-7) == 2     # tail 4e-7 > 5e-7 * 1e-7*...
    assert O.truncation_rank(np.array([1.0, 1e-3, 1e-9]), 1e-6) == 2
    assert O.truncation_rank(np.array([1.0, 1e-3, 1e-9]), 1e-2) == 1
    assert O.truncation_rank(np.zeros(3), 1e-6) == 0


def test_round_reproduces_prescribed_singular_values():
    m1, m2, k = 70, 55, 9
    rng = np.random.default_rng(8)
    Q1, _ = np.linalg.qr(rng.standard_normal((m1, k)))
    Q2, _ = np.linalg.qr(rng.standard_normal((m2, k)))
    sig = 10.0 ** -np.arange(k, dtype=float)
    Mx = rng.standard_normal((k, k))
    # L diag(d) R^T with a non-orthogonal split of Q1 diag(sig) Q2^T
    L = Q1 @ np.diag(sig) @ Mx
    R = Q2 @ np.linalg.inv(Mx).T
    U, s, V, ok = O.lr_round(L, np.ones(k), R, 1e-5, 64)
    assert ok and len(s) == 5
    assert np.allclose(s, sig[:5], rtol=1e-9)
    assert np.allclose(U.T @ U, np.eye(5), atol=1e-13)
    X = Q1 @ np.diag(sig) @ Q2.T
    u2, s2, v2 = O.svd_truncate(X, 1e-5)
    assert np.allclose(s2, s, rtol=1e-9)
    assert np.linalg.norm((U * s) @ V.T - (u2 * s2) @ v2.T) < 1e-12


# ---------------------------------------------------------------- end to end
def test_parseval_error_matches_spatial_error():
    m = 64
    U, V = inputs.separable_random(m, 4, seed=9)
    Uo, s, Vo, _ = O.lr_poisson2d(U, V, "5pt", 1e-4)
    X = (Uo * s) @ Vo.T
    Xs = O.solve_full(U @ V.T, "5pt")
    e_sp = np.linalg.norm(X - Xs) / np.linalg.norm(Xs)
    assert math.isclose(O.rel_error_freq(Uo, s, Vo, U, V, "5pt"), e_sp, rel_tol=1e-6)


def test_lowrank_residual_matches_dense_residual():
    m = 32
    U, V = inputs.separable_random(m, 3, seed=10)
    for kind in O.KINDS:
        Uo, s, Vo, _ = O.lr_poisson2d(U, V, kind, 1e-5)
        X = (Uo * s) @ Vo.T
        F = U @ V.T
        dense = np.linalg.norm(O.apply_operator(X, kind) - F) / np.linalg.norm(F)
        assert math.isclose(O.lowrank_residual(Uo, s, Vo, U, V, kind), dense, rel_tol=1e-6)


@pytest.mark.parametrize("kind", O.KINDS)
def test_lowrank_solve_m256_accuracy_and_rank(kind):
    # n = 256, rank-8 random separable RHS, eps = 1e-10: error <= 10 eps against
    # the full-grid solve, and the rank is within a few of the optimal eps-rank.
    m, eps = 256, 1e-10
    U, V = inputs.separable_random(m, 8, seed=0)
    Uo, s, Vo, info = O.lr_poisson2d(U, V, kind, eps)
    assert info.ok
    Xs = O.solve_full(U @ V.T, kind)
    X = (Uo * s) @ Vo.T
    assert np.linalg.norm(X - Xs) <= 10 * eps * np.linalg.norm(Xs)
    _, sopt, _ = O.svd_truncate(Xs, eps)
    assert len(sopt) <= info.rank <= len(sopt) + 4
    assert np.allclose(Uo.T @ Uo, np.eye(info.rank), atol=1e-12)


def test_lr_truncate_oracle():
    m = 80
    rng = np.random.default_rng(12)
    U, V = rng.standard_normal((m, 6)), rng.standard_normal((m, 6))
    U = np.hstack([U, U[:, :2] * 1e-9])       # numerically rank 6 + tiny
    V = np.hstack([V, V[:, :2]])
    Uo, so, Vo, ok = O.lr_truncate(U, None, V, 1e-6, 64)
    assert ok and len(so) == 6
    X = U @ V.T
    assert np.linalg.norm((Uo * so) @ Vo.T - X) <= 1e-6 * np.linalg.norm(X)
