"""Pins of the 3D Tucker oracle (oracle/tucker3d.py) against facts outside
it: LAPACK eigenvalues and a dense solve of the assembled 7-point operator,
a closed-form eigenfunction solution, exact recovery of a tensor of known
Tucker rank, the higher-order SVD's all-orthogonality and error bound, and
the low-rank solve against the full-format one by brute force."""
import numpy as np
import pytest

from oracle import poisson_lowrank as P
from oracle import tucker3d as T
from paper_1306_2150_gb300 import inputs


def test_7point_eigenvalues_are_sums_of_1d_ones():
    n = (3, 4, 5)
    ev = np.sort(np.linalg.eigvalsh(T.dense_operator3(*n)))
    mu = [P.eig_second_difference(k) * (k + 1) ** 2 for k in n]
    ref = np.sort((mu[0][:, None, None] + mu[1][None, :, None] + mu[2][None, None, :]).ravel())
    assert np.allclose(ev, ref, rtol=1e-12, atol=0)
    assert np.allclose(T.mu(7), P.eig_second_difference(7) * 64, rtol=1e-14)


def test_stencil_matches_the_assembled_operator():
    X = np.random.default_rng(1).standard_normal((4, 5, 6))
    A = T.dense_operator3(4, 5, 6)
    assert np.allclose(T.apply_operator3(X).ravel(), A @ X.ravel(), rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("n", [(5, 6, 7), (8, 8, 8)])
def test_full_solve_matches_dense_lu(n):
    F = np.random.default_rng(2).standard_normal(n)
    X = T.solve_full3(F)
    Xd = np.linalg.solve(T.dense_operator3(*n), F.ravel()).reshape(n)
    assert np.allclose(X, Xd, rtol=0, atol=1e-12 * np.abs(Xd).max())


def test_eigenfunction_is_solved_exactly_at_rank_one():
    # F = sin(a pi x) sin(b pi y) sin(c pi z) is an eigenfunction of the
    # discrete operator with eigenvalue mu_a + mu_b + mu_c (closed form)
    n, (a, b, c) = 40, (2, 5, 9)
    x = inputs.grid(n)
    s = [np.sin(q * np.pi * x)[:, None] for q in (a, b, c)]
    G = np.ones((1, 1, 1))
    res = T.lr_poisson3d(G, s[0], s[1], s[2], 1e-10)
    lam = sum(4.0 * (n + 1) ** 2 * np.sin(q * np.pi / (2 * (n + 1))) ** 2 for q in (a, b, c))
    X = T.tucker_full(res.G, *res.U)
    ref = np.einsum("i,j,k->ijk", s[0][:, 0], s[1][:, 0], s[2][:, 0]) / lam
    assert res.G.shape == (1, 1, 1)
    assert np.linalg.norm(X - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.linalg.norm(T.apply_operator3(X) - np.einsum("i,j,k->ijk", *[v[:, 0] for v in s])) <= 1e-9 * lam * np.linalg.norm(X)


def test_frequency_tensor_entries_are_the_transformed_rhs_over_the_symbol():
    G, U1, U2, U3 = inputs.tucker_random((9, 10, 11), (2, 3, 2), seed=4)
    F = T.tucker_full(G, U1, U2, U3)
    X = T.FreqTensor(G, P.dst1(U1), P.dst1(U2), P.dst1(U3))
    ref = T.dst3(T.solve_full3(F))            # Xh = S X S S, from the full solve
    got = X.block(np.arange(9), np.arange(10), np.arange(11))
    assert np.allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    assert np.allclose(X.fibre(1, 3, 7), ref[3, :, 7], rtol=0, atol=1e-13 * np.abs(ref).max())
    assert np.allclose(X.fibre(2, 8, 0), ref[8, 0, :], rtol=0, atol=1e-13 * np.abs(ref).max())


def test_cross_recovers_a_tensor_of_known_tucker_rank():
    rng = np.random.default_rng(7)
    ranks = (3, 4, 5)
    U = [np.linalg.qr(rng.standard_normal((n, r)))[0] for n, r in zip((30, 31, 32), ranks)]
    A = T.tucker_full(rng.standard_normal(ranks), *U)
    cr = T.tucker_cross(T.DenseTensor(A), 1e-12)
    Y = T.tucker_full(cr.C, *cr.Q)
    assert np.linalg.norm(Y - A) <= 1e-11 * np.linalg.norm(A)
    assert [q.shape[1] for q in cr.Q] == list(ranks)
    # interpolation: Y equals A on the index grid
    assert np.allclose(Y[np.ix_(*cr.I)], A[np.ix_(*cr.I)], rtol=0, atol=1e-12 * np.abs(A).max())


def test_hosvd_rounding_is_all_orthogonal_and_within_its_bound():
    rng = np.random.default_rng(3)
    # a core with decaying multilinear spectrum in orthonormal bases
    C = rng.standard_normal((12, 10, 9)) * np.exp(-np.arange(12))[:, None, None] * np.exp(-0.7 * np.arange(10))[None, :, None]
    Qs = [np.linalg.qr(rng.standard_normal((n, r)))[0] for n, r in zip((40, 41, 42), C.shape)]
    # nothing dropped: the core is all-orthogonal (De Lathauwer et al. 2000),
    # the row norms of each unfolding are that mode's singular values
    G, Us, sig = T.hosvd_round(C, Qs, 0.0)
    assert G.shape == C.shape
    for mode in range(3):
        unf = np.moveaxis(G, mode, 0).reshape(G.shape[mode], -1)
        gram = unf @ unf.T
        assert np.allclose(gram, np.diag(np.diag(gram)), atol=1e-12 * np.abs(gram).max())
        assert np.allclose(np.sqrt(np.diag(gram)), sig[mode], rtol=1e-10)
    for eps in (1e-2, 1e-5, 1e-9):
        G, Us, sig = T.hosvd_round(C, Qs, eps)
        full = T.tucker_full(C, *Qs)
        err = np.linalg.norm(T.tucker_full(G, *Us) - full) / np.linalg.norm(full)
        assert err <= eps
        for mode in range(3):
            assert np.allclose(Us[mode].T @ Us[mode], np.eye(G.shape[mode]), atol=1e-13)
            # each kept rank is the smallest whose dropped tail fits its share
            s = sig[mode]
            R = G.shape[mode]
            assert np.sqrt(np.sum(s[R:] ** 2)) <= eps * np.linalg.norm(C) / np.sqrt(3)
            assert R == 0 or np.sqrt(np.sum(s[R - 1:] ** 2)) > eps * np.linalg.norm(C) / np.sqrt(3)


@pytest.mark.parametrize("eps", [1e-6, 1e-10])
@pytest.mark.parametrize("case", ["smooth", "random", "uneven"])
def test_lowrank_solve_within_10_eps_of_the_full_solve(case, eps):
    if case == "smooth":
        G, U1, U2, U3 = inputs.smooth3d(48, eps)
    elif case == "random":
        G, U1, U2, U3 = inputs.tucker_random(40, 6, seed=5)
    else:
        G, U1, U2, U3 = inputs.tucker_random((47, 66, 75), (2, 5, 3), seed=6)
    F = T.tucker_full(G, U1, U2, U3)
    res = T.lr_poisson3d(G, U1, U2, U3, eps)
    assert res.cross.converged
    assert T.rel_error_full(res, F) <= 10 * eps
    for U in res.U:
        assert np.allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-12)


def test_smooth_rhs_generator_matches_its_function():
    for n in (16, 40):
        G, U1, U2, U3 = inputs.smooth3d(n, 1e-6)
        F = T.tucker_full(G, U1, U2, U3)
        D = inputs.smooth3d_dense(n)
        assert np.linalg.norm(F - D) <= 2e-6 * np.linalg.norm(D)
        assert max(G.shape) <= 24


def test_zero_rhs_rounds_to_the_empty_tucker_tensor():
    G, U1, U2, U3 = inputs.tucker_random(20, 2, seed=1)
    res = T.lr_poisson3d(np.zeros_like(G), U1, U2, U3, 1e-6)
    assert res.cross.converged and res.G.shape == (0, 0, 0)
    assert all(U.shape == (20, 0) for U in res.U)


@pytest.mark.parametrize("n", [(1, 1, 1), (2, 3, 5), (7, 1, 4)])
def test_tiny_grids_are_solved_to_rounding_error(n):
    # grids smaller than the ranks: the cross spans the whole tensor
    rhs = inputs.tucker_random(n, (1, 1, 1), seed=2)
    res = T.lr_poisson3d(*rhs, 1e-10)
    assert T.rel_error_full(res, T.tucker_full(*rhs)) <= 1e-13
