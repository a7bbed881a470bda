"""Pins of the Stokes oracle (oracle/stokes.py) against facts outside it:
the assembled saddle system, the paper's statement on the Schur spectrum
(Section 2), the kernel modes, the semi-staggered Laplacian of the Poisson
oracle, and the momentum and divergence equations."""
import numpy as np
import pytest

from oracle import poisson_lowrank as P
from oracle import stokes as S


@pytest.mark.parametrize("n", [4, 7, 10])
def test_laplacian_from_gradients_is_the_semi_operator(n):
    m = n - 1
    U = np.random.default_rng(n).standard_normal((m, m))
    A = P.dense_operator(m, "semi")
    assert np.allclose(S.laplace(U, n).reshape(-1, order="F"), A @ U.reshape(-1, order="F"), rtol=0, atol=1e-9 * n * n)


@pytest.mark.parametrize("n", [6, 8, 11])
def test_schur_spectrum_matches_the_paper(n):
    # Section 2: two zero eigenvalues in 2D, (n-2)^2 eigenvalues equal to 1,
    # the rest in [0, 1]
    ev = np.linalg.eigvalsh(S.schur_dense(n))
    assert np.sum(np.abs(ev) < 1e-10) == 2
    assert np.sum(np.abs(ev - 1.0) < 1e-10) == (n - 2) ** 2
    assert ev.min() > -1e-10 and ev.max() < 1.0 + 1e-10


@pytest.mark.parametrize("n", [5, 8])
def test_kernel_modes_are_annihilated_by_the_gradient(n):
    for K in S.kernel_modes(n):
        assert np.abs(S.bx(K, n)).max() < 1e-13 and np.abs(S.by(K, n)).max() < 1e-13
        assert abs(np.linalg.norm(K) - 1.0) < 1e-14


@pytest.mark.parametrize("n", [6, 9])
def test_uzawa_matches_the_assembled_saddle_system(n):
    rng = np.random.default_rng(n)
    f1 = rng.standard_normal((n - 1, n - 1))
    f2 = rng.standard_normal((n - 1, n - 1))
    res = S.uzawa_cg(f1, f2, n, tol=1e-13)
    u, v, p = S.saddle_dense(f1, f2, n)
    assert np.allclose(res.u, u, atol=1e-10) and np.allclose(res.v, v, atol=1e-10)
    assert np.allclose(res.p, p, atol=1e-9 * max(1.0, np.abs(p).max()))


def compatible_g(n, seed):
    """A low-rank divergence right-hand side orthogonal to the pressure's
    kernel modes (the part B^T u can meet)."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(np.stack([np.ones(n), (-1.0) ** np.arange(n)], axis=1))
    gu, gv = rng.standard_normal((n, 2)), rng.standard_normal((n, 2))
    gu -= Q @ (Q.T @ gu)
    return gu @ gv.T


@pytest.mark.parametrize("n", [6, 8, 16])
def test_uzawa_with_divergence_rhs_matches_the_assembled_saddle_system(n):
    # B^T u = g (Eq. flr:stprob with a second right-hand side; Schur
    # right-hand side B^T A^-1 f - g, reading G5), against the dense saddle
    # solve; the velocity's divergence is g and the momentum equation holds
    rng = np.random.default_rng(100 + n)
    f1 = rng.standard_normal((n - 1, n - 1))
    f2 = rng.standard_normal((n - 1, n - 1))
    g = compatible_g(n, n)
    res = S.uzawa_cg(f1, f2, n, tol=1e-13, g=g)
    u, v, p = S.saddle_dense(f1, f2, n, g=g)
    assert np.allclose(res.u, u, atol=1e-10) and np.allclose(res.v, v, atol=1e-10)
    assert np.allclose(res.p, p, atol=1e-9 * max(1.0, np.abs(p).max()))
    assert np.linalg.norm(S.bt(res.u, res.v, n) - g) <= 1e-10 * np.linalg.norm(g)
    m1 = S.laplace(res.u, n) + S.bx(res.p, n) - f1
    assert np.linalg.norm(m1) <= 1e-9 * np.linalg.norm(f1)
    assert res.resid <= 1e-12


def test_uzawa_solution_satisfies_momentum_and_divergence():
    n = 24
    (a1, b1), (a2, b2) = S.body_force(n)
    f1, f2 = a1 @ b1.T, a2 @ b2.T
    res = S.uzawa_cg(f1, f2, n, tol=1e-12)
    assert res.resid <= 1e-12
    m1 = S.laplace(res.u, n) + S.bx(res.p, n) - f1
    m2 = S.laplace(res.v, n) + S.by(res.p, n) - f2
    assert np.linalg.norm(m1) <= 1e-9 * np.linalg.norm(f1) and np.linalg.norm(m2) <= 1e-9 * np.linalg.norm(f2)
    assert np.linalg.norm(S.bt(res.u, res.v, n)) <= 1e-11 * np.linalg.norm(S.bt(S.laplace_solve(f1, n), S.laplace_solve(f2, n), n))


def test_cg_iterations_do_not_grow_with_the_grid():
    # Section 2: CG works on the complement of the kernel, where the Schur
    # operator is bounded away from 0 independently of h
    its = []
    for n in (16, 32, 64):
        (a1, b1), (a2, b2) = S.body_force(n)
        its.append(S.uzawa_cg(a1 @ b1.T, a2 @ b2.T, n, tol=1e-8).iters)
    assert max(its) <= min(its) + 6, its


def test_zero_force_gives_the_zero_solution():
    res = S.uzawa_cg(np.zeros((7, 7)), np.zeros((7, 7)), 8)
    assert res.iters == 0 and res.resid == 0.0
    assert not np.any(res.u) and not np.any(res.v) and not np.any(res.p)
