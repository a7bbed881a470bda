"""Pins of the exponential-sum oracle (oracle/expsum.py): the quadrature
against 1/lambda by brute force over the spectrum interval, and the solve
against the exact solution."""
import numpy as np
import pytest

from oracle import expsum as E
from oracle import poisson_lowrank as P
from paper_1306_2150_gb300 import inputs


@pytest.mark.parametrize("eps", [1e-4, 1e-7, 1e-10])
@pytest.mark.parametrize("m", [64, 1024, 16384])
def test_sinc_quadrature_reaches_eps_over_the_spectrum(m, eps):
    a, _ = P.symbol(m, "5pt")
    lo, hi = 2.0 * a.min(), 2.0 * a.max()
    t, w = E.sinc_exp_sum(lo, hi, eps)
    lam = np.geomspace(lo, hi, 4001)
    approx = np.exp(-np.outer(lam, t)) @ w
    assert np.max(np.abs(approx * lam - 1.0)) <= 2 * eps


def test_sinc_quadrature_is_exact_for_the_integral_it_samples():
    # the nodes and weights are those of the trapezoidal rule for the
    # substituted integral: w_k = tau t_k with log t_k equally spaced
    t, w = E.sinc_exp_sum(10.0, 1e6, 1e-8)
    tau = np.diff(np.log(t))
    assert np.allclose(tau, tau[0]) and np.allclose(w / t, tau[0])


@pytest.mark.parametrize("m", [64, 255])
def test_expsum_solve_matches_the_exact_solution(m):
    eps = 1e-7
    U, V = inputs.separable_random(m, 4, seed=3)
    Ux, s, Vx, q = E.expsum_solve(U, V, eps)
    assert q > 10
    assert P.rel_error_freq(Ux, s, Vx, U, V, "5pt") <= 10 * eps
