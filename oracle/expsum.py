"""Plain FP64 CPU oracle for the exponential-sum solver, the comparison
method of Section 4.1 ("known approaches": 1/lambda approximated by a sum of
exponentials, so that the inverse of a Kronecker sum becomes a short sum of
Kronecker products).

TEST INFRASTRUCTURE ONLY: imported by tests/ and the CPU legs of bench.py,
never by the CUDA library.

For the 5-point kind Lambda_ij = mu_i + mu_j, so exp(-t Lambda_ij) =
exp(-t mu_i) exp(-t mu_j) and, with 1/lambda ~ sum_q w_q exp(-t_q lambda),

    Xh ~ sum_q w_q (E_q Uh) (E_q Vh)^T,   E_q = diag(exp(-t_q mu)),

a low-rank matrix of rank (number of terms) x r, rounded at eps (Section 3).
The paper does not print its exponential sum; the one used here is the sinc
(trapezoidal) quadrature of

    1/lambda = int_{-inf}^{inf} exp(s - lambda e^s) ds          (t = e^s)

with step tau and nodes s_k = s_min + k tau (Stenger, "Numerical Methods
Based on Sinc and Analytic Functions", 1993; the same rule written out for
1/lambda by Hackbusch, "Hierarchical Matrices", 2015): t_k = e^{s_k},
w_k = tau e^{s_k}.  The semi-staggered symbol a_i b_j + b_i a_j does not
split into a sum of a function of i and one of j, so this baseline is for
the 5-point kind only.
"""
from __future__ import annotations

import math

import numpy as np

from . import poisson_lowrank as P


def sinc_exp_sum(lam_min: float, lam_max: float, eps: float):
    """(t, w) with |1/lambda - sum_k w_k exp(-t_k lambda)| <= ~eps / lambda on
    [lam_min, lam_max].  Step from the trapezoidal rule's error for an
    integrand analytic in the strip |Im s| < pi/2, exp(-2 pi (pi/2) / tau),
    with a factor 32 for its constant (measured: without it the error is
    about 16 eps); the left end where the neglected tail e^{s} lam_max <=
    eps / 4, the right end where the integrand exp(s - lam_min e^s) falls
    below eps / lam_max."""
    tau = math.pi * math.pi / (math.log(1.0 / eps) + math.log(32.0))
    s_min = math.log(eps / (4.0 * lam_max))
    s_max = math.log((math.log(lam_max / eps) + 2.0) / lam_min)
    k = np.arange(0, int(math.ceil((s_max - s_min) / tau)) + 1)
    s = s_min + k * tau
    t = np.exp(s)
    return t, tau * t


def expsum_solve(U: np.ndarray, V: np.ndarray, eps: float):
    """The exponential-sum low-rank solve of the 5-point problem
    (U, s, V with orthonormal factors).  The quadrature is built for
    eps / 10 so that it stays below the rounding's tolerance."""
    m = U.shape[0]
    a, _ = P.symbol(m, "5pt")
    t, w = sinc_exp_sum(2.0 * a.min(), 2.0 * a.max(), eps / 10.0)
    Uh, Vh = P.dst1(U), P.dst1(V)
    L = np.hstack([np.exp(-tk * a)[:, None] * Uh * wk for tk, wk in zip(t, w)])
    R = np.hstack([np.exp(-tk * a)[:, None] * Vh for tk in t])
    Ur, s, Vr, _ = P.lr_round(L, np.ones(L.shape[1]), R, eps, L.shape[1])
    return P.dst1(Ur), s, P.dst1(Vr), len(t)
