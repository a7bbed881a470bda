"""Low-rank Uzawa Stokes solve (Section 2, Section 5) through the C ABI
against the full-format oracle (oracle/stokes.py)."""
import numpy as np
import pytest

from oracle import stokes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lr():
    from paper_1306_2150_gb300 import build, lr as lrmod
    build.build()
    lrmod.load()
    return lrmod


@pytest.fixture(scope="module")
def h(lr):
    handle = lr.Handle()
    yield handle
    handle.close()


def dense(t):
    U, s, V = (x.detach().cpu().numpy() for x in t)
    return (U * s) @ V.T


def body_force_dev(n):
    (a1, b1), (a2, b2) = S.body_force(n)
    return [(torch.from_numpy(a1).cuda(), torch.from_numpy(b1).cuda()),
            (torch.from_numpy(a2).cuda(), torch.from_numpy(b2).cuda())], (a1 @ b1.T, a2 @ b2.T)


@pytest.mark.parametrize("n", [16, 64, 256])
@pytest.mark.parametrize("prec,eps,tol,acc", [("fp64", 1e-10, 1e-9, 1e-7), ("mixed", 1e-7, 1e-6, 2e-5)])
def test_stokes_matches_oracle(lr, h, n, prec, eps, tol, acc):
    fdev, (f1, f2) = body_force_dev(n)
    res = lr.lr_stokes_uzawa(h, n, fdev, tol_div=tol, eps=eps, prec=prec)
    assert res.status == lr.LR_OK, h.last_error()
    assert len(res.history) == res.iters + 1 and res.history[0] == 1.0 and res.history[-1] <= tol
    ref = S.uzawa_cg(f1, f2, n, tol=1e-13)
    u, v, p = dense(res.u[0]), dense(res.u[1]), dense(res.p)
    for a, b in ((u, ref.u), (v, ref.v), (p, ref.p)):
        assert np.linalg.norm(a - b) <= acc * np.linalg.norm(b), (np.linalg.norm(a - b) / np.linalg.norm(b))
    # divergence of the returned velocity, recomputed by the oracle: the CG
    # stops on the Schur residual (tol); the velocity's own rounding at eps
    # adds up to about n eps through B^T (a difference over h)
    div = np.linalg.norm(S.bt(u, v, n)) / np.linalg.norm(S.bt(S.laplace_solve(f1, n), S.laplace_solve(f2, n), n))
    bound = 5 * tol + 2 * n * (max(eps, 1e-6) if prec == "mixed" else eps)  # mixed inner solves run at >= 1e-6
    assert div <= bound and res.resid <= bound, (div, res.resid)
    # the pressure has no kernel component beyond the rounding that follows
    # the projection (relative eps; the modes have unit norm)
    for K in S.kernel_modes(n):
        assert abs(np.sum(p * K)) <= max(1e-8, 2 * eps) * np.linalg.norm(p)


@pytest.mark.parametrize("n,eps,tol", [(16, 1e-10, 1e-9), (64, 1e-7, 1e-6)])
@pytest.mark.parametrize("gmres", [False, True])
def test_stokes_with_divergence_rhs_matches_oracle(lr, h, n, eps, tol, gmres):
    # B^T u = g (Schur right-hand side B^T A^-1 f - g, reading G5), a smooth g
    # of rank 2 (cell centres) with its kernel components removed, against the
    # full-format oracle; a smooth g keeps the pressure of low rank
    fdev, (f1, f2) = body_force_dev(n)
    xc = (np.arange(n) + 0.5) / n
    Q, _ = np.linalg.qr(np.stack([np.ones(n), (-1.0) ** np.arange(n)], axis=1))
    gu = np.stack([np.cos(2 * np.pi * xc), xc - 0.3], axis=1)
    gv = np.stack([np.sin(np.pi * xc), np.cos(3 * np.pi * xc) * (1 + xc)], axis=1)
    gu -= Q @ (Q.T @ gu)
    g = gu @ gv.T
    gdev = (torch.from_numpy(np.asfortranarray(gu)).cuda(), torch.from_numpy(np.asfortranarray(gv)).cuda())
    # (the pressure's rank with g is about 30 at n = 64 and eps = 1e-8: the
    # tighter levels would need sums of more than 64 columns)
    res = lr.lr_stokes_uzawa(h, n, fdev, tol_div=tol, eps=eps, prec="fp64", g=gdev, gmres=gmres, maxit=400)
    assert res.status == lr.LR_OK, h.last_error()
    ref = S.uzawa_cg(f1, f2, n, tol=1e-13, g=g)
    u, v, p = dense(res.u[0]), dense(res.u[1]), dense(res.p)
    for a, b in ((u, ref.u), (v, ref.v), (p, ref.p)):
        assert np.linalg.norm(a - b) <= 100 * tol * np.linalg.norm(b), (np.linalg.norm(a - b) / np.linalg.norm(b))
    div = np.linalg.norm(S.bt(u, v, n) - g)
    scale = np.linalg.norm(S.bt(S.laplace_solve(f1, n), S.laplace_solve(f2, n), n) - g)
    bound = 5 * tol + 2 * n * eps
    assert div <= bound * scale and res.resid <= bound, (div / scale, res.resid)


def test_stokes_iterations_independent_of_h(lr, h):
    its = []
    for n in (64, 256, 1024):
        fdev, _ = body_force_dev(n)
        res = lr.lr_stokes_uzawa(h, n, fdev, tol_div=1e-6, eps=1e-8, prec="fp64")
        assert res.status == lr.LR_OK
        its.append(res.iters)
    assert max(its) <= min(its) + 6, its


def test_stokes_rejects_bad_arguments(lr, h):
    import ctypes
    fdev, _ = body_force_dev(16)
    o = lr._options(1e-7, "fp64", "semi", 64, 1.0, 16, 0, 0, 0)
    st = lr.load().lr_stokes_uzawa(h.ptr, 3, 16, None, None, None, None, 1e-6, 10, ctypes.byref(o), None, None, None)
    assert st == lr.LR_EINVAL


@pytest.mark.parametrize("n", [16, 64, 256])
@pytest.mark.parametrize("prec,eps,tol,acc", [("fp64", 1e-10, 1e-9, 1e-7), ("mixed", 1e-7, 1e-6, 2e-5)])
def test_stokes_gmres_matches_oracle(lr, h, n, prec, eps, tol, acc):
    # Section 5: inexact GMRES with adaptive accuracy of the Schur products
    fdev, (f1, f2) = body_force_dev(n)
    res = lr.lr_stokes_uzawa(h, n, fdev, tol_div=tol, eps=eps, prec=prec, gmres=True)
    assert res.status == lr.LR_OK, h.last_error()
    assert len(res.history) == res.iters + 1 and res.history[0] == 1.0
    ref = S.uzawa_cg(f1, f2, n, tol=1e-13)
    u, v, p = dense(res.u[0]), dense(res.u[1]), dense(res.p)
    for a, b in ((u, ref.u), (v, ref.v), (p, ref.p)):
        assert np.linalg.norm(a - b) <= acc * np.linalg.norm(b), (np.linalg.norm(a - b) / np.linalg.norm(b))
    div = np.linalg.norm(S.bt(u, v, n)) / np.linalg.norm(S.bt(S.laplace_solve(f1, n), S.laplace_solve(f2, n), n))
    bound = 5 * tol + 2 * n * (max(eps, 1e-6) if prec == "mixed" else eps)
    assert div <= bound, div
    # GMRES minimises the residual over the Krylov space CG works in: within
    # one restart cycle (20 vectors) it needs no more iterations than CG, up
    # to the inexact products; a restart costs part of the space
    if prec == "mixed":
        return  # float32 products are less accurate than asked (B^T amplifies their error): more restarts
    cg = lr.lr_stokes_uzawa(h, n, fdev, tol_div=tol, eps=eps, prec=prec)
    if cg.iters < 20:
        assert res.iters <= cg.iters + 3, (res.iters, cg.iters)
    else:
        assert res.iters <= 2 * cg.iters, (res.iters, cg.iters)


@pytest.mark.parametrize("gmres", [False, True])
def test_stokes_resumes_from_a_saved_pressure(lr, h, gmres):
    # checkpoint / resume: a loose solve's pressure, passed back in, is the
    # initial guess; the resumed solve reaches the tight tolerance in fewer
    # iterations than a solve from zero and agrees with the oracle
    n = 64
    fdev, (f1, f2) = body_force_dev(n)
    loose = lr.lr_stokes_uzawa(h, n, fdev, tol_div=1e-4, eps=1e-10, prec="fp64", gmres=gmres)
    assert loose.status == lr.LR_OK, h.last_error()
    saved = tuple(t.clone() for t in loose.p)
    full = lr.lr_stokes_uzawa(h, n, fdev, tol_div=1e-9, eps=1e-10, prec="fp64", gmres=gmres)
    res = lr.lr_stokes_uzawa(h, n, fdev, tol_div=1e-9, eps=1e-10, prec="fp64", gmres=gmres, p0=saved)
    assert res.status == lr.LR_OK, h.last_error()
    assert res.iters < full.iters, (res.iters, full.iters)
    if not gmres:
        assert res.history[0] < 1e-3  # CG starts from the saved iterate's residual
    ref = S.uzawa_cg(f1, f2, n, tol=1e-13)
    p = dense(res.p)
    assert np.linalg.norm(p - ref.p) <= 1e-7 * np.linalg.norm(ref.p)


def test_stokes_mixed_reaches_the_tolerance_at_larger_n(lr, h):
    # config 4's tolerance at n = 1024: the mixed path runs the velocity solves
    # of the Schur products in float64 when the accuracy they need (a tenth of
    # eps) is below what float32 solves resolve, so CG reaches tol_div in about
    # as many iterations as the float64 path
    n, eps, tol = 1024, 1e-7, 1e-6
    fdev, _ = body_force_dev(n)
    mixed = lr.lr_stokes_uzawa(h, n, fdev, tol_div=tol, eps=eps, prec="mixed", maxit=60)
    assert mixed.status == lr.LR_OK, h.last_error()
    fp64 = lr.lr_stokes_uzawa(h, n, fdev, tol_div=tol, eps=eps, prec="fp64", maxit=60)
    assert fp64.status == lr.LR_OK
    assert mixed.history[-1] <= tol and abs(mixed.iters - fp64.iters) <= 2, (mixed.iters, fp64.iters)
