"""GPU parity: the CUDA path through the C ABI against the CPU FP64 oracle.

Tolerances: float64 results within 10 eps (relative Frobenius, the solve's
stated accuracy target) and transforms within a few ulps times log M; float32
(mixed) transforms within 2e-6 relative; pivot indices and ranks of the FP64
path on the 256-point random separable problem bit-exact.
"""
import math

import numpy as np
import pytest

from oracle import poisson_lowrank as O
from paper_1306_2150_gb300 import inputs

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


def cuda(a):
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def npy(t):
    return t.detach().cpu().numpy()


def solve(lr, h, U, V, **kw):
    res = lr.lr_poisson2d(h, cuda(U), cuda(V), **kw)
    torch.cuda.synchronize()
    return res, npy(res.U), npy(res.s), npy(res.V)


# ------------------------------------------------------------------ forward / inverse DST
@pytest.mark.parametrize("m", [1, 2, 3, 31, 256, 1000, 2048, 2049, 5000])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_dst1_matches_oracle(lr, h, m, prec):
    X = np.random.default_rng(m).standard_normal((m, 3))
    Y = npy(lr.lr_dst1(h, cuda(X), prec))
    Yo = O.dst1(X)
    err = np.linalg.norm(Y - Yo, axis=0) / np.linalg.norm(Yo, axis=0)
    tol = 1e-14 * max(1.0, math.log2(2 * m)) if prec == "fp64" else 2e-6
    assert err.max() <= tol, err


@pytest.mark.parametrize("m", [16384, 65536])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_dst1_full_size_sampled(lr, h, m, prec):
    X = np.random.default_rng(7).standard_normal((m, 2))
    Y = npy(lr.lr_dst1(h, cuda(X), prec))
    nx = np.linalg.norm(X[:, 0])
    tol = 1e-13 if prec == "fp64" else 3e-6
    for k in (0, 1, 2, 1000, m // 2, m - 2, m - 1):
        assert abs(Y[k, 0] - O.dst1_entry(X[:, 0], k)) <= tol * nx
    # orthogonality: the transform is an involution up to rounding
    Z = npy(lr.lr_dst1(h, cuda(Y), prec))
    assert np.linalg.norm(Z - X) <= (1e-13 if prec == "fp64" else 5e-6) * np.linalg.norm(X)


# ------------------------------------------------------------------ solve
def test_m256_r8_fp64_pivots_ranks_bitexact(lr, h):
    m, r, eps = 256, 8, 1e-10
    U, V = inputs.separable_random(m, r, seed=0)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec="fp64")
    assert res.status == lr.LR_OK
    ou, os_, ov, info = O.lr_poisson2d(U, V, "5pt", eps)
    assert res.info.aca_steps == info.cross.k
    assert res.pivots_I == info.cross.I
    assert res.pivots_J == info.cross.J
    assert res.info.rank == info.rank
    err = O.rel_error_freq(Uo, s, Vo, U, V, "5pt")
    assert err <= 10 * eps
    assert np.allclose(s, os_, rtol=1e-9, atol=1e-12 * os_[0])
    assert np.abs(Uo.T @ Uo - np.eye(len(s))).max() < 1e-12


def test_dense_lu_n32(lr, h):
    # the n = 32 dense LU check, on the GPU result
    m, r, eps = 32, 8, 1e-10
    U, V = inputs.separable_random(m, r, seed=0)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec="fp64")
    X = (Uo * s) @ Vo.T
    Xd = O.solve_dense(U @ V.T, "5pt")
    assert np.linalg.norm(X - Xd) <= 10 * eps * np.linalg.norm(Xd)


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-10), ("fp64", 1e-6), ("mixed", 1e-6)])
@pytest.mark.parametrize("m", [256, 1000, 4096])
def test_random_separable_accuracy(lr, h, m, prec, eps):
    U, V = inputs.separable_random(m, 8, seed=m)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec=prec)
    assert res.status == lr.LR_OK
    assert O.rel_error_freq(Uo, s, Vo, U, V, "5pt") <= 10 * eps


@pytest.mark.parametrize("m", [1024, 4096])
@pytest.mark.parametrize("prec,eps", [("fp64", 1e-10), ("fp64", 1e-6), ("mixed", 1e-6)])
def test_smooth_sum_accuracy(lr, h, m, prec, eps):
    U, V = inputs.smooth_sum(m, eps)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec=prec)
    assert res.status == lr.LR_OK
    assert O.rel_error_freq(Uo, s, Vo, U, V, "5pt") <= 10 * eps


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_size_16384(lr, h, prec):
    # the benchmarked workload: n = 16384, eps = 1e-6, exact error by Parseval
    m, eps = 16384, 1e-6
    U, V = inputs.smooth_sum(m, eps)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec=prec)
    assert res.status == lr.LR_OK
    assert O.rel_error_freq(Uo, s, Vo, U, V, "5pt", block=1024) <= 10 * eps


def test_full_size_65536_sampled_rows(lr, h):
    m, eps = 65536, 1e-6
    U, V = inputs.smooth_sum(m, eps)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec="mixed")
    assert res.status == lr.LR_OK
    rows = np.unique(np.concatenate([np.arange(64), np.linspace(0, m - 1, 192).astype(int)]))
    assert O.rel_error_freq(Uo, s, Vo, U, V, "5pt", rows=rows) <= 10 * eps


def test_semistaggered_operator(lr, h):
    m, eps = 255, 1e-10
    U, V = inputs.separable_random(m, 6, seed=3)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec="fp64", op="semi")
    assert res.status == lr.LR_OK
    ou, os_, ov, info = O.lr_poisson2d(U, V, "semi", eps)
    assert res.pivots_I == info.cross.I and res.pivots_J == info.cross.J
    assert res.info.rank == info.rank
    Xs = O.solve_full(U @ V.T, "semi")
    X = (Uo * s) @ Vo.T
    assert np.linalg.norm(X - Xs) <= 10 * eps * np.linalg.norm(Xs)



@pytest.mark.parametrize("kind", ["5pt", "semi"])
@pytest.mark.parametrize("cs", [0, 1, 3])
def test_probe_restart_fp64_bitexact(lr, h, kind, cs):
    # Block-diagonal Xh (Section 4.2 cross, reading G7 of the stop rule): the
    # cross converges on block A, a residual probe lands in block B and the
    # loop restarts at its row.  Pivots, probe rounds, steps and rank of the
    # float64 path equal the oracle's; the error is within 10 eps.
    m, eps = 128, 1e-6
    Uh, Vh = inputs.block_diagonal_freq(m, 32)
    U, V = O.dst1(Uh), O.dst1(Vh)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec="fp64", op=kind, cluster_size=cs)
    assert res.status == lr.LR_OK
    ou, os_, ov, info = O.lr_poisson2d(U, V, kind, eps)
    assert info.cross.probe_rounds == 2
    assert res.info.probe_rounds == info.cross.probe_rounds
    assert res.info.aca_steps == info.cross.k
    assert res.pivots_I == info.cross.I and res.pivots_J == info.cross.J
    assert res.info.rank == info.rank
    assert O.rel_error_freq(Uo, s, Vo, U, V, kind) <= 10 * eps


def test_probe_restart_mixed(lr, h):
    m, eps = 4096, 1e-6
    Uh, Vh = inputs.block_diagonal_freq(m, 1024)
    U, V = O.dst1(Uh), O.dst1(Vh)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec="mixed")
    assert res.status == lr.LR_OK
    assert res.info.probe_rounds >= 2
    assert max(res.pivots_I) >= 1024
    assert O.rel_error_freq(Uo, s, Vo, U, V, "5pt") <= 10 * eps


# ------------------------------------------------------------------ edges
@pytest.mark.parametrize("m", [1, 2, 3, 5])
def test_tiny_grids(lr, h, m):
    U, V = inputs.separable_random(m, 1, seed=m)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=1e-12, prec="fp64")
    X = (Uo * s) @ Vo.T
    Xd = O.solve_dense(U @ V.T, "5pt")
    assert np.linalg.norm(X - Xd) <= 1e-11 * np.linalg.norm(Xd)


def test_eigenfunction_is_rank_one(lr, h):
    m = 777
    x = np.arange(1, m + 1) / (m + 1)
    u, v = np.sin(3 * np.pi * x)[:, None], np.sin(5 * np.pi * x)[:, None]
    res, Uo, s, Vo = solve(lr, h, u, v, eps=1e-10, prec="fp64")
    assert res.info.rank == 1
    assert O.rel_error_freq(Uo, s, Vo, u, v, "5pt") <= 1e-12


def test_zero_rhs_gives_rank_zero(lr, h):
    m = 300
    U = np.zeros((m, 2))
    V = np.ones((m, 2))
    res, Uo, s, Vo = solve(lr, h, U, V, eps=1e-8, prec="fp64")
    assert res.status == lr.LR_OK and res.info.rank == 0


def test_max_rank_rhs(lr, h):
    m, eps = 2000, 1e-6
    U, V = inputs.separable_random(m, 64, seed=5)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec="mixed")
    assert res.status == lr.LR_OK
    assert O.rel_error_freq(Uo, s, Vo, U, V, "5pt") <= 10 * eps


def test_step_cap_returns_enoconv_with_partial_result(lr, h):
    m = 1024
    U, V = inputs.separable_random(m, 8, seed=1)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=1e-10, prec="fp64", rmax=3)
    assert res.status == lr.LR_ENOCONV
    assert res.info.aca_steps == 3 and res.info.converged == 0 and 1 <= res.info.rank <= 3


def test_output_capacity_cut(lr, h):
    m = 512
    U, V = inputs.separable_random(m, 8, seed=2)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=1e-10, prec="fp64", rmax_out=4)
    assert res.status == lr.LR_ENOCONV and res.info.cut == 1 and res.info.rank == 4


@pytest.mark.parametrize("cs", [1, 2, 4, 8, 16])
def test_cluster_sizes_agree(lr, h, cs):
    m, eps = 3000, 1e-10
    U, V = inputs.separable_random(m, 6, seed=9)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec="fp64", cluster_size=cs)
    ou, os_, ov, info = O.lr_poisson2d(U, V, "5pt", eps)
    assert res.pivots_I == info.cross.I and res.pivots_J == info.cross.J
    assert O.rel_error_freq(Uo, s, Vo, U, V, "5pt") <= 10 * eps


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_repeat_runs_bitwise_identical(lr, h, prec):
    U, V = inputs.separable_random(5000, 10, seed=4)
    a = solve(lr, h, U, V, eps=1e-8, prec=prec)
    b = solve(lr, h, U, V, eps=1e-8, prec=prec)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


def test_async_mode_then_info(lr, h):
    U, V = inputs.separable_random(700, 5, seed=6)
    Ut, Vt = cuda(U), cuda(V)
    out = (lr.colmajor_empty(700, 64), torch.empty(64, dtype=torch.float64, device="cuda"),
           lr.colmajor_empty(700, 64))
    assert lr.lr_poisson2d(h, Ut, Vt, eps=1e-9, prec="fp64", async_=True, out=out) is None
    torch.cuda.synchronize()
    info, pi, pj = lr.lr_get_info(h)
    R = info.rank
    assert info.converged == 1 and R > 0
    err = O.rel_error_freq(npy(out[0][:, :R]), npy(out[1][:R]), npy(out[2][:, :R]), U, V, "5pt")
    assert err <= 1e-8


def test_workspace_limit_gives_enomem_and_handle_recovers(lr):
    # allocation failure on the host side: a workspace request above the
    # handle's cap returns LR_ENOMEM before any launch; lifting the cap, the
    # same handle solves the problem
    m = 16384
    U, V = inputs.smooth_sum(m, 1e-6)
    Ut, Vt = cuda(U), cuda(V)
    with lr.Handle() as h2:
        lr.lr_set_workspace_limit(h2, 1 << 20)
        res = lr.lr_poisson2d(h2, Ut, Vt, eps=1e-6, prec="mixed", check=False)
        assert res.status == lr.LR_ENOMEM
        assert "limit" in h2.last_error()
        b = lr.Batch([(torch.from_numpy(U), torch.from_numpy(V))] * 2)
        assert lr.lr_poisson2d_batched(h2, b, eps=1e-6, check=False) == lr.LR_ENOMEM
        x = np.arange(1, 1024) / 1024
        fdev = [(cuda(np.sin(np.pi * x)[:, None]), cuda(np.cos(np.pi * x)[:, None]))] * 2
        assert lr.lr_stokes_uzawa(h2, 1024, fdev, check=False).status == lr.LR_ENOMEM
        lr.lr_set_workspace_limit(h2, 0)
        res = lr.lr_poisson2d(h2, Ut, Vt, eps=1e-6, prec="mixed")
        torch.cuda.synchronize()
        assert res.status == lr.LR_OK
        rows = np.unique(np.linspace(0, m - 1, 64).astype(int))
        assert O.rel_error_freq(npy(res.U), npy(res.s), npy(res.V), U, V, "5pt", rows=rows) <= 1e-5


def test_invalid_arguments(lr, h):
    import ctypes
    U = lr.colmajor_empty(100, 2)
    U.fill_(1.0)
    Uo = lr.colmajor_empty(100, 8)
    s = torch.empty(8, dtype=torch.float64, device="cuda")
    lib = lr.load()
    o = lr.lr_options_default()

    def call(rhs_r=2, ld=100, eps=1e-6, rmax=8, uptr=None, opt_rmax=64):
        o.eps = eps
        o.rmax = opt_rmax
        rhs = lr.LrMat(100, 100, rhs_r, rhs_r, ld, uptr or U.data_ptr(), None, U.data_ptr())
        sol = lr.LrMat(100, 100, 0, rmax, 100, Uo.data_ptr(), s.data_ptr(), Uo.data_ptr())
        return lib.lr_poisson2d(h.ptr, ctypes.byref(rhs), ctypes.byref(sol), ctypes.byref(o))

    assert call(rhs_r=0) == lr.LR_EINVAL
    assert call(rhs_r=65) == lr.LR_EINVAL
    assert call(ld=99) == lr.LR_EINVAL
    assert call(eps=0.0) == lr.LR_EINVAL
    assert call(eps=float("nan")) == lr.LR_EINVAL
    assert call(rmax=0) == lr.LR_EINVAL
    assert call(opt_rmax=65) == lr.LR_EINVAL
    assert call(uptr=U.data_ptr() + 8) == lr.LR_EINVAL
    assert "16-byte" in h.last_error()


# ------------------------------------------------------------------ rounding
def test_truncate_matches_oracle(lr, h):
    m1, m2, k = 500, 430, 12
    rng = np.random.default_rng(13)
    U = rng.standard_normal((m1, k)) * (10.0 ** -np.arange(k))
    V = rng.standard_normal((m2, k))
    Ut, st, Vt, status = lr.lr_truncate(h, cuda(U), None, cuda(V), 1e-6)
    torch.cuda.synchronize()
    uo, so, vo, ok = O.lr_truncate(U, None, V, 1e-6, 64)
    assert status == lr.LR_OK
    assert len(npy(st)) == len(so)
    assert np.allclose(npy(st), so, rtol=1e-10)
    X = U @ V.T
    Xg = (npy(Ut) * npy(st)) @ npy(Vt).T
    assert np.linalg.norm(Xg - X) <= 1.01e-6 * np.linalg.norm(X)
    assert np.abs(npy(Ut).T @ npy(Ut) - np.eye(len(so))).max() < 1e-10


# ------------------------------------------------------------------ refinement
@pytest.mark.parametrize("m,kind", [(256, "random"), (1024, "smooth"), (4096, "smooth"), (16384, "smooth")])
def test_mixed_with_refinement_reaches_1e10(lr, h, m, kind):
    # float32 sampling alone stalls near 1e-7; float64 residual refinement
    # (automatic below eps = 1e-7) brings the mixed path to 10 eps
    eps = 1e-10
    U, V = inputs.separable_random(m, 8, seed=0) if kind == "random" else inputs.smooth_sum(m, eps)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec="mixed")
    assert res.status == lr.LR_OK
    assert 1 <= res.info.refine_rounds <= 6
    rows = None if m <= 4096 else np.unique(np.linspace(0, m - 1, 512).astype(int))
    assert O.rel_error_freq(Uo, s, Vo, U, V, "5pt", rows=rows) <= 10 * eps
    assert np.abs(Uo.T @ Uo - np.eye(len(s))).max() < 1e-10
    assert np.abs(Vo.T @ Vo - np.eye(len(s))).max() < 1e-10
    assert np.all(np.diff(s) <= 0)


def test_refinement_off_is_limited_by_float32(lr, h):
    m, eps = 1024, 1e-10
    U, V = inputs.smooth_sum(m, eps)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec="mixed", refine=-1)
    assert res.info.refine_rounds == 0
    e_plain = O.rel_error_freq(Uo, s, Vo, U, V, "5pt")
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec="mixed", refine=2)
    e_ref = O.rel_error_freq(Uo, s, Vo, U, V, "5pt")
    assert e_ref <= 10 * eps < e_plain


def test_refinement_semistaggered(lr, h):
    m, eps = 2048, 1e-10
    U, V = inputs.smooth_sum(m, eps)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec="mixed", op="semi")
    assert res.status == lr.LR_OK and res.info.refine_rounds >= 1
    assert O.rel_error_freq(Uo, s, Vo, U, V, "semi") <= 10 * eps


# ------------------------------------------------------------------ cluster transform variant
@pytest.mark.parametrize("m", [2049, 4096, 5000, 16384, 65536])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cluster_transform_variant(lr, h, m, prec):
    # one thread-block cluster per column (CS = 2, 2, 4, 8, 16 CTAs; float64 at
    # m = 65536 needs more shared memory than the variant uses and falls back
    # to the four-step transform)
    eps = 1e-6 if prec == "mixed" else 1e-10
    U, V = inputs.smooth_sum(m, eps)
    res, Uo, s, Vo = solve(lr, h, U, V, eps=eps, prec=prec, cluster_dst=True)
    assert res.status == lr.LR_OK
    rows = None if m <= 5000 else np.unique(np.linspace(0, m - 1, 256).astype(int))
    assert O.rel_error_freq(Uo, s, Vo, U, V, "5pt", rows=rows) <= 10 * eps
    ref, Ur, sr, Vr = solve(lr, h, U, V, eps=eps, prec=prec)
    assert abs(len(s) - len(sr)) <= 1


# ------------------------------------------------------------------ full-grid solver (crossover reference)
@pytest.mark.parametrize("m", [1, 2, 3, 31, 256, 1000, 2049, 5000])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["5pt", "semi"])
def test_full_grid_matches_oracle(lr, h, m, prec, kind):
    F = np.random.default_rng(m + 7).standard_normal((m, m))
    X = npy(lr.lr_poisson2d_full(h, cuda(F), prec=prec, op=kind))
    Xo = O.solve_full(F, kind)
    err = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
    tol = 1e-13 * max(1.0, math.log2(m)) if prec == "fp64" else 3e-6
    assert err <= tol, err


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_grid_agrees_with_lowrank_at_16384(lr, h, prec):
    m = 16384
    U, V = inputs.smooth_sum(m, 1e-12)
    Ud, Vd = cuda(U), cuda(V)
    F = torch.from_numpy(np.asfortranarray(U @ V.T)).T.cuda().T   # exact float64 product on the host
    X = lr.lr_poisson2d_full(h, F, prec=prec)
    del F
    res = lr.lr_poisson2d(h, Ud, Vd, eps=1e-12, prec="fp64")
    # whole sampled rows: the low-rank solution's error (<= 10 eps in the
    # Frobenius norm) is not uniform over single entries (it is relatively
    # largest in the corners, where X is smallest)
    rows = np.unique(np.linspace(0, m - 1, 300).astype(np.int64))
    Xs = npy(X[torch.from_numpy(rows).cuda()])
    Ul, sl, Vl = npy(res.U), npy(res.s), npy(res.V)
    Xl = (Ul[rows] * sl) @ Vl.T                # sampled rows of the low-rank solution, on the host
    err = np.linalg.norm(Xs - Xl) / np.linalg.norm(Xl)
    assert err <= (1e-10 if prec == "fp64" else 1e-5), err


# ------------------------------------------------------------------ exponential-sum baseline
@pytest.mark.parametrize("m,kind", [(64, "random"), (255, "random"), (1024, "smooth"), (4096, "smooth")])
def test_expsum_matches_oracle(lr, h, m, kind):
    from oracle import expsum as E
    eps = 1e-7
    U, V = inputs.separable_random(m, 4, seed=3) if kind == "random" else inputs.smooth_sum(m, eps)
    Ux, s, Vx, q = lr.lr_poisson2d_expsum(h, cuda(U), cuda(V), eps=eps)
    t, _ = E.sinc_exp_sum(2 * O.symbol(m, "5pt")[0].min(), 2 * O.symbol(m, "5pt")[0].max(), eps / 10)
    assert q == len(t)
    assert O.rel_error_freq(npy(Ux), npy(s), npy(Vx), U, V, "5pt") <= 10 * eps
    assert np.abs(npy(Ux).T @ npy(Ux) - np.eye(len(s))).max() < 1e-10
