"""Low-rank 3D Poisson solve in Tucker format (Section 3, Eq. flr:tucker;
Sections 4.1-4.2 in three dimensions) through the C ABI, against the oracle
(oracle/tucker3d.py): the exact full-format solution where the full tensor
fits, frequency-space slices of it at the benchmark sizes, and the oracle's
own low-rank solve (ranks)."""
import ctypes

import numpy as np
import pytest

from oracle import poisson_lowrank as P
from oracle import tucker3d as T
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


def to_dev(G, U1, U2, U3):
    return (torch.from_numpy(np.ascontiguousarray(G)).cuda(),
            *[torch.from_numpy(np.asfortranarray(U)).cuda() for U in (U1, U2, U3)])


def host(res):
    return res.G.cpu().numpy(), [U.cpu().numpy() for U in res.U]


def check_orthonormal(Us):
    for U in Us:
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 1e-11


@pytest.mark.parametrize("eps", [1e-6, 1e-10])
@pytest.mark.parametrize("case", ["smooth48", "random40", "uneven", "smooth128"])
def test_tucker3d_matches_the_full_solve(lr, h, case, eps):
    if case == "smooth48":
        rhs = inputs.smooth3d(48, eps)
    elif case == "smooth128":
        rhs = inputs.smooth3d(128, eps)
    elif case == "random40":
        rhs = inputs.tucker_random(40, 6, seed=5)
    else:
        rhs = inputs.tucker_random((47, 66, 75), (2, 5, 3), seed=6)
    res = lr.lr_poisson3d_tucker(h, *to_dev(*rhs), eps=eps)
    assert res.status == lr.LR_OK, h.last_error()
    G, Us = host(res)
    check_orthonormal(Us)
    F = T.tucker_full(*rhs)
    Xs = T.solve_full3(F)
    X = T.tucker_full(G, *Us)
    err = np.linalg.norm(X - Xs) / np.linalg.norm(Xs)
    assert err <= 10 * eps, err
    # the oracle's low-rank solve of the same right-hand side keeps ranks
    # within a few of these (its pivots may differ in near-ties)
    ref = T.lr_poisson3d(*rhs, eps)
    for k in range(3):
        assert abs(G.shape[k] - ref.G.shape[k]) <= 3, (G.shape, ref.G.shape)


@pytest.mark.parametrize("n", [256, 512, 1024])
def test_tucker3d_benchmark_sizes_on_sampled_slices(lr, h, n):
    eps = 1e-6
    rhs = inputs.smooth3d(n, eps)
    res = lr.lr_poisson3d_tucker(h, *to_dev(*rhs), eps=eps)
    assert res.status == lr.LR_OK, h.last_error()
    G, Us = host(res)
    check_orthonormal(Us)
    slices = sorted({0, 1, 2, 5, n // 7, n // 3, n // 2, n - 1})
    err = T.rel_error_freq_sampled(G, Us, *rhs, slices)
    assert err <= 10 * eps, err


def test_eigenfunction_gives_rank_one(lr, h):
    n, (a, b, c) = 64, (3, 7, 20)
    x = inputs.grid(n)
    s = [np.sin(q * np.pi * x)[:, None] for q in (a, b, c)]
    res = lr.lr_poisson3d_tucker(h, *to_dev(np.ones((1, 1, 1)), *s), eps=1e-10)
    assert res.status == lr.LR_OK, h.last_error()
    G, Us = host(res)
    assert G.shape == (1, 1, 1)
    lam = sum(4.0 * (n + 1) ** 2 * np.sin(q * np.pi / (2 * (n + 1))) ** 2 for q in (a, b, c))
    X = T.tucker_full(G, *Us)
    ref = np.einsum("i,j,k->ijk", s[0][:, 0], s[1][:, 0], s[2][:, 0]) / lam
    assert np.linalg.norm(X - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("n", [(1, 1, 1), (2, 3, 5), (7, 1, 4)])
def test_tiny_and_degenerate_grids(lr, h, n):
    rhs = inputs.tucker_random(n, (1, 1, 1), seed=2)
    res = lr.lr_poisson3d_tucker(h, *to_dev(*rhs), eps=1e-10)
    assert res.status == lr.LR_OK, h.last_error()
    G, Us = host(res)
    F = T.tucker_full(*rhs)
    Xs = T.solve_full3(F)
    X = T.tucker_full(G, *Us)
    assert np.linalg.norm(X - Xs) <= 1e-9 * np.linalg.norm(Xs)


def test_zero_rhs_gives_rank_zero(lr, h):
    G, U1, U2, U3 = inputs.tucker_random(20, 2, seed=1)
    res = lr.lr_poisson3d_tucker(h, *to_dev(np.zeros_like(G), U1, U2, U3), eps=1e-6)
    assert res.status == lr.LR_OK, h.last_error()
    assert tuple(res.G.shape) == (0, 0, 0) and all(U.shape[1] == 0 for U in res.U)


def test_repeated_runs_are_bitwise_identical(lr, h):
    rhs = inputs.smooth3d(96, 1e-8)
    d = to_dev(*rhs)
    a = host(lr.lr_poisson3d_tucker(h, *d, eps=1e-8))
    b = host(lr.lr_poisson3d_tucker(h, *d, eps=1e-8))
    assert np.array_equal(a[0], b[0]) and all(np.array_equal(x, y) for x, y in zip(a[1], b[1]))


def test_invalid_arguments_are_rejected(lr, h):
    lib = lr.load()
    G, U1, U2, U3 = to_dev(*inputs.tucker_random(16, 2, seed=1))
    outs = [lr.colmajor_empty(16, 16, "cuda") for _ in range(3)]
    Go = torch.empty(16 ** 3, dtype=torch.float64, device="cuda")

    def call(mut=None, prec="fp64"):
        rhs, sol = lr.LrTucker(), lr.LrTucker()
        for k, U in enumerate((U1, U2, U3)):
            rhs.n[k] = 16; rhs.r[k] = 2; rhs.rmax[k] = 2; rhs.ld[k] = 16; rhs.U[k] = U.data_ptr()
            sol.n[k] = 16; sol.rmax[k] = 16; sol.ld[k] = 16; sol.U[k] = outs[k].data_ptr()
        rhs.G = G.data_ptr()
        sol.G = Go.data_ptr()
        if mut:
            mut(rhs, sol)
        o = lr._options(1e-6, prec, "5pt", 64, 1.0, 16, 0, 0, 0)
        return lib.lr_poisson3d_tucker(h.ptr, ctypes.byref(rhs), ctypes.byref(sol), ctypes.byref(o))

    assert call() == lr.LR_OK
    assert call(prec="mixed") == lr.LR_OK
    assert call(prec=7) == lr.LR_EINVAL
    assert call(lambda r, s: r.r.__setitem__(0, 0)) == lr.LR_EINVAL
    assert call(lambda r, s: r.r.__setitem__(1, 65)) == lr.LR_EINVAL
    assert call(lambda r, s: r.n.__setitem__(2, 0)) == lr.LR_EINVAL
    assert call(lambda r, s: s.n.__setitem__(0, 15)) == lr.LR_EINVAL
    assert call(lambda r, s: r.ld.__setitem__(0, 15)) == lr.LR_EINVAL
    assert call(lambda r, s: s.rmax.__setitem__(2, 0)) == lr.LR_EINVAL
    assert call(lambda r, s: setattr(r, "G", None)) == lr.LR_EINVAL


@pytest.mark.parametrize("case", ["smooth48", "random40", "uneven", "smooth128"])
def test_tucker3d_mixed_matches_the_full_solve(lr, h, case):
    # float32 transforms and float32 Jacobi in the HOSVD cores, eps = 1e-6
    eps = 1e-6
    if case == "smooth48":
        rhs = inputs.smooth3d(48, eps)
    elif case == "smooth128":
        rhs = inputs.smooth3d(128, eps)
    elif case == "random40":
        rhs = inputs.tucker_random(40, 6, seed=5)
    else:
        rhs = inputs.tucker_random((47, 66, 75), (2, 5, 3), seed=6)
    res = lr.lr_poisson3d_tucker(h, *to_dev(*rhs), eps=eps, prec="mixed")
    assert res.status == lr.LR_OK, h.last_error()
    G, Us = host(res)
    for U in Us:
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 1e-5
    F = T.tucker_full(*rhs)
    Xs = T.solve_full3(F)
    X = T.tucker_full(G, *Us)
    err = np.linalg.norm(X - Xs) / np.linalg.norm(Xs)
    assert err <= 10 * eps, err


def test_tucker3d_mixed_rejects_tight_eps(lr, h):
    with pytest.raises(lr.LrError):
        lr.lr_poisson3d_tucker(h, *to_dev(*inputs.tucker_random(16, 2, seed=1)), eps=1e-9, prec="mixed")
