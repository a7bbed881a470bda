"""lr_truncate_noalloc: the rounding without any allocation, for callers that
cannot call cudaMalloc (code inside another framework's memory pool, or
latency-critical loops where cudaMalloc may stall and cudaFree synchronises
the device).  It must give the results of lr_truncate, call after call, even
though every call reuses the same static scratch array.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lr():
    from paper_1306_2150_gb300 import build, lr as lrmod
    build.build()
    lrmod.load()
    return lrmod


def _noalloc(lr, U, s, V, eps, rmax):
    """Call lr_truncate_noalloc through the C ABI on copies of the inputs."""
    n1, r = U.shape
    n2 = V.shape[0]
    ld = max(n1, n2)
    ld += ld & 1
    Uw = torch.zeros((r, ld), dtype=torch.float64, device="cuda")
    Vw = torch.zeros((r, ld), dtype=torch.float64, device="cuda")
    Uw[:, :n1].copy_(torch.from_numpy(U.T.copy()))
    Vw[:, :n2].copy_(torch.from_numpy(V.T.copy()))
    sw = torch.from_numpy(s.copy()).cuda()
    X = lr.LrMat(n1, n2, r, r, ld, Uw.data_ptr(), sw.data_ptr(), Vw.data_ptr())
    stream = torch.cuda.current_stream().cuda_stream
    st = lr.load().lr_truncate_noalloc(ctypes.byref(X), float(eps), int(rmax), ctypes.c_void_p(stream))
    R = X.r
    return st, Uw[:R, :n1].cpu().numpy().T, sw[:R].cpu().numpy(), Vw[:R, :n2].cpu().numpy().T


def _problem(seed, n1, n2, k):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((n1, k)) * (10.0 ** -np.linspace(0, 9, k))
    V = rng.standard_normal((n2, k))
    s = rng.uniform(0.5, 2.0, k)
    return U, s, V


def test_noalloc_truncate_matches_lr_truncate_twice(lr):
    h = lr.Handle()
    try:
        # two calls in a row on different shapes: the second must not see
        # anything the first left in the shared scratch
        for seed, (n1, n2, k, eps) in enumerate([(700, 530, 14, 1e-7), (3000, 2900, 40, 1e-10)]):
            U, s, V = _problem(seed, n1, n2, k)
            st, Un, sn, Vn = _noalloc(lr, U, s, V, eps, 64)
            Ue, se, Ve, ste = lr.lr_truncate(h, torch.from_numpy(U).cuda(), torch.from_numpy(s).cuda(),
                                             torch.from_numpy(V).cuda(), eps)
            torch.cuda.synchronize()
            assert st == lr.LR_OK and ste == lr.LR_OK
            Ue, se, Ve = Ue.cpu().numpy(), se.cpu().numpy(), Ve.cpu().numpy()
            assert len(sn) == len(se)
            assert np.allclose(sn, se, rtol=1e-10, atol=0)
            Xn = (Un * sn) @ Vn.T
            Xe = (Ue * se) @ Ve.T
            assert np.linalg.norm(Xn - Xe) <= 1e-12 * np.linalg.norm(Xe)
            assert np.abs(Un.T @ Un - np.eye(len(sn))).max() < 1e-10
    finally:
        h.close()


def test_noalloc_truncate_matches_oracle(lr):
    # Against the oracle's rounding (Section 3: QR of both factors, SVD of the
    # core, truncation at eps): the kept rank may differ by one where a
    # singular value sits at the cutoff; the singular values agree to 1e-10 of
    # the largest and the rounded matrices to the truncation tolerance.
    from oracle import poisson_lowrank as O
    for seed, (n1, n2, k, eps) in enumerate([(700, 530, 14, 1e-7), (3000, 2900, 40, 1e-10), (129, 65, 64, 1e-6)]):
        U, s, V = _problem(10 + seed, n1, n2, k)
        st, Un, sn, Vn = _noalloc(lr, U, s, V, eps, 64)
        Uo, so, Vo, ok = O.lr_truncate(U, s, V, eps, 64)
        assert st == lr.LR_OK and ok
        assert abs(len(sn) - len(so)) <= 1
        q = min(len(sn), len(so))
        assert np.abs(sn[:q] - so[:q]).max() <= 1e-10 * so[0]
        Xn = (Un * sn) @ Vn.T
        Xo = (Uo * so) @ Vo.T
        assert np.linalg.norm(Xn - Xo) <= 10 * eps * np.linalg.norm(Xo)


def test_noalloc_cut_to_rmax(lr):
    # more columns needed than rmax: LR_ENOCONV with the leading rmax kept
    from oracle import poisson_lowrank as O
    U, s, V = _problem(3, 500, 400, 12)
    st, Un, sn, Vn = _noalloc(lr, U, s, V, 1e-12, 5)
    Uo, so, Vo, ok = O.lr_truncate(U, s, V, 1e-12, 5)
    assert st == lr.LR_ENOCONV and not ok
    assert len(sn) == 5
    assert np.abs(sn - so).max() <= 1e-10 * so[0]


def test_noalloc_rejects_rank_beyond_static_limit(lr):
    U, s, V = _problem(5, 200, 200, 65)
    st, *_ = _noalloc(lr, U, s, V, 1e-6, 64)
    assert st == lr.LR_EINVAL
