"""Maxvol row selection (lr_maxvol) through the C ABI against the CPU oracle:
seeded Gaussian matrices from one row to several grid strides of rows and
k = 1..64, the cross skeletons of the low-rank solve (starting from the ACA
row pivots) at n = 1024 and at the benchmark's n = 16384, the swap cap, and
the error statuses.

Where every decision of the oracle is clear of a tie (largest against
runner-up, and against 1 + delta, by a relative 1e-9), the rows and the swap
count must be identical; otherwise both results must be (1 + delta)-dominant
by a fresh solve."""
import numpy as np
import pytest

from oracle import maxvol as M
from oracle import poisson_lowrank as O
from paper_1306_2150_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MARGIN = 1e-9


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


def _gauss(m, k, seed):
    return inputs.normal(seed, m * k).reshape(k, m).T.copy()


def _dev(lr, C):
    out = lr.colmajor_empty(C.shape[0], C.shape[1])
    out.copy_(torch.from_numpy(C))
    return out


def _clear_of_ties(log, delta, maxswaps):
    for q, (_, _, big, second, outside) in enumerate(log):
        last = q == len(log) - 1
        if not last or big > 1.0 + delta:
            if q < maxswaps and not (big > (1.0 + delta) * (1 + MARGIN) and big - second > MARGIN * big):
                return False
        else:
            if not outside < (1.0 + delta) * (1 - MARGIN):
                return False
    return True


def _check(lr, h, C, rows0, delta, maxswaps):
    ro, no, bo, log = M.maxvol(C, rows0, delta, maxswaps, trace=True)
    rg, ng, bg, st = lr.lr_maxvol(h, _dev(lr, C), rows0, delta, maxswaps)
    torch.cuda.synchronize()
    capped = bo > 1.0 + delta
    assert st == (lr.LR_ENOCONV if capped else lr.LR_OK)
    assert sorted(set(rg)) == sorted(rg) and all(0 <= r < C.shape[0] for r in rg)
    if _clear_of_ties(log, delta, maxswaps):
        assert rg == ro and ng == no
        assert bg == pytest.approx(bo, rel=1e-10, abs=1e-12)
    if not capped:
        Bg = M.coefficients(C, rg)
        assert np.abs(Bg).max() <= (1.0 + delta) * (1 + 1e-9)
    return ro, no


@pytest.mark.parametrize("m,k,delta,seed", [
    (1, 1, 0.0, 1), (7, 1, 0.0, 2), (37, 5, 0.0, 3), (1000, 7, 1e-2, 4), (4099, 16, 1e-2, 5),
    (20000, 64, 5e-2, 6), (100003, 9, 1e-2, 7), (257, 33, 0.0, 8)])
def test_gaussian_matches_oracle(lr, h, m, k, delta, seed):
    C = _gauss(m, k, seed)
    _, nswaps = _check(lr, h, C, list(range(k)), delta, 16 * k)
    if m > 2 * k:
        assert nswaps > 0


def test_start_rows_anywhere(lr, h):
    C = _gauss(3000, 12, 9)
    rows0 = [2999, 5, 1500, 77, 2000, 1, 640, 641, 1200, 2500, 30, 900]
    _check(lr, h, C, rows0, 1e-2, 200)


@pytest.mark.parametrize("n", [1024, 16384])
def test_cross_skeleton_from_aca_pivots(lr, h, n):
    # the columns of the cross of Section 4.2 for the smooth right-hand side,
    # row pivots refined from those the ACA chose
    U, V = inputs.smooth_sum(n, 1e-6)
    _, _, _, info = O.lr_poisson2d(U, V, "5pt", 1e-6)
    cr = info.cross
    C = np.ascontiguousarray(cr.C)
    for delta in (1e-2, 0.0):
        rows, nswaps = _check(lr, h, C, list(cr.I), delta, 200)
        vol0 = abs(np.linalg.det(C[list(cr.I), :]))
        assert abs(np.linalg.det(C[rows, :])) >= vol0 * (1 - 1e-12)


def test_swap_cap(lr, h):
    C = _gauss(5000, 10, 10)
    ro, no, bo = M.maxvol(C, list(range(10)), 0.0, 3)
    assert no == 3 and bo > 1.0
    rg, ng, bg, st = lr.lr_maxvol(h, _dev(lr, C), list(range(10)), 0.0, 3)
    assert st == lr.LR_ENOCONV and ng == 3 and rg == ro
    rg, ng, bg, st = lr.lr_maxvol(h, _dev(lr, C), list(range(10)), 0.0, 0)
    assert st == lr.LR_ENOCONV and ng == 0 and rg == list(range(10))
    assert bg == pytest.approx(np.abs(M.coefficients(C, range(10))).max(), rel=1e-10)


def test_error_statuses(lr, h):
    C = _gauss(200, 4, 11)
    with pytest.raises(lr.LrError) as e:
        lr.lr_maxvol(h, _dev(lr, C), [0, 1, 2, 2], 1e-2)
    assert e.value.status == lr.LR_EINVAL
    with pytest.raises(lr.LrError) as e:
        lr.lr_maxvol(h, _dev(lr, C), [0, 1, 2, 200], 1e-2)
    assert e.value.status == lr.LR_EINVAL
    Cs = C.copy()
    Cs[3] = 0.0  # C[[0, 1, 2, 3], :] singular: a zero row stays exactly zero under elimination
    with pytest.raises(lr.LrError) as e:
        lr.lr_maxvol(h, _dev(lr, Cs), [0, 1, 2, 3], 1e-2)
    assert e.value.status == lr.LR_EINVAL
    Cn = C.copy()
    Cn[50, 2] = np.nan
    with pytest.raises(lr.LrError) as e:
        lr.lr_maxvol(h, _dev(lr, Cn), [0, 1, 2, 3], 1e-2)
    assert e.value.status == lr.LR_ENONFINITE
    big = _gauss(100, 65, 12)
    with pytest.raises(lr.LrError) as e:
        lr.lr_maxvol(h, _dev(lr, big), list(range(65)), 1e-2)
    assert e.value.status == lr.LR_EINVAL
    # the handle stays usable after every error
    rg, ng, bg, st = lr.lr_maxvol(h, _dev(lr, C), [0, 1, 2, 3], 1e-2)
    assert st == lr.LR_OK
