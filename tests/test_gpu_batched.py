"""Batched solves (many independent right-hand sides of uneven size and rank)
and CUDA-graph replay, through the C ABI, against single solves and the
CPU oracle."""
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


def npy(t):
    return t.detach().cpu().numpy()


def _problems(count, n_lo, n_hi, r_hi, seed):
    out = []
    for n, r, s in inputs.batch_problems(count, n_lo, n_hi, r_hi, seed):
        U, V = inputs.separable_random(n, r, s)
        out.append((U, V))
    return out


@pytest.mark.parametrize("prec,eps", [("mixed", 1e-6), ("fp64", 1e-9)])
def test_batched_equals_single_solves_and_oracle(lr, h, prec, eps):
    probs = _problems(20, 300, 3000, 32, seed=3)
    batch = lr.Batch([(torch.from_numpy(U), torch.from_numpy(V)) for U, V in probs])
    st = lr.lr_poisson2d_batched(h, batch, eps=eps, prec=prec)
    torch.cuda.synchronize()
    assert st == lr.LR_OK and all(s == lr.LR_OK for s in batch.status)
    for i, (U, V) in enumerate(probs):
        Ub, sb, Vb = (npy(t) for t in batch.result(i))
        # the batch gives each cross about 2048 indices per CTA; with that
        # cluster size a single solve runs the same kernels on the same
        # shapes, hence gives bitwise the same result
        cs = max(1, min(16, (U.shape[0] + 2047) // 2048))
        single = lr.lr_poisson2d(h, torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda(), eps=eps, prec=prec,
                                 cluster_size=cs)
        torch.cuda.synchronize()
        assert np.array_equal(Ub, npy(single.U)) and np.array_equal(sb, npy(single.s))
        assert O.rel_error_freq(Ub, sb, Vb, U, V, "5pt") <= 10 * eps


def test_batched_graph_replay_tracks_new_data(lr, h):
    probs = _problems(12, 512, 2048, 16, seed=11)
    batch = lr.Batch([(torch.from_numpy(U), torch.from_numpy(V)) for U, V in probs])
    for rep in range(3):
        if rep == 2:  # new right-hand sides in the same device buffers
            for (U, V), (Ud, Vd) in zip(probs, batch.rhs):
                Ud.mul_(-2.0)
        st = lr.lr_poisson2d_batched(h, batch, eps=1e-6, prec="mixed", graph=True)
        torch.cuda.synchronize()
        assert st == lr.LR_OK
        for i, (U, V) in enumerate(probs):
            Ub, sb, Vb = (npy(t) for t in batch.result(i))
            scale = -2.0 if rep == 2 else 1.0
            assert O.rel_error_freq(Ub, sb, Vb, scale * U, V, "5pt") <= 1e-5


def test_single_solve_graph_replay(lr, h):
    m, eps = 4096, 1e-6
    U, V = inputs.smooth_sum(m, eps)
    Ud, Vd = torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda()
    out = (lr.colmajor_empty(m, 64), torch.empty(64, dtype=torch.float64, device="cuda"), lr.colmajor_empty(m, 64))
    ref = lr.lr_poisson2d(h, Ud, Vd, eps=eps, prec="mixed")
    for _ in range(3):
        res = lr.lr_poisson2d(h, Ud, Vd, eps=eps, prec="mixed", graph=True, out=out)
        torch.cuda.synchronize()
        assert res.status == lr.LR_OK
        assert np.array_equal(npy(res.U), npy(ref.U)) and np.array_equal(npy(res.s), npy(ref.s))


def test_batch_of_uneven_log_uniform_problems_converges(lr, h):
    # the 512-problem batch recipe, scaled to 64 problems for test time:
    # n log-uniform in [512, 16384], r uniform in {1..32}, eps = 1e-6
    probs = _problems(64, 512, 16384, 32, seed=3)
    batch = lr.Batch([(torch.from_numpy(U), torch.from_numpy(V)) for U, V in probs])
    st = lr.lr_poisson2d_batched(h, batch, eps=1e-6, prec="mixed", graph=True)
    torch.cuda.synchronize()
    assert st == lr.LR_OK
    assert all(s == lr.LR_OK for s in batch.status)
    for i in range(64):
        U, V = probs[i]
        Ub, sb, Vb = (npy(t) for t in batch.result(i))
        rows = np.unique(np.linspace(0, U.shape[0] - 1, 128).astype(int))
        assert O.rel_error_freq(Ub, sb, Vb, U, V, "5pt", rows=rows) <= 1e-5, i


# ------------------------------------------------------------------ autotuning (tuned-shape lookup, tiles, cluster sizes)
def test_autotune_single_then_lookup(lr, h):
    m, eps = 16384, 1e-6
    U, V = inputs.smooth_sum(m, eps)
    Ud, Vd = torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda()
    t = lr.lr_autotune(h, Ud, Vd, eps=eps, prec="mixed", reps=3)
    assert 1 <= t["cluster_size"] <= 16 and t["log_tile"] in (0, 10, 11, 12) and t["transform"] in (0, 1)
    assert t["candidates"] >= 2 and 0 < t["ms_best"] <= t["ms_default"] * 1.0001
    # a solve with cluster_size 0 now uses the tuned size, and gives bitwise
    # the result of an explicit solve with that size
    a = lr.lr_poisson2d(h, Ud, Vd, eps=eps, prec="mixed")
    assert a.info.cluster_size == t["cluster_size"]
    b = lr.lr_poisson2d(h, Ud, Vd, eps=eps, prec="mixed", cluster_size=t["cluster_size"])
    assert np.array_equal(npy(a.U), npy(b.U)) and np.array_equal(npy(a.s), npy(b.s))
    rows = np.unique(np.linspace(0, m - 1, 256).astype(int))
    assert O.rel_error_freq(npy(a.U), npy(a.s), npy(a.V), U, V, "5pt", rows=rows) <= 10 * eps


def test_autotune_batched(lr, h):
    probs = _problems(16, 512, 4096, 16, seed=5)
    batch = lr.Batch([(torch.from_numpy(U), torch.from_numpy(V)) for U, V in probs])
    t = lr.lr_autotune_batched(h, batch, eps=1e-6, prec="mixed", reps=2)
    assert t["batch_indices_per_cta"] in (1024, 2048, 4096, 8192) and t["candidates"] == 4
    st = lr.lr_poisson2d_batched(h, batch, eps=1e-6, prec="mixed")
    torch.cuda.synchronize()
    assert st == lr.LR_OK
    for i, (U, V) in enumerate(probs):
        Ub, sb, Vb = (npy(x) for x in batch.result(i))
        assert O.rel_error_freq(Ub, sb, Vb, U, V, "5pt") <= 1e-5
