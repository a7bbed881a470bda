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
    # the stream form: each problem is the single-solve launch chain
    probs = _problems(20, 300, 3000, 32, seed=3)
    batch = lr.Batch([(torch.from_numpy(U), torch.from_numpy(V)) for U, V in probs])
    st = lr.lr_poisson2d_batched(h, batch, eps=eps, prec=prec, streams=True)
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


@pytest.mark.parametrize("prec,eps", [("mixed", 1e-6), ("fp64", 1e-9), ("fp64", 1e-6)])
def test_phased_batch_matches_oracle(lr, h, prec, eps):
    # the phase-batched form on uneven problems: small-path (M <= 4096) and
    # four-step transforms, single-CTA and clustered crosses (4096 indices per
    # CTA by default: m > 4096 takes 2 or more CTAs).  Mixed: every problem within
    # 10 eps of the exact solution.  Float64: the oracle's rank and singular
    # values, and its error (the cross stop rule at tol = eps leaves some of
    # these random problems slightly above 10 eps at eps = 1e-9, in the
    # oracle as on the GPU)
    probs = _problems(24, 300, 12000, 32, seed=13)
    batch = lr.Batch([(torch.from_numpy(U), torch.from_numpy(V)) for U, V in probs])
    st = lr.lr_poisson2d_batched(h, batch, eps=eps, prec=prec)
    torch.cuda.synchronize()
    assert st == lr.LR_OK and all(s == lr.LR_OK for s in batch.status)
    info, _, _ = lr.lr_get_info(h)
    assert info.launches <= 16  # 4 + 4 transform launches, <= 5 cluster-size groups, 3 rounding
    for i, (U, V) in enumerate(probs):
        Ub, sb, Vb = (npy(t) for t in batch.result(i))
        rows = None if U.shape[0] <= 4096 else np.unique(np.linspace(0, U.shape[0] - 1, 256).astype(int))
        err = O.rel_error_freq(Ub, sb, Vb, U, V, "5pt", rows=rows)
        if prec == "mixed":
            assert err <= 10 * eps, i
            continue
        ou, os_, ov, inf = O.lr_poisson2d(U, V, "5pt", eps)
        assert len(sb) == inf.rank, i
        assert np.allclose(sb, os_, rtol=1e-8, atol=1e-11 * os_[0]), i
        assert err <= max(10 * eps, 1.1 * O.rel_error_freq(ou, os_, ov, U, V, "5pt", rows=rows)), i


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_phased_batch_probe_restart_and_edge_problems(lr, h, prec):
    # a block-diagonal problem whose second block only a residual probe finds
    # (Section 4.2, reading G7), an eigenfunction (zero rows), tiny grids and
    # a zero right-hand side, in one batch; float64 ranks equal the oracle's
    eps = 1e-6
    Uh, Vh = inputs.block_diagonal_freq(128, 32)
    x = np.arange(1, 31) / 31
    probs = [(O.dst1(Uh), O.dst1(Vh)),
             (np.sin(3 * np.pi * x)[:, None], (np.sin(np.pi * x) + 0.3 * np.sin(2 * np.pi * x))[:, None]),
             inputs.separable_random(1, 1, seed=1), inputs.separable_random(2, 2, seed=2),
             inputs.separable_random(5, 3, seed=5), (np.zeros((64, 2)), np.ones((64, 2))),
             inputs.separable_random(4097, 7, seed=9)]
    probs = [(np.asfortranarray(a), np.asfortranarray(b)) for a, b in probs]
    batch = lr.Batch([(torch.from_numpy(a), torch.from_numpy(b)) for a, b in probs])
    lr.lr_poisson2d_batched(h, batch, eps=eps, prec=prec, check=False)
    torch.cuda.synchronize()
    for i, (U, V) in enumerate(probs):
        Ub, sb, Vb = (npy(t) for t in batch.result(i))
        if not U.any():
            assert len(sb) == 0 and batch.status[i] == lr.LR_OK
            continue
        assert batch.status[i] == lr.LR_OK, i
        assert O.rel_error_freq(Ub, sb, Vb, U, V, "5pt") <= 10 * eps, i
        if prec == "fp64":
            assert len(sb) == O.lr_poisson2d(U, V, "5pt", eps)[3].rank, i


def test_phased_batch_one_pass_transform_long_orders(lr, h):
    # float32 batches with enough columns take the one-pass transform: orders
    # with M = 2^13 (two columns per CTA), 2^14 and 2^15 (one and two residue
    # classes) and M = 2^16, 2^17 (four and eight residues, inputs folded);
    # every problem within 10 eps on sampled rows
    eps = 1e-6
    ms = [2500, 4097, 9000, 16385, 20000, 40000, 65536]
    probs = [inputs.separable_random(m, 6, seed=40 + i) for i, m in enumerate(ms)]
    probs.append((np.zeros((9000, 2), order="F"), np.ones((9000, 2), order="F")))  # rank 0: no live column
    batch = lr.Batch([(torch.from_numpy(U), torch.from_numpy(V)) for U, V in probs])
    st = lr.lr_poisson2d_batched(h, batch, eps=eps, prec="mixed")
    torch.cuda.synchronize()
    assert st == lr.LR_OK and all(s == lr.LR_OK for s in batch.status)
    assert batch.c_sol[len(probs) - 1].r == 0
    for i, (U, V) in enumerate(probs[:-1]):
        Ub, sb, Vb = (npy(t) for t in batch.result(i))
        rows = np.unique(np.linspace(0, U.shape[0] - 1, 128).astype(int))
        assert O.rel_error_freq(Ub, sb, Vb, U, V, "5pt", rows=rows) <= 10 * eps, (i, ms[i])


def test_phased_batch_one_pass_transform_semistaggered(lr, h):
    # the semi-staggered operator (reading G1) through the one-pass transform
    # and the register-resident cross, mixed, every problem within 10 eps
    eps = 1e-6
    probs = [inputs.separable_random(m, 8, seed=60 + i) for i, m in enumerate([5000, 7000, 12000, 16383, 4500])]
    batch = lr.Batch([(torch.from_numpy(U), torch.from_numpy(V)) for U, V in probs])
    st = lr.lr_poisson2d_batched(h, batch, eps=eps, prec="mixed", op="semi")
    torch.cuda.synchronize()
    assert st == lr.LR_OK
    for i, (U, V) in enumerate(probs):
        Ub, sb, Vb = (npy(t) for t in batch.result(i))
        rows = np.unique(np.linspace(0, U.shape[0] - 1, 128).astype(int))
        assert O.rel_error_freq(Ub, sb, Vb, U, V, "semi", rows=rows) <= 10 * eps, i


def test_phased_batch_headline_shape(lr, h):
    # the benchmark's shape: m = 16384 smooth right-hand sides (4 CTAs per
    # problem at the default 4096 indices per CTA), mixed precision, graph
    m, eps = 16384, 1e-6
    U, V = inputs.smooth_sum(m, eps)
    probs = [(U * (1.0 + p / 8), V) for p in range(8)]
    batch = lr.Batch([(torch.from_numpy(np.asfortranarray(a)), torch.from_numpy(b)) for a, b in probs])
    for _ in range(2):
        st = lr.lr_poisson2d_batched(h, batch, eps=eps, prec="mixed", graph=True)
        torch.cuda.synchronize()
        assert st == lr.LR_OK
    rows = np.unique(np.linspace(0, m - 1, 192).astype(int))
    for i, (a, b) in enumerate(probs):
        Ub, sb, Vb = (npy(t) for t in batch.result(i))
        assert O.rel_error_freq(Ub, sb, Vb, a, b, "5pt", rows=rows) <= 10 * eps, i


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


@pytest.mark.parametrize("streams", [False, True])
def test_batch_of_uneven_log_uniform_problems_converges(lr, h, streams):
    # the 512-problem batch recipe, scaled to 64 problems for test time:
    # n log-uniform in [512, 16384], r uniform in {1..32}, eps = 1e-6
    probs = _problems(64, 512, 16384, 32, seed=3)
    batch = lr.Batch([(torch.from_numpy(U), torch.from_numpy(V)) for U, V in probs])
    st = lr.lr_poisson2d_batched(h, batch, eps=1e-6, prec="mixed", graph=True, streams=streams)
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


@pytest.mark.parametrize("streams", [False, True])
def test_autotune_batched(lr, h, streams):
    probs = _problems(16, 512, 4096, 16, seed=5)
    batch = lr.Batch([(torch.from_numpy(U), torch.from_numpy(V)) for U, V in probs])
    t = lr.lr_autotune_batched(h, batch, eps=1e-6, prec="mixed", reps=2, streams=streams)
    allowed = (1024, 2048, 4096, 8192) if streams else (2048, 4096, 8192, 16384)
    assert t["batch_indices_per_cta"] in allowed and t["candidates"] == 4
    st = lr.lr_poisson2d_batched(h, batch, eps=1e-6, prec="mixed", streams=streams)
    torch.cuda.synchronize()
    assert st == lr.LR_OK
    for i, (U, V) in enumerate(probs):
        Ub, sb, Vb = (npy(x) for x in batch.result(i))
        assert O.rel_error_freq(Ub, sb, Vb, U, V, "5pt") <= 1e-5


def test_async_batch_then_status(lr, h):
    # LR_FLAG_ASYNC: the call returns before the stream finishes; after a
    # synchronisation lr_batched_status gives the ranks and statuses the
    # synchronous call reports, and the factors equal the synchronous ones
    probs = _problems(10, 300, 6000, 12, seed=21)
    sync_b = lr.Batch([(torch.from_numpy(U), torch.from_numpy(V)) for U, V in probs])
    async_b = lr.Batch([(torch.from_numpy(U), torch.from_numpy(V)) for U, V in probs])
    assert lr.lr_poisson2d_batched(h, sync_b, eps=1e-6, prec="mixed") == lr.LR_OK
    assert lr.lr_poisson2d_batched(h, async_b, eps=1e-6, prec="mixed", async_=True) == lr.LR_OK
    torch.cuda.synchronize()
    assert lr.lr_batched_status(h, async_b) == lr.LR_OK
    for i in range(len(probs)):
        assert async_b.c_sol[i].r == sync_b.c_sol[i].r > 0 and async_b.status[i] == lr.LR_OK
        for a, b in zip(async_b.result(i), sync_b.result(i)):
            assert torch.equal(a, b)
    # a larger batch than the last call is rejected
    big = lr.Batch([(torch.from_numpy(U), torch.from_numpy(V)) for U, V in probs + probs[:1]])
    assert lr.lr_batched_status(h, big, check=False) == lr.LR_EINVAL
