"""The multi-rank (replica) path of bench.py on CPU: two gloo ranks combine
their timings by a max over ranks and count every rank's solves; the
reference arm runs on rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    res = {"mixed": {"ms": 1.0 + rank}, "fp64": {"ms": 5.0 - rank}, "batch_mixed": {"ms_step": 3.0 + 2 * rank, "batch": 64},
           "batch_fp64": {"ms_step": 9.0}, "e2e_batch": {"ms_step": 4.0 + rank, "batch": 64}}
    bench.combine_ranks(res, world, "cpu")
    out.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_count_all_solves():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29517
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        res = got[r]
        assert res["mixed"]["ms"] == 2.0 and res["fp64"]["ms"] == 5.0
        assert res["batch_mixed"]["ms_step"] == 5.0 and res["e2e_batch"]["ms_step"] == 5.0
        assert res["batch_mixed"]["batch"] == 128 and res["e2e_batch"]["batch"] == 128


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                         capture_output=True, text=True, env=env, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_reference_arm_prints_the_oracle_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--n", "1024", "--cpu-seconds", "1"],
                         capture_output=True, text=True, env=env, timeout=300)
    assert out.returncode == 0, out.stderr[-500:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
