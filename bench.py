"""Benchmark: ms per 2D low-rank Poisson solve (n = 16384, eps = 1e-6).

A solve is the full low-rank solve (forward DST of the factors, cross
approximation in frequency space, rounding, inverse DST) of the 5-point
Dirichlet Poisson problem on a 16384 x 16384 interior grid, right-hand side
f = 1/(1+x+y) + 0.5 sin(3 pi x) exp(-2y) in factored form compressed to eps.

One step = one batch of --batch independent solves of that problem (each with
its own right-hand side and output buffers), run by lr_poisson2d_batched in
mixed precision as one replayed CUDA graph; the headline value is whole-job
throughput, step time / batch, in ms per solve.  The single-solve latency of
the mixed and the float64 paths is measured in the same run (with per-phase
CUDA events).  Inputs are resident on the device; L2 is flushed (a 512 MiB
write) between timed steps, outside the timed events.

--impl reference times the CPU FP64 oracle on the host cores (the reference
arm of this benchmark).  With torchrun (N > 1) every rank runs independent
replicas of the solve (the single solve does not shard); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 16384
EPS = 1e-6
EPS_TIGHT = 1e-10
METRIC = "ms per 2D low-rank Poisson solve (n=16384, eps=1e-6), mixed vs FP64; % roofline"
WORKLOAD = "lowrank_poisson2d_5pt_n16384_eps1e-6_smooth_rhs"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=N_GRID)
    p.add_argument("--batch", type=int, default=64)
    p.add_argument("--batch-sweep", type=int, nargs="*", default=[16, 72, 152],
                   help="other batch sizes of the mixed batched step (ms per solve, context)")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--crossover", type=int, nargs="*", default=[256, 1024, 4096, 16384],
                   help="grid sizes of the full-grid vs low-rank comparison")
    p.add_argument("--expsum", type=int, nargs="*", default=[1024, 16384],
                   help="grid sizes of the exponential-sum vs cross comparison")
    p.add_argument("--maxvol", type=int, nargs="*", default=[16, 64],
                   help="ranks k of the maxvol row selection timed at m = n (none: skip)")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the untuned launch shapes (for profiler runs, whose per-launch overhead "
                        "would skew the tuner's timings)")
    p.add_argument("--stokes", type=int, nargs="*", default=[1024, 4096, 8192],
                   help="cells per direction of the low-rank Uzawa Stokes runs")
    p.add_argument("--stokes-gmres", type=int, nargs="*", default=[],
                   help="cells per direction of the Stokes runs with inexact GMRES (Section 5) besides CG")
    p.add_argument("--uneven", type=int, default=512,
                   help="problems in the uneven batch (n log-uniform in [512, 16384], r in 1..32; 0: skip)")
    p.add_argument("--tucker", type=int, nargs="*", default=[128, 256, 512, 1024],
                   help="grid sizes of the 3D Tucker solves (eps = 1e-6, float64)")
    p.add_argument("--sweep", type=int, nargs="*", default=[1024, 4096, 16384, 65536],
                   help="grid sizes of the single-solve sweep (eps 1e-6 and 1e-10, float64 and mixed)")
    p.add_argument("--cpu-worker", action="store_true", help=argparse.SUPPRESS)
    return p.parse_args()


# ---------------------------------------------------------------- CPU oracle
def cpu_worker(n: int, seconds: float, steps: int):
    """Time the oracle's low-rank solve; prints one JSON line."""
    import numpy as np
    from oracle import poisson_lowrank as O
    from paper_1306_2150_gb300 import inputs
    U, V = inputs.smooth_sum(n, EPS)
    times = []
    t_end = time.perf_counter() + seconds
    while len(times) < max(1, steps) or time.perf_counter() < t_end:
        t0 = time.perf_counter()
        O.lr_poisson2d(U, V, "5pt", EPS)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end and len(times) >= 1:
            break
    print(json.dumps({"ms": 1e3 * statistics.median(times), "solves": len(times),
                      "total_s": sum(times), "rank_in": U.shape[1]}))
    _ = np


def run_cpu_baseline(n: int, seconds: float, steps: int = 1) -> dict:
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[v] = "1"
    env.pop("RANK", None)
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", "--n", str(n),
                          "--cpu-seconds", str(seconds), "--steps", str(steps)],
                         capture_output=True, text=True, env=env, cwd=ROOT)
    line = [l for l in out.stdout.splitlines() if l.startswith("{")]
    if out.returncode != 0 or not line:
        return {"error": (out.stderr or out.stdout)[-300:]}
    r = json.loads(line[-1])
    return {"value": round(r["ms"], 3), "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": f"{r['solves']} oracle low-rank solves at n={n} (scipy DST-I + numpy cross "
                      f"+ numpy QR/SVD), single thread, median"}


def run_cpu_baseline_all_cores(n: int, seconds: float) -> dict:
    """The oracle's low-rank solve on every host core at once: one
    single-threaded worker process per core, each timing solves for about
    `seconds`; ms per solve = the slowest worker's wall time / all solves."""
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")  # no fork after the GPU was touched
        with cf.ProcessPoolExecutor(max_workers=cores, mp_context=ctx) as ex:
            res = list(ex.map(_cpu_all_worker, [(n, seconds)] * cores))
    except Exception as e:  # pragma: no cover
        return {"error": str(e)[-200:]}
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    solves = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return {"value": round(1e3 * wall / solves, 3), "unit": "ms", "cores": cores, "kind": "oracle",
            "sample": f"{solves} oracle low-rank solves at n={n} on {cores} worker processes "
                      f"(one single-threaded solver per core), {wall:.1f} s wall"}


def _cpu_all_worker(arg):
    n, seconds = arg
    sys.path.insert(0, ROOT)
    from oracle import poisson_lowrank as O
    from paper_1306_2150_gb300 import inputs
    U, V = inputs.smooth_sum(n, EPS)
    t0 = time.perf_counter()
    count = 0
    while count < 1 or time.perf_counter() - t0 < seconds:
        O.lr_poisson2d(U, V, "5pt", EPS)
        count += 1
    return count, time.perf_counter() - t0


def rel_error_sampled(res_U, res_s, res_V, U, V, rows: int = 256, kind: str = "5pt") -> float:
    """Relative Frobenius error of a GPU result against the exact discrete
    solution, from the oracle's Parseval evaluation on `rows` evenly spaced
    frequency rows (all rows when the grid is smaller)."""
    import numpy as np
    from oracle import poisson_lowrank as O
    Uo = res_U.detach().cpu().numpy() if hasattr(res_U, "cpu") else res_U
    so = res_s.detach().cpu().numpy() if hasattr(res_s, "cpu") else res_s
    Vo = res_V.detach().cpu().numpy() if hasattr(res_V, "cpu") else res_V
    Un = U.numpy() if hasattr(U, "numpy") else U
    Vn = V.numpy() if hasattr(V, "numpy") else V
    m = Un.shape[0]
    idx = None if m <= rows else np.unique(np.linspace(0, m - 1, rows).astype(int))
    return float(O.rel_error_freq(Uo, so, Vo, Un, Vn, kind, rows=idx))


# ---------------------------------------------------------------- clocks
class Clocks:
    """SM clock and clock-event (throttle) reasons sampled while a timed region
    runs: every 2 ms from NVML on a thread (read-only queries), else from
    nvidia-smi (100 ms).  The JSON line carries the summary; LR_BENCH_CLOCKS_DIR
    (default: the system's temporary directory) receives the raw nvidia-smi
    samples."""
    # NVML clock-event reason bits
    REASONS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.thread = None
        self.samples = []  # (sm MHz, max sm MHz, reason bits)
        self.path = os.path.join(os.environ.get("LR_BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"lr_bench_clocks_rank{index}.csv")

    def _nvml_start(self) -> bool:
        import ctypes
        import threading
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return False
            dev = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(dev)) != 0:
                return False
            reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        except Exception:
            return False
        self.stop = threading.Event()
        clk, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()

        def run():
            while not self.stop.is_set():
                if (lib.nvmlDeviceGetClockInfo(dev, 1, ctypes.byref(clk)) == 0
                        and lib.nvmlDeviceGetMaxClockInfo(dev, 1, ctypes.byref(mx)) == 0
                        and reasons_fn(dev, ctypes.byref(rs)) == 0):
                    self.samples.append((clk.value, mx.value, rs.value))
                time.sleep(0.002)

        self.thread = threading.Thread(target=run, daemon=True)
        self.thread.start()
        time.sleep(0.01)  # first sample before the region starts
        return True

    def __enter__(self):
        if self._nvml_start():
            return self
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.thread:
            self.stop.set()
            self.thread.join(timeout=5)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        if self.thread:
            if not self.samples:
                return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
            reasons = {nm for nm, bit in self.REASONS.items() if any(r & bit for _, _, r in self.samples)}
            return {"sm_mhz": statistics.median(c for c, _, _ in self.samples),
                    "sm_max_mhz": max(m for _, m, _ in self.samples), "reasons": sorted(reasons),
                    "samples": len(self.samples), "source": "nvml, 2 ms"}
        try:
            rows = [l.split(",") for l in open(self.path).read().splitlines() if l.strip()]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi, 100 ms"}


# ---------------------------------------------------------------- ncu traffic
# DRAM bytes per launch of each phase's kernel at this workload, from the
# committed ncu summaries; null once the kernel source has changed since.  The
# source hash covers the kernel's whole translation unit: the .cu file and the
# headers it includes, in this order, concatenated.
BATCH_TU = ["paper_1306_2150_gb300/csrc/" + f for f in
            ("batch.cu", "fft_common.cuh", "fft_inplace.cuh", "lr_internal.h", "lr_common.cuh")]
TRAFFIC_FILES = {
    "cross": ("profiles/batch_cross_f32_n16384_b64.md", BATCH_TU),
    "forward_dst": ("profiles/batch_dst_forward_f32_n16384_b64.md", BATCH_TU),
    "inverse_dst": ("profiles/batch_dst_inverse_f32_n16384_b64.md", BATCH_TU),
    "rounding": ("profiles/batch_rounding_f32_n16384_b64.md", BATCH_TU),
}


def source_hash(files) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(phase: str):
    import re
    ent = TRAFFIC_FILES.get(phase)
    if not ent:
        return None
    try:
        text = open(os.path.join(ROOT, ent[0])).read()
        src = source_hash(ent[1])
    except OSError:
        return None
    mb = re.search(r"dram_bytes_per_launch:\s*([0-9]+)", text)
    mh = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    if not mb or not mh or mh.group(1) != src:
        return None
    return int(mb.group(1))


# ---------------------------------------------------------------- GPU arm
def algorithmic_bytes(n: int, r: int, k: int, R: int, w: int) -> dict:
    """Bytes each phase must move at minimum (inputs read once, outputs written
    once; no scratch): forward DST reads U, V (float64) and writes Uh, Vh (w);
    the cross reads Uh, Vh and writes the k-column skeleton C, R; the inverse
    DST reads the R kept columns of both factors (w) and writes float64."""
    return {"forward_dst": 2 * n * r * (8 + w), "cross": 2 * n * (r + k) * w,
            "rounding": 2 * k * k * 8 + 2 * n * (k + R) * w, "inverse_dst": 2 * n * R * (w + 8)}


def gpu_arm(args, rank: int, world: int) -> dict | None:
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1306_2150_gb300 import inputs, lr

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    n = args.n
    U, V = inputs.smooth_sum(n, EPS)
    r = U.shape[1]
    Ud = torch.from_numpy(U).cuda()
    Vd = torch.from_numpy(V).cuda()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    h = lr.Handle(stream)
    out = (lr.colmajor_empty(n, 64), torch.empty(64, dtype=torch.float64, device="cuda"),
           lr.colmajor_empty(n, 64))
    results = {"autotune": {}}
    # launch shapes tuned on this problem before anything is timed
    for prec in ("mixed", "fp64"):
        if not args.no_autotune:
            results["autotune"][prec] = lr.lr_autotune(h, Ud, Vd, eps=EPS, prec=prec, reps=3)
    for prec in ("mixed", "fp64"):
        for _ in range(args.warmup):
            lr.lr_poisson2d(h, Ud, Vd, eps=EPS, prec=prec, out=out)
        res = lr.lr_poisson2d(h, Ud, Vd, eps=EPS, prec=prec, out=out, timing=True)
        phases = lr.lr_get_phase_times(h)
        info = res.info
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        ph = []
        clocks = Clocks(torch.cuda.current_device())
        with clocks:
            for i in range(args.steps):
                flush.fill_(i & 0xFF)
                ev[i][0].record(stream)
                lr.lr_poisson2d(h, Ud, Vd, eps=EPS, prec=prec, out=out, async_=True,
                                timing=True)
                ev[i][1].record(stream)
                stream.synchronize()
                ph.append(lr.lr_get_phase_times(h))
            torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        per = [a.elapsed_time(b) for a, b in ev]
        info2, _, _ = lr.lr_get_info(h)
        # end-to-end through the C ABI from pinned host memory, result back
        Uh = torch.from_numpy(U).pin_memory()
        Vh = torch.from_numpy(V).pin_memory()
        Ub = torch.empty_like(Ud)
        Vb = torch.empty_like(Vd)
        host_out = torch.empty((2 * n * 64 + 64,), dtype=torch.float64).pin_memory()
        e2e = []
        for i in range(max(3, args.steps // 2)):
            flush.fill_(i & 0xFF)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            Ub.copy_(Uh, non_blocking=True)
            Vb.copy_(Vh, non_blocking=True)
            rr = lr.lr_poisson2d(h, Ub, Vb, eps=EPS, prec=prec, out=out)
            R = rr.info.rank
            host_out[: n * R].view(R, n).copy_(out[0][:, :R].t(), non_blocking=True)
            host_out[n * R: 2 * n * R].view(R, n).copy_(out[2][:, :R].t(), non_blocking=True)
            host_out[2 * n * R: 2 * n * R + R].copy_(out[1][:R], non_blocking=True)
            b.record(stream)
            stream.synchronize()
            e2e.append(a.elapsed_time(b))
        R = info2.rank
        # accuracy of the timed result (outside the timed region)
        lr.lr_poisson2d(h, Ud, Vd, eps=EPS, prec=prec, out=out)
        err = rel_error_sampled(out[0][:, :R], out[1][:R], out[2][:, :R], U, V)
        results[prec] = {
            "rel_err": err,
            "ms": statistics.median(per), "ms_mean": statistics.mean(per), "per_step": per,
            "phases": {k: statistics.median([p[k] for p in ph]) for k in ph[0]},
            "rank": R, "aca_steps": info2.aca_steps, "launches": info2.launches,
            "cluster_size": info2.cluster_size, "clocks": clocks.summary(),
            "e2e_ms": statistics.median(e2e),
            "h2d": 2 * n * r * 8, "d2h": (2 * n * R + R) * 8,
            "r": r, "first_phases": phases, "status": res.status, "info_rank": info.rank,
        }
    # ---- eps = 1e-10 (the second tolerance of the n-sweep): float64 against
    # mixed precision with float64 residual refinement, single solves
    U2, V2 = inputs.smooth_sum(n, EPS_TIGHT)
    U2d, V2d = torch.from_numpy(U2).cuda(), torch.from_numpy(V2).cuda()
    for prec in ("fp64", "mixed"):
        for _ in range(max(2, args.warmup // 2)):
            lr.lr_poisson2d(h, U2d, V2d, eps=EPS_TIGHT, prec=prec, out=out)
        per = []
        for i in range(max(3, args.steps // 4)):
            flush.fill_(i & 0xFF)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rr = lr.lr_poisson2d(h, U2d, V2d, eps=EPS_TIGHT, prec=prec, out=out)
            b.record(stream)
            stream.synchronize()
            per.append(a.elapsed_time(b))
        results["tight_" + prec] = {"ms": statistics.median(per), "rank": rr.info.rank, "r": U2.shape[1],
                                    "refine_rounds": rr.info.refine_rounds, "status": rr.status,
                                    "rel_err": rel_error_sampled(rr.U, rr.s, rr.V, U2, V2)}
    # ---- the n-sweep of single solves: eps 1e-6 and 1e-10, float64 and mixed
    # (mixed at 1e-10 with float64 refinement), each with its error
    results["sweep"] = []
    for ns in args.sweep:
        for eps_s in (EPS, EPS_TIGHT):
            Us, Vs = inputs.smooth_sum(ns, eps_s)
            Usd, Vsd = torch.from_numpy(Us).cuda(), torch.from_numpy(Vs).cuda()
            outs = (lr.colmajor_empty(ns, 64), torch.empty(64, dtype=torch.float64, device="cuda"),
                    lr.colmajor_empty(ns, 64))
            row = {"n": ns, "eps": eps_s, "rhs_rank": Us.shape[1]}
            for prec in ("fp64", "mixed"):
                rr = lr.lr_poisson2d(h, Usd, Vsd, eps=eps_s, prec=prec, out=outs)
                per = []
                for i in range(3):
                    flush.fill_(i & 0xFF)
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    rr = lr.lr_poisson2d(h, Usd, Vsd, eps=eps_s, prec=prec, out=outs)
                    b.record(stream)
                    stream.synchronize()
                    per.append(a.elapsed_time(b))
                row[prec] = {"ms": round(statistics.median(per), 4), "rank": rr.info.rank, "status": rr.status,
                             "refine_rounds": rr.info.refine_rounds,
                             "rel_err": float(f"{rel_error_sampled(rr.U, rr.s, rr.V, Us, Vs):.3e}")}
            results["sweep"].append(row)
            del Usd, Vsd, outs
    # ---- crossover against the full-grid solver X = S((S F S)/Lambda)S on the
    # dense grid (same smooth right-hand side, single solves, 3 timed each)
    results["crossover"] = []
    for nc in args.crossover:
        Uc, Vc = inputs.smooth_sum(nc, EPS)
        Ucd, Vcd = torch.from_numpy(Uc).cuda(), torch.from_numpy(Vc).cuda()
        Fc = lr.as_colmajor(Ucd @ Vcd.T)
        Xc = lr.colmajor_empty(nc, nc)
        outc = (lr.colmajor_empty(nc, 64), torch.empty(64, dtype=torch.float64, device="cuda"),
                lr.colmajor_empty(nc, 64))
        row = {"n": nc}
        for prec in ("mixed", "fp64"):
            for kind, fn in (("full_grid", lambda: lr.lr_poisson2d_full(h, Fc, prec=prec, out=Xc)),
                             ("lowrank", lambda: lr.lr_poisson2d(h, Ucd, Vcd, eps=EPS, prec=prec, out=outc))):
                fn()
                per = []
                for i in range(3):
                    flush.fill_(i & 0xFF)
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    fn()
                    b.record(stream)
                    stream.synchronize()
                    per.append(a.elapsed_time(b))
                row[f"{kind}_{prec}_ms"] = round(statistics.median(per), 4)
        results["crossover"].append(row)
        del Fc, Xc
        torch.cuda.empty_cache()
    # ---- low-rank Uzawa Stokes (semi-staggered grids, body force of rank 1
    # per component, truncation eps = 1e-7, stop at the Schur residual 1e-6)
    results["stokes"] = []
    for ns in list(args.stokes) + [g for g in args.stokes_gmres if g not in args.stokes]:
        x = np.arange(1, ns) / ns
        fs = [(torch.from_numpy(np.sin(np.pi * x)[:, None]).cuda(), torch.from_numpy(np.cos(np.pi * x)[:, None]).cuda()),
              (torch.from_numpy(-np.cos(np.pi * x)[:, None]).cuda(),
               torch.from_numpy((np.sin(np.pi * x) * (1.0 + x))[:, None]).cuda())]
        row = {"n": ns}
        variants = [("mixed", False), ("fp64", False)]
        if ns in args.stokes_gmres:
            variants += [("fp64", True), ("mixed", True)]
        for prec, gm in variants:
            mi = 60 if prec == "mixed" else 200  # mixed stalls above n = 256 (float32 noise through B^T)
            lr.lr_stokes_uzawa(h, ns, fs, tol_div=1e-6, eps=1e-7, prec=prec, maxit=mi, check=False,
                               gmres=gm)  # warm-up
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            flush.fill_(1)
            a.record(stream)
            rs = lr.lr_stokes_uzawa(h, ns, fs, tol_div=1e-6, eps=1e-7, prec=prec, maxit=mi, check=False, gmres=gm)
            b.record(stream)
            stream.synchronize()
            ok = rs.status == lr.LR_OK
            row[prec + ("_gmres" if gm else "")] = {"ms": round(a.elapsed_time(b), 3) if ok else None,
                         "converged": ok, "iters": rs.iters, "status": rs.status,
                         "cg_residual": rs.history[-1],
                         "velocity_divergence": rs.resid, "pressure_rank": int(rs.p[1].shape[0]),
                         "velocity_ranks": [int(c[1].shape[0]) for c in rs.u]}
        results["stokes"].append(row)
    # ---- 3D Poisson in Tucker format (7-point operator, smooth right-hand
    # side exp(-(x+2y+3z)) + 1/sqrt(r^2 + 0.01), eps = 1e-6, float64)
    results["tucker"] = []
    for nt in args.tucker:
        G3, A1, A2, A3 = inputs.smooth3d(nt, 1e-6)
        d3 = (torch.from_numpy(G3).cuda(), *[torch.from_numpy(np.asfortranarray(A)).cuda() for A in (A1, A2, A3)])
        row = {"n": nt, "rhs_ranks": list(G3.shape)}
        for prec in ("fp64", "mixed"):
            r0 = lr.lr_poisson3d_tucker(h, *d3, eps=1e-6, check=False, prec=prec)
            per = []
            for i in range(3):
                flush.fill_(i & 0xFF)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                torch.cuda.nvtx.range_push(f"tucker3d_{prec}_n{nt}")  # profiler range (ncu --nvtx-include)
                a.record(stream)
                r0 = lr.lr_poisson3d_tucker(h, *d3, eps=1e-6, check=False, prec=prec)
                b.record(stream)
                stream.synchronize()
                torch.cuda.nvtx.range_pop()
                per.append(a.elapsed_time(b))
            row[prec] = {"ms": round(statistics.median(per), 3), "status": r0.status,
                         "solution_ranks": list(r0.G.shape), "cross_steps": r0.steps,
                         "probe_rounds": r0.probe_rounds}
        results["tucker"].append(row)
    # ---- exponential-sum baseline against the cross (n = 1024, eps = 1e-7,
    # float64, the paper's comparison point)
    results["expsum"] = []
    for ne in args.expsum:
        Ue, Ve = inputs.smooth_sum(ne, 1e-7)
        Ued, Ved = torch.from_numpy(Ue).cuda(), torch.from_numpy(Ve).cuda()
        oute = (lr.colmajor_empty(ne, 64), torch.empty(64, dtype=torch.float64, device="cuda"),
                lr.colmajor_empty(ne, 64))
        row = {"n": ne, "eps": 1e-7}
        for kind, fn in (("expsum_fp64", lambda: lr.lr_poisson2d_expsum(h, Ued, Ved, eps=1e-7)),
                         ("cross_fp64", lambda: lr.lr_poisson2d(h, Ued, Ved, eps=1e-7, prec="fp64", out=oute)),
                         ("cross_mixed", lambda: lr.lr_poisson2d(h, Ued, Ved, eps=1e-7, prec="mixed", out=oute,
                                                                 refine=-1))):
            r0 = fn()
            per = []
            for i in range(3):
                flush.fill_(i & 0xFF)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                r0 = fn()
                b.record(stream)
                stream.synchronize()
                per.append(a.elapsed_time(b))
            row[kind + "_ms"] = round(statistics.median(per), 4)
            if kind == "expsum_fp64":
                row["expsum_terms"] = r0[3]
                row["expsum_rank"] = int(r0[1].shape[0])
        results["expsum"].append(row)
    # ---- maxvol row selection (the quasi-optimal pivots that Section 4.2
    # cites): seeded Gaussian m x k with m = n, rows 0..k-1 to start,
    # delta = 1e-2; one synchronous call, events around it.  Bytes: C read and
    # B written by the coefficient kernel, B read and written by each swap.
    results["maxvol"] = []
    for kv in args.maxvol:
        mv_m = args.n
        Cm = lr.colmajor_empty(mv_m, kv)
        Cm.copy_(torch.from_numpy(inputs.normal(41 + kv, mv_m * kv).reshape(kv, mv_m).T.copy()))
        r0 = lr.lr_maxvol(h, Cm, list(range(kv)), 1e-2)
        per = []
        for i in range(3):
            flush.fill_(i & 0xFF)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r0 = lr.lr_maxvol(h, Cm, list(range(kv)), 1e-2)
            b.record(stream)
            stream.synchronize()
            per.append(a.elapsed_time(b))
        ms = statistics.median(per)
        byts = mv_m * kv * 8 * (2 + 2 * r0[1])
        results["maxvol"].append({
            "m": mv_m, "k": kv, "delta": 1e-2, "ms": round(ms, 4), "swaps": r0[1], "bmax": round(r0[2], 6),
            "status": r0[3], "algorithmic_bytes": byts, "gbs": round(byts / (ms * 1e-3) / 1e9, 1),
            "note": "one launch per swap over an L2-resident B, the record read between groups of 32 swaps: "
                    "bound by launch and host round-trip latency, not by HBM"})
    # ---- the uneven batch: problems with n log-uniform in [512, 16384], r
    # uniform in 1..32 and random separable factors (seed 3), eps = 1e-6; one
    # batched call (one CUDA graph) in each precision against a loop of
    # single float64 solves
    results["uneven"] = {}
    if args.uneven > 0:
        specs = inputs.batch_problems(args.uneven, 512, 16384, 32, seed=3)
        uprobs = []
        for (nn, rr, sd) in specs:
            Uu, Vu = inputs.separable_random(nn, rr, seed=sd)
            uprobs.append((torch.from_numpy(Uu), torch.from_numpy(Vu)))
        ub = lr.Batch(uprobs)
        row = {"problems": len(specs), "n_min": min(x[0] for x in specs), "n_max": max(x[0] for x in specs),
               "r_min": min(x[1] for x in specs), "r_max": max(x[1] for x in specs),
               "unknowns_total": int(sum(x[0] * x[0] for x in specs))}
        for prec in ("mixed", "fp64"):
            for streams in (False, True):
                tag = prec + ("_streams" if streams else "")
                for _ in range(2):
                    lr.lr_poisson2d_batched(h, ub, eps=EPS, prec=prec, graph=True, streams=streams)
                per = []
                for i in range(3):
                    flush.fill_(i & 0xFF)
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    lr.lr_poisson2d_batched(h, ub, eps=EPS, prec=prec, graph=True, async_=True, streams=streams)
                    b.record(stream)
                    stream.synchronize()
                    per.append(a.elapsed_time(b))
                info_u, _, _ = lr.lr_get_info(h)
                row["batched_" + tag + "_ms"] = round(statistics.median(per), 3)
                row["launches_" + tag] = info_u.launches
                lr.lr_poisson2d_batched(h, ub, eps=EPS, prec=prec, graph=True, streams=streams, check=False)
                row["status_" + tag] = sorted(set(int(ub.status[i]) for i in range(len(specs))))
                # accuracy of every 16th problem, on sampled rows
                errs = [rel_error_sampled(*ub.result(i), *uprobs[i], rows=128) for i in range(0, len(specs), 16)]
                row["max_rel_err_" + tag] = max(errs)
                row["checked_" + tag] = len(errs)
        flush.fill_(7)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        a.record(stream)
        for (Uu, Vu), o in zip(ub.rhs, ub.out):
            lr.lr_poisson2d(h, Uu, Vu, eps=EPS, prec="fp64", out=o, check=False)
        b.record(stream)
        stream.synchronize()
        row["loop_single_fp64_ms"] = round(a.elapsed_time(b), 3)
        row["loop_single_fp64_wall_ms"] = round((time.perf_counter() - t0) * 1e3, 3)
        row["batched_mixed_speedup_over_loop"] = round(row["loop_single_fp64_ms"] / row["batched_mixed_ms"], 2)
        results["uneven"] = row
        del ub, uprobs
    # ---- throughput: batches of independent solves, one CUDA graph per batch
    # (phase-batched launches), the per-problem stream form beside it
    B = args.batch
    probs = [(torch.from_numpy(U) * (1.0 + p / B), torch.from_numpy(V)) for p in range(B)]
    for prec in ("mixed", "fp64"):
        batch = lr.Batch(probs)
        if not args.no_autotune:
            results["autotune"]["batch_" + prec] = lr.lr_autotune_batched(h, batch, eps=EPS, prec=prec, reps=2)
        for _ in range(args.warmup):
            lr.lr_poisson2d_batched(h, batch, eps=EPS, prec=prec, graph=True)
        torch.cuda.synchronize()
        per = []
        clocks = Clocks(torch.cuda.current_device())
        with clocks:
            for i in range(args.steps if prec == "mixed" else max(3, args.steps // 4)):
                flush.fill_(i & 0xFF)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                lr.lr_poisson2d_batched(h, batch, eps=EPS, prec=prec, graph=True, async_=True)
                b.record(stream)
                stream.synchronize()
                per.append(a.elapsed_time(b))
        info, _, _ = lr.lr_get_info(h)
        ranks = [batch.c_sol[i].r for i in range(B)]
        # accuracy of the timed results (outside the timed region): the first,
        # middle and last problem on sampled rows
        errs = [rel_error_sampled(*batch.result(p), *probs[p]) for p in sorted({0, B // 2, B - 1})]
        # per-phase device time of one batched step (events between the
        # phases; not a graph replay)
        ph = []
        for i in range(max(3, args.steps // 4)):
            flush.fill_(i & 0xFF)
            lr.lr_poisson2d_batched(h, batch, eps=EPS, prec=prec, timing=True)
            ph.append(lr.lr_get_phase_times(h))
        # the per-problem stream form of the same batch
        for _ in range(2):
            lr.lr_poisson2d_batched(h, batch, eps=EPS, prec=prec, graph=True, streams=True)
        per_s = []
        for i in range(max(3, args.steps // 4)):
            flush.fill_(i & 0xFF)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lr.lr_poisson2d_batched(h, batch, eps=EPS, prec=prec, graph=True, async_=True, streams=True)
            b.record(stream)
            stream.synchronize()
            per_s.append(a.elapsed_time(b))
        results["batch_" + prec] = {"ms_step": statistics.median(per), "per_step": per, "batch": B,
                                    "launches": info.launches, "clocks": clocks.summary(),
                                    "ranks": sorted(set(ranks)), "max_rel_err": max(errs),
                                    "checked": len(errs),
                                    "phases": {k: statistics.median([p[k] for p in ph]) for k in ph[0]},
                                    "streams_ms_step": statistics.median(per_s)}
        del batch
    # ---- the same step at other batch sizes (mixed, graph replay; context for
    # the choice of 64: at two CTAs per SM and four per problem 72 clusters
    # fit one wave of the cross, and the transforms fill the SMs in whole
    # columns)
    results["batch_sweep"] = []
    for Bs in args.batch_sweep:
        sp = [(torch.from_numpy(U) * (1.0 + p / Bs), torch.from_numpy(V)) for p in range(Bs)]
        sb = lr.Batch(sp)
        for _ in range(3):
            lr.lr_poisson2d_batched(h, sb, eps=EPS, prec="mixed", graph=True)
        per = []
        for i in range(5):
            flush.fill_(i & 0xFF)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lr.lr_poisson2d_batched(h, sb, eps=EPS, prec="mixed", graph=True, async_=True)
            b.record(stream)
            stream.synchronize()
            per.append(a.elapsed_time(b))
        err = rel_error_sampled(*sb.result(Bs - 1), *sp[Bs - 1])
        results["batch_sweep"].append({"batch": Bs, "ms_step": round(statistics.median(per), 4),
                                       "ms_per_solve": round(statistics.median(per) / Bs, 5),
                                       "rel_err_last": float(f"{err:.3e}")})
        del sb
    # ---- end to end through the C ABI: host factors in, host factors out.
    # Every step copies all 64 problems' U and V from one pinned host buffer
    # into one device buffer (the batch's input factors are views of it),
    # solves, gathers every problem's kept factors and singular values on the
    # device (one kernel) and copies them to pinned host memory.  The solves run
    # back to back on one stream; a step's input copy (on a copy stream) and
    # its gather and read-back (on a third stream) overlap the neighbouring
    # steps' solves; the time is the whole run over the three streams.
    sizes = [2 * n * U.shape[1] for U, _ in probs]
    hin = torch.empty(sum(sizes), dtype=torch.float64).pin_memory()
    off = 0
    for (U, V), sz in zip(probs, sizes):
        r = U.shape[1]
        hin[off: off + n * r].copy_(U.t().reshape(-1))
        hin[off + n * r: off + sz].copy_(V.t().reshape(-1))
        off += sz
    # streams: solves (back to back), input copies, gathers and read-backs;
    # two input, output and gather buffers (one per step parity), one handle
    # per parity, both on the solve stream
    cs_, xs_, gs_ = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    e2e_h = [lr.Handle(cs_) for _ in range(2)]
    dins, e2e_b, houts, obufs, sbufs = [], [], [], [], []
    for k2 in range(2):
        din = torch.empty(sum(sizes), dtype=torch.float64, device="cuda")
        views, off = [], 0
        for (U, V), sz in zip(probs, sizes):
            r = U.shape[1]
            views.append((din[off: off + n * r].view(r, n).t(), din[off + n * r: off + sz].view(r, n).t()))
            off += sz
        dins.append(din)
        # outputs of all problems in one buffer, [problem][U columns, V columns][n], so
        # that the kept columns are gathered by one index_select
        obuf = torch.empty((B, 128, n), dtype=torch.float64, device="cuda")
        sbuf = torch.empty((B, 64), dtype=torch.float64, device="cuda")
        bb = lr.Batch(views)
        for p in range(B):
            Uo, Vo, so = obuf[p, :64].t(), obuf[p, 64:].t(), sbuf[p]
            bb.out[p] = (Uo, so, Vo)
            bb.c_sol[p] = lr.LrMat(n, n, 0, 64, n, Uo.data_ptr(), so.data_ptr(), Vo.data_ptr())
        obufs.append(obuf)
        sbufs.append(sbuf)
        e2e_b.append(bb)
        houts.append((torch.empty((2 * 64 * B, n), dtype=torch.float64).pin_memory(),
                      torch.empty(64 * B, dtype=torch.float64).pin_memory()))
    torch.cuda.synchronize()
    for k2 in range(2):
        dins[k2].copy_(hin)
        for _ in range(max(2, args.warmup)):
            lr.lr_poisson2d_batched(e2e_h[k2], e2e_b[k2], eps=EPS, prec="mixed", graph=True)
    torch.cuda.synchronize()
    h2d = d2h = 0
    # gather indices through pinned memory (a pageable copy would block the host
    # until the gather stream reached it); a parity's buffer is rewritten only
    # after its previous gather, which the next solve of that parity waits for
    idx_host = [torch.empty(2 * 64 * B, dtype=torch.int64).pin_memory() for _ in range(2)]
    sidx_host = [torch.empty(64 * B, dtype=torch.int64).pin_memory() for _ in range(2)]
    ev_solved = [None, None]    # solve of the step of this parity done (inputs and outputs in use until then)
    ev_gathered = [None, None]  # its outputs gathered (the next solve of this parity may overwrite them)

    def finish(k2):
        """The last solve of parity k2 is done: its ranks, then gather and read back."""
        nonlocal d2h
        ev_solved[k2].synchronize()
        lr.lr_batched_status(e2e_h[k2], e2e_b[k2])
        ranks = np.array([e2e_b[k2].c_sol[p].r for p in range(B)])
        cols = np.concatenate([np.r_[p * 128 + np.arange(R), p * 128 + 64 + np.arange(R)]
                               for p, R in enumerate(ranks)]).astype(np.int64)
        svals = np.concatenate([p * 64 + np.arange(R) for p, R in enumerate(ranks)]).astype(np.int64)
        idx_host[k2][: len(cols)].numpy()[:] = cols
        sidx_host[k2][: len(svals)].numpy()[:] = svals
        with torch.cuda.stream(gs_):
            ci = idx_host[k2][: len(cols)].cuda(non_blocking=True)
            si = sidx_host[k2][: len(svals)].cuda(non_blocking=True)
            kept = obufs[k2].view(B * 128, n).index_select(0, ci)
            sk = sbufs[k2].view(-1).index_select(0, si)
            ev_gathered[k2] = torch.cuda.Event()
            ev_gathered[k2].record(gs_)
            houts[k2][0][: kept.shape[0]].copy_(kept, non_blocking=True)
            houts[k2][1][: sk.shape[0]].copy_(sk, non_blocking=True)
        d2h = (kept.numel() + sk.numel()) * 8

    def run(nsteps):
        for i in range(nsteps):
            k2 = i % 2
            with torch.cuda.stream(xs_):  # inputs of this parity: free once its last solve is done
                if ev_solved[k2] is not None:
                    xs_.wait_event(ev_solved[k2])
                dins[k2].copy_(hin, non_blocking=True)
                ev_in = torch.cuda.Event()
                ev_in.record(xs_)
            cs_.wait_event(ev_in)
            if ev_gathered[k2] is not None:  # outputs of this parity gathered
                cs_.wait_event(ev_gathered[k2])
            lr.lr_poisson2d_batched(e2e_h[k2], e2e_b[k2], eps=EPS, prec="mixed", graph=True, async_=True)
            ev_solved[k2] = torch.cuda.Event()
            ev_solved[k2].record(cs_)
            if i > 0:
                finish(1 - k2)
        finish((nsteps - 1) % 2)

    run(4)  # warm-up of the whole pipeline (gather buffers, graph replays)
    nsteps = max(8, args.steps)
    flush.fill_(3)
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(cs_)
    xs_.wait_event(t_start)
    gs_.wait_event(t_start)
    run(nsteps)
    cs_.wait_stream(gs_)
    cs_.wait_stream(xs_)
    t_end.record(cs_)
    t_end.synchronize()
    h2d = dins[0].numel() * 8
    e2e = [t_start.elapsed_time(t_end) / nsteps]
    errs_e2e = [rel_error_sampled(*e2e_b[k2].result(B - 1), *probs[B - 1]) for k2 in range(2)]
    for hh in e2e_h:
        hh.close()
    results["e2e_batch"] = {"ms_step": statistics.median(e2e), "h2d": h2d, "d2h": d2h, "batch": B,
                            "steps": nsteps, "max_rel_err": max(errs_e2e)}
    h.close()
    return results


# Timed quantities of a rank's results: the slowest rank sets the job's time.
RANK_TIMES = (("mixed", "ms"), ("fp64", "ms"), ("batch_mixed", "ms_step"), ("batch_fp64", "ms_step"),
              ("e2e_batch", "ms_step"))


def combine_ranks(res: dict, world: int, device: str) -> dict:
    """Replicas (one independent batch per rank, no collective on the data
    path): the max over ranks of every timed quantity, and whole-job unit
    counts, since every rank solved its own batch.  One all-reduce on the
    initialised process group (NCCL on the GPU machine, gloo in the CPU tests)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([res[a][b] for a, b in RANK_TIMES], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    for (a, b), v in zip(RANK_TIMES, t.tolist()):
        res[a][b] = v
    res["batch_mixed"]["batch"] *= world
    res["e2e_batch"]["batch"] *= world
    return res


def main():
    args = parse()
    if args.cpu_worker:
        cpu_worker(args.n, args.cpu_seconds, args.steps)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        # The reference arm is the CPU oracle: rank 0 alone runs it.
        if rank != 0:
            return
        cb = run_cpu_baseline_all_cores(args.n, max(5.0, args.cpu_seconds))
        line = {"impl": "reference", "metric": METRIC, "value": cb.get("value"), "unit": "ms",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": cb.get("value"), "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": args.n, "eps": EPS, "operator": "5pt",
                           "rhs": "1/(1+x+y)+0.5 sin(3 pi x) exp(-2y), compressed to eps"},
                "cpu_baseline": cb,
                "e2e": {"value": cb.get("value"), "unit": "ms", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    res = gpu_arm(args, rank, world)
    if world > 1:
        combine_ranks(res, world, "cuda")
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    import json as _j
    peaks = {}
    try:
        peaks = _j.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    mx, f64 = res["mixed"], res["fp64"]
    bm, bf, eb = res["batch_mixed"], res["batch_fp64"], res["e2e_batch"]
    n = args.n
    ph = mx["phases"]
    B = bm["batch"] // world
    value = bm["ms_step"] / bm["batch"]  # whole-job throughput: ms per solve
    alg = algorithmic_bytes(n, mx["r"], mx["aca_steps"], mx["rank"], 4)
    alg_total = sum(alg.values())
    # dominant phase of the timed batched step (each phase one or a few
    # launches over all B problems of a rank): its algorithmic bytes over its
    # CUDA-event time
    bph = bm["phases"]
    dom = max(("forward_dst", "cross", "rounding", "inverse_dst"), key=lambda k: bph[k])
    byts = B * alg[dom]
    achieved = byts / (bph[dom] * 1e-3) / 1e9
    # every phase against HBM; the transforms also against the FP32 FMA peak
    # (152 SMs x 128 lanes x 2 flops x 2.07 GHz = 80.5 TFLOP/s): 5 H log2 H
    # flops per H-point FFT, two per residue class, M / H classes per column
    M = 1 << max(6, (2 * n - 1 - 1).bit_length())
    H = min(M, 16384)
    fft_flops_col = (M // H) * 2 * 5 * H * (H.bit_length() - 1)
    fp32_peak = 152 * 128 * 2 * 2.07e9
    cols = {"forward_dst": 2 * mx["r"], "inverse_dst": 2 * mx["rank"]}
    phase_roof = {}
    for k in ("forward_dst", "cross", "rounding", "inverse_dst"):
        gbs = B * alg[k] / (bph[k] * 1e-3) / 1e9
        ent = {"ms": round(bph[k], 4), "algorithmic_bytes": B * alg[k], "gbs": round(gbs, 2),
               "hbm_frac": round(gbs / hbm, 5), "traffic": committed_traffic(k)}
        if k in cols:
            fl = B * cols[k] * fft_flops_col
            ent.update({"fft_flops": fl, "fp32_tflops": round(fl / (bph[k] * 1e-3) / 1e12, 3),
                        "fp32_frac": round(fl / (bph[k] * 1e-3) / fp32_peak, 4)})
        phase_roof[k] = ent
    acc = {"single_mixed": mx["rel_err"], "single_fp64": f64["rel_err"],
           "batch_mixed_max": bm["max_rel_err"], "batch_fp64_max": bf["max_rel_err"],
           "tight_fp64": res["tight_fp64"]["rel_err"], "tight_mixed_refined": res["tight_mixed"]["rel_err"]}
    un = res.get("uneven") or {}
    for key in ("mixed", "fp64", "mixed_streams", "fp64_streams"):
        if "max_rel_err_" + key in un:
            acc["uneven_" + key + "_max"] = un["max_rel_err_" + key]
    bound = {k: (EPS_TIGHT if k.startswith("tight") else EPS) for k in acc}
    acc_line = {k: float(f"{v:.3e}") for k, v in acc.items()}
    acc_line["within_10eps"] = all(acc[k] <= 10 * bound[k] for k in acc)
    acc_line["note"] = ("relative Frobenius error against the exact discrete solution (oracle, Parseval, "
                        "256 sampled frequency rows at n=16384); eps=1e-6 rows against 10*eps, eps=1e-10 rows "
                        "against 10*1e-10")
    line = {
        "metric": METRIC, "value": round(value, 5), "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(bm["ms_step"], 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "eps": EPS, "operator": "5pt", "batch": B,
                   "rhs_rank": mx["r"], "solution_rank": mx["rank"], "cross_steps": mx["aca_steps"],
                   "l2": "flushed (512 MiB write) between timed steps",
                   "replicas_per_gpu": 1, "parallelism": "replicas" if world > 1 else "single"},
        "batched_fp64": {"value": round(bf["ms_step"] / bm["batch"], 5), "unit": "ms per solve"},
        "batched_phases_ms": {"mixed": {k: round(v, 4) for k, v in bph.items()},
                              "fp64": {k: round(v, 4) for k, v in bf["phases"].items()}},
        "batched_stream_form": {"mixed": round(bm["streams_ms_step"] / B, 5),
                                "fp64": round(bf["streams_ms_step"] / B, 5), "unit": "ms per solve",
                                "note": "one launch chain per problem over 32 streams (the previous form)"},
        "accuracy": acc_line,
        "single_solve": {
            "mixed": {"value": round(mx["ms"], 4), "unit": "ms",
                      "phases_ms": {k: round(v, 4) for k, v in ph.items()}},
            "fp64": {"value": round(f64["ms"], 4), "unit": "ms", "rank": f64["rank"],
                     "cross_steps": f64["aca_steps"],
                     "phases_ms": {k: round(v, 4) for k, v in f64["phases"].items()}}},
        "eps_1e-10_single_solve": {
            "fp64_ms": round(res["tight_fp64"]["ms"], 4),
            "mixed_refined_ms": round(res["tight_mixed"]["ms"], 4),
            "refine_rounds": res["tight_mixed"]["refine_rounds"],
            "rank": {"fp64": res["tight_fp64"]["rank"], "mixed": res["tight_mixed"]["rank"]},
            "rhs_rank": res["tight_fp64"]["r"]},
        "single_solve_sweep": res["sweep"],
        "crossover_full_grid_vs_lowrank": res["crossover"],
        "stokes_uzawa_lowrank": res["stokes"],
        "expsum_vs_cross": res["expsum"],
        "maxvol": res.get("maxvol", []),
        "tucker3d": res["tucker"],
        "uneven_batch": res["uneven"],
        "batch_size_sweep": res.get("batch_sweep", []),
        "mixed_batched_over_fp64_single": round(f64["ms"] / value, 2),
        "mixed_batched_over_fp64_batched": round(bf["ms_step"] / bm["ms_step"], 2),
        "batched_effective_gbs": round(alg_total * B / (bm["ms_step"] * 1e-3) / 1e9, 2),
        "roofline": {"bound": "hbm", "kernel": "batched " + dom, "achieved": round(achieved, 2),
                     "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 5),
                     "traffic": committed_traffic(dom), "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": byts, "launch_ms": round(bph[dom], 4),
                     "problems_per_launch": B},
        "phase_rooflines": phase_roof,
        "autotune": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                     for k, v in res["autotune"].items()},
        "e2e": {"value": round(eb["ms_step"] / eb["batch"], 5), "unit": "ms", "h2d_bytes_per_step": eb["h2d"],
                "d2h_bytes_per_step": eb["d2h"], "steps": eb.get("steps"),
                "max_rel_err": float(f"{eb.get('max_rel_err', float('nan')):.3e}"),
                "note": "pinned host factors in, kept factors out, every step; solves back to back on one "
                        "stream, each step's input copy and gather/read-back on two more streams overlap the "
                        "neighbouring solves"},
        "gpu_launches": bm["launches"] * args.steps,
        "clocks": bm["clocks"],
    }
    if not args.no_cpu_baseline and world == 1:
        cb = run_cpu_baseline_all_cores(n, args.cpu_seconds)
        cb["single_core"] = run_cpu_baseline(n, args.cpu_seconds)
        line["cpu_baseline"] = cb
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
