"""Thin ctypes binding of liblrpoisson.so (C ABI in include/lrpoisson.h).

Argument marshalling only: every numerical step runs in the library's CUDA
kernels.  PyTorch supplies device memory and the stream.  Factor matrices are
float64 CUDA tensors of shape (rows, cols) stored column-major
(``t.stride(0) == 1``), which is the layout the C ABI expects.

There is no CPU fallback: if the compiled library is missing, ``load()``
raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblrpoisson.so")

LR_OK, LR_EINVAL, LR_ENOMEM, LR_ENOCONV, LR_ETIMEOUT, LR_ECUDA, LR_ENONFINITE = range(7)
LR_FP64, LR_MIXED = 0, 1
LR_OP_5PT, LR_OP_SEMISTAGGERED = 0, 1
LR_FLAG_ASYNC = 1
LR_FLAG_TIMING = 2
LR_FLAG_GRAPH = 4
LR_FLAG_CLUSTER_DST = 8
LR_FLAG_GMRES = 16
LR_FLAG_BATCH_STREAMS = 32
PHASES = ("forward_dst", "cross", "rounding", "inverse_dst")

PRECISIONS = {"fp64": LR_FP64, "mixed": LR_MIXED}
OPERATORS = {"5pt": LR_OP_5PT, "semi": LR_OP_SEMISTAGGERED}

# Every function the header declares (checked against the header by the tests).
EXPORTS = ("lr_options_default", "lr_create", "lr_set_stream", "lr_destroy",
           "lr_last_error", "lr_status_string", "lr_dst1", "lr_poisson2d",
           "lr_truncate", "lr_get_info", "lr_get_phase_times", "lr_truncate_noalloc",
           "lr_poisson2d_batched", "lr_autotune", "lr_autotune_batched", "lr_poisson2d_full",
           "lr_stokes_uzawa", "lr_poisson2d_expsum", "lr_poisson3d_tucker", "lr_set_workspace_limit",
           "lr_batched_status", "lr_maxvol")


class LrMat(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int), ("r", ctypes.c_int),
                ("rmax", ctypes.c_int), ("ld", ctypes.c_int),
                ("U", ctypes.c_void_p), ("s", ctypes.c_void_p), ("V", ctypes.c_void_p)]


class LrTucker(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("r", ctypes.c_int * 3), ("rmax", ctypes.c_int * 3),
                ("ld", ctypes.c_int * 3), ("G", ctypes.c_void_p), ("U", ctypes.c_void_p * 3)]


class LrOptions(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("op", ctypes.c_int), ("eps", ctypes.c_double),
                ("rmax", ctypes.c_int), ("aca_tol_factor", ctypes.c_double),
                ("probes", ctypes.c_int), ("seed", ctypes.c_ulonglong),
                ("flags", ctypes.c_uint), ("cluster_size", ctypes.c_int), ("refine", ctypes.c_int)]


class LrTune(ctypes.Structure):
    _fields_ = [("cluster_size", ctypes.c_int), ("log_tile", ctypes.c_int), ("transform", ctypes.c_int),
                ("batch_indices_per_cta", ctypes.c_int), ("candidates", ctypes.c_int),
                ("ms_best", ctypes.c_double), ("ms_default", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class LrInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("aca_steps", ctypes.c_int), ("rank", ctypes.c_int),
                ("converged", ctypes.c_int), ("cut", ctypes.c_int),
                ("probe_rounds", ctypes.c_int), ("zero_rows", ctypes.c_int),
                ("cluster_size", ctypes.c_int), ("launches", ctypes.c_int),
                ("norm_est", ctypes.c_double),
                ("sigma0", ctypes.c_double),
                ("refine_rounds", ctypes.c_int), ("pad", ctypes.c_int),
                ("refine_corr", ctypes.c_double)]


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load the compiled library (once).  Raises RuntimeError if it is absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} not found: build it with `python -m paper_1306_2150_gb300.build` "
                           "(there is no CPU fallback)")
    try:  # torch first: it loads the CUDA runtime the library links against
        import torch  # noqa: F401
    except Exception:
        pass
    lib = ctypes.CDLL(p)
    c_int, c_void_p, c_double = ctypes.c_int, ctypes.c_void_p, ctypes.c_double
    lib.lr_options_default.argtypes = [ctypes.POINTER(LrOptions)]
    lib.lr_options_default.restype = None
    lib.lr_create.argtypes = [ctypes.POINTER(c_void_p), c_void_p]
    lib.lr_create.restype = c_int
    lib.lr_set_stream.argtypes = [c_void_p, c_void_p]
    lib.lr_set_stream.restype = c_int
    lib.lr_set_workspace_limit.argtypes = [c_void_p, ctypes.c_size_t]
    lib.lr_set_workspace_limit.restype = c_int
    lib.lr_destroy.argtypes = [c_void_p]
    lib.lr_destroy.restype = c_int
    lib.lr_last_error.argtypes = [c_void_p]
    lib.lr_last_error.restype = ctypes.c_char_p
    lib.lr_status_string.argtypes = [c_int]
    lib.lr_status_string.restype = ctypes.c_char_p
    lib.lr_dst1.argtypes = [c_void_p, c_int, c_int, c_void_p, c_int, c_void_p, c_int, c_int]
    lib.lr_dst1.restype = c_int
    lib.lr_poisson2d.argtypes = [c_void_p, ctypes.POINTER(LrMat), ctypes.POINTER(LrMat),
                                 ctypes.POINTER(LrOptions)]
    lib.lr_poisson2d.restype = c_int
    lib.lr_truncate.argtypes = [c_void_p, ctypes.POINTER(LrMat), c_double, c_int]
    lib.lr_truncate.restype = c_int
    lib.lr_maxvol.argtypes = [c_void_p, c_void_p, c_int, c_int, c_int, c_double, c_int,
                              ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_double)]
    lib.lr_maxvol.restype = c_int
    lib.lr_get_info.argtypes = [c_void_p, ctypes.POINTER(LrInfo), ctypes.POINTER(c_int),
                                ctypes.POINTER(c_int), c_int]
    lib.lr_get_info.restype = c_int
    lib.lr_get_phase_times.argtypes = [c_void_p, ctypes.POINTER(c_double), c_int]
    lib.lr_get_phase_times.restype = c_int
    lib.lr_truncate_noalloc.argtypes = [ctypes.POINTER(LrMat), c_double, c_int, c_void_p]
    lib.lr_truncate_noalloc.restype = c_int
    lib.lr_poisson2d_batched.argtypes = [c_void_p, c_int, ctypes.POINTER(LrMat), ctypes.POINTER(LrMat),
                                         ctypes.POINTER(LrOptions), ctypes.POINTER(c_int)]
    lib.lr_poisson2d_batched.restype = c_int
    lib.lr_batched_status.argtypes = [c_void_p, c_int, ctypes.POINTER(LrMat), ctypes.POINTER(c_int)]
    lib.lr_batched_status.restype = c_int
    lib.lr_autotune.argtypes = [c_void_p, ctypes.POINTER(LrMat), ctypes.POINTER(LrOptions), c_int,
                                ctypes.POINTER(LrTune)]
    lib.lr_autotune.restype = c_int
    lib.lr_poisson2d_full.argtypes = [c_void_p, c_int, c_void_p, c_int, c_void_p, c_int,
                                      ctypes.POINTER(LrOptions)]
    lib.lr_poisson2d_full.restype = c_int
    lib.lr_stokes_uzawa.argtypes = [c_void_p, c_int, c_int, ctypes.POINTER(LrMat), ctypes.POINTER(LrMat),
                                    ctypes.POINTER(LrMat), ctypes.POINTER(LrMat), c_double, c_int,
                                    ctypes.POINTER(LrOptions), ctypes.POINTER(c_int), ctypes.POINTER(c_double),
                                    ctypes.POINTER(c_double)]
    lib.lr_stokes_uzawa.restype = c_int
    lib.lr_poisson3d_tucker.argtypes = [c_void_p, ctypes.POINTER(LrTucker), ctypes.POINTER(LrTucker),
                                        ctypes.POINTER(LrOptions)]
    lib.lr_poisson3d_tucker.restype = c_int
    lib.lr_poisson2d_expsum.argtypes = [c_void_p, ctypes.POINTER(LrMat), ctypes.POINTER(LrMat),
                                        ctypes.POINTER(LrOptions), ctypes.POINTER(c_int)]
    lib.lr_poisson2d_expsum.restype = c_int
    lib.lr_autotune_batched.argtypes = [c_void_p, c_int, ctypes.POINTER(LrMat), ctypes.POINTER(LrMat),
                                        ctypes.POINTER(LrOptions), c_int, ctypes.POINTER(LrTune)]
    lib.lr_autotune_batched.restype = c_int
    if path is None:
        _lib = lib
    return lib


class LrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


def status_string(s: int) -> str:
    return load().lr_status_string(int(s)).decode()


def lr_options_default() -> LrOptions:
    o = LrOptions()
    load().lr_options_default(ctypes.byref(o))
    return o


class Handle:
    """lr_create / lr_destroy around a CUDA stream (torch's current stream by
    default)."""

    def __init__(self, stream=None):
        import torch
        lib = load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        ptr = ctypes.c_void_p()
        st = lib.lr_create(ctypes.byref(ptr), ctypes.c_void_p(stream.cuda_stream))
        if st != LR_OK:
            raise LrError(st, "lr_create failed")
        self.ptr = ptr

    def last_error(self) -> str:
        return load().lr_last_error(self.ptr).decode()

    def close(self):
        if getattr(self, "ptr", None):
            load().lr_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def colmajor_empty(rows: int, cols: int, device="cuda"):
    """float64 tensor of shape (rows, cols), column-major, 16-byte aligned
    columns (leading dimension rounded up to an even count)."""
    import torch
    ld = rows + (rows & 1)
    return torch.empty((max(cols, 1), ld), dtype=torch.float64, device=device).t()[:rows, :cols]


def as_colmajor(t):
    import torch
    if t.dtype != torch.float64:
        t = t.to(torch.float64)
    if t.dim() == 1:
        t = t[:, None]
    if t.stride(0) == 1 and t.stride(1) >= t.shape[0] and t.stride(1) % 2 == 0 \
            and t.data_ptr() % 16 == 0:
        return t
    out = colmajor_empty(t.shape[0], t.shape[1], t.device)
    out.copy_(t)
    return out


def _ld(t) -> int:
    return int(t.stride(1)) if t.shape[1] > 1 else max(int(t.stride(1)), t.shape[0])


@dataclass
class SolveResult:
    U: object
    s: object
    V: object
    info: LrInfo
    status: int
    pivots_I: list
    pivots_J: list


def _options(eps, prec, op, rmax, aca_tol_factor, probes, seed, flags, cluster_size, refine=0) -> LrOptions:
    o = lr_options_default()
    o.refine = int(refine)
    o.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    o.op = OPERATORS[op] if isinstance(op, str) else int(op)
    o.eps = float(eps)
    o.rmax = int(rmax)
    o.aca_tol_factor = float(aca_tol_factor)
    o.probes = int(probes)
    o.seed = int(seed)
    o.flags = int(flags)
    o.cluster_size = int(cluster_size)
    return o


def lr_poisson2d(h: Handle, U, V, eps: float = 1e-6, prec="mixed", op="5pt", rmax: int = 64,
                 rmax_out: int = 64, aca_tol_factor: float = 1.0, probes: int = 16, seed: int = 0,
                 cluster_size: int = 0, async_: bool = False, out=None, check: bool = True,
                 timing: bool = False, graph: bool = False, refine: int = 0, cluster_dst: bool = False):
    """Low-rank solve of A X = U V^T.  Returns SolveResult with the solution
    factors (views of rank R) unless ``async_`` (then read lr_get_info after
    synchronising the stream).  ``out`` = (Uo, s, Vo) preallocated outputs."""
    U = as_colmajor(U)
    V = as_colmajor(V)
    m, r = U.shape
    if V.shape != (m, r):
        raise ValueError("U and V must have the same shape")
    if U.stride(1) != V.stride(1):
        V2 = colmajor_empty(m, r, V.device)
        V2.copy_(V)
        V = V2
        if U.stride(1) != V.stride(1):
            U2 = colmajor_empty(m, r, U.device)
            U2.copy_(U)
            U = U2
    if out is None:
        import torch
        Uo = colmajor_empty(m, rmax_out, U.device)
        Vo = colmajor_empty(m, rmax_out, U.device)
        s = torch.empty(rmax_out, dtype=torch.float64, device=U.device)
    else:
        Uo, s, Vo = out
    rhs = LrMat(m, m, r, r, _ld(U), U.data_ptr(), None, V.data_ptr())
    sol = LrMat(m, m, 0, Uo.shape[1], _ld(Uo), Uo.data_ptr(), s.data_ptr(), Vo.data_ptr())
    if _ld(Vo) != _ld(Uo):
        raise ValueError("output factors need the same leading dimension")
    flags = (LR_FLAG_ASYNC if async_ else 0) | (LR_FLAG_TIMING if timing else 0) | \
        (LR_FLAG_GRAPH if graph else 0) | (LR_FLAG_CLUSTER_DST if cluster_dst else 0)
    o = _options(eps, prec, op, rmax, aca_tol_factor, probes, seed, flags, cluster_size, refine)
    st = load().lr_poisson2d(h.ptr, ctypes.byref(rhs), ctypes.byref(sol), ctypes.byref(o))
    if async_:
        if st != LR_OK:
            raise LrError(st, h.last_error())
        return None
    if check and st not in (LR_OK, LR_ENOCONV):
        raise LrError(st, h.last_error())
    info, pi, pj = lr_get_info(h)
    R = sol.r
    return SolveResult(Uo[:, :R], s[:R], Vo[:, :R], info, st, pi, pj)


def lr_set_workspace_limit(h: Handle, nbytes: int) -> None:
    """Cap the handle's device workspace (0: no cap); larger needs give LR_ENOMEM."""
    st = load().lr_set_workspace_limit(h.ptr, int(nbytes))
    if st != LR_OK:
        raise LrError(st, "lr_set_workspace_limit failed")


def lr_get_info(h: Handle, cap: int = 64):
    info = LrInfo()
    pi = (ctypes.c_int * cap)()
    pj = (ctypes.c_int * cap)()
    st = load().lr_get_info(h.ptr, ctypes.byref(info), pi, pj, cap)
    if st != LR_OK:
        raise LrError(st, "lr_get_info failed")
    k = min(info.aca_steps, cap)
    return info, list(pi[:k]), list(pj[:k])


def lr_dst1(h: Handle, X, prec="fp64", out=None):
    """Orthonormal DST-I of every column of X (float64 CUDA, column-major)."""
    X = as_colmajor(X)
    m, n = X.shape
    Y = colmajor_empty(m, n, X.device) if out is None else out
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    st = load().lr_dst1(h.ptr, m, n, X.data_ptr(), _ld(X), Y.data_ptr(), _ld(Y), p)
    if st != LR_OK:
        raise LrError(st, h.last_error())
    return Y


def lr_truncate(h: Handle, U, s, V, eps: float, rmax: int = 64):
    """Rounding of U diag(s) V^T (s None: ones).  Returns (U, s, V, status)
    with the kept rank."""
    import torch
    U = as_colmajor(U)
    V = as_colmajor(V)
    n1, r = U.shape
    n2 = V.shape[0]
    ld = max(_ld(U), _ld(V))
    ld += ld & 1
    Uw = torch.empty((r, ld), dtype=torch.float64, device=U.device).t()
    Vw = torch.empty((r, ld), dtype=torch.float64, device=U.device).t()
    Uw[:n1].copy_(U)
    Vw[:n2].copy_(V)
    sw = torch.ones(r, dtype=torch.float64, device=U.device) if s is None else \
        s.to(torch.float64).clone().contiguous()
    X = LrMat(n1, n2, r, r, ld, Uw.data_ptr(), sw.data_ptr(), Vw.data_ptr())
    st = load().lr_truncate(h.ptr, ctypes.byref(X), float(eps), int(rmax))
    if st not in (LR_OK, LR_ENOCONV):
        raise LrError(st, h.last_error())
    R = X.r
    return Uw[:n1, :R], sw[:R], Vw[:n2, :R], st


def lr_maxvol(h: Handle, C, rows, delta: float = 1e-2, maxswaps: int | None = None):
    """Maxvol row selection on C (CUDA float64, m x k, column-major) from the
    starting rows ``rows``.  Returns (rows, nswaps, bmax, status); status is
    LR_OK or LR_ENOCONV (swap cap reached), other statuses raise."""
    C = as_colmajor(C)
    m, k = C.shape
    if maxswaps is None:
        maxswaps = 16 * k
    arr = (ctypes.c_int * k)(*[int(r) for r in rows])
    ns = ctypes.c_int(0)
    bm = ctypes.c_double(0.0)
    st = load().lr_maxvol(h.ptr, C.data_ptr(), m, k, _ld(C), float(delta), int(maxswaps), arr,
                          ctypes.byref(ns), ctypes.byref(bm))
    if st not in (LR_OK, LR_ENOCONV):
        raise LrError(st, h.last_error())
    return list(arr), ns.value, bm.value, st


def lr_get_phase_times(h: Handle) -> dict:
    """Per-phase milliseconds of the last solve run with ``timing=True``."""
    ms = (ctypes.c_double * len(PHASES))()
    st = load().lr_get_phase_times(h.ptr, ms, len(PHASES))
    if st != LR_OK:
        raise LrError(st, h.last_error())
    return dict(zip(PHASES, list(ms)))


class Batch:
    """Device buffers of a batch of problems for lr_poisson2d_batched: the
    right-hand sides (column-major float64) and preallocated outputs."""

    def __init__(self, problems, rmax_out: int = 64, device="cuda"):
        import torch
        self.rhs, self.out = [], []
        for U, V in problems:
            U = as_colmajor(U.to(device) if hasattr(U, "to") else torch.from_numpy(U).to(device))
            V = as_colmajor(V.to(device) if hasattr(V, "to") else torch.from_numpy(V).to(device))
            if U.stride(1) != V.stride(1):
                V2 = colmajor_empty(V.shape[0], V.shape[1], device)
                V2.copy_(V)
                V = V2
            m = U.shape[0]
            Uo, Vo = colmajor_empty(m, rmax_out, device), colmajor_empty(m, rmax_out, device)
            s = torch.empty(rmax_out, dtype=torch.float64, device=device)
            self.rhs.append((U, V))
            self.out.append((Uo, s, Vo))
        n = len(problems)
        self.c_rhs = (LrMat * n)()
        self.c_sol = (LrMat * n)()
        for i, ((U, V), (Uo, s, Vo)) in enumerate(zip(self.rhs, self.out)):
            m, r = U.shape
            self.c_rhs[i] = LrMat(m, m, r, r, _ld(U), U.data_ptr(), None, V.data_ptr())
            self.c_sol[i] = LrMat(m, m, 0, Uo.shape[1], _ld(Uo), Uo.data_ptr(), s.data_ptr(), Vo.data_ptr())
        self.status = (ctypes.c_int * n)()

    def __len__(self):
        return len(self.rhs)

    def result(self, i):
        R = self.c_sol[i].r
        Uo, s, Vo = self.out[i]
        return Uo[:, :R], s[:R], Vo[:, :R]


def lr_batched_status(h: Handle, batch: Batch, check: bool = True) -> int:
    """Ranks and statuses of the last asynchronous lr_poisson2d_batched on h
    (after the caller synchronised its stream) into ``batch``."""
    st = load().lr_batched_status(h.ptr, len(batch), batch.c_sol, batch.status)
    if check and st not in (LR_OK, LR_ENOCONV):
        raise LrError(st, h.last_error())
    return st


def lr_poisson2d_batched(h: Handle, batch: Batch, eps: float = 1e-6, prec="mixed", op="5pt",
                         rmax: int = 64, aca_tol_factor: float = 1.0, probes: int = 16, seed: int = 0,
                         cluster_size: int = 0, async_: bool = False, graph: bool = False,
                         check: bool = True, streams: bool = False, timing: bool = False) -> int:
    """Solve every problem of ``batch``; returns the lr_status of the call
    (per-problem statuses in ``batch.status``, results via ``batch.result``).
    ``streams`` selects the per-problem launch chains over internal streams
    instead of the phase-batched launches."""
    flags = (LR_FLAG_ASYNC if async_ else 0) | (LR_FLAG_GRAPH if graph else 0) | \
        (LR_FLAG_BATCH_STREAMS if streams else 0) | (LR_FLAG_TIMING if timing else 0)
    o = _options(eps, prec, op, rmax, aca_tol_factor, probes, seed, flags, cluster_size)
    st = load().lr_poisson2d_batched(h.ptr, len(batch), batch.c_rhs, batch.c_sol, ctypes.byref(o),
                                     batch.status)
    if check and st not in (LR_OK, LR_ENOCONV):
        raise LrError(st, h.last_error())
    return st


def lr_autotune(h: Handle, U, V, eps: float = 1e-6, prec="mixed", op="5pt", rmax: int = 64,
                reps: int = 5) -> dict:
    """Time launch-shape candidates of lr_poisson2d on (U, V) and keep the
    fastest in the handle for this order, precision and operator kind."""
    U = as_colmajor(U)
    V = as_colmajor(V)
    if U.stride(1) != V.stride(1):
        V2 = colmajor_empty(V.shape[0], V.shape[1], V.device)
        V2.copy_(V)
        V = V2
    m, r = U.shape
    rhs = LrMat(m, m, r, r, _ld(U), U.data_ptr(), None, V.data_ptr())
    o = _options(eps, prec, op, rmax, 1.0, 16, 0, 0, 0)
    t = LrTune()
    st = load().lr_autotune(h.ptr, ctypes.byref(rhs), ctypes.byref(o), int(reps), ctypes.byref(t))
    if st != LR_OK:
        raise LrError(st, h.last_error())
    return t.as_dict()


def lr_autotune_batched(h: Handle, batch: Batch, eps: float = 1e-6, prec="mixed", op="5pt", rmax: int = 64,
                        reps: int = 3, streams: bool = False) -> dict:
    """Time the indices-per-CTA candidates of lr_poisson2d_batched on ``batch``
    and keep the fastest in the handle for this precision (``streams``: tune
    the per-problem stream form instead of the phase-batched form)."""
    o = _options(eps, prec, op, rmax, 1.0, 16, 0, LR_FLAG_BATCH_STREAMS if streams else 0, 0)
    t = LrTune()
    st = load().lr_autotune_batched(h.ptr, len(batch), batch.c_rhs, batch.c_sol, ctypes.byref(o), int(reps),
                                    ctypes.byref(t))
    if st != LR_OK:
        raise LrError(st, h.last_error())
    return t.as_dict()


def lr_poisson2d_full(h: Handle, F, prec="mixed", op="5pt", out=None):
    """Full-grid solve of A X = F (dense m x m, float64 on the device):
    X = S ((S F S) / Lambda) S.  Returns X (column-major float64)."""
    F = as_colmajor(F)
    m = F.shape[0]
    if F.shape != (m, m):
        raise ValueError("F must be square")
    X = colmajor_empty(m, m, F.device) if out is None else out
    o = _options(1e-6, prec, op, 64, 1.0, 16, 0, 0, 0)
    st = load().lr_poisson2d_full(h.ptr, m, F.data_ptr(), _ld(F), X.data_ptr(), _ld(X), ctypes.byref(o))
    if st != LR_OK:
        raise LrError(st, h.last_error())
    return X


@dataclass
class StokesResult:
    u: list          # [(U, s, V) for the x and y velocity components]
    p: tuple         # (U, s, V) of the pressure
    iters: int
    resid: float
    status: int
    history: list    # ||r_k|| / ||r_0|| of the CG residual, k = 0..iters


def lr_stokes_uzawa(h: Handle, n: int, f, tol_div: float = 1e-6, maxit: int = 200, eps: float = 1e-7,
                    prec="mixed", rmax_out: int = 64, check: bool = True, gmres: bool = False,
                    p0=None, g=None) -> StokesResult:
    """Low-rank Uzawa solve of the 2D Stokes problem on n x n cells; ``f`` is
    [(U1, V1), (U2, V2)], the body-force components at the (n-1)^2 interior
    vertices in factored form (device float64); ``g`` (optional) the
    divergence right-hand side (Ug, Vg) on the n x n cell centres."""
    import torch
    m = n - 1
    c_f = (LrMat * 2)()
    c_u = (LrMat * 2)()
    keep, outs = [], []
    for k, (U, V) in enumerate(f):
        U = as_colmajor(U)
        V = as_colmajor(V)
        if U.stride(1) != V.stride(1):
            V2 = colmajor_empty(V.shape[0], V.shape[1], V.device)
            V2.copy_(V)
            V = V2
        keep += [U, V]
        c_f[k] = LrMat(m, m, U.shape[1], U.shape[1], _ld(U), U.data_ptr(), None, V.data_ptr())
        Uo, Vo = colmajor_empty(m, rmax_out, U.device), colmajor_empty(m, rmax_out, U.device)
        so = torch.empty(rmax_out, dtype=torch.float64, device=U.device)
        outs.append((Uo, so, Vo))
        c_u[k] = LrMat(m, m, 0, rmax_out, _ld(Uo), Uo.data_ptr(), so.data_ptr(), Vo.data_ptr())
    dev = keep[0].device
    Up, Vp = colmajor_empty(n, rmax_out, dev), colmajor_empty(n, rmax_out, dev)
    sp = torch.empty(rmax_out, dtype=torch.float64, device=dev)
    r0 = 0
    if p0 is not None:  # resume from a saved pressure (U, s, V)
        U0, s0, V0 = p0
        r0 = U0.shape[1]
        Up[:, :r0].copy_(U0)
        Vp[:, :r0].copy_(V0)
        sp[:r0].copy_(s0)
    c_p = LrMat(n, n, r0, rmax_out, _ld(Up), Up.data_ptr(), sp.data_ptr(), Vp.data_ptr())
    o = _options(eps, prec, "semi", 64, 1.0, 16, 0, LR_FLAG_GMRES if gmres else 0, 0)
    c_g = None
    if g is not None:
        Ug, Vg = as_colmajor(g[0]), as_colmajor(g[1])
        if Ug.stride(1) != Vg.stride(1):
            V2 = colmajor_empty(Vg.shape[0], Vg.shape[1], Vg.device)
            V2.copy_(Vg)
            Vg = V2
        keep += [Ug, Vg]
        c_g = LrMat(n, n, Ug.shape[1], Ug.shape[1], _ld(Ug), Ug.data_ptr(), None, Vg.data_ptr())
    iters = ctypes.c_int(0)
    resid = ctypes.c_double(0.0)
    hist = (ctypes.c_double * (int(maxit) + 1))()
    st = load().lr_stokes_uzawa(h.ptr, 2, n, c_f, ctypes.byref(c_g) if c_g is not None else None, c_u,
                                ctypes.byref(c_p), float(tol_div), int(maxit),
                                ctypes.byref(o), ctypes.byref(iters), ctypes.byref(resid), hist)
    if check and st not in (LR_OK, LR_ENOCONV):
        raise LrError(st, h.last_error())
    u = [(Uo[:, :c_u[k].r], so[:c_u[k].r], Vo[:, :c_u[k].r]) for k, (Uo, so, Vo) in enumerate(outs)]
    return StokesResult(u, (Up[:, :c_p.r], sp[:c_p.r], Vp[:, :c_p.r]), iters.value, resid.value, st,
                        list(hist[:iters.value + 1]))


def lr_poisson2d_expsum(h: Handle, U, V, eps: float = 1e-7, rmax_out: int = 64):
    """Exponential-sum solve of the 5-point problem (float64); returns
    (U, s, V, number of quadrature terms)."""
    import torch
    U = as_colmajor(U)
    V = as_colmajor(V)
    if U.stride(1) != V.stride(1):
        V2 = colmajor_empty(V.shape[0], V.shape[1], V.device)
        V2.copy_(V)
        V = V2
    m, r = U.shape
    Uo, Vo = colmajor_empty(m, rmax_out, U.device), colmajor_empty(m, rmax_out, U.device)
    so = torch.empty(rmax_out, dtype=torch.float64, device=U.device)
    rhs = LrMat(m, m, r, r, _ld(U), U.data_ptr(), None, V.data_ptr())
    sol = LrMat(m, m, 0, rmax_out, _ld(Uo), Uo.data_ptr(), so.data_ptr(), Vo.data_ptr())
    o = _options(eps, "fp64", "5pt", 64, 1.0, 16, 0, 0, 0)
    q = ctypes.c_int(0)
    st = load().lr_poisson2d_expsum(h.ptr, ctypes.byref(rhs), ctypes.byref(sol), ctypes.byref(o), ctypes.byref(q))
    if st not in (LR_OK,):
        raise LrError(st, h.last_error())
    R = sol.r
    return Uo[:, :R], so[:R], Vo[:, :R], q.value


@dataclass
class TuckerResult:
    G: object        # core (R0, R1, R2), device float64
    U: list          # factors n_k x R_k with orthonormal columns
    steps: int       # cross steps
    probe_rounds: int
    status: int


def lr_poisson3d_tucker(h: Handle, G, U1, U2, U3, eps: float = 1e-6, rmax: int = 64, rmax_out: int = 64,
                        aca_tol_factor: float = 1.0, probes: int = 16, seed: int = 0,
                        check: bool = True, prec="fp64") -> TuckerResult:
    """Low-rank 3D solve: the right-hand side in Tucker format, core G
    (r0, r1, r2) and factors U_k (n_k x r_k), device float64 tensors; prec
    "mixed" runs the transforms and the rounding cores' Jacobi in float32."""
    import torch
    G = G.contiguous()
    Us = []
    for U in (U1, U2, U3):
        U = as_colmajor(U)
        if _ld(U) % 2:
            U2_ = colmajor_empty(U.shape[0], U.shape[1], U.device)
            U2_.copy_(U)
            U = U2_
        Us.append(U)
    dev = G.device
    ns = [U.shape[0] for U in Us]
    rs = list(G.shape)
    outs = [colmajor_empty(n, rmax_out, dev) for n in ns]
    Go = torch.empty(rmax_out ** 3, dtype=torch.float64, device=dev)
    rhs = LrTucker()
    sol = LrTucker()
    for k in range(3):
        rhs.n[k] = ns[k]; rhs.r[k] = rs[k]; rhs.rmax[k] = rs[k]; rhs.ld[k] = _ld(Us[k]); rhs.U[k] = Us[k].data_ptr()
        sol.n[k] = ns[k]; sol.r[k] = 0; sol.rmax[k] = rmax_out; sol.ld[k] = _ld(outs[k]); sol.U[k] = outs[k].data_ptr()
    rhs.G = G.data_ptr()
    sol.G = Go.data_ptr()
    o = _options(eps, prec, "5pt", rmax, aca_tol_factor, probes, seed, 0, 0)
    st = load().lr_poisson3d_tucker(h.ptr, ctypes.byref(rhs), ctypes.byref(sol), ctypes.byref(o))
    if check and st not in (LR_OK,):
        raise LrError(st, h.last_error())
    R = [sol.r[k] for k in range(3)]
    info = LrInfo()
    load().lr_get_info(h.ptr, ctypes.byref(info), None, None, 0)
    steps, pr = info.aca_steps, info.probe_rounds
    return TuckerResult(Go[:R[0] * R[1] * R[2]].view(R[0], R[1], R[2]) if min(R) > 0 else Go[:0].view(0, 0, 0),
                        [outs[k][:, :R[k]] for k in range(3)], steps, pr, st)
