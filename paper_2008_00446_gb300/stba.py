"""Thin ctypes binding of libstba.so (include/stba.h).

Argument marshalling only: every step of the LM iteration runs in the library's CUDA kernels.  Arrays may
be NumPy arrays or PyTorch tensors (CPU or CUDA); CUDA tensors are passed as device pointers, everything
else as host pointers.  The functions carry the C names; `Context` owns a `stba_ctx*`.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

_LIB = None

STBA_FP64, STBA_MIXED = 0, 1
STBA_SOLVER_CLUSTERS, STBA_SOLVER_PCG_FULL, STBA_SOLVER_PCG_CLUSTERS = 0, 1, 2
STBA_FACTOR_UPDATE_DEFAULT, STBA_FACTOR_UPDATE_SIMT, STBA_FACTOR_UPDATE_TENSOR = 0, 1, 2
STBA_FACTOR_PANEL_DEFAULT, STBA_FACTOR_PANEL_STACKED, STBA_FACTOR_PANEL_SPLIT, STBA_FACTOR_PANEL_PERSISTENT = 0, 1, 2, 3
STBA_PAIR_BLOCKS_DEFAULT, STBA_PAIR_BLOCKS_STORED, STBA_PAIR_BLOCKS_RECOMPUTE = 0, 1, 2
# stba_autotune's candidates: name -> (factor_tile, factor_update, factor_panel)
AUTOTUNE_CANDIDATES = {"64_split_tensor": (64, 2, 2), "64_split_simt": (64, 1, 2), "64_stacked_simt": (64, 1, 1),
                       "32_stacked_simt": (32, 1, 1), "64_persistent": (64, 1, 3), "64_stacked_tensor": (64, 2, 1)}
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of device memory", 4: "not SPD",
          5: "non-finite value", 6: "timeout", 7: "invalid state"}

# every symbol the header declares
EXPORTS = ["stba_default_options", "stba_create", "stba_set_clusters", "stba_lm_iteration", "stba_solve",
           "stba_cost", "stba_get_params", "stba_set_params", "stba_get_state", "stba_set_state",
           "stba_last_step", "stba_problem_info", "stba_get_cluster_system", "stba_set_timing",
           "stba_stage_times", "stba_destroy", "stba_status_string", "stba_last_error", "stba_cost_noalloc",
           "stba_record", "stba_adjoint", "stba_graph_create", "stba_graph_edges", "stba_graph_cluster",
           "stba_graph_cluster_batch", "stba_graph_destroy", "stba_cluster_sgc", "stba_autotune", "stba_measure_peaks", "stba_set_shard", "stba_shard_owned"]


# transport of the sharded iteration: (user, data, count, dtype 0 = FP64 / 1 = FP32, stream) -> 0 on success
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                 ctypes.c_void_p)


class StbaOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("correction", ctypes.c_int32), ("lambda0", ctypes.c_double),
                ("lambda_min", ctypes.c_double), ("correction_lambda", ctypes.c_double),
                ("ftol", ctypes.c_double), ("gtol", ctypes.c_double), ("xtol", ctypes.c_double),
                ("refine_steps", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("linear_solver", ctypes.c_int32), ("pcg_max_iter", ctypes.c_int32), ("pcg_tol", ctypes.c_double),
                ("huber_a", ctypes.c_double), ("factor_tile", ctypes.c_int32), ("factor_update", ctypes.c_int32),
                ("factor_panel", ctypes.c_int32), ("solve_cluster", ctypes.c_int32),
                ("pair_blocks", ctypes.c_int32), ("factor_fp64", ctypes.c_int32)]


class StbaIterInfo(ctypes.Structure):
    _fields_ = [("F_before", ctypes.c_double), ("F_after", ctypes.c_double), ("lambda_used", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("grad_inf", ctypes.c_double), ("dx_norm", ctypes.c_double),
                ("x_norm", ctypes.c_double), ("accepted", ctypes.c_int32), ("stop", ctypes.c_int32),
                ("corrected", ctypes.c_int32), ("failed_clusters", ctypes.c_int32),
                ("boosted_pivots", ctypes.c_int32), ("linear_iterations", ctypes.c_int32),
                ("iteration", ctypes.c_int64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["lambda"] = d.pop("lambda_")
        for k in ("accepted", "stop", "corrected"):
            d[k] = bool(d[k])
        return d


class StbaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libstba.so (building it with nvcc first when absent or stale).  Raises if it cannot."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libstba.so not found at {_build.LIB}; run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    sig = {
        "stba_default_options": (None, [ctypes.POINTER(StbaOptions)]),
        "stba_create": (I32, [P, I64, P, I64, P, P, P, I64, P, ctypes.POINTER(StbaOptions), P, ctypes.POINTER(P)]),
        "stba_set_clusters": (I32, [P, P]),
        "stba_lm_iteration": (I32, [P, ctypes.POINTER(StbaIterInfo)]),
        "stba_solve": (I32, [P, I32, ctypes.POINTER(StbaIterInfo)]),
        "stba_cost": (I32, [P, ctypes.POINTER(D)]),
        "stba_get_params": (I32, [P, P, P]),
        "stba_set_params": (I32, [P, P, P]),
        "stba_get_state": (I32, [P, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(I64)]),
        "stba_set_state": (I32, [P, D, D, I64]),
        "stba_last_step": (I32, [P, P, P]),
        "stba_problem_info": (I32, [P, ctypes.POINTER(I64), I32]),
        "stba_get_cluster_system": (I32, [P, I32, P, P, ctypes.POINTER(I64)]),
        "stba_set_timing": (I32, [P, I32]),
        "stba_stage_times": (I32, [P, ctypes.POINTER(ctypes.c_float), I32, ctypes.POINTER(I32)]),
        "stba_destroy": (None, [P]),
        "stba_status_string": (ctypes.c_char_p, [I32]),
        "stba_last_error": (ctypes.c_char_p, [P]),
        "stba_cost_noalloc": (I32, [P, I64, P, I64, P, P, P, I64, P, P]),
        "stba_record": (I32, [P, I32]),
        "stba_adjoint": (I32, [P, P, P, P, P, P]),
        "stba_graph_create": (I32, [I64, I64, P, P, I64, ctypes.POINTER(P)]),
        "stba_graph_edges": (I32, [P, ctypes.POINTER(I64), P, P, P]),
        "stba_graph_cluster": (I32, [P, I32, D, ctypes.c_uint64, P, ctypes.POINTER(I32)]),
        "stba_graph_cluster_batch": (I32, [P, I32, D, ctypes.c_uint64, I32, P, P]),
        "stba_graph_destroy": (None, [P]),
        "stba_cluster_sgc": (I32, [P, I32, D, ctypes.c_uint64, I32, P, P]),
        "stba_autotune": (I32, [P, I32, ctypes.POINTER(I32), ctypes.POINTER(ctypes.c_float)]),
        "stba_measure_peaks": (I32, [P, I32, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "stba_set_shard": (I32, [P, I32, I32, ALLREDUCE_FN, P, I32]),
        "stba_shard_owned": (I32, [P, P, ctypes.POINTER(I32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


# ----------------------------------------------------------------------------------------------------------
# marshalling helpers
# ----------------------------------------------------------------------------------------------------------
def _ptr(a, dtype, keep):
    """Pointer to a contiguous array of `dtype`; keeps converted copies alive in `keep`."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            tdt = {np.float64: torch.float64, np.int32: torch.int32, np.float32: torch.float32}[dtype]
            t = a.detach().to(tdt).contiguous()
            keep.append(t)
            return ctypes.c_void_p(t.data_ptr())
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    keep.append(arr)
    return ctypes.c_void_p(arr.ctypes.data)


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


def stba_default_options(**overrides) -> StbaOptions:
    o = StbaOptions()
    load().stba_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Context:
    """Owns one stba_ctx*.  Use the module functions below or the methods of the same names."""

    def __init__(self, handle, m, n, q):
        self.handle = handle
        self.m, self.n, self.q = m, n, q

    def _check(self, status):
        if status != 0:
            msg = load().stba_last_error(self.handle).decode()
            raise StbaError(status, msg)

    def close(self):
        if self.handle:
            load().stba_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def stba_create(cameras, points, obs_cam, obs_pt, obs_uv, cluster_assignment, options=None, stream=None,
                **option_overrides) -> Context:
    L = load()
    keep = []
    m, n, q = len(cameras), len(points), len(obs_cam)
    opt = options if options is not None else stba_default_options(**option_overrides)
    h = ctypes.c_void_p()
    st = L.stba_create(_ptr(cameras, np.float64, keep), m, _ptr(points, np.float64, keep), n,
                       _ptr(obs_cam, np.int32, keep), _ptr(obs_pt, np.int32, keep), _ptr(obs_uv, np.float64, keep),
                       q, _ptr(cluster_assignment, np.int32, keep), ctypes.byref(opt), _stream_handle(stream),
                       ctypes.byref(h))
    if st != 0:
        raise StbaError(st, L.stba_last_error(None).decode())
    return Context(h, m, n, q)


def stba_set_clusters(ctx: Context, cluster_assignment):
    keep = []
    ctx._check(load().stba_set_clusters(ctx.handle, _ptr(cluster_assignment, np.int32, keep)))


def stba_lm_iteration(ctx: Context, want_info=True):
    info = StbaIterInfo()
    ctx._check(load().stba_lm_iteration(ctx.handle, ctypes.byref(info) if want_info else None))
    return info.as_dict() if want_info else None


def stba_solve(ctx: Context, max_iter: int):
    info = StbaIterInfo()
    ctx._check(load().stba_solve(ctx.handle, int(max_iter), ctypes.byref(info)))
    return info.as_dict()


def stba_cost(ctx: Context) -> float:
    F = ctypes.c_double()
    ctx._check(load().stba_cost(ctx.handle, ctypes.byref(F)))
    return F.value


def stba_get_params(ctx: Context, cameras=None, points=None):
    """Copies the parameters into the given arrays (NumPy or torch, host or device) or new NumPy arrays."""
    cams = cameras if cameras is not None else np.empty((ctx.m, 9))
    pts = points if points is not None else np.empty((ctx.n, 3))
    ctx._check(load().stba_get_params(ctx.handle, ctypes.c_void_p(_data_ptr(cams)), ctypes.c_void_p(_data_ptr(pts))))
    return cams, pts


def stba_set_params(ctx: Context, cameras=None, points=None):
    keep = []
    pc = _ptr(cameras, np.float64, keep) if cameras is not None else None
    pp = _ptr(points, np.float64, keep) if points is not None else None
    ctx._check(load().stba_set_params(ctx.handle, pc, pp))


def stba_get_state(ctx: Context):
    lam, F, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    ctx._check(load().stba_get_state(ctx.handle, ctypes.byref(lam), ctypes.byref(F), ctypes.byref(it)))
    return lam.value, F.value, it.value


def stba_set_state(ctx: Context, lam: float, F: float = -1.0, iteration: int = 0):
    ctx._check(load().stba_set_state(ctx.handle, float(lam), float(F), int(iteration)))


def stba_last_step(ctx: Context):
    dc = np.empty((ctx.m, 9))
    dp = np.empty((ctx.n, 3))
    ctx._check(load().stba_last_step(ctx.handle, ctypes.c_void_p(dc.ctypes.data), ctypes.c_void_p(dp.ctypes.data)))
    return dc, dp


def stba_problem_info(ctx: Context):
    keys = ["m", "n", "q", "l", "nv", "max_dim", "device_bytes", "build_items", "launches_per_iter",
            "pair_instances", "factor_flops", "s_lower_elems"]
    out = (ctypes.c_int64 * len(keys))()
    ctx._check(load().stba_problem_info(ctx.handle, out, len(keys)))
    return dict(zip(keys, list(out)))


def stba_get_cluster_system(ctx: Context, k: int):
    dim = ctypes.c_int64()
    ctx._check(load().stba_get_cluster_system(ctx.handle, int(k), None, None, ctypes.byref(dim)))
    S = np.empty((dim.value, dim.value))
    b = np.empty(dim.value)
    ctx._check(load().stba_get_cluster_system(ctx.handle, int(k), ctypes.c_void_p(S.ctypes.data),
                                              ctypes.c_void_p(b.ctypes.data), ctypes.byref(dim)))
    return S, b


def stba_set_timing(ctx: Context, on: bool):
    ctx._check(load().stba_set_timing(ctx.handle, int(bool(on))))


def stba_stage_times(ctx: Context):
    ms = (ctypes.c_float * 16)()
    cnt = ctypes.c_int32()
    ctx._check(load().stba_stage_times(ctx.handle, ms, 16, ctypes.byref(cnt)))
    return list(ms)[: cnt.value]


def _noalloc_check(cameras, points, obs_cam, obs_pt, obs_uv, F_out):
    """Validation of stba_cost_noalloc's arguments, before anything reaches the device.  Shapes come first
    (the library sizes every device read from them), then dtype, contiguity, and one CUDA device for all."""
    import torch
    args = (("cameras", cameras, torch.float64), ("points", points, torch.float64), ("obs_cam", obs_cam, torch.int32),
            ("obs_pt", obs_pt, torch.int32), ("obs_uv", obs_uv, torch.float64), ("F_out", F_out, torch.float64))
    for name, t, _ in args:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"stba_cost_noalloc: {name} must be a torch tensor")
    m, n, q = cameras.shape[0] if cameras.dim() else -1, points.shape[0] if points.dim() else -1, \
        obs_cam.shape[0] if obs_cam.dim() else -1
    want = (("cameras", cameras, (m, 9)), ("points", points, (n, 3)), ("obs_cam", obs_cam, (q,)),
            ("obs_pt", obs_pt, (q,)), ("obs_uv", obs_uv, (q, 2)))
    for name, t, shape in want:
        if tuple(t.shape) != shape or min(shape) < 1:
            raise ValueError(f"stba_cost_noalloc: {name} has shape {tuple(t.shape)}, expected {shape} with m, n, q >= 1")
    if F_out.numel() < 1:
        raise ValueError("stba_cost_noalloc: F_out must hold at least one float64")
    for name, t, dt in args:
        if t.dtype != dt or not t.is_contiguous():
            raise TypeError(f"stba_cost_noalloc: {name} must be a contiguous {dt} tensor "
                            "(nothing is converted here, since a conversion would allocate)")
    for name, t, _ in args:
        if not t.is_cuda or t.device != F_out.device:
            raise TypeError(f"stba_cost_noalloc: every tensor must be on one CUDA device ({name} is on {t.device}, "
                            f"F_out on {F_out.device})")
    return m, n, q


def stba_cost_noalloc(cameras, points, obs_cam, obs_pt, obs_uv, F_out, stream=None):
    """F(x) into the device scalar F_out without any device allocation by the library.  Every array must
    already be a contiguous CUDA tensor of the right shape and dtype (float64 / int32) on one device: nothing
    is converted or copied here, since a conversion would allocate.  The call runs with that device current
    (its static scratch and, by default, its current stream)."""
    import torch
    m, n, q = _noalloc_check(cameras, points, obs_cam, obs_pt, obs_uv, F_out)
    with torch.cuda.device(F_out.device):
        st = load().stba_cost_noalloc(ctypes.c_void_p(cameras.data_ptr()), m, ctypes.c_void_p(points.data_ptr()), n,
                                      ctypes.c_void_p(obs_cam.data_ptr()), ctypes.c_void_p(obs_pt.data_ptr()),
                                      ctypes.c_void_p(obs_uv.data_ptr()), q, ctypes.c_void_p(F_out.data_ptr()),
                                      _stream_handle(stream))
    if st != 0:
        raise StbaError(st, "stba_cost_noalloc failed")


def stba_measure_peaks(reps=5, stream=None):
    """Measured FP32 CUDA-core and dense TF32 tensor-core rates of the current GPU: (fp32_tflops, tf32_tflops)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    st = load().stba_measure_peaks(_stream_handle(stream), int(reps), ctypes.byref(a), ctypes.byref(b))
    if st != 0:
        raise StbaError(st, "stba_measure_peaks failed")
    return a.value, b.value


def gloo_allreduce(group=None):
    """A transport for stba_set_shard over torch.distributed (e.g. the gloo backend): sums a host NumPy array
    over the ranks in place."""
    import torch
    import torch.distributed as dist

    def allreduce(arr):
        dist.all_reduce(torch.from_numpy(arr), group=group)
    return allreduce


def stba_set_shard(ctx: Context, rank: int, world: int, allreduce=None):
    """Sharded iteration (one process per rank, each with its own context): this rank builds, factors and
    solves only its clusters; `allreduce(arr)` sums a NumPy array in place over the ranks (the library stages
    the exchanged values in host memory).  world = 1 returns to the single-process iteration."""
    if world > 1:
        if allreduce is None:
            raise ValueError("a sharded iteration needs a transport (allreduce)")

        def cb(user, data, count, dtype, stream):
            try:
                ct = ctypes.c_double if dtype == 0 else ctypes.c_float
                allreduce(np.ctypeslib.as_array(ctypes.cast(data, ctypes.POINTER(ct)), shape=(int(count),)))
                return 0
            except Exception:   # reported to the library as a failed exchange
                return 1
        fn = ALLREDUCE_FN(cb)
    else:
        fn = ALLREDUCE_FN()
    ctx._shard_cb = fn   # the library keeps the pointer; the Python object must outlive the context's use of it
    ctx._check(load().stba_set_shard(ctx.handle, int(rank), int(world), fn, None, 1))


def stba_shard_owned(ctx: Context) -> np.ndarray:
    """Clusters of the current assignment owned by this rank (0 / 1 per cluster)."""
    l = ctypes.c_int32()
    ctx._check(load().stba_shard_owned(ctx.handle, None, ctypes.byref(l)))
    out = np.zeros(l.value, np.int32)
    ctx._check(load().stba_shard_owned(ctx.handle, ctypes.c_void_p(out.ctypes.data), ctypes.byref(l)))
    return out


def stba_autotune(ctx: Context, iterations=5):
    """Times the candidate factorisations (AUTOTUNE_CANDIDATES, in order) and keeps the fastest:
    (name of the kept candidate or None, {candidate: ms per iteration})."""
    choice = ctypes.c_int32()
    names = list(AUTOTUNE_CANDIDATES)
    ms = (ctypes.c_float * len(names))()
    ctx._check(load().stba_autotune(ctx.handle, int(iterations), ctypes.byref(choice), ms))
    return (names[choice.value] if choice.value >= 0 else None), {nm: ms[i] for i, nm in enumerate(names)}


def stba_record(ctx: Context, max_iter: int):
    """Start (or restart, or with 0 free) the tape of the next `max_iter` iterations for stba_adjoint."""
    ctx._check(load().stba_record(ctx.handle, int(max_iter)))


def stba_adjoint(ctx: Context, dL_dcams, dL_dpts=None):
    """Reverse-mode derivative of the recorded iterations.  Returns (dL/d obs_uv [q][2] in input order,
    dL/d cameras0 [m][9], dL/d points0 [n][3]) as float64 arrays: CUDA tensors on the device of dL_dcams
    when it is a CUDA tensor, NumPy arrays otherwise."""
    keep = []
    pc = _ptr(dL_dcams, np.float64, keep)
    pp = _ptr(dL_dpts, np.float64, keep) if dL_dpts is not None else None
    on_cuda = False
    try:
        import torch
        on_cuda = isinstance(dL_dcams, torch.Tensor) and dL_dcams.is_cuda
    except ImportError:
        pass
    if on_cuda:
        import torch
        dev = dL_dcams.device
        gq = torch.empty((ctx.q, 2), dtype=torch.float64, device=dev)
        gc = torch.empty((ctx.m, 9), dtype=torch.float64, device=dev)
        gp = torch.empty((ctx.n, 3), dtype=torch.float64, device=dev)
        ptrs = [ctypes.c_void_p(t.data_ptr()) for t in (gq, gc, gp)]
    else:
        gq, gc, gp = np.empty((ctx.q, 2)), np.empty((ctx.m, 9)), np.empty((ctx.n, 3))
        ptrs = [ctypes.c_void_p(a.ctypes.data) for a in (gq, gc, gp)]
    ctx._check(load().stba_adjoint(ctx.handle, pc, pp, *ptrs))
    return gq, gc, gp


def stba_destroy(ctx: Context):
    ctx.close()


def _data_ptr(a):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            assert a.is_contiguous() and a.dtype == torch.float64
            return a.data_ptr()
    except ImportError:
        pass
    assert isinstance(a, np.ndarray) and a.flags.c_contiguous and a.dtype == np.float64
    return a.ctypes.data


# ----------------------------------------------------------------------------------------------------------
# autograd
# ----------------------------------------------------------------------------------------------------------
def _autograd_function():
    import torch

    class STBAFunction(torch.autograd.Function):
        """(cameras_K, points_K) = K STBA LM iterations from (cameras0, points0) on the observations obs_uv.

        forward: one context, a tape of K iterations (the cluster assignment of iteration t is
        cluster_seq[t], or cluster_seq itself when it is one assignment).  backward: stba_adjoint, the
        derivative with the damping, clusters and accept flags of the forward run held fixed.  Gradients
        come back in the dtype of each input."""

        @staticmethod
        def forward(fctx, cameras0, points0, obs_uv, obs_cam, obs_pt, cluster_seq, iters, options):
            seq = cluster_seq
            per_iter = getattr(seq, "ndim", 1) == 2
            first = seq[0] if per_iter else seq
            sctx = stba_create(cameras0, points0, obs_cam, obs_pt, obs_uv, first, options=options)
            stba_record(sctx, int(iters))
            for t in range(int(iters)):
                if per_iter and t > 0:
                    stba_set_clusters(sctx, seq[t])
                stba_lm_iteration(sctx, want_info=False)
            dev = cameras0.device
            cams = torch.empty((sctx.m, 9), dtype=torch.float64, device=dev)
            pts = torch.empty((sctx.n, 3), dtype=torch.float64, device=dev)
            stba_get_params(sctx, cams, pts)
            fctx.stba = sctx
            fctx.dtypes = (cameras0.dtype, points0.dtype, obs_uv.dtype)
            return cams.to(cameras0.dtype), pts.to(points0.dtype)

        @staticmethod
        def backward(fctx, g_cams, g_pts):
            dev = g_cams.device if g_cams is not None else g_pts.device
            gc_in = (g_cams if g_cams is not None else torch.zeros((fctx.stba.m, 9), device=dev)).to(torch.float64)
            gp_in = g_pts.to(torch.float64) if g_pts is not None else None
            gq, gc, gp = stba_adjoint(fctx.stba, gc_in.contiguous(), gp_in.contiguous() if gp_in is not None else None)
            tc, tp, tq = fctx.dtypes
            return gc.to(tc), gp.to(tp), gq.to(tq), None, None, None, None, None

    return STBAFunction


def stba_differentiable(cameras0, points0, obs_uv, obs_cam, obs_pt, cluster_seq, iters, options=None):
    """K STBA iterations as a differentiable function of (cameras0, points0, obs_uv) (torch tensors)."""
    global _STBA_FN
    if _STBA_FN is None:
        _STBA_FN = _autograd_function()
    return _STBA_FN.apply(cameras0, points0, obs_uv, obs_cam, obs_pt, cluster_seq, iters, options)


_STBA_FN = None


# ----------------------------------------------------------------------------------------------------------
# camera graph and stochastic graph clustering (host only)
# ----------------------------------------------------------------------------------------------------------
class CameraGraph:
    """Owns one stba_graph* (stba_graph_create)."""

    def __init__(self, handle, m):
        self.handle = handle
        self.m = m

    def close(self):
        if self.handle:
            load().stba_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _graph_check(status):
    if status != 0:
        raise StbaError(status, load().stba_last_error(None).decode())


def stba_graph_create(m, n, obs_cam, obs_pt) -> CameraGraph:
    c = np.ascontiguousarray(obs_cam, dtype=np.int32)
    p = np.ascontiguousarray(obs_pt, dtype=np.int32)
    h = ctypes.c_void_p()
    _graph_check(load().stba_graph_create(int(m), int(n), ctypes.c_void_p(c.ctypes.data),
                                          ctypes.c_void_p(p.ctypes.data), len(c), ctypes.byref(h)))
    return CameraGraph(h, int(m))


def stba_graph_edges(g: CameraGraph):
    """(i, j, w) arrays of the edges, i < j."""
    E = ctypes.c_int64()
    _graph_check(load().stba_graph_edges(g.handle, ctypes.byref(E), None, None, None))
    i = np.empty(E.value, np.int32)
    j = np.empty(E.value, np.int32)
    w = np.empty(E.value, np.int64)
    _graph_check(load().stba_graph_edges(g.handle, ctypes.byref(E), ctypes.c_void_p(i.ctypes.data),
                                         ctypes.c_void_p(j.ctypes.data), ctypes.c_void_p(w.ctypes.data)))
    return i, j, w


def stba_graph_cluster(g: CameraGraph, gamma=100, beta=10.0, seed=0):
    """(assignment [m] int32, number of clusters)."""
    out = np.empty(g.m, np.int32)
    l = ctypes.c_int32()
    _graph_check(load().stba_graph_cluster(g.handle, int(gamma), float(beta), int(seed),
                                           ctypes.c_void_p(out.ctypes.data), ctypes.byref(l)))
    return out, l.value


def stba_graph_cluster_batch(g: CameraGraph, count, gamma=100, beta=10.0, seed=0):
    """(assignments [count][m] int32, cluster counts [count])."""
    out = np.empty((int(count), g.m), np.int32)
    l = np.empty(int(count), np.int32)
    _graph_check(load().stba_graph_cluster_batch(g.handle, int(gamma), float(beta), int(seed), int(count),
                                                 ctypes.c_void_p(out.ctypes.data), ctypes.c_void_p(l.ctypes.data)))
    return out, l


def stba_cluster_sgc(ctx: Context, count=1, gamma=100, beta=10.0, seed=0):
    """count clusterings of the context's camera graph: (assignments [count][m], cluster counts [count])."""
    out = np.empty((int(count), ctx.m), np.int32)
    l = np.empty(int(count), np.int32)
    ctx._check(load().stba_cluster_sgc(ctx.handle, int(gamma), float(beta), int(seed), int(count),
                                       ctypes.c_void_p(out.ctypes.data), ctypes.c_void_p(l.ctypes.data)))
    return out, l
