"""ctypes binding of the C ABI in include/irk.h (argument marshalling only).

Every function below calls the entry point of the same name in libirk.so;
all numerical work runs in the library's CUDA kernels.  Arrays may be NumPy
arrays (host memory) or torch tensors (host or CUDA memory); they must be
float64 and contiguous.  Importing this module raises if the library has not
been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

# IRK_LIBRARY selects another build of the same library (the bounds-checked
# one, _lib/libirk_bounds.so); the default is the optimised build.
_LIB_PATH = os.environ.get("IRK_LIBRARY") or _build.LIB

IRK_OK = 0
IRK_ERR_INVALID = 1
IRK_ERR_NOMEM = 2
IRK_ERR_CUDA = 3
IRK_ERR_NEWTON_DIVERGED = 4
IRK_ERR_NEWTON_MAXIT = 5
IRK_ERR_KRYLOV_BREAKDOWN = 6
IRK_ERR_TIMEOUT = 7
IRK_ERR_NO_DEVICE = 8

IRK_GAUSS, IRK_RADAU_IIA, IRK_LOBATTO_IIIC, IRK_SDIRK = 0, 1, 2, 3
IRK_BASIS_SCHUR, IRK_BASIS_EIGEN = 0, 1
FAMILY_NAMES = {"gauss": IRK_GAUSS, "radau": IRK_RADAU_IIA, "lobatto": IRK_LOBATTO_IIIC,
                "sdirk": IRK_SDIRK}
IRK_OP_DIFFUSION_1D, IRK_OP_BURGERS_1D, IRK_OP_BURGERS_2D, IRK_OP_VSF_2D = 0, 1, 2, 3
IRK_MASS_IDENTITY, IRK_MASS_DAE = 0, 1
IRK_MG_FP64, IRK_MG_FP32, IRK_MG_BF16 = 0, 1, 2

OP_NAMES = {"diffusion1d": IRK_OP_DIFFUSION_1D, "burgers1d": IRK_OP_BURGERS_1D,
            "burgers2d": IRK_OP_BURGERS_2D, "vsf": IRK_OP_VSF_2D}


class IrkConfig(C.Structure):
    _fields_ = [
        ("family", C.c_int), ("stages", C.c_int), ("op", C.c_int), ("mass", C.c_int),
        ("n", C.c_int), ("length", C.c_double), ("nu", C.c_double), ("forcing", C.c_int),
        ("newton_rtol", C.c_double), ("newton_maxit", C.c_int),
        ("krylov_rtol", C.c_double), ("krylov_restart", C.c_int), ("krylov_maxit", C.c_int),
        ("nonlinear_variant", C.c_int), ("gamma_mode", C.c_int),
        ("mg_precision", C.c_int), ("mg_levels", C.c_int), ("mg_pre", C.c_int),
        ("mg_post", C.c_int), ("mg_coarse_sweeps", C.c_int), ("mg_omega", C.c_double),
        ("profile", C.c_int), ("use_graphs", C.c_int), ("initial_guess", C.c_int),
        ("basis", C.c_int), ("mg_shifted_sweeps", C.c_int), ("mg_coarse_reduction", C.c_double),
        ("mg_coarse_smoother", C.c_int), ("dirk_sequential", C.c_int), ("dae_solver", C.c_int),
        ("mg_tile_rows", C.c_int),
        ("mg_fuse_transfer", C.c_int),
    ]


class IrkStats(C.Structure):
    _fields_ = [
        ("steps", C.c_int), ("newton_its", C.c_int), ("krylov_its", C.c_int),
        ("prec_apps", C.c_int), ("vcycles", C.c_int), ("max_newton_its", C.c_int),
        ("final_rel_res", C.c_double), ("kernel_launches", C.c_longlong),
        ("outer_its", C.c_int), ("poisson_vcycles", C.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class IrkKernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_longlong), ("ms", C.c_double),
                ("bytes", C.c_double), ("flops", C.c_double)]


class IrkServerStats(C.Structure):
    _fields_ = [
        ("submitted", C.c_longlong), ("completed", C.c_longlong), ("failed", C.c_longlong),
        ("steps", C.c_longlong), ("wall_s", C.c_double), ("steps_per_s", C.c_double),
        ("p50_step_ms", C.c_double), ("p99_step_ms", C.c_double), ("max_step_ms", C.c_double),
        ("p50_request_ms", C.c_double), ("p99_request_ms", C.c_double),
        ("p50_queue_ms", C.c_double), ("p99_queue_ms", C.c_double),
        ("peak_active", C.c_int), ("slots", C.c_int),
        ("budget_bytes", C.c_size_t), ("peak_bytes", C.c_size_t),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class IrkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with "
                          "`python -m paper_2101_01776_gb300.build` (needs nvcc)")
    lib = C.CDLL(_LIB_PATH)
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    P = C.POINTER
    sig = {
        "irk_config_default": (None, [P(IrkConfig)]),
        "irk_create": (i, [P(IrkConfig), vp, i, vp, P(vp)]),
        "irk_step": (i, [vp, d, d, i, P(IrkStats)]),
        "irk_get_state": (i, [vp, vp, i]),
        "irk_set_state": (i, [vp, vp, i]),
        "irk_set_state_keep_stages": (i, [vp, vp, i]),
        "irk_get_stages": (i, [vp, vp, i]),
        "irk_set_stages": (i, [vp, vp, i]),
        "irk_stage_residual": (i, [vp, d, d, vp, vp, i]),
        "irk_stage_jacobian_apply": (i, [vp, d, vp, vp, vp, i]),
        "irk_tableau": (i, [i, i, vp, vp, vp, vp, vp, vp, vp]),
        "irk_transform": (i, [i, i, i, vp, vp, vp, vp, vp]),
        "irk_get_config": (i, [vp, P(IrkConfig)]),
        "irk_autotune": (i, [vp, d, d, i, P(IrkConfig)]),
        "irk_kernel_stats": (i, [vp, P(IrkKernelStat), i, P(i)]),
        "irk_reset_kernel_stats": (i, [vp]),
        "irk_device_bytes": (sz, [vp]),
        "irk_last_error": (C.c_char_p, [vp]),
        "irk_status_string": (C.c_char_p, [i]),
        "irk_destroy": (None, [vp]),
        "irk_stage_residual_noalloc": (i, [i, i, d, d, i, vp, d, vp, vp, vp, vp, vp]),
        "irk_measure_alu_peak": (i, [i, vp, P(d)]),
        "irk_config_device_bytes": (sz, [P(IrkConfig)]),
        "irk_create_in": (i, [P(IrkConfig), vp, i, vp, vp, sz, P(vp)]),
        "irk_server_create": (i, [i, sz, P(vp)]),
        "irk_server_create_batched": (i, [i, i, i, sz, P(vp)]),
        "irk_server_submit": (i, [vp, P(IrkConfig), vp, d, d, i, P(C.c_longlong)]),
        "irk_server_wait": (i, [vp, C.c_longlong, vp, P(IrkStats), vp]),
        "irk_server_stats_get": (i, [vp, P(IrkServerStats)]),
        "irk_server_destroy": (None, [vp]),
        "irk_debug_bounds": (C.c_longlong, [i, C.c_char_p, sz]),
        "irk_batch_create": (i, [i, vp, P(vp)]),
        "irk_batch_instance_bytes": (sz, [P(IrkConfig)]),
        "irk_batch_add": (i, [vp, P(IrkConfig), vp, i, d, vp, sz, P(i)]),
        "irk_batch_step": (i, [vp, vp, vp]),
        "irk_batch_get_state": (i, [vp, i, vp, i]),
        "irk_batch_get_stages": (i, [vp, i, vp, i]),
        "irk_batch_remove": (i, [vp, i]),
        "irk_batch_count": (i, [vp]),
        "irk_batch_last_error": (C.c_char_p, [vp]),
        "irk_batch_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()
EXPORTED = (
    "irk_config_default", "irk_create", "irk_step", "irk_get_state", "irk_set_state",
    "irk_get_stages", "irk_set_stages", "irk_stage_residual", "irk_stage_jacobian_apply", "irk_tableau",
    "irk_kernel_stats", "irk_reset_kernel_stats", "irk_device_bytes", "irk_last_error",
    "irk_status_string", "irk_destroy", "irk_stage_residual_noalloc",
    "irk_config_device_bytes", "irk_create_in", "irk_server_create", "irk_server_submit",
    "irk_server_wait", "irk_server_stats_get", "irk_server_destroy", "irk_transform",
    "irk_get_config", "irk_autotune", "irk_set_state_keep_stages", "irk_debug_bounds",
    "irk_measure_alu_peak", "irk_batch_create", "irk_batch_instance_bytes", "irk_batch_add",
    "irk_batch_step", "irk_batch_get_state", "irk_batch_get_stages", "irk_batch_remove",
    "irk_batch_count", "irk_batch_last_error", "irk_batch_destroy", "irk_server_create_batched",
)


def status_string(st: int) -> str:
    return LIB.irk_status_string(st).decode()


def irk_config_default(**overrides) -> IrkConfig:
    cfg = IrkConfig()
    LIB.irk_config_default(C.byref(cfg))
    for k, v in overrides.items():
        if k == "op" and isinstance(v, str):
            v = OP_NAMES[v]
        if k == "family" and isinstance(v, str):
            v = FAMILY_NAMES[v]
        if not hasattr(cfg, k):
            raise AttributeError(f"irk_config has no field {k!r}")
        setattr(cfg, k, v)
    if "op" in overrides and "mass" not in overrides:
        cfg.mass = IRK_MASS_DAE if cfg.op == IRK_OP_VSF_2D else IRK_MASS_IDENTITY
    return cfg


def _ptr(x):
    """(address, on_device) of a contiguous float64 NumPy array or torch tensor."""
    if hasattr(x, "data_ptr"):  # torch tensor
        if not x.is_contiguous() or str(x.dtype) != "torch.float64":
            raise ValueError("tensor must be contiguous float64")
        return C.c_void_p(x.data_ptr()), int(x.is_cuda)
    import numpy as np
    if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
        raise ValueError("array must be a contiguous float64 numpy array")
    return C.c_void_p(x.ctypes.data), 0


def _nbytes(x) -> int:
    return x.numel() * x.element_size() if hasattr(x, "data_ptr") else x.nbytes


def _state_len(cfg) -> int:
    """Values of one state vector: ncomp * n^dim (the 2D operators carry two fields)."""
    two_d = cfg.op in (IRK_OP_BURGERS_2D, IRK_OP_VSF_2D)
    return (2 if two_d else 1) * cfg.n ** (2 if two_d else 1)


def _need(x, count: int, what: str):
    """The library copies `count` float64 values through the pointer: refuse a
    smaller buffer here instead of letting the copy run past its end."""
    if _nbytes(x) < 8 * count:
        raise ValueError(f"{what} holds {_nbytes(x) // 8} float64 values; {count} are needed")


def _need_state(cfg, u0):
    # only for a valid config (device bytes > 0); irk_create reports the others
    if LIB.irk_config_device_bytes(C.byref(cfg)) > 0:
        _need(u0, _state_len(cfg), "u0")


# handle address -> (state values, stages); op, n and stages are fixed at
# irk_create, and irk_destroy drops the entry
_HANDLE_SIZES = {}


def _handle_len(h, stages: bool) -> int:
    key = getattr(h, "value", h)
    if key not in _HANDLE_SIZES:
        cfg = irk_get_config(h)
        _HANDLE_SIZES[key] = (_state_len(cfg), cfg.stages)
    n, s = _HANDLE_SIZES[key]
    return n * (s if stages else 1)


def _check(st: int, handle=None):
    if st != IRK_OK:
        msg = LIB.irk_last_error(handle).decode(errors="replace")
        raise IrkError(st, msg)


def irk_create(cfg: IrkConfig, u0, stream=None):
    """Return an opaque handle (c_void_p).  stream: torch.cuda.Stream, raw handle or None."""
    h = C.c_void_p()
    p, dev = _ptr(u0)
    _need_state(cfg, u0)
    sp = None
    if stream is not None:
        sp = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(LIB.irk_create(C.byref(cfg), p, dev, sp, C.byref(h)))
    return h


def irk_step(h, t_n: float, dt: float, nsteps: int = 1) -> IrkStats:
    st = IrkStats()
    _check(LIB.irk_step(h, t_n, dt, nsteps, C.byref(st)), h)
    return st


def irk_get_state(h, dst):
    p, dev = _ptr(dst)
    _need(dst, _handle_len(h, False), "dst")
    _check(LIB.irk_get_state(h, p, dev), h)
    return dst


def irk_set_state(h, src):
    p, dev = _ptr(src)
    _need(src, _handle_len(h, False), "src")
    _check(LIB.irk_set_state(h, p, dev), h)


def irk_set_state_keep_stages(h, src):
    p, dev = _ptr(src)
    _need(src, _handle_len(h, False), "src")
    _check(LIB.irk_set_state_keep_stages(h, p, dev), h)


def irk_get_stages(h, dst):
    p, dev = _ptr(dst)
    _need(dst, _handle_len(h, True), "dst")
    _check(LIB.irk_get_stages(h, p, dev), h)
    return dst


def irk_set_stages(h, src):
    p, dev = _ptr(src)
    _need(src, _handle_len(h, True), "src")
    _check(LIB.irk_set_stages(h, p, dev), h)


def irk_stage_residual(h, t_n: float, dt: float, K, F):
    pk, dk = _ptr(K)
    pf, df = _ptr(F)
    if dk != df:
        raise ValueError("K and F must live in the same memory space")
    n = _handle_len(h, True)
    _need(K, n, "K")
    _need(F, n, "F")
    _check(LIB.irk_stage_residual(h, t_n, dt, pk, pf, dk), h)
    return F


def irk_stage_jacobian_apply(h, dt: float, K, V, JV):
    (pk, dk), (pv, dv), (pj, dj) = _ptr(K), _ptr(V), _ptr(JV)
    if not (dk == dv == dj):
        raise ValueError("K, V and JV must live in the same memory space")
    n = _handle_len(h, True)
    for x, what in ((K, "K"), (V, "V"), (JV, "JV")):
        _need(x, n, what)
    _check(LIB.irk_stage_jacobian_apply(h, dt, pk, pv, pj, dk), h)
    return JV


def irk_stage_residual_noalloc(op, n: int, length: float, nu: float, stages: int, A, dt: float,
                               u, K, F, fnorm, stream=None):
    """Stage residual and ||F|| with no device allocation (all tensors on the
    device; A a host float64 array).  Enqueued on `stream`; not synchronised."""
    import numpy as np
    if isinstance(op, str):
        op = OP_NAMES[op]
    A = np.ascontiguousarray(A, dtype=np.float64)
    ptrs = [_ptr(x) for x in (u, K, F, fnorm)]
    if not all(dev for _, dev in ptrs):
        raise ValueError("u, K, F and fnorm must be device tensors")
    devices = {x.device for x in (u, K, F, fnorm)}
    if len(devices) != 1:
        raise ValueError("u, K, F and fnorm must live on one device")
    two_d = op in (IRK_OP_BURGERS_2D, IRK_OP_VSF_2D)
    npts = n ** (2 if two_d else 1) if isinstance(n, int) and n > 0 else 0
    # sizes matter only for calls the library would run: a known op, 1..5
    # stages, n a power of two >= 8 and at most 2^20 points (its scratch
    # limit); it rejects the others before touching any buffer
    if op in (IRK_OP_DIFFUSION_1D, IRK_OP_BURGERS_1D, IRK_OP_BURGERS_2D, IRK_OP_VSF_2D) and \
            1 <= stages <= 5 and npts and n >= 8 and not (n & (n - 1)) and npts <= 1 << 20:
        L = (2 if two_d else 1) * npts
        _need(A, stages * stages, "A")
        _need(u, L, "u")
        _need(K, stages * L, "K")
        _need(F, stages * L, "F")
        _need(fnorm, 1, "fnorm")
    sp = None
    if stream is not None:
        sp = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    import torch
    with torch.cuda.device(u.device):  # the library runs on the current device
        st = LIB.irk_stage_residual_noalloc(op, n, length, nu, stages, A.ctypes.data, dt,
                                            *[p for p, _ in ptrs], sp)
    if st != IRK_OK:
        raise IrkError(st, "irk_stage_residual_noalloc rejected the call (see stderr)")


def irk_measure_alu_peak(precision: int = 0, stream=None) -> float:
    """Measured FMA throughput of the current device in TFLOP/s (0 = FP64, 1 = FP32)."""
    sp = None
    if stream is not None:
        sp = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    out = C.c_double()
    _check(LIB.irk_measure_alu_peak(precision, sp, C.byref(out)))
    return out.value


def irk_config_device_bytes(cfg: IrkConfig) -> int:
    return int(LIB.irk_config_device_bytes(C.byref(cfg)))


def irk_create_in(cfg: IrkConfig, u0, arena_ptr: int, arena_bytes: int, stream=None):
    h = C.c_void_p()
    p, dev = _ptr(u0)
    _need_state(cfg, u0)
    sp = None
    if stream is not None:
        sp = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(LIB.irk_create_in(C.byref(cfg), p, dev, sp, C.c_void_p(arena_ptr), arena_bytes,
                             C.byref(h)))
    return h


def irk_server_create(slots: int, budget_bytes: int = 0):
    s = C.c_void_p()
    _check(LIB.irk_server_create(slots, budget_bytes, C.byref(s)))
    return s


def irk_server_create_batched(capacity: int, budget_bytes: int = 0, stream_slots: int = 0,
                              stream_min_n: int = 0):
    s = C.c_void_p()
    _check(LIB.irk_server_create_batched(capacity, stream_slots, stream_min_n, budget_bytes,
                                         C.byref(s)))
    return s


# (server address, request id) -> (state values, steps) of each submitted
# request, so that irk_server_wait hands the library buffers of the right size
_SUBMITTED = {}


def irk_server_submit(s, cfg: IrkConfig, u0, t0: float, dt: float, nsteps: int) -> int:
    import numpy as np
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    _need_state(cfg, u0)
    rid = C.c_longlong()
    _check(LIB.irk_server_submit(s, C.byref(cfg), u0.ctypes.data, t0, dt, nsteps, C.byref(rid)))
    _SUBMITTED[(getattr(s, "value", s), rid.value)] = (_state_len(cfg), nsteps)
    return rid.value


def irk_server_wait(s, rid: int, shape, nsteps: int):
    """(final state, IrkStats, per-step wall ms) of request rid (host arrays)."""
    import numpy as np
    out = np.empty(shape)
    known = _SUBMITTED.pop((getattr(s, "value", s), rid), None)
    if known is not None:
        _need(out, known[0], "shape")
        nsteps = known[1]
    st = IrkStats()
    ms = np.empty(max(nsteps, 1))
    code = LIB.irk_server_wait(s, rid, out.ctypes.data, C.byref(st), ms.ctypes.data)
    if code != IRK_OK:
        raise IrkError(code, f"request {rid} failed")
    return out, st, ms[:nsteps]


def irk_server_stats_get(s) -> dict:
    o = IrkServerStats()
    _check(LIB.irk_server_stats_get(s, C.byref(o)))
    return o.as_dict()


def irk_server_destroy(s):
    LIB.irk_server_destroy(s)


def irk_tableau(s: int, family: int = IRK_GAUSS):
    """Host-only tableau and real Schur form: dict of numpy arrays."""
    import numpy as np
    A, Q, R = (np.zeros((s, s)) for _ in range(3))
    b, c = np.zeros(s), np.zeros(s)
    bs = np.zeros(s, dtype=np.int32)
    nb = C.c_int()
    _check(LIB.irk_tableau(family, s, A.ctypes.data, b.ctypes.data, c.ctypes.data,
                           Q.ctypes.data, R.ctypes.data, bs.ctypes.data, C.byref(nb)))
    return {"A": A, "b": b, "c": c, "Q0": Q, "R0": R, "block_sizes": list(bs[:nb.value])}


def irk_transform(s: int, family: int = IRK_GAUSS, basis: int = IRK_BASIS_SCHUR):
    """Host-only A0^{-1} = T R T^{-1} in either basis: dict of numpy arrays."""
    import numpy as np
    T, Ti, R = (np.zeros((s, s)) for _ in range(3))
    bs = np.zeros(s, dtype=np.int32)
    nb = C.c_int()
    _check(LIB.irk_transform(family, s, basis, T.ctypes.data, Ti.ctypes.data, R.ctypes.data,
                             bs.ctypes.data, C.byref(nb)))
    return {"T": T, "Tinv": Ti, "R": R, "block_sizes": list(bs[:nb.value])}


def irk_get_config(h) -> IrkConfig:
    cfg = IrkConfig()
    _check(LIB.irk_get_config(h, C.byref(cfg)), h)
    return cfg


def irk_autotune(h, t_n: float, dt: float, steps: int = 2) -> IrkConfig:
    cfg = IrkConfig()
    _check(LIB.irk_autotune(h, t_n, dt, steps, C.byref(cfg)), h)
    return cfg


def irk_debug_bounds(selftest: bool = False):
    """(hits, message) of the bounds-checked build's device records since the
    last call; hits is -1 in the normal build and -2 after a CUDA error."""
    buf = C.create_string_buffer(256)
    hits = LIB.irk_debug_bounds(int(selftest), buf, len(buf))
    return hits, buf.value.decode(errors="replace")


def irk_kernel_stats(h):
    arr = (IrkKernelStat * 64)()
    n = C.c_int()
    _check(LIB.irk_kernel_stats(h, arr, 64, C.byref(n)), h)
    return [{"name": arr[k].name.decode(), "launches": arr[k].launches, "ms": arr[k].ms,
             "bytes": arr[k].bytes, "flops": arr[k].flops} for k in range(n.value)]


def irk_reset_kernel_stats(h):
    _check(LIB.irk_reset_kernel_stats(h), h)


def irk_device_bytes(h) -> int:
    return int(LIB.irk_device_bytes(h))


def irk_last_error(h=None) -> str:
    return LIB.irk_last_error(h).decode(errors="replace")


def irk_destroy(h):
    _HANDLE_SIZES.pop(getattr(h, "value", h), None)
    LIB.irk_destroy(h)


class IrkSolver:
    """Owning wrapper around one handle (marshalling only)."""

    def __init__(self, u0, stream=None, **cfg):
        self.cfg = irk_config_default(**cfg)
        self.h = irk_create(self.cfg, u0, stream)

    @property
    def ncomp(self):
        return 2 if self.cfg.op in (IRK_OP_BURGERS_2D, IRK_OP_VSF_2D) else 1

    @property
    def shape(self):
        d = 2 if self.cfg.op in (IRK_OP_BURGERS_2D, IRK_OP_VSF_2D) else 1
        return (self.ncomp,) + (self.cfg.n,) * d

    def step(self, t_n, dt, nsteps=1):
        return irk_step(self.h, t_n, dt, nsteps)

    def state(self, out=None):
        import numpy as np
        if out is None:
            out = np.empty(self.shape)
        return irk_get_state(self.h, out)

    def set_state(self, src):
        irk_set_state(self.h, src)

    def set_stages(self, src):
        irk_set_stages(self.h, src)

    def stages(self, out=None):
        import numpy as np
        if out is None:
            out = np.empty((self.cfg.stages,) + self.shape)
        return irk_get_stages(self.h, out)

    def close(self):
        if self.h is not None:
            irk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class IrkBatch:
    """Owning wrapper around an irk_batch (include/irk_batch.h): many 2D
    Burgers problems of different sizes stepped together (marshalling only)."""

    def __init__(self, capacity: int, stream=None):
        self.capacity = capacity
        self.b = C.c_void_p()
        sp = None
        if stream is not None:
            sp = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        st = LIB.irk_batch_create(capacity, sp, C.byref(self.b))
        if st != IRK_OK:
            raise IrkError(st, "irk_batch_create failed")
        self.shapes = {}

    def _check(self, st):
        if st != IRK_OK:
            raise IrkError(st, LIB.irk_batch_last_error(self.b).decode(errors="replace"))

    @staticmethod
    def instance_bytes(cfg: IrkConfig) -> int:
        return LIB.irk_batch_instance_bytes(C.byref(cfg))

    def add(self, u0, dt: float, arena_ptr: int = 0, arena_bytes: int = 0, **cfg) -> int:
        c = irk_config_default(**cfg)
        p, dev = _ptr(u0)
        _need(u0, 2 * c.n * c.n, "u0")
        slot = C.c_int(-1)
        self._check(LIB.irk_batch_add(self.b, C.byref(c), p, dev, dt,
                                      C.c_void_p(arena_ptr) if arena_ptr else None, arena_bytes,
                                      C.byref(slot)))
        self.shapes[slot.value] = ((2, c.n, c.n), c.stages)
        return slot.value

    def step(self):
        """One step of every resident instance; returns {slot: (status, stats dict)}."""
        stats = (IrkStats * self.capacity)()
        status = (C.c_int * self.capacity)()
        self._check(LIB.irk_batch_step(self.b, stats, status))
        return {k: (status[k], stats[k].as_dict()) for k in self.shapes}

    def state(self, slot: int, out=None):
        import numpy as np
        if out is None:
            out = np.empty(self.shapes[slot][0])
        p, dev = _ptr(out)
        _need(out, int(np.prod(self.shapes[slot][0])), "out")
        self._check(LIB.irk_batch_get_state(self.b, slot, p, dev))
        return out

    def stages(self, slot: int, out=None):
        import numpy as np
        shape, s = self.shapes[slot]
        if out is None:
            out = np.empty((s,) + shape)
        p, dev = _ptr(out)
        _need(out, s * int(np.prod(shape)), "out")
        self._check(LIB.irk_batch_get_stages(self.b, slot, p, dev))
        return out

    def remove(self, slot: int):
        self._check(LIB.irk_batch_remove(self.b, slot))
        self.shapes.pop(slot, None)

    def count(self) -> int:
        return LIB.irk_batch_count(self.b)

    def close(self):
        if self.b:
            LIB.irk_batch_destroy(self.b)
            self.b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
