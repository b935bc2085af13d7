"""Python binding of libnbody.so, the GB300 direct-summation gravity library.

The functions here carry the C ABI's names (``include/nbody.h``) and only
marshal arguments: every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: if ``libnbody.so`` is missing or cannot be
loaded, the first call raises ``RuntimeError`` (build it with
``python paper_2509_19294_gb300/build.py`` or ``__graft_entry__.build()``).

Arrays may be torch tensors (CUDA or CPU) or numpy arrays, float64 and
C-contiguous, in the C-ABI layout: positions/velocities/accelerations
``[3, n]``, masses and potentials ``[n]``.  CPU arrays are staged through
device buffers by the library itself.  ``stream`` defaults to torch's current
CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libnbody.so")

NBODY_OK = 0
NBODY_EINVAL = -1
NBODY_ENOMEM = -2
NBODY_ECUDA = -3
NBODY_ENONFINITE = -4
NBODY_ETIMEOUT = -5
NBODY_ESTATE = -6
NBODY_EUNSUPPORTED = -7
NBODY_ETOOBIG = -8
NBODY_NOALLOC_MAX_N = 262144

NBODY_F64 = 0
NBODY_F32C = 1

NBODY_FLAG_AUTOTUNE = 1
NBODY_FLAG_PROFILE = 2
NBODY_FLAG_CHECK_FINITE = 4
NBODY_FLAG_NO_GRAPH = 8
NBODY_FLAG_TRACE = 16
NBODY_TRACE_CAP = 65536

EXPORTED = ("nbody_init", "nbody_destroy", "nbody_forces", "nbody_step", "nbody_energy",
            "nbody_tune", "nbody_get_tiles", "nbody_tiles_supported", "nbody_profile_read",
            "nbody_kernel_launches", "nbody_strerror", "nbody_last_error_message",
            "nbody_forces_noalloc", "nbody_forces_jerk",
            "nbody_step_hermite", "nbody_get_jerk_tiles", "nbody_set_jerk_tiles",
            "nbody_block_start", "nbody_block_advance", "nbody_block_state", "nbody_block_trace")


class NBodyTiles(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("p", ctypes.c_int32), ("tj", ctypes.c_int32),
                ("split", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]


class NBodyConfig(ctypes.Structure):
    _fields_ = [("n_total", ctypes.c_int64), ("n_clusters", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("cluster_offsets", ctypes.POINTER(ctypes.c_int64)),
                ("eps", ctypes.POINTER(ctypes.c_double)), ("G", ctypes.c_double),
                ("reorder_every", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("tiles", NBodyTiles), ("max_device_bytes", ctypes.c_int64)]


class NBodyError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        msg = f"{where}: {nbody_strerror(code)} ({code})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libnbody.so (once).  Raises RuntimeError if it is not built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it first (no CPU fallback exists)")
        lib = ctypes.CDLL(path)
        vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.nbody_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(NBodyConfig), vp]
        lib.nbody_init.restype = ctypes.c_int
        lib.nbody_destroy.argtypes = [vp]
        lib.nbody_destroy.restype = None
        lib.nbody_forces.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.nbody_forces.restype = ctypes.c_int
        lib.nbody_step.argtypes = [vp, vp, vp, vp, vp, vp, d, i32, vp, vp]
        lib.nbody_step.restype = ctypes.c_int
        lib.nbody_energy.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.nbody_energy.restype = ctypes.c_int
        lib.nbody_tune.argtypes = [vp, vp]
        lib.nbody_tune.restype = ctypes.c_int
        lib.nbody_get_tiles.argtypes = [vp, ctypes.POINTER(NBodyTiles)]
        lib.nbody_get_tiles.restype = ctypes.c_int
        lib.nbody_tiles_supported.argtypes = [ctypes.POINTER(NBodyTiles), ctypes.c_int]
        lib.nbody_tiles_supported.restype = ctypes.c_int
        lib.nbody_profile_read.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(i64), ctypes.c_int]
        lib.nbody_profile_read.restype = ctypes.c_int
        lib.nbody_kernel_launches.argtypes = [vp]
        lib.nbody_kernel_launches.restype = i64
        lib.nbody_strerror.argtypes = [ctypes.c_int]
        lib.nbody_strerror.restype = ctypes.c_char_p
        lib.nbody_last_error_message.argtypes = [vp]
        lib.nbody_last_error_message.restype = ctypes.c_char_p
        lib.nbody_forces_noalloc.argtypes = [i64, vp, vp, d, d, vp, vp, vp]
        lib.nbody_forces_noalloc.restype = ctypes.c_int
        lib.nbody_forces_jerk.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        lib.nbody_forces_jerk.restype = ctypes.c_int
        lib.nbody_step_hermite.argtypes = [vp, vp, vp, vp, vp, vp, vp, d, i32, vp, vp]
        lib.nbody_step_hermite.restype = ctypes.c_int
        lib.nbody_get_jerk_tiles.argtypes = [vp, ctypes.POINTER(NBodyTiles)]
        lib.nbody_get_jerk_tiles.restype = ctypes.c_int
        lib.nbody_set_jerk_tiles.argtypes = [vp, ctypes.POINTER(NBodyTiles)]
        lib.nbody_set_jerk_tiles.restype = ctypes.c_int
        lib.nbody_block_start.argtypes = [vp, vp, vp, vp, vp, vp, vp, d, d, d, d, vp]
        lib.nbody_block_start.restype = ctypes.c_int
        lib.nbody_block_advance.argtypes = [vp, vp, vp, vp, vp, vp, vp, d, ctypes.POINTER(i64),
                                            ctypes.POINTER(i64), vp]
        lib.nbody_block_advance.restype = ctypes.c_int
        lib.nbody_block_state.argtypes = [vp, vp, vp, vp]
        lib.nbody_block_state.restype = ctypes.c_int
        lib.nbody_block_trace.argtypes = [vp, vp, i64, i64, vp]
        lib.nbody_block_trace.restype = ctypes.c_int
        _lib = lib
        return lib


def nbody_strerror(code: int) -> str:
    try:
        return load().nbody_strerror(int(code)).decode()
    except RuntimeError:
        return f"status {code}"


class Context:
    """Handle of one nbody_ctx plus the sizes the binding needs."""

    def __init__(self, handle, n_total: int, n_clusters: int, mode: int):
        self.handle = handle
        self.n = n_total
        self.n_clusters = n_clusters
        self.mode = mode

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        nbody_destroy(self)

    def __del__(self):
        try:
            nbody_destroy(self)
        except Exception:
            pass


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def _ptr(a, shape, name, keep):
    """Device or host address of a float64 C-contiguous array of the given shape."""
    if a is None:
        return None
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous() or tuple(a.shape) != shape:
                raise ValueError(f"{name}: need a contiguous float64 tensor of shape {shape}, "
                                 f"got {a.dtype} {tuple(a.shape)}")
            keep.append(a)
            return ctypes.c_void_p(a.data_ptr())
    except ImportError:
        pass
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.shape != shape:
            raise ValueError(f"{name}: need a C-contiguous float64 array of shape {shape}, "
                             f"got {a.dtype} {a.shape}")
        keep.append(a)
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"{name}: unsupported array type {type(a)}")


def _check(ctx, rc, where):
    if rc != NBODY_OK:
        detail = ""
        if ctx is not None and getattr(ctx, "handle", None):
            detail = load().nbody_last_error_message(ctx.handle).decode()
        raise NBodyError(rc, where, detail)


def nbody_init(n_total: int, eps, mode: int = NBODY_F32C, G: float = 1.0, cluster_offsets=None,
               reorder_every: int = 0, flags: int = 0, tiles=None, max_device_bytes: int = 0,
               stream=None) -> Context:
    """Create a context (see nbody_init in nbody.h).  eps: scalar or one per cluster;
    max_device_bytes: cap on the context's device memory (0 = none)."""
    lib = load()
    if cluster_offsets is None:
        offsets = np.array([0, n_total], np.int64)
    else:
        offsets = np.ascontiguousarray(cluster_offsets, dtype=np.int64)
    ncl = len(offsets) - 1
    eps_arr = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, np.float64), (ncl,)))
    cfg = NBodyConfig()
    cfg.n_total = int(n_total)
    cfg.n_clusters = ncl
    cfg.mode = int(mode)
    cfg.cluster_offsets = offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    cfg.eps = eps_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cfg.G = float(G)
    cfg.reorder_every = int(reorder_every)
    cfg.flags = int(flags)
    cfg.max_device_bytes = int(max_device_bytes)
    if tiles is not None:
        t = tuple(tiles) + (0,) * (5 - len(tiles))
        cfg.tiles = NBodyTiles(*[int(x) for x in t])
    h = ctypes.c_void_p()
    rc = lib.nbody_init(ctypes.byref(h), ctypes.byref(cfg), _stream(stream))
    _check(None, rc, "nbody_init")
    return Context(h, int(n_total), ncl, int(mode))


def nbody_destroy(ctx: Context) -> None:
    if ctx is not None and ctx.handle:
        load().nbody_destroy(ctx.handle)
        ctx.handle = None


def nbody_forces(ctx: Context, pos, mass, acc, pot=None, stream=None) -> None:
    n = ctx.n
    keep = []
    rc = load().nbody_forces(ctx.handle, _ptr(pos, (3, n), "pos", keep),
                             _ptr(mass, (n,), "mass", keep), _ptr(acc, (3, n), "acc", keep),
                             _ptr(pot, (n,), "pot", keep), _stream(stream))
    _check(ctx, rc, "nbody_forces")


def nbody_step(ctx: Context, pos, vel, mass, acc, pot, dt: float, nsteps: int, diag=None,
               stream=None) -> None:
    n = ctx.n
    keep = []
    rc = load().nbody_step(ctx.handle, _ptr(pos, (3, n), "pos", keep),
                           _ptr(vel, (3, n), "vel", keep), _ptr(mass, (n,), "mass", keep),
                           _ptr(acc, (3, n), "acc", keep), _ptr(pot, (n,), "pot", keep),
                           float(dt), int(nsteps),
                           _ptr(diag, (int(nsteps), ctx.n_clusters, 9), "diag", keep),
                           _stream(stream))
    _check(ctx, rc, "nbody_step")


def nbody_forces_jerk(ctx: Context, pos, vel, mass, acc, jerk, pot=None, stream=None) -> None:
    """Acceleration, jerk and potential (see nbody_forces_jerk in nbody.h)."""
    n = ctx.n
    keep = []
    rc = load().nbody_forces_jerk(ctx.handle, _ptr(pos, (3, n), "pos", keep),
                                  _ptr(vel, (3, n), "vel", keep), _ptr(mass, (n,), "mass", keep),
                                  _ptr(acc, (3, n), "acc", keep), _ptr(jerk, (3, n), "jerk", keep),
                                  _ptr(pot, (n,), "pot", keep), _stream(stream))
    _check(ctx, rc, "nbody_forces_jerk")


def nbody_step_hermite(ctx: Context, pos, vel, mass, acc, jerk, pot, dt: float, nsteps: int,
                       diag=None, stream=None) -> None:
    """Fourth-order Hermite steps (see nbody_step_hermite in nbody.h)."""
    n = ctx.n
    keep = []
    rc = load().nbody_step_hermite(ctx.handle, _ptr(pos, (3, n), "pos", keep),
                                   _ptr(vel, (3, n), "vel", keep), _ptr(mass, (n,), "mass", keep),
                                   _ptr(acc, (3, n), "acc", keep), _ptr(jerk, (3, n), "jerk", keep),
                                   _ptr(pot, (n,), "pot", keep), float(dt), int(nsteps),
                                   _ptr(diag, (int(nsteps), ctx.n_clusters, 9), "diag", keep),
                                   _stream(stream))
    _check(ctx, rc, "nbody_step_hermite")


def nbody_block_start(ctx: Context, pos, vel, mass, acc, jerk, pot, dt_max: float, dt_min: float,
                      eta: float, eta_s: float, stream=None) -> None:
    """Start individual block time steps (see nbody_block_start in nbody.h)."""
    n = ctx.n
    keep = []
    rc = load().nbody_block_start(ctx.handle, _ptr(pos, (3, n), "pos", keep),
                                  _ptr(vel, (3, n), "vel", keep), _ptr(mass, (n,), "mass", keep),
                                  _ptr(acc, (3, n), "acc", keep), _ptr(jerk, (3, n), "jerk", keep),
                                  _ptr(pot, (n,), "pot", keep), float(dt_max), float(dt_min),
                                  float(eta), float(eta_s), _stream(stream))
    _check(ctx, rc, "nbody_block_start")


def nbody_block_advance(ctx: Context, pos, vel, mass, acc, jerk, pot, t_end: float, stream=None):
    """Block steps until t_end; returns (block steps, single-particle evaluations) so far."""
    n = ctx.n
    keep = []
    blocks, evals = ctypes.c_int64(), ctypes.c_int64()
    rc = load().nbody_block_advance(ctx.handle, _ptr(pos, (3, n), "pos", keep),
                                    _ptr(vel, (3, n), "vel", keep), _ptr(mass, (n,), "mass", keep),
                                    _ptr(acc, (3, n), "acc", keep), _ptr(jerk, (3, n), "jerk", keep),
                                    _ptr(pot, (n,), "pot", keep), float(t_end), ctypes.byref(blocks),
                                    ctypes.byref(evals), _stream(stream))
    _check(ctx, rc, "nbody_block_advance")
    return blocks.value, evals.value


def nbody_block_state(ctx: Context, stream=None):
    """(t[n], dt[n]) of every particle."""
    t = np.empty(ctx.n, np.float64)
    dt = np.empty(ctx.n, np.float64)
    rc = load().nbody_block_state(ctx.handle, ctypes.c_void_p(t.ctypes.data),
                                  ctypes.c_void_p(dt.ctypes.data), _stream(stream))
    _check(ctx, rc, "nbody_block_state")
    return t, dt


def nbody_block_trace(ctx: Context, first: int, last: int, stream=None):
    """Steps first .. last (counted from 1, NBODY_FLAG_TRACE): (seconds, active
    particles) of each, from trace records first - 1 .. last."""
    count = last - first + 2
    out = np.empty(2 * count, np.uint64)
    rc = load().nbody_block_trace(ctx.handle, ctypes.c_void_p(out.ctypes.data), first - 1, count,
                                  _stream(stream))
    _check(ctx, rc, "nbody_block_trace")
    rec = out.reshape(count, 2)
    return np.diff(rec[:, 0].astype(np.int64)) * 1e-9, rec[1:, 1].astype(np.int64)


def nbody_get_jerk_tiles(ctx: Context):
    t = NBodyTiles()
    _check(ctx, load().nbody_get_jerk_tiles(ctx.handle, ctypes.byref(t)), "nbody_get_jerk_tiles")
    return (t.block, t.p, t.tj, t.split, t.ctas_per_sm)


def nbody_set_jerk_tiles(ctx: Context, tiles) -> None:
    t = tuple(tiles) + (0,) * (5 - len(tiles))
    tt = NBodyTiles(*[int(x) for x in t])
    _check(ctx, load().nbody_set_jerk_tiles(ctx.handle, ctypes.byref(tt)), "nbody_set_jerk_tiles")


def nbody_energy(ctx: Context, pos, vel, mass, pot, stream=None) -> np.ndarray:
    """Return [n_clusters, 9]: K, W, E, Px, Py, Pz, Lx, Ly, Lz per cluster."""
    n = ctx.n
    keep = []
    out = np.empty((ctx.n_clusters, 9), np.float64)
    rc = load().nbody_energy(ctx.handle, _ptr(pos, (3, n), "pos", keep),
                             _ptr(vel, (3, n), "vel", keep), _ptr(mass, (n,), "mass", keep),
                             _ptr(pot, (n,), "pot", keep), ctypes.c_void_p(out.ctypes.data),
                             _stream(stream))
    _check(ctx, rc, "nbody_energy")
    return out


def nbody_tune(ctx: Context, stream=None) -> None:
    _check(ctx, load().nbody_tune(ctx.handle, _stream(stream)), "nbody_tune")


def nbody_get_tiles(ctx: Context):
    """(block, p, tj, split, ctas_per_sm) of the F32C kernel in use."""
    t = NBodyTiles()
    _check(ctx, load().nbody_get_tiles(ctx.handle, ctypes.byref(t)), "nbody_get_tiles")
    return (t.block, t.p, t.tj, t.split, t.ctas_per_sm)


def nbody_tiles_supported():
    """Compiled (block, p, tj, ctas_per_sm) shapes."""
    lib = load()
    n = lib.nbody_tiles_supported(None, 0)
    arr = (NBodyTiles * n)()
    lib.nbody_tiles_supported(arr, n)
    return [(t.block, t.p, t.tj, t.ctas_per_sm) for t in arr]


def nbody_profile_read(ctx: Context, reset: bool = False):
    """(total ms, launches) of the force kernel since the last reset (NBODY_FLAG_PROFILE)."""
    ms = ctypes.c_double()
    cnt = ctypes.c_int64()
    rc = load().nbody_profile_read(ctx.handle, ctypes.byref(ms), ctypes.byref(cnt), int(reset))
    _check(ctx, rc, "nbody_profile_read")
    return ms.value, cnt.value


def nbody_kernel_launches(ctx: Context) -> int:
    return int(load().nbody_kernel_launches(ctx.handle))


def nbody_forces_noalloc(pos, mass, eps: float, acc, pot=None, G: float = 1.0, stream=None) -> None:
    """Forces of one system without any allocation (see nbody_forces_noalloc in nbody.h).

    For callers that cannot allocate device memory when they compute forces:
    the library uses a fixed scratch array compiled into libnbody.so instead of
    a context.  All arrays must already be on the device; n is at most
    NBODY_NOALLOC_MAX_N.  Calls share the scratch, so do not let two of them
    run concurrently on the GPU.
    """
    n = int(mass.shape[0])
    keep = []
    rc = load().nbody_forces_noalloc(n, _ptr(pos, (3, n), "pos", keep),
                                     _ptr(mass, (n,), "mass", keep), float(eps), float(G),
                                     _ptr(acc, (3, n), "acc", keep), _ptr(pot, (n,), "pot", keep),
                                     _stream(stream))
    _check(None, rc, "nbody_forces_noalloc")
