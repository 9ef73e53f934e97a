"""Thin ctypes binding of include/pplbm.h (argument marshalling only).

Every function here forwards to the CUDA library ``_lib/libpplbm.so``; there
is no CPU path.  PyTorch is used for two pieces of plumbing only: device
memory (the library allocates through torch's caching allocator) and the
CUDA stream the library queues its kernels on.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpplbm.so")

LBM_OK = 0
LBM_PENDING = 1
LBM_ERR_ARG = -1
LBM_ERR_OOM = -2
LBM_ERR_CUDA = -3
LBM_ERR_NUMERIC = -4
LBM_ERR_TIMEOUT = -5
LBM_ERR_STATE = -6
LBM_ERR_UNKNOWN_TICKET = -7
LBM_ERR_CAPACITY = -8
LBM_NOALLOC_MAX_COUNT = 1073741824

LBM_STORE_F32 = 0
LBM_STORE_F32_DEV = 1
LBM_STORE_F16_DEV = 2
LBM_EOS_F64 = 0
LBM_EOS_DF = 1
LBM_EOS_F32 = 2
LBM_COLL_BGK = 0
LBM_COLL_MRT = 1
LBM_EOS_KIND_CS = 0
LBM_EOS_KIND_VDW = 1
LBM_KERNEL_AUTO = 0
LBM_KERNEL_PLAIN = 1
LBM_KERNEL_TMA = 2
LBM_SCHED_AUTO = 0
LBM_SCHED_TWO_PASS = 1
LBM_SCHED_FUSED = 2


class LatticeDesc(ctypes.Structure):
    """lbm_lattice_desc."""

    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("tau", ctypes.c_double), ("G", ctypes.c_double),
                ("eps", ctypes.c_double), ("sigma", ctypes.c_double), ("T", ctypes.c_double),
                ("eos_a", ctypes.c_double), ("eos_b", ctypes.c_double),
                ("eos_c", ctypes.c_double), ("eos_k", ctypes.c_double),
                ("rho0", ctypes.c_double),
                ("storage", ctypes.c_int32), ("eos_precision", ctypes.c_int32),
                ("m2_trace_variant", ctypes.c_int32), ("collision", ctypes.c_int32),
                ("mrt_rates", ctypes.c_double * 9), ("eos_kind", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class RuntimeOpts(ctypes.Structure):
    """lbm_runtime_opts."""

    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
                ("stream", ctypes.c_void_p), ("tile_x", ctypes.c_int32),
                ("tile_y", ctypes.c_int32), ("grid_ctas", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("graph_steps", ctypes.c_int32),
                ("kernel_variant", ctypes.c_int32), ("sites_per_thread", ctypes.c_int32)]


class ServerOpts(ctypes.Structure):
    """lbm_server_opts."""

    _fields_ = [("arena_bytes", ctypes.c_size_t), ("max_resident", ctypes.c_int32),
                ("chunk_steps", ctypes.c_int32), ("max_request_sites", ctypes.c_int64),
                ("target_resident_sites", ctypes.c_int64), ("storage", ctypes.c_int32), ("eos_precision", ctypes.c_int32),
                ("kernel_variant", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32),
                ("sites_per_thread", ctypes.c_int32), ("with_velocity", ctypes.c_int32),
                ("max_width", ctypes.c_int32), ("chunk_ms", ctypes.c_double),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    """lbm_server_stats."""

    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("queued", ctypes.c_int32),
                ("resident", ctypes.c_int32), ("site_steps", ctypes.c_int64),
                ("busy_s", ctypes.c_double), ("arena_bytes", ctypes.c_int64),
                ("arena_in_use", ctypes.c_int64), ("launches", ctypes.c_int64)]


class KernelStat(ctypes.Structure):
    """lbm_kernel_stat."""

    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("bytes_per_launch", ctypes.c_double)]


class Info(ctypes.Structure):
    """lbm_info_t."""

    _fields_ = [("sites", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32),
                ("n_tiles", ctypes.c_int32), ("grid_ctas", ctypes.c_int32),
                ("psi_tile_x", ctypes.c_int32), ("psi_tile_y", ctypes.c_int32),
                ("psi_n_tiles", ctypes.c_int32), ("psi_grid_ctas", ctypes.c_int32),
                ("psi_variant", ctypes.c_int32), ("collide_variant", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("n_lattices", ctypes.c_int32),
                ("spt", ctypes.c_int32), ("psi_spt", ctypes.c_int32),
                ("tensor_map", ctypes.c_int32)]


# Every symbol include/pplbm.h declares, with (restype, argtypes).
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "lbm_desc_default": (None, [ctypes.POINTER(LatticeDesc), ctypes.c_int32, ctypes.c_int32]),
    "lbm_create": (ctypes.c_int, [ctypes.POINTER(LatticeDesc), ctypes.c_int32,
                                  ctypes.POINTER(RuntimeOpts), ctypes.POINTER(_vp)]),
    "lbm_init": (ctypes.c_int, [_vp, ctypes.c_int32, _dp, _dp, _dp]),
    "lbm_step": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "lbm_moments": (ctypes.c_int, [_vp, ctypes.c_int32, _dp, _dp, _dp, _dp]),
    "lbm_mass": (ctypes.c_int, [_vp, ctypes.c_int32, _dp]),
    "lbm_sync": (ctypes.c_int, [_vp]),
    "lbm_status_detail": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32)]),
    "lbm_destroy": (None, [_vp]),
    "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "lbm_last_error": (ctypes.c_char_p, [_vp]),
    "lbm_profile": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "lbm_profile_read": (ctypes.c_int, [_vp, ctypes.POINTER(KernelStat), ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_int32)]),
    "lbm_launch_count": (ctypes.c_int64, [_vp]),
    "lbm_info": (ctypes.c_int, [_vp, ctypes.POINTER(Info)]),
    "lbm_autotune": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "lbm_inject_copy_timeout": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "lbm_selfcheck": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int32]),
    "lbm_selfcheck_arith": (ctypes.c_int, [ctypes.POINTER(ctypes.c_float), ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_float),
                                           ctypes.POINTER(ctypes.c_float)]),
    "lbm_selfcheck_psi": (ctypes.c_int, [ctypes.POINTER(LatticeDesc), ctypes.POINTER(ctypes.c_float),
                                         ctypes.c_int64, ctypes.POINTER(ctypes.c_float),
                                         ctypes.POINTER(ctypes.c_double)]),
    "lbm_mass_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_server_opts_default": (None, [ctypes.POINTER(ServerOpts)]),
    "lbm_server_create": (ctypes.c_int, [ctypes.POINTER(ServerOpts), ctypes.POINTER(_vp)]),
    "lbm_submit": (ctypes.c_int, [_vp, ctypes.POINTER(LatticeDesc), _dp, ctypes.c_int64,
                                  ctypes.POINTER(ctypes.c_uint64)]),
    "lbm_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, _dp, _dp, _dp, _dp]),
    "lbm_server_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(ServerStats)]),
    "lbm_server_destroy": (None, [_vp]),
}

_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library; raises if it was not built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(f"CUDA library {path} is missing: run "
                                  "paper_2003_07968_gb300.build.build() first")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class LbmError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        msg = f"{where}: {lbm_strerror(code)} ({code})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


def lbm_strerror(code: int) -> str:
    return load().lbm_strerror(int(code)).decode()


def _check(rc: int, where: str, h=None) -> int:
    if rc < 0:
        detail = load().lbm_last_error(h.ptr).decode() if h is not None else ""
        raise LbmError(rc, where, detail)
    return rc


# --------------------------------------------------------------- torch plumbing
class _TorchAllocator:
    """Device memory for the library from torch's caching allocator."""

    def __init__(self, device):
        import torch

        self.torch = torch
        self.device = device
        self.live = {}
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, _ctx):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:  # out of memory: the library reports LBM_ERR_OOM
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ptr, _nbytes, _ctx):
        self.live.pop(int(ptr), None)


class Handle:
    """An lbm_handle* plus the Python objects that must outlive it."""

    def __init__(self, ptr, stream, allocator, descs):
        self.ptr = ptr
        self.stream = stream  # torch.cuda.Stream the kernels run on
        self.allocator = allocator
        self.descs = descs

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                lbm_destroy(self)
            except Exception:
                pass


def lbm_desc_default(nx: int, ny: int, **kw) -> LatticeDesc:
    """lbm_desc_default, then the given fields; eos_kind=LBM_EOS_KIND_VDW
    also sets the reduced van der Waals constants a, b, c (3, 1/3, 8/3)
    unless they are given too."""
    d = LatticeDesc()
    load().lbm_desc_default(ctypes.byref(d), int(nx), int(ny))
    if kw.get("eos_kind") == LBM_EOS_KIND_VDW:
        d.eos_a, d.eos_b, d.eos_c = 3.0, 1.0 / 3.0, 8.0 / 3.0
    for k, v in kw.items():
        if k == "mrt_rates":
            for i in range(9):
                d.mrt_rates[i] = float(v[i])
        else:
            if not hasattr(d, k):
                raise AttributeError(k)
            setattr(d, k, v)
    return d


def lbm_create(descs, tile=None, grid_ctas=0, schedule=LBM_SCHED_AUTO, graph_steps=0,
               stream=None, device=None, kernel_variant=LBM_KERNEL_AUTO,
               sites_per_thread=0, allocator=None) -> Handle:
    """Create a handle over one descriptor or a list of them.  ``tile`` =
    (tile_x, tile_y) fixes both passes' tiles, with ``sites_per_thread``.
    ``allocator``: an object with ctypes callbacks ``alloc`` and ``free``
    (default: torch's caching allocator)."""
    import torch

    if isinstance(descs, LatticeDesc):
        descs = [descs]
    n = len(descs)
    arr = (LatticeDesc * n)(*descs)
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    if stream is None:
        stream = torch.cuda.Stream(device=dev)
    alloc = allocator if allocator is not None else _TorchAllocator(dev)
    o = RuntimeOpts()
    o.alloc, o.free, o.alloc_ctx = alloc.alloc, alloc.free, None
    o.stream = stream.cuda_stream
    o.tile_x, o.tile_y = (tile or (0, 0))
    o.grid_ctas, o.schedule, o.graph_steps = grid_ctas, schedule, graph_steps
    o.kernel_variant = kernel_variant
    o.sites_per_thread = sites_per_thread
    out = ctypes.c_void_p()
    with torch.cuda.device(dev):
        rc = load().lbm_create(arr, n, ctypes.byref(o), ctypes.byref(out))
    _check(rc, "lbm_create")
    return Handle(out, stream, alloc, list(descs))


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def lbm_init(h: Handle, lattice: int, rho, ux=None, uy=None) -> None:
    d = h.descs[lattice]
    shp = (d.ny, d.nx)
    r, x, y = _f64(rho, shp), _f64(ux, shp), _f64(uy, shp)
    _check(load().lbm_init(h.ptr, lattice, _ptr(r), _ptr(x), _ptr(y)), "lbm_init", h)
    # pageable host arrays were copied before lbm_init returned


def lbm_step(h: Handle, nsteps: int) -> None:
    _check(load().lbm_step(h.ptr, int(nsteps)), "lbm_step", h)


def _pinned_empty(shape) -> np.ndarray:
    """FP64 host array in page-locked memory from torch's pinned-memory
    allocator (cached, so repeated calls reuse blocks): the library's
    device-to-host copies into it run at the link's rate, where pageable
    memory is staged by the driver at a fraction of it (4.9 ms against
    0.2 ms for a 2048^2 field)."""
    import torch

    return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()


def lbm_moments(h: Handle, lattice: int, rho=True, u=True, mass=True, out=None) -> dict:
    """rho, ux, uy ([ny, nx] FP64) and mass of one lattice.  ``out`` may hold
    preallocated host arrays under the same keys; the arrays made here are
    page-locked."""
    d = h.descs[lattice]
    shp = (d.ny, d.nx)
    out = dict(out or {})
    if rho and "rho" not in out:
        out["rho"] = _pinned_empty(shp)
    if u:
        if "ux" not in out:
            out["ux"] = _pinned_empty(shp)
        if "uy" not in out:
            out["uy"] = _pinned_empty(shp)
    m = ctypes.c_double(0.0)
    rc = load().lbm_moments(h.ptr, lattice, _ptr(out.get("rho") if rho else None),
                            _ptr(out.get("ux") if u else None), _ptr(out.get("uy") if u else None),
                            ctypes.byref(m) if mass else None)
    _check(rc, "lbm_moments", h)
    if mass:
        out["mass"] = m.value
    return out


def lbm_mass(h: Handle, lattice: int) -> float:
    m = ctypes.c_double(0.0)
    _check(load().lbm_mass(h.ptr, lattice, ctypes.byref(m)), "lbm_mass", h)
    return m.value


def lbm_sync(h: Handle) -> None:
    _check(load().lbm_sync(h.ptr), "lbm_sync", h)


def lbm_status_detail(h: Handle) -> int:
    i = ctypes.c_int32(-1)
    _check(load().lbm_status_detail(h.ptr, ctypes.byref(i)), "lbm_status_detail", h)
    return i.value


def lbm_destroy(h: Handle) -> None:
    if h.ptr:
        load().lbm_destroy(h.ptr)
        h.ptr = None


def lbm_profile(h: Handle, on: bool) -> None:
    _check(load().lbm_profile(h.ptr, 1 if on else 0), "lbm_profile", h)


def lbm_profile_read(h: Handle) -> list[dict]:
    arr = (KernelStat * 8)()
    n = ctypes.c_int32(0)
    _check(load().lbm_profile_read(h.ptr, arr, 8, ctypes.byref(n)), "lbm_profile_read", h)
    return [dict(name=arr[i].name.decode(), launches=arr[i].launches,
                 total_ms=arr[i].total_ms, bytes_per_launch=arr[i].bytes_per_launch)
            for i in range(n.value)]


def lbm_launch_count(h: Handle) -> int:
    return int(load().lbm_launch_count(h.ptr))


def lbm_info(h: Handle) -> dict:
    i = Info()
    _check(load().lbm_info(h.ptr, ctypes.byref(i)), "lbm_info", h)
    return {k: getattr(i, k) for k, _ in Info._fields_}


def lbm_mass_noalloc(values_ptr: int, count: int, offset: float, mass_out_ptr: int,
                     stream_ptr: int) -> int:
    """FP64 sum of `count` FP32 device values plus `offset` into the device
    double at `mass_out_ptr`, queued on `stream_ptr`; allocates nothing.
    Returns the status code (raises on errors)."""
    return _check(load().lbm_mass_noalloc(values_ptr, int(count), float(offset), mass_out_ptr,
                                          stream_ptr), "lbm_mass_noalloc")


def lbm_selfcheck() -> tuple[int, str]:
    buf = ctypes.create_string_buffer(512)
    rc = load().lbm_selfcheck(buf, 512)
    return rc, buf.value.decode()


def lbm_inject_copy_timeout(h: Handle, tile: int) -> None:
    """Arm the failure-detection test of the single pass for the next step."""
    _check(load().lbm_inject_copy_timeout(h.ptr, int(tile)), "lbm_inject_copy_timeout", h)


def lbm_selfcheck_psi(desc: LatticeDesc, rho) -> tuple[np.ndarray, np.ndarray]:
    """(psi, radicand) of the step kernels for the FP32 densities ``rho`` with
    the constants of ``desc`` (radicand: float-float arithmetic only)."""
    v = np.ascontiguousarray(rho, dtype=np.float32).ravel()
    psi = np.empty_like(v)
    rad = np.empty(v.size, dtype=np.float64)
    fp = ctypes.POINTER(ctypes.c_float)
    _check(load().lbm_selfcheck_psi(ctypes.byref(desc), v.ctypes.data_as(fp),
                                    ctypes.c_int64(v.size), psi.ctypes.data_as(fp),
                                    rad.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "lbm_selfcheck_psi")
    return psi, rad


def lbm_selfcheck_arith(x) -> tuple[np.ndarray, np.ndarray]:
    """The step kernels' 1/x and sqrt(x) for float32 values x (GPU)."""
    v = np.ascontiguousarray(x, dtype=np.float32).ravel()
    r = np.empty_like(v)
    q = np.empty_like(v)
    fp = ctypes.POINTER(ctypes.c_float)
    _check(load().lbm_selfcheck_arith(v.ctypes.data_as(fp), ctypes.c_int64(v.size),
                                      r.ctypes.data_as(fp), q.ctypes.data_as(fp)),
           "lbm_selfcheck_arith")
    return r, q


def lbm_autotune(h: Handle, repeats: int = 3) -> dict:
    _check(load().lbm_autotune(h.ptr, int(repeats)), "lbm_autotune", h)
    return lbm_info(h)


# --------------------------------------------------------------- serving
class Server:
    """An lbm_server*; the lattices' shapes are remembered per ticket so
    lbm_poll can size its outputs."""

    def __init__(self, ptr):
        self.ptr = ptr
        self.shapes = {}

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                lbm_server_destroy(self)
            except Exception:
                pass


def lbm_server_opts_default(**kw) -> ServerOpts:
    o = ServerOpts()
    load().lbm_server_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def lbm_server_create(opts: ServerOpts | None = None, device=None) -> Server:
    """A server whose device memory comes from torch's caching allocator,
    unless ``opts`` already name an allocator."""
    import torch

    o = opts if opts is not None else lbm_server_opts_default()
    alloc = None
    if not o.alloc:
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        alloc = _TorchAllocator(dev)
        o.alloc, o.free, o.alloc_ctx = alloc.alloc, alloc.free, None
    out = ctypes.c_void_p()
    _check(load().lbm_server_create(ctypes.byref(o), ctypes.byref(out)), "lbm_server_create")
    srv = Server(out)
    srv.alloc = alloc  # keeps the callbacks alive as long as the server
    return srv


def lbm_submit(s: Server, desc: LatticeDesc, rho, nsteps: int) -> int:
    r = _f64(rho, (desc.ny, desc.nx))
    t = ctypes.c_uint64(0)
    _check(load().lbm_submit(s.ptr, ctypes.byref(desc), _ptr(r), int(nsteps), ctypes.byref(t)),
           "lbm_submit")
    s.shapes[t.value] = (desc.ny, desc.nx)
    return t.value


def lbm_poll(s: Server, ticket: int, u: bool = True):
    """None while pending; else dict(rho, ux, uy, latency_s).  Raises LbmError
    for a failed request (its code in .code)."""
    shp = s.shapes.get(ticket, (1, 1))
    rho = np.empty(shp)
    ux = np.empty(shp) if u else None
    uy = np.empty(shp) if u else None
    lat = ctypes.c_double(0.0)
    rc = load().lbm_poll(s.ptr, ctypes.c_uint64(ticket), _ptr(rho), _ptr(ux), _ptr(uy),
                         ctypes.byref(lat))
    if rc == LBM_PENDING:
        return None
    s.shapes.pop(ticket, None)
    _check(rc, "lbm_poll")
    return {"rho": rho, "ux": ux, "uy": uy, "latency_s": lat.value}


def lbm_server_get_stats(s: Server) -> dict:
    st = ServerStats()
    _check(load().lbm_server_get_stats(s.ptr, ctypes.byref(st)), "lbm_server_get_stats")
    return {k: getattr(st, k) for k, _ in ServerStats._fields_}


def lbm_server_destroy(s: Server) -> None:
    if s.ptr:
        load().lbm_server_destroy(s.ptr)
        s.ptr = None
