"""ctypes binding of the C ABI in ``include/flints.h`` (argument marshalling only).

Every step of the lensing remap runs in the CUDA library ``_lib/libflints.so``;
this module only converts torch tensors and numpy arrays to pointers, sizes
and streams.  There is no CPU fallback: if the library is missing or cannot
be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libflints.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "flints.h")

FLINTS_FP64 = 0
FLINTS_MIXED = 1
FLINTS_SPIN2_AUGMENTED = 1  # spin 2: widely linear estimator with xi+ and xi-
FLINTS_ROTATE_TO_TARGET = 2  # spin 2: P in the frame at n, not n'
FLINTS_NO_VARIANCE = 4
FLINTS_FORCE_FALLBACK = 256  # testing aid: mixed plans re-solve every point in FP64
ST_NUGGET, ST_FALLBACK, ST_WINDOW, ST_FAILED, ST_POLE, ST_INPUT = 1, 2, 4, 8, 16, 32


class FlintsError(RuntimeError):
    pass


class _Stats(ctypes.Structure):
    _fields_ = [("points", ctypes.c_int64), ("nugget", ctypes.c_int64), ("fallback", ctypes.c_int64),
                ("window", ctypes.c_int64), ("failed", ctypes.c_int64)]


class _Info(ctypes.Structure):
    _fields_ = [("nside", ctypes.c_int64), ("lmax", ctypes.c_int), ("spin", ctypes.c_int), ("K", ctypes.c_int),
                ("precision", ctypes.c_int), ("t_max", ctypes.c_double), ("n_intervals", ctypes.c_int),
                ("xi0", ctypes.c_double), ("search_radius", ctypes.c_double), ("device_bytes", ctypes.c_int64)]


class _PaperInfo(ctypes.Structure):
    _fields_ = [("nside", ctypes.c_int64), ("nside_coarse", ctypes.c_int64), ("y", ctypes.c_int), ("K", ctypes.c_int),
                ("slots", ctypes.c_int64), ("t_max", ctypes.c_double), ("n_intervals", ctypes.c_int),
                ("xi0", ctypes.c_double), ("table_bytes", ctypes.c_int64), ("max_pair_t", ctypes.c_double),
                ("nugget_slots", ctypes.c_int64), ("failed_slots", ctypes.c_int64), ("points", ctypes.c_int64),
                ("window", ctypes.c_int64), ("precision", ctypes.c_int), ("spin", ctypes.c_int),
                ("flags", ctypes.c_uint), ("device_bytes", ctypes.c_int64)]


class LaunchCfg(ctypes.Structure):
    """flints_launch_cfg: warps per block, blocks per SM cap, targets per warp tile (0 = default)."""
    _fields_ = [("warps_per_block", ctypes.c_int), ("blocks_per_sm", ctypes.c_int), ("tile_points", ctypes.c_int)]

    def key(self):
        return (self.warps_per_block, self.blocks_per_sm, self.tile_points)


class _Job(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("first", ctypes.c_int64), ("count", ctypes.c_int64),
                ("map", ctypes.c_void_p), ("defl", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("var", ctypes.c_void_p), ("status", ctypes.c_void_p)]


_lib = None


def header_functions() -> list[str]:
    """Names of the functions declared in include/flints.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(flints_[a-z0-9_]+)\s*\(", txt)))


def load_library(path: str = LIB_PATH):
    """Load libflints.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FlintsError(f"{path} is missing: build it with paper_1003_4984_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i64, c_int, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    lib.flints_plan.argtypes = [ctypes.POINTER(vp), i64, c_int, dp, dp, c_int, c_int, c_int, ctypes.c_uint, vp]
    lib.flints_lens_spin0.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.flints_lens_spin2.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.flints_lens_range.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, vp]
    lib.flints_stencil.argtypes = [vp, i64, i64, vp, vp, vp, vp]
    lib.flints_supersample.argtypes = [vp, i64, i64, i64, vp, vp, vp, vp, vp]
    lib.flints_lens_batch.argtypes = [ctypes.POINTER(_Job), c_int, vp]
    lib.flints_get_stats.argtypes = [vp, ctypes.POINTER(_Stats), vp]
    lib.flints_reset_stats.argtypes = [vp, vp]
    lib.flints_get_info.argtypes = [vp, ctypes.POINTER(_Info)]
    lib.flints_get_table.argtypes = [vp, c_int, dp, dp, vp]
    lib.flints_last_error.restype = ctypes.c_char_p
    lib.flints_free.argtypes = [vp]
    lib.flints_free.restype = None
    lib.flints_plan_set_launch.argtypes = [vp, ctypes.POINTER(LaunchCfg)]
    lib.flints_plan_set_launch.restype = c_int
    lib.flints_batch_create.argtypes = [ctypes.POINTER(vp), c_int]
    lib.flints_batch_stage.argtypes = [vp, ctypes.POINTER(_Job), c_int, c_int]
    lib.flints_batch_launch.argtypes = [vp, ctypes.POINTER(LaunchCfg), vp]
    lib.flints_batch_run.argtypes = [vp, ctypes.POINTER(_Job), c_int, ctypes.POINTER(LaunchCfg), vp]
    lib.flints_batch_free.argtypes = [vp]
    lib.flints_batch_free.restype = None
    for name in ("flints_batch_create", "flints_batch_stage", "flints_batch_launch", "flints_batch_run"):
        getattr(lib, name).restype = c_int
    lib.flints_lens_noalloc.argtypes = [i64, c_int, dp, dp, c_int, c_int, c_int, i64, i64, vp, vp, vp, vp, vp, vp]
    lib.flints_lens_noalloc.restype = c_int
    lib.flints_noalloc_last_error.restype = ctypes.c_char_p
    lib.flints_measure_fma_peak.argtypes = [c_int, c_int, dp, vp]
    lib.flints_measure_fma_peak.restype = c_int
    lib.flints_measure_last_error.restype = ctypes.c_char_p
    lib.flints_synth_plan.argtypes = [ctypes.POINTER(vp), i64, c_int, c_int, c_int, vp]
    lib.flints_synth_plan.restype = c_int
    lib.flints_synthesize.argtypes = [vp, vp, vp, vp, vp]
    lib.flints_synthesize.restype = c_int
    lib.flints_synth_free.argtypes = [vp]
    lib.flints_synth_free.restype = None
    lib.flints_synth_last_error.restype = ctypes.c_char_p
    lib.flints_paper_plan.argtypes = [ctypes.POINTER(vp), i64, c_int, dp, dp, c_int, c_int, c_int, ctypes.c_uint, vp]
    lib.flints_paper_lens.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, vp]
    lib.flints_paper_supersample.argtypes = [vp, i64, i64, i64, vp, vp, vp, vp, vp]
    lib.flints_paper_get_info.argtypes = [vp, ctypes.POINTER(_PaperInfo), vp]
    lib.flints_paper_tables.argtypes = [vp, vp, vp, vp, vp]
    for name in ("flints_paper_plan", "flints_paper_lens", "flints_paper_supersample", "flints_paper_get_info",
                 "flints_paper_tables"):
        getattr(lib, name).restype = c_int
    lib.flints_paper_free.argtypes = [vp]
    lib.flints_paper_free.restype = None
    lib.flints_paper_last_error.restype = ctypes.c_char_p
    for name in ("flints_plan", "flints_lens_spin0", "flints_lens_spin2", "flints_lens_range", "flints_stencil",
                 "flints_lens_batch", "flints_get_stats", "flints_reset_stats", "flints_get_info",
                 "flints_get_table"):
        getattr(lib, name).restype = c_int
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise FlintsError(f"flints error {rc}: {_lib.flints_last_error().decode()}")


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream) -> int | None:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dev_f64(t, shape, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise FlintsError(f"{name} must be a contiguous float64 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise FlintsError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def _dev_buf(t, n: int, name: str, dtype: str = "float64"):
    """A contiguous CUDA tensor of ``dtype`` with at least ``n`` elements: the check for
    buffers the library reads or writes through a raw pointer (a host tensor's address
    handed to a kernel would be an invalid device access)."""
    import torch

    if (not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != getattr(torch, dtype)
            or not t.is_contiguous()):
        raise FlintsError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if t.numel() < n:
        raise FlintsError(f"{name} holds {t.numel()} elements, the call needs {n}")
    return t


@dataclass
class Info:
    nside: int
    lmax: int
    spin: int
    K: int
    precision: int
    t_max: float
    n_intervals: int
    xi0: float
    search_radius: float
    device_bytes: int


class Plan:
    """A lensing plan: spectrum, resolution, spin, stencil size and precision.

    ``precision`` is "fp64" or "mixed".  Creating the plan tabulates xi on the
    current CUDA device (Sec. 2.5 steps 1-2).
    """

    def __init__(self, nside: int, cl, cl_bb=None, spin: int = 0, K: int = 32, precision: str = "fp64",
                 flags: int = 0, stream=None):
        lib = load_library()
        cl = np.ascontiguousarray(cl, dtype=np.float64)
        lmax = cl.size - 1
        bb = None if cl_bb is None else np.ascontiguousarray(cl_bb, dtype=np.float64)
        if bb is not None and bb.size != cl.size:
            raise FlintsError("cl_bb must have the same length as cl")
        prec = {"fp64": FLINTS_FP64, "mixed": FLINTS_MIXED}[precision]
        h = ctypes.c_void_p()
        dp = ctypes.POINTER(ctypes.c_double)
        _check(lib.flints_plan(ctypes.byref(h), int(nside), int(lmax), cl.ctypes.data_as(dp),
                               bb.ctypes.data_as(dp) if bb is not None else None, int(spin), int(K), prec,
                               int(flags), _stream(stream)))
        self._h = h
        self.nside, self.lmax, self.spin, self.K, self.precision = int(nside), lmax, int(spin), int(K), precision
        self.npix = 12 * self.nside * self.nside

    @property
    def handle(self) -> int:
        return self._h.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.flints_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ queries
    def info(self) -> Info:
        i = _Info()
        _check(_lib.flints_get_info(self._h, ctypes.byref(i)))
        return Info(i.nside, i.lmax, i.spin, i.K, i.precision, i.t_max, i.n_intervals, i.xi0, i.search_radius,
                    i.device_bytes)

    def device_bytes(self) -> int:
        """Device memory the plan holds, as the library counted its allocations."""
        return self.info().device_bytes

    def table(self, which: int = 0, stream=None):
        n = self.info().n_intervals + 1
        f = np.empty(n)
        g = np.empty(n)
        dp = ctypes.POINTER(ctypes.c_double)
        _check(_lib.flints_get_table(self._h, which, f.ctypes.data_as(dp), g.ctypes.data_as(dp), _stream(stream)))
        return f, g

    def stats(self, stream=None) -> dict:
        s = _Stats()
        _check(_lib.flints_get_stats(self._h, ctypes.byref(s), _stream(stream)))
        return {k: getattr(s, k) for k, _ in _Stats._fields_}

    def reset_stats(self, stream=None):
        _check(_lib.flints_reset_stats(self._h, _stream(stream)))

    def set_launch(self, cfg: "LaunchCfg | None"):
        """Launch shape of this plan's lens launches (None: library defaults)."""
        self.launch_cfg = cfg
        _check(_lib.flints_plan_set_launch(self._h, ctypes.byref(cfg) if cfg is not None else None))

    # ------------------------------------------------------------- compute
    def lens(self, map_, defl, out=None, var=None, status=None, first: int = 0, count: int | None = None,
             stream=None):
        """Lens targets [first, first+count) (default: the whole map) on the GPU.

        ``map_`` (Npix,) or (Npix, 2), ``defl`` (count, 2): float64 CUDA tensors.
        Returns (out, var, status) tensors (created when not given).
        """
        import torch

        if count is None:
            count = self.npix - first
        comp = (self.npix,) if self.spin == 0 else (self.npix, 2)
        _dev_f64(map_, comp, "map")
        _dev_f64(defl, (count, 2), "defl")
        oshape = (count,) if self.spin == 0 else (count, 2)
        dev = map_.device
        if out is None:
            out = torch.empty(oshape, dtype=torch.float64, device=dev)
        _dev_f64(out, oshape, "out")
        if var is not None:
            _dev_f64(var, (count,), "var")
        if status is not None and (status.dtype != torch.uint8 or not status.is_cuda or status.numel() != count
                                   or not status.is_contiguous()):
            raise FlintsError("status must be a contiguous uint8 CUDA tensor of length count")
        _check(_lib.flints_lens_range(self._h, int(first), int(count), _ptr(map_), _ptr(defl), _ptr(out), _ptr(var),
                                      _ptr(status), _stream(stream)))
        return out, var, status

    def supersample(self, map_, nside_out: int, out=None, var=None, status=None, first: int = 0,
                    count: int | None = None, stream=None):
        """Interpolate the map at the centres of RING pixels [first, first+count) of an
        Nside = ``nside_out`` grid (no deflection; flints_supersample)."""
        import torch

        npix_out = 12 * int(nside_out) ** 2
        if count is None:
            count = npix_out - first
        comp = (self.npix,) if self.spin == 0 else (self.npix, 2)
        _dev_f64(map_, comp, "map")
        oshape = (count,) if self.spin == 0 else (count, 2)
        if out is None:
            out = torch.empty(oshape, dtype=torch.float64, device=map_.device)
        _dev_f64(out, oshape, "out")
        if var is not None:
            _dev_f64(var, (count,), "var")
        if status is not None and (status.dtype != torch.uint8 or not status.is_cuda or status.numel() != count
                                   or not status.is_contiguous()):
            raise FlintsError("status must be a contiguous uint8 CUDA tensor of length count")
        _check(_lib.flints_supersample(self._h, int(nside_out), int(first), int(count), _ptr(map_), _ptr(out),
                                       _ptr(var), _ptr(status), _stream(stream)))
        return out, var, status

    def lens_full(self, map_, defl, out, var=None, stream=None):
        """Whole-map entry point (flints_lens_spin0 / flints_lens_spin2)."""
        comp = (self.npix,) if self.spin == 0 else (self.npix, 2)
        _dev_f64(map_, comp, "map")
        _dev_f64(defl, (self.npix, 2), "defl")
        _dev_f64(out, comp, "out")
        if var is not None:
            _dev_f64(var, (self.npix,), "var")
        if self.spin == 1:  # spin-1 plans use the range entry point over the whole map
            _check(_lib.flints_lens_range(self._h, 0, self.npix, _ptr(map_), _ptr(defl), _ptr(out), _ptr(var), None,
                                          _stream(stream)))
            return out, var
        fn = _lib.flints_lens_spin0 if self.spin == 0 else _lib.flints_lens_spin2
        _check(fn(self._h, _ptr(map_), _ptr(defl), _ptr(out), _ptr(var), _stream(stream)))
        return out, var

    def stencil(self, defl, first: int = 0, count: int | None = None, stream=None):
        """K nearest RING pixels of each displaced target: int64 (count, K) and status."""
        import torch

        if count is None:
            count = self.npix - first
        _dev_f64(defl, (count, 2), "defl")
        idx = torch.empty((count, self.K), dtype=torch.int64, device=defl.device)
        st = torch.empty(count, dtype=torch.uint8, device=defl.device)
        _check(_lib.flints_stencil(self._h, int(first), int(count), _ptr(defl), _ptr(idx), _ptr(st),
                                   _stream(stream)))
        return idx, st


def _job_array(jobs):
    arr = (_Job * max(1, len(jobs)))()
    for k, (plan, first, count, m, d, o, v, s) in enumerate(jobs):
        if int(count) > 0:  # the library reads and writes these through raw device pointers
            two = 1 if plan.spin == 0 else 2
            _dev_buf(m, plan.npix * two, f"job {k}: map")
            _dev_buf(d, 2 * int(count), f"job {k}: defl")
            _dev_buf(o, int(count) * two, f"job {k}: out")
            if v is not None:
                _dev_buf(v, int(count), f"job {k}: var")
            if s is not None:
                _dev_buf(s, int(count), f"job {k}: status", "uint8")
        arr[k] = _Job(plan.handle, first, count, _ptr(m), _ptr(d), _ptr(o), _ptr(v), _ptr(s))
    return arr


class Batch:
    """Persistent batched launch over many plans' target ranges (flints_batch_*).

    ``stage`` writes the job table on the host only; ``launch`` is stream work
    only (upload, queue reset, kernels) and can be captured in a CUDA graph.
    Jobs are tuples (plan, first, count, map, defl, out, var, status).
    """

    def __init__(self, max_jobs: int):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.flints_batch_create(ctypes.byref(h), int(max_jobs)))
        self._h = h
        self._keep = None

    def stage(self, jobs, tile_points: int = 0):
        self._keep = list(jobs)  # the caller's tensors must outlive the launches
        arr = _job_array(jobs)
        _check(_lib.flints_batch_stage(self._h, arr, len(jobs), int(tile_points)))

    def launch(self, cfg: "LaunchCfg | None" = None, stream=None):
        _check(_lib.flints_batch_launch(self._h, ctypes.byref(cfg) if cfg is not None else None, _stream(stream)))

    def run(self, jobs, cfg: "LaunchCfg | None" = None, stream=None):
        self.stage(jobs, cfg.tile_points if cfg is not None else 0)
        self.launch(cfg, stream)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.flints_batch_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lens_batch(jobs, stream=None):
    """Run several (plan, first, count, map, defl, out, var, status) jobs through flints_lens_batch."""
    load_library()
    _check(_lib.flints_lens_batch(_job_array(jobs), len(jobs), _stream(stream)))


def lens_host(plan: Plan, map_host: np.ndarray, defl_host: np.ndarray, first: int = 0, count: int | None = None,
              stream=None):
    """Host-buffer convenience: copy inputs to the device, lens, copy value and variance back."""
    import torch

    if count is None:
        count = plan.npix - first
    m = torch.from_numpy(np.ascontiguousarray(map_host, dtype=np.float64)).cuda(non_blocking=True)
    d = torch.from_numpy(np.ascontiguousarray(defl_host, dtype=np.float64)).cuda(non_blocking=True)
    var = torch.empty(count, dtype=torch.float64, device=m.device)
    out, var, _ = plan.lens(m, d, var=var, first=first, count=count, stream=stream)
    return out.cpu().numpy(), var.cpu().numpy()


def measure_fma_peak(precision: str = "mixed", iters: int | None = None, stream=None) -> float:
    """flints_measure_fma_peak: measured multiply-add throughput (TFLOP/s) of the FP32
    pipe (``"mixed"``) or the FP64 pipe (``"fp64"``) of the current device."""
    lib = load_library()
    if iters is None:
        iters = 20000 if precision == "mixed" else 400
    out = ctypes.c_double()
    rc = lib.flints_measure_fma_peak({"fp64": FLINTS_FP64, "mixed": FLINTS_MIXED}[precision], int(iters),
                                     ctypes.byref(out), _stream(stream))
    if rc != 0:
        raise FlintsError(f"flints error {rc}: {lib.flints_measure_last_error().decode()}")
    return out.value


def lens_noalloc(nside: int, cl, map_, defl, out, var=None, status=None, cl_bb=None, spin: int = 0, K: int = 32,
                 precision: str = "fp64", first: int = 0, count: int | None = None, stream=None):
    """flints_lens_noalloc: lens without any device allocation by the library.

    For callers that cannot call cudaMalloc (serving runtimes that own all device
    memory in their own pool, hosts that forbid library allocations): every
    buffer is the caller's; the library's working memory is a fixed device array
    shared by all calls, so calls must not overlap on the GPU.  The call copies
    ``cl`` from host memory and synchronises ``stream`` once.  The first call on
    a device looks up the array's device address; make it before any stream
    capture begins.
    """
    lib = load_library()
    npix = 12 * int(nside) * int(nside)
    if count is None:
        count = npix - first
    if int(count) > 0:
        two = 1 if int(spin) == 0 else 2
        _dev_buf(map_, npix * two, "map")
        _dev_buf(defl, 2 * int(count), "defl")
        _dev_buf(out, int(count) * two, "out")
        if var is not None:
            _dev_buf(var, int(count), "var")
        if status is not None:
            _dev_buf(status, int(count), "status", "uint8")
    cl = np.ascontiguousarray(cl, dtype=np.float64)
    bb = None if cl_bb is None else np.ascontiguousarray(cl_bb, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    prec = {"fp64": FLINTS_FP64, "mixed": FLINTS_MIXED}[precision]
    rc = lib.flints_lens_noalloc(int(nside), cl.size - 1, cl.ctypes.data_as(dp),
                                 bb.ctypes.data_as(dp) if bb is not None else None, int(spin), int(K), prec,
                                 int(first), int(count), _ptr(map_), _ptr(defl), _ptr(out), _ptr(var), _ptr(status),
                                 _stream(stream))
    if rc != 0:
        raise FlintsError(f"flints error {rc}: {lib.flints_noalloc_last_error().decode()}")
    return out, var, status


class Synth:
    """GPU harmonic synthesis (flints_synth_plan / flints_synthesize): band-limited
    RING maps from a_lm.  Spin 0: T; spin 1, 2: (Re P, Im P) of P = -sum (E + iB) sY_lm."""

    def __init__(self, nside: int, lmax: int, spin: int = 0, precision: str = "mixed", stream=None):
        lib = load_library()
        self.nside, self.lmax, self.spin = int(nside), int(lmax), int(spin)
        self.npix = 12 * self.nside * self.nside
        prec = {"fp64": FLINTS_FP64, "mixed": FLINTS_MIXED}[precision]
        h = ctypes.c_void_p()
        rc = lib.flints_synth_plan(ctypes.byref(h), self.nside, self.lmax, self.spin, prec, _stream(stream))
        if rc != 0:
            raise FlintsError(f"flints error {rc}: {lib.flints_synth_last_error().decode()}")
        self._h = h

    def _alm(self, a, name):
        import torch

        if a is None:
            return None
        if not (isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.complex128
                and tuple(a.shape) == (self.lmax + 1, self.lmax + 1) and a.is_contiguous()):
            raise FlintsError(f"{name} must be a contiguous complex128 CUDA tensor of shape (lmax+1, lmax+1)")
        return a

    def run(self, alm, blm=None, out=None, stream=None):
        import torch

        alm = self._alm(alm, "alm")
        blm = self._alm(blm, "blm")
        shape = (self.npix,) if self.spin == 0 else (self.npix, 2)
        if out is None:
            out = torch.empty(shape, dtype=torch.float64, device=alm.device)
        _dev_f64(out, shape, "out")
        lib = load_library()
        rc = lib.flints_synthesize(self._h, _ptr(alm), _ptr(blm), _ptr(out), _stream(stream))
        if rc != 0:
            raise FlintsError(f"flints error {rc}: {lib.flints_synth_last_error().decode()}")
        return out

    def close(self):
        if getattr(self, "_h", None):
            load_library().flints_synth_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PaperPlan:
    """The paper's stencil with tabulated inverses (flints_paper_*): level-y
    pixel-centred stencil of 9 * 4^(y-1) pixels, L^-1 (the factor of S^-1)
    tabulated per symmetry class of central pixels, two triangular
    matrix-vector products per target (spin 0; precision "fp64" or "mixed",
    the per-target arithmetic in double-float on the FP32 pipe)."""

    def __init__(self, nside: int, cl, y: int = 1, precision: str = "fp64", spin: int = 0, cl_bb=None,
                 augmented: bool = False, stream=None):
        lib = load_library()
        cl = np.ascontiguousarray(cl, dtype=np.float64)
        bb = None if cl_bb is None else np.ascontiguousarray(cl_bb, dtype=np.float64)
        if bb is not None and bb.size != cl.size:
            raise FlintsError("cl_bb must have the length of cl")
        self.nside, self.y, self.precision, self.spin = int(nside), int(y), precision, int(spin)
        prec = {"fp64": FLINTS_FP64, "mixed": FLINTS_MIXED}[precision]
        dp = ctypes.POINTER(ctypes.c_double)
        h = ctypes.c_void_p()
        self.augmented = bool(augmented)
        rc = lib.flints_paper_plan(ctypes.byref(h), self.nside, cl.size - 1, cl.ctypes.data_as(dp),
                                   None if bb is None else bb.ctypes.data_as(dp), self.y, self.spin, prec,
                                   FLINTS_SPIN2_AUGMENTED if augmented else 0, _stream(stream))
        if rc != 0:
            raise FlintsError(f"flints error {rc}: {lib.flints_paper_last_error().decode()}")
        self._h = h
        i = self.info()
        self.nside_coarse, self.K, self.slots = i["nside_coarse"], i["K"], i["slots"]

    def _raise(self, rc):
        if rc != 0:
            raise FlintsError(f"flints error {rc}: {load_library().flints_paper_last_error().decode()}")

    def info(self, stream=None) -> dict:
        inf = _PaperInfo()
        self._raise(load_library().flints_paper_get_info(self._h, ctypes.byref(inf), _stream(stream)))
        return {name: getattr(inf, name) for name, _ in _PaperInfo._fields_}

    def _outputs(self, map_, count, out, var, status):
        import torch

        two = (2,) if self.spin != 0 else ()
        _dev_f64(map_, (12 * self.nside * self.nside,) + two, "map")
        if out is None:
            out = torch.empty((count,) + two, dtype=torch.float64, device=map_.device)
        if var is None:
            var = torch.empty(count, dtype=torch.float64, device=map_.device)
        _dev_f64(out, (count,) + two, "out")
        _dev_f64(var, (count,), "var")
        if status is not None and (status.dtype != torch.uint8 or tuple(status.shape) != (count,)
                                   or not status.is_cuda or not status.is_contiguous()):
            raise FlintsError("status must be a contiguous uint8 CUDA tensor of shape (count,)")
        return out, var

    def lens(self, map_, defl, first: int = 0, count: int | None = None, out=None, var=None, status=None,
             stream=None):
        """Lensed values at pixels first .. first+count-1 displaced along defl[(count, 2)]."""
        if count is None:
            count = 12 * self.nside * self.nside - first
        _dev_f64(defl, (count, 2), "defl")
        out, var = self._outputs(map_, count, out, var, status)
        self._raise(load_library().flints_paper_lens(self._h, first, count, _ptr(map_), _ptr(defl), _ptr(out),
                                                     _ptr(var), _ptr(status), _stream(stream)))
        return out, var

    def supersample(self, map_, nside_out: int, first: int = 0, count: int | None = None, out=None, var=None,
                    status=None, stream=None):
        """Values at the centres of pixels first .. first+count-1 of the grid nside_out."""
        if count is None:
            count = 12 * nside_out * nside_out - first
        out, var = self._outputs(map_, count, out, var, status)
        self._raise(load_library().flints_paper_supersample(self._h, nside_out, first, count, _ptr(map_), _ptr(out),
                                                            _ptr(var), _ptr(status), _stream(stream)))
        return out, var

    def tables(self, stream=None):
        """(members (12 Nc^2, K) int32, slot (12 Nc^2,) int32, linv (slots, len) float64) device
        copies; linv holds L^-1 packed by columns (K = 9, len 45) or in the lane-step layout of
        include/flints.h (K = 36, len 704); None for mixed plans."""
        import torch

        npc = 12 * self.nside_coarse * self.nside_coarse
        mem = torch.empty((npc, self.K), dtype=torch.int32, device="cuda")
        slot = torch.empty(npc, dtype=torch.int32, device="cuda")
        linv = None
        if self.precision == "fp64":  # mixed plans keep only double-float blocks
            n_l = 704 if self.K == 36 else self.K * (self.K + 1) // 2
            shape = (self.slots, n_l) if self.spin == 0 else (self.slots, n_l, 2)  # complex for spin 1, 2
            if self.augmented:  # the real 2K x 2K factor packed by columns
                shape = (self.slots, (2 * self.K) * (2 * self.K + 1) // 2)
            linv = torch.empty(shape, dtype=torch.float64, device="cuda")
        self._raise(load_library().flints_paper_tables(self._h, _ptr(mem), _ptr(slot), _ptr(linv), _stream(stream)))
        return mem, slot, linv

    def close(self):
        if getattr(self, "_h", None):
            load_library().flints_paper_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
