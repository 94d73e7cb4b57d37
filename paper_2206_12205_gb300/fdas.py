"""ctypes binding to libfdas (include/fdas.h): the same entry points, argument marshalling only.

Every step of the path runs in libfdas' CUDA kernels.  torch tensors supply device memory
and streams; this module checks their device, dtype and size, passes raw pointers, and
turns fdas_status codes into exceptions.  If the library is missing this module raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

FDAS_OK, FDAS_E_INVALID, FDAS_E_UNSUPPORTED, FDAS_E_NOMEM, FDAS_E_CUDA, FDAS_E_OVERFLOW, FDAS_E_TIMEOUT, FDAS_E_STATE = range(8)
FDAS_FP32, FDAS_BF16, FDAS_BF16_SPLIT, FDAS_FP16_SCALED, FDAS_BF16_DIRECT, FDAS_FP8_DIRECT = 0, 1, 2, 3, 4, 5
FDAS_DEV_PEAK_OVERFLOW, FDAS_DEV_TIMEOUT = 0x1, 0x2
PRECISIONS = {"fp32": FDAS_FP32, "bf16": FDAS_BF16, "bf16_split": FDAS_BF16_SPLIT, "fp16_scaled": FDAS_FP16_SCALED,
              "bf16_direct": FDAS_BF16_DIRECT, "fp8_direct": FDAS_FP8_DIRECT}

# every symbol include/fdas.h declares
EXPORTED = (
    "fdas_plan", "fdas_plan_get_info", "fdas_make_templates", "fdas_spectrum", "fdas_plane",
    "fdas_peaks", "fdas_search", "fdas_get_templates", "fdas_device_status", "fdas_last_error",
    "fdas_destroy", "fdas_status_string", "fdas_version", "fdas_profile_enable", "fdas_profile_read",
    "fdas_plane_static", "fdas_interp_power", "fdas_refine",
    "fdas_batch_plan", "fdas_batch_autotune", "fdas_batch_make_templates", "fdas_batch_search",
    "fdas_batch_get_info", "fdas_batch_series_info", "fdas_batch_device_status", "fdas_batch_last_error",
    "fdas_batch_set_lanes",
    "fdas_batch_destroy", "fdas_band_max", "fdas_check_timeout", "fdas_levels_order",
)
REFINE_MAX_STEPS = 1000
STATIC_SCRATCH_BYTES = 40 << 20
STAGES = ("spectrum", "segments", "correlate", "peaks")

CAND_DTYPE = np.dtype([("r", "<f8"), ("z", "<f8")])   # fdas_cand
PEAK_DTYPE = np.dtype([("series", "<u4"), ("r", "<u4"), ("zi", "<i2"), ("harm", "u1"),
                       ("pad", "u1"), ("power", "<f4")])
assert PEAK_DTYPE.itemsize == 16


class FdasError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {status_string(status)} ({status})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


class _Config(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int64), ("zmax", ctypes.c_int32), ("taps", ctypes.c_int32),
                ("seg_len", ctypes.c_int32), ("precision", ctypes.c_int32), ("max_harm", ctypes.c_int32),
                ("thr", ctypes.c_float * 5), ("max_peaks", ctypes.c_int32), ("sigma2", ctypes.c_double),
                ("norm_block", ctypes.c_int32), ("harm_mode", ctypes.c_int32)]


class _Info(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int64), ("K", ctypes.c_int32), ("seg_valid", ctypes.c_int32),
                ("n_seg", ctypes.c_int64), ("plane_elem_bytes", ctypes.c_int32), ("plane_bytes", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_size_t), ("cells", ctypes.c_int64)]


class _Profile(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int64), ("launches", ctypes.c_int64), ("n_timed", ctypes.c_int64 * 4),
                ("ms", ctypes.c_double * 4), ("n_timed_peaks", ctypes.c_int64 * 2), ("ms_peaks", ctypes.c_double * 2),
                ("level1_fused", ctypes.c_int64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libfdas.so from the package's _build directory (built by __graft_entry__.build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"libfdas.so is not built ({path}); run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    V, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    S = ctypes.c_int
    sig = {
        "fdas_plan": (S, [ctypes.POINTER(_Config), ctypes.POINTER(V), ctypes.POINTER(SZ)]),
        "fdas_plan_get_info": (S, [V, ctypes.POINTER(_Info)]),
        "fdas_make_templates": (S, [V, V]),
        "fdas_spectrum": (S, [V, V, V, V, V, V]),
        "fdas_plane": (S, [V, V, V, V, V]),
        "fdas_peaks": (S, [V, V, V, V, V, V]),
        "fdas_search": (S, [V, V, V, V, V, V, V]),
        "fdas_get_templates": (S, [V, V, V]),
        "fdas_device_status": (S, [V, ctypes.POINTER(I32), ctypes.c_int]),
        "fdas_check_timeout": (S, [V, I64, V]),
        "fdas_levels_order": (S, [V, V, I64, ctypes.POINTER(I64)]),
        "fdas_last_error": (ctypes.c_char_p, [V]),
        "fdas_destroy": (None, [V]),
        "fdas_status_string": (ctypes.c_char_p, [S]),
        "fdas_version": (ctypes.c_int, []),
        "fdas_profile_enable": (S, [V, ctypes.c_int]),
        "fdas_profile_read": (S, [V, ctypes.POINTER(_Profile), ctypes.c_int]),
        "fdas_plane_static": (S, [V, V, V, V]),
        "fdas_interp_power": (S, [V, V, V, V, I32, I32, V, V]),
        "fdas_refine": (S, [V, V, V, I32, I32, V, V, V, V]),
        "fdas_batch_plan": (S, [ctypes.POINTER(_Config), I32, ctypes.POINTER(V), ctypes.POINTER(SZ)]),
        "fdas_batch_autotune": (S, [V, ctypes.c_char_p, V]),
        "fdas_batch_make_templates": (S, [V, V]),
        "fdas_batch_search": (S, [V, V, V, V, V, V]),
        "fdas_batch_get_info": (S, [V, ctypes.POINTER(I32), ctypes.POINTER(SZ), ctypes.POINTER(I64),
                                    ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "fdas_batch_series_info": (S, [V, I32, ctypes.POINTER(_Info), ctypes.POINTER(_Config), ctypes.POINTER(I64),
                                       ctypes.POINTER(I64), ctypes.POINTER(I32)]),
        "fdas_batch_device_status": (S, [V, ctypes.POINTER(I32), ctypes.c_int]),
        "fdas_batch_last_error": (ctypes.c_char_p, [V]),
        "fdas_batch_destroy": (None, [V]),
        "fdas_batch_set_lanes": (S, [V, I32, ctypes.POINTER(SZ)]),
        "fdas_band_max": (S, [V, V, V, V, I32, V, V, V, V, V]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _ = I64
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().fdas_status_string(int(status)).decode()


def fdas_version() -> int:
    return int(load().fdas_version())


# ----------------------------------------------------------------------------- helpers
def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> Optional[int]:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _dev_ptr(t, name: str, dtype=None, min_bytes: int = 0) -> int:
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    nbytes = t.numel() * t.element_size()
    if nbytes < min_bytes:
        raise ValueError(f"{name}: {nbytes} bytes < required {min_bytes}")
    return int(t.data_ptr())


def _check(status: int, where: str, plan=None):
    if status != FDAS_OK:
        detail = ""
        if plan is not None and plan.handle:
            detail = (load().fdas_last_error(plan.handle) or b"").decode()
        raise FdasError(status, where, detail)


@dataclasses.dataclass
class PlanInfo:
    nb: int
    K: int
    seg_valid: int
    n_seg: int
    plane_elem_bytes: int
    plane_bytes: int
    workspace_bytes: int
    cells: int


class Plan:
    """Owns an fdas_plan_t.  Create with fdas_plan(); freed by fdas_destroy() or GC."""

    def __init__(self, handle: int, cfg: dict, info: PlanInfo):
        self.handle = handle
        self.cfg = cfg
        self.info = info

    @property
    def precision(self) -> int:
        return self.cfg["precision"]

    def plane_dtype(self):
        torch = _torch()
        return torch.float32 if self.info.plane_elem_bytes == 4 else torch.bfloat16

    def __del__(self):
        try:
            fdas_destroy(self)
        except Exception:
            pass


def make_config(n_samples: int, zmax: int, taps: int, seg_len: int, precision="fp32", max_harm: int = 1,
                thr: Sequence[float] = (30.0,) * 5, max_peaks: int = 1 << 16, sigma2: float = 0.0,
                norm_block: int = 0, harm_mode: int = 0) -> dict:
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    thr = list(thr) + [float(thr[-1])] * (5 - len(thr))
    return dict(n_samples=int(n_samples), zmax=int(zmax), taps=int(taps), seg_len=int(seg_len),
                precision=int(precision), max_harm=int(max_harm), thr=[float(v) for v in thr[:5]],
                max_peaks=int(max_peaks), sigma2=float(sigma2), norm_block=int(norm_block),
                harm_mode=int(harm_mode))


# ----------------------------------------------------------------------------- entry points
def _to_config(cfg: dict, c: "_Config"):
    for k in ("n_samples", "zmax", "taps", "seg_len", "precision", "max_harm", "max_peaks", "sigma2"):
        setattr(c, k, cfg[k])
    c.norm_block = int(cfg.get("norm_block", 0))
    c.harm_mode = int(cfg.get("harm_mode", 0))
    for i, v in enumerate(cfg["thr"]):
        c.thr[i] = v


def _from_config(c: "_Config") -> dict:
    d = {k: getattr(c, k) for k in ("n_samples", "zmax", "taps", "seg_len", "precision", "max_harm", "max_peaks",
                                     "sigma2", "norm_block", "harm_mode")}
    d["thr"] = [float(c.thr[i]) for i in range(5)]
    return d


def fdas_plan(cfg: dict) -> Plan:
    lib = load()
    c = _Config()
    _to_config(cfg, c)
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    _check(lib.fdas_plan(ctypes.byref(c), ctypes.byref(h), ctypes.byref(ws)), "fdas_plan")
    inf = _Info()
    _check(lib.fdas_plan_get_info(h, ctypes.byref(inf)), "fdas_plan_get_info")
    info = PlanInfo(inf.nb, inf.K, inf.seg_valid, inf.n_seg, inf.plane_elem_bytes, inf.plane_bytes,
                    inf.workspace_bytes, inf.cells)
    return Plan(h.value, dict(cfg), info)


def fdas_make_templates(plan: Plan, stream=None):
    _check(load().fdas_make_templates(plan.handle, _stream_ptr(stream)), "fdas_make_templates", plan)


def fdas_spectrum(plan: Plan, series, workspace, xhat, sigma2=None, stream=None):
    torch = _torch()
    n = plan.cfg["n_samples"]
    args = (plan.handle,
            _dev_ptr(series, "series", torch.float32, 4 * n),
            _dev_ptr(workspace, "workspace", None, plan.info.workspace_bytes),
            _dev_ptr(xhat, "xhat", torch.float32, 8 * plan.info.nb),
            _dev_ptr(sigma2, "sigma2", torch.float64, 8) if sigma2 is not None else None,
            _stream_ptr(stream))
    _check(load().fdas_spectrum(*args), "fdas_spectrum", plan)


def fdas_plane(plan: Plan, xhat, workspace, plane, stream=None):
    torch = _torch()
    args = (plan.handle,
            _dev_ptr(xhat, "xhat", torch.float32, 8 * plan.info.nb),
            _dev_ptr(workspace, "workspace", None, plan.info.workspace_bytes),
            _dev_ptr(plane, "plane", plan.plane_dtype(), plan.info.plane_bytes),
            _stream_ptr(stream))
    _check(load().fdas_plane(*args), "fdas_plane", plan)


def fdas_plane_static(plan: Plan, xhat, plane, stream=None):
    """fdas_plane without a workspace: for callers that may not allocate device memory at call
    time (stream capture, pre-reserved real-time pipelines, hosts owning the memory pool).
    Its scratch is a library-owned static device array; concurrent calls race on it."""
    torch = _torch()
    args = (plan.handle,
            _dev_ptr(xhat, "xhat", torch.float32, 8 * plan.info.nb),
            _dev_ptr(plane, "plane", plan.plane_dtype(), plan.info.plane_bytes),
            _stream_ptr(stream))
    _check(load().fdas_plane_static(*args), "fdas_plane_static", plan)


def fdas_peaks(plan: Plan, plane, workspace, peaks, npeaks, stream=None):
    torch = _torch()
    args = (plan.handle,
            _dev_ptr(plane, "plane", plan.plane_dtype(), plan.info.plane_bytes),
            _dev_ptr(workspace, "workspace", None, plan.info.workspace_bytes),
            _dev_ptr(peaks, "peaks", torch.uint8, 16 * plan.cfg["max_peaks"]) if peaks is not None else None,
            _dev_ptr(npeaks, "npeaks", torch.int32, 4),
            _stream_ptr(stream))
    _check(load().fdas_peaks(*args), "fdas_peaks", plan)


def fdas_search(plan: Plan, series, workspace, plane, peaks, npeaks, stream=None):
    torch = _torch()
    n = plan.cfg["n_samples"]
    args = (plan.handle,
            _dev_ptr(series, "series", torch.float32, 4 * n),
            _dev_ptr(workspace, "workspace", None, plan.info.workspace_bytes),
            _dev_ptr(plane, "plane", plan.plane_dtype(), plan.info.plane_bytes),
            _dev_ptr(peaks, "peaks", torch.uint8, 16 * plan.cfg["max_peaks"]) if peaks is not None else None,
            _dev_ptr(npeaks, "npeaks", torch.int32, 4),
            _stream_ptr(stream))
    _check(load().fdas_search(*args), "fdas_search", plan)


def _points(pts, name: str, n=None) -> int:
    """A float64 tensor of shape (n, 2) holding (r, z) rows, as fdas_cand records."""
    torch = _torch()
    if pts.dim() != 2 or pts.shape[1] != 2:
        raise ValueError(f"{name}: expected shape (n, 2), got {tuple(pts.shape)}")
    if n is not None and pts.shape[0] != n:
        raise ValueError(f"{name}: expected {n} rows, got {pts.shape[0]}")
    return _dev_ptr(pts, name, torch.float64)


def fdas_interp_power(plan: Plan, xhat, pts, out, k0=None, fp64: bool = False, stream=None):
    """Interpolated power and gradient at the (n, 2) points pts into out (n, 3): P, dP/dr, dP/dz."""
    torch = _torch()
    n = int(pts.shape[0])
    args = (plan.handle,
            _dev_ptr(xhat, "xhat", torch.float32, 8 * plan.info.nb),
            _points(pts, "pts"),
            _dev_ptr(k0, "k0", torch.int64, 8 * n) if k0 is not None else None,
            n, 1 if fp64 else 0,
            _dev_ptr(out, "out", torch.float64, 24 * n),
            _stream_ptr(stream))
    _check(load().fdas_interp_power(*args), "fdas_interp_power", plan)


def fdas_refine(plan: Plan, xhat, cands_in, steps: int, cands_out, power=None, evals=None, stream=None):
    """Gradient-ascent refinement of (n, 2) seeds; power (n, 3) and evals (n,) are optional outputs."""
    torch = _torch()
    n = int(cands_in.shape[0])
    args = (plan.handle,
            _dev_ptr(xhat, "xhat", torch.float32, 8 * plan.info.nb),
            _points(cands_in, "cands_in"),
            n, int(steps),
            _points(cands_out, "cands_out", n),
            _dev_ptr(power, "power", torch.float64, 24 * n) if power is not None else None,
            _dev_ptr(evals, "evals", torch.int32, 4 * n) if evals is not None else None,
            _stream_ptr(stream))
    _check(load().fdas_refine(*args), "fdas_refine", plan)


def fdas_band_max(plan: Plan, plane, lo: Sequence[int], hi: Sequence[int], stream=None):
    """Band maxima of a plane: (value float32[n], r int64[n], zi int32[n]) device tensors."""
    torch = _torch()
    n = len(lo)
    dev = plane.device
    value = torch.empty(n, dtype=torch.float32, device=dev)
    r = torch.empty(n, dtype=torch.int64, device=dev)
    zi = torch.empty(n, dtype=torch.int32, device=dev)
    scratch = torch.empty(max(1, 3 * n), dtype=torch.int64, device=dev)
    hlo = np.ascontiguousarray(np.asarray(lo, dtype=np.int64))
    hhi = np.ascontiguousarray(np.asarray(hi, dtype=np.int64))
    if hlo.shape != hhi.shape:
        raise ValueError("lo and hi must have the same length")
    args = (plan.handle,
            _dev_ptr(plane, "plane", plan.plane_dtype(), plan.info.plane_bytes),
            hlo.ctypes.data, hhi.ctypes.data, n,
            _dev_ptr(scratch, "scratch", torch.int64),
            _dev_ptr(value, "value", torch.float32), _dev_ptr(r, "r", torch.int64), _dev_ptr(zi, "zi", torch.int32),
            _stream_ptr(stream))
    _check(load().fdas_band_max(*args), "fdas_band_max", plan)   # pageable bounds are staged before it returns
    return value, r, zi


def fdas_get_templates(plan: Plan, out, stream=None):
    torch = _torch()
    K, S = plan.info.K, plan.cfg["seg_len"]
    _check(load().fdas_get_templates(plan.handle, _dev_ptr(out, "out", torch.float32, 8 * K * S),
                                     _stream_ptr(stream)), "fdas_get_templates", plan)


def fdas_levels_order(plan: Plan) -> np.ndarray:
    """The order of level 2's (row << 16 | 4-chunk block) entries the level search takes (host)."""
    lib = load()
    n = ctypes.c_int64(0)
    _check(lib.fdas_levels_order(plan.handle, None, 0, ctypes.byref(n)), "fdas_levels_order", plan)
    out = np.zeros(n.value, dtype=np.uint32)
    _check(lib.fdas_levels_order(plan.handle, out.ctypes.data, out.size, ctypes.byref(n)), "fdas_levels_order", plan)
    return out


def fdas_check_timeout(plan: Plan, max_cycles: int, stream=None):
    """Launch the bounded-wait self-check (sets FDAS_DEV_TIMEOUT after max_cycles SM cycles)."""
    _check(load().fdas_check_timeout(plan.handle, int(max_cycles), _stream_ptr(stream)), "fdas_check_timeout", plan)


def fdas_device_status(plan: Plan, clear: bool = True) -> int:
    bits = ctypes.c_int32(0)
    _check(load().fdas_device_status(plan.handle, ctypes.byref(bits), 1 if clear else 0), "fdas_device_status", plan)
    return int(bits.value)


def fdas_profile_enable(plan: Plan, enable: bool = True):
    _check(load().fdas_profile_enable(plan.handle, 1 if enable else 0), "fdas_profile_enable", plan)


def fdas_profile_read(plan: Plan, reset: bool = True) -> dict:
    """Per-stage event times (ms, summed) and launch counts since the last reset."""
    pr = _Profile()
    _check(load().fdas_profile_read(plan.handle, ctypes.byref(pr), 1 if reset else 0), "fdas_profile_read", plan)
    return {"calls": int(pr.calls), "launches": int(pr.launches),
            "ms": {STAGES[i]: float(pr.ms[i]) for i in range(4)},
            "n_timed": {STAGES[i]: int(pr.n_timed[i]) for i in range(4)},
            "peaks_kernels": {name: {"ms": float(pr.ms_peaks[i]), "n_timed": int(pr.n_timed_peaks[i])}
                              for i, name in enumerate(("k4_level1", "k4_levels"))},
            "level1_fused": int(pr.level1_fused)}


def fdas_destroy(plan: Plan):
    if plan.handle:
        load().fdas_destroy(plan.handle)
        plan.handle = None


# ----------------------------------------------------------------------------- batches
def _check_batch(status: int, where: str, batch=None):
    if status != FDAS_OK:
        detail = ""
        if batch is not None and batch.handle:
            detail = (load().fdas_batch_last_error(batch.handle) or b"").decode()
        raise FdasError(status, where, detail)


@dataclasses.dataclass
class BatchSeries:
    info: PlanInfo
    cfg: dict
    sample_offset: int
    peak_offset: int
    group: int


class Batch:
    """Owns an fdas_batch_t.  Create with fdas_batch_plan(); freed by fdas_batch_destroy() or GC."""

    def __init__(self, handle: int):
        self.handle = handle
        self.refresh()

    def refresh(self):
        lib = load()
        n, ws = ctypes.c_int32(), ctypes.c_size_t()
        ts, tp, tc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check_batch(lib.fdas_batch_get_info(self.handle, ctypes.byref(n), ctypes.byref(ws), ctypes.byref(ts),
                                             ctypes.byref(tp), ctypes.byref(tc)), "fdas_batch_get_info", self)
        self.n_series, self.workspace_bytes = int(n.value), int(ws.value)
        self.total_samples, self.total_peaks, self.total_cells = int(ts.value), int(tp.value), int(tc.value)
        self.series = []
        for i in range(self.n_series):
            inf, c = _Info(), _Config()
            so, po, g = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
            _check_batch(lib.fdas_batch_series_info(self.handle, i, ctypes.byref(inf), ctypes.byref(c), ctypes.byref(so),
                                                    ctypes.byref(po), ctypes.byref(g)), "fdas_batch_series_info", self)
            self.series.append(BatchSeries(PlanInfo(inf.nb, inf.K, inf.seg_valid, inf.n_seg, inf.plane_elem_bytes,
                                                    inf.plane_bytes, inf.workspace_bytes, inf.cells),
                                           _from_config(c), int(so.value), int(po.value), int(g.value)))

    def __del__(self):
        try:
            fdas_batch_destroy(self)
        except Exception:
            pass


def fdas_batch_plan(cfgs: Sequence[dict]) -> Batch:
    arr = (_Config * len(cfgs))()
    for i, cfg in enumerate(cfgs):
        _to_config(cfg, arr[i])
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    _check_batch(load().fdas_batch_plan(arr, len(cfgs), ctypes.byref(h), ctypes.byref(ws)), "fdas_batch_plan")
    return Batch(h.value)


def fdas_batch_autotune(batch: Batch, cache_path: Optional[str] = None, stream=None):
    path = cache_path.encode() if cache_path else None
    _check_batch(load().fdas_batch_autotune(batch.handle, path, _stream_ptr(stream)), "fdas_batch_autotune", batch)
    batch.refresh()


def fdas_batch_set_lanes(batch: Batch, lanes: int) -> int:
    """Concurrent lanes of the batch's graph; returns the new workspace size in bytes."""
    ws = ctypes.c_size_t()
    _check_batch(load().fdas_batch_set_lanes(batch.handle, int(lanes), ctypes.byref(ws)), "fdas_batch_set_lanes", batch)
    batch.refresh()
    return int(ws.value)


def fdas_batch_make_templates(batch: Batch, stream=None):
    _check_batch(load().fdas_batch_make_templates(batch.handle, _stream_ptr(stream)), "fdas_batch_make_templates",
                 batch)


def fdas_batch_search(batch: Batch, series, workspace, peaks, npeaks, stream=None):
    torch = _torch()
    args = (batch.handle,
            _dev_ptr(series, "series", torch.float32, 4 * batch.total_samples),
            _dev_ptr(workspace, "workspace", None, batch.workspace_bytes),
            _dev_ptr(peaks, "peaks", torch.uint8, 16 * batch.total_peaks) if batch.total_peaks > 0 else None,
            _dev_ptr(npeaks, "npeaks", torch.int32, 4 * batch.n_series),
            _stream_ptr(stream))
    _check_batch(load().fdas_batch_search(*args), "fdas_batch_search", batch)


def fdas_batch_device_status(batch: Batch, clear: bool = True) -> int:
    bits = ctypes.c_int32(0)
    _check_batch(load().fdas_batch_device_status(batch.handle, ctypes.byref(bits), 1 if clear else 0),
                 "fdas_batch_device_status", batch)
    return int(bits.value)


def fdas_batch_destroy(batch: Batch):
    if batch.handle:
        load().fdas_batch_destroy(batch.handle)
        batch.handle = None


# ----------------------------------------------------------------------------- conveniences
def peaks_to_numpy(peaks_u8, npeaks: int) -> np.ndarray:
    """View the first npeaks records of a uint8 peak buffer (device or host) as PEAK_DTYPE."""
    a = peaks_u8[: 16 * npeaks].cpu().numpy() if hasattr(peaks_u8, "cpu") else np.asarray(peaks_u8)[: 16 * npeaks]
    return a.view(PEAK_DTYPE).copy()


class Search:
    """One configured series search with its device buffers (torch-owned)."""

    def __init__(self, cfg: dict, device="cuda", stream=None):
        torch = _torch()
        self.plan = fdas_plan(cfg)
        self.device = torch.device(device)
        fdas_make_templates(self.plan, stream)
        inf = self.plan.info
        self.workspace = torch.empty(inf.workspace_bytes, dtype=torch.uint8, device=self.device)
        self.plane = torch.empty(inf.cells, dtype=self.plan.plane_dtype(), device=self.device)
        self.xhat = torch.empty(2 * inf.nb, dtype=torch.float32, device=self.device)
        self.sigma2 = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.peaks = torch.zeros(16 * max(1, cfg["max_peaks"]), dtype=torch.uint8, device=self.device)
        self.npeaks = torch.zeros(1, dtype=torch.int32, device=self.device)

    def plane_2d(self):
        return self.plane.view(self.plan.info.K, self.plan.info.nb)

    def search(self, series, stream=None):
        fdas_search(self.plan, series, self.workspace, self.plane, self.peaks, self.npeaks, stream)

    def spectrum(self, series, stream=None):
        fdas_spectrum(self.plan, series, self.workspace, self.xhat, self.sigma2, stream)
        return self.xhat

    def plane_from_spectrum(self, xhat, stream=None):
        fdas_plane(self.plan, xhat, self.workspace, self.plane, stream)
        return self.plane

    def find_peaks(self, stream=None):
        fdas_peaks(self.plan, self.plane, self.workspace, self.peaks, self.npeaks, stream)

    def peak_list(self) -> np.ndarray:
        n = int(self.npeaks.item())
        n = min(n, self.plan.cfg["max_peaks"])
        return peaks_to_numpy(self.peaks, n)
