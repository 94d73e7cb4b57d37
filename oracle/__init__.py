"""FP64 CPU oracle for the FDAS hot path (arXiv:2206.12205) -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference
legs may import this package.  The product library never loads it, and it shares no code
with the CUDA path: the arithmetic lives in ``fdas_oracle.c`` (plain C, FP64), compiled with
gcc into ``oracle/_build/liboracle.so``; this module only marshals numpy arrays.

What each function computes, and the paper passage it follows, is stated beside it in
``fdas_oracle.c``.  Pins that tie it to the paper and to mathematics live in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdas_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

PEAK_DTYPE = np.dtype([("h", np.int32), ("zi", np.int32), ("r", np.int64), ("power", np.float64)])


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, OpenMP over plane rows)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
           "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "orc_fft": (ctypes.c_int, [P, i64, ctypes.c_int]),
            "orc_spectrum": (ctypes.c_int, [P, i64, f64, P, P]),
            "orc_spectrum_local": (ctypes.c_int, [P, i64, i64, P]),
            "orc_e4m3": (f64, [f64]),
            "orc_plane_fp8": (ctypes.c_int, [P, i64, ctypes.c_int, ctypes.c_int, P, P]),
            "orc_plane_fp8_cells": (ctypes.c_int, [P, i64, ctypes.c_int, ctypes.c_int, P, i64, P, P, P]),
            "orc_fresnel": (None, [f64, P, P]),
            "orc_response": (None, [f64, f64, P]),
            "orc_response_quad": (None, [f64, f64, P]),
            "orc_response_moments_quad": (None, [f64, f64, P, P, P]),
            "orc_templates": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, P]),
            "orc_plane": (ctypes.c_int, [P, i64, ctypes.c_int, ctypes.c_int, P, P]),
            "orc_plane_cells": (ctypes.c_int, [P, i64, ctypes.c_int, ctypes.c_int, P, i64, P, P, P]),
            "orc_peaks_f32": (ctypes.c_int, [P, i64, ctypes.c_int, ctypes.c_int, P, i64, P, P, P, P, P]),
            "orc_peaks_anch_f32": (ctypes.c_int, [P, i64, ctypes.c_int, ctypes.c_int, P, i64, P, P, P, P, P]),
            "orc_peaks_anch_f64": (ctypes.c_int, [P, i64, ctypes.c_int, ctypes.c_int, P, i64, P, P, P, P, P]),
            "orc_peaks_f64": (ctypes.c_int, [P, i64, ctypes.c_int, ctypes.c_int, P, i64, P, P, P, P, P]),
            "orc_interp_power": (None, [P, i64, ctypes.c_int, f64, f64, P, P, P]),
            "orc_interp_power_at": (None, [P, i64, ctypes.c_int, i64, f64, f64, P, P, P]),
            "orc_refine_many": (None, [P, i64, ctypes.c_int, i64, P, ctypes.c_int, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def fft(a, sign: int = -1) -> np.ndarray:
    """Unscaled radix-2 complex FFT; sign -1 forward, +1 inverse."""
    b = np.array(a, dtype=np.complex128, copy=True)
    if _load().orc_fft(_p(b), b.size, int(sign)) != 0:
        raise ValueError("fft length must be a power of two")
    return b


def spectrum(x, sigma2: float = 0.0):
    """Normalised spectrum Xhat[0..N/2) of a real float32 series and the sigma^2 used."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    nb = x.size // 2
    out = np.empty(nb, dtype=np.complex128)
    s2 = ctypes.c_double(0.0)
    if _load().orc_spectrum(_p(x), x.size, float(sigma2), _p(out), ctypes.byref(s2)) != 0:
        raise ValueError("series length must be a power of two >= 4")
    return out, s2.value


def spectrum_local(x, block: int):
    """Spectrum with robust local normalisation: each block of `block` bins scaled by
    sqrt(2 ln 2 / median |X_k|^2) over the block (orc_spectrum_local)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    nb = x.size // 2
    out = np.empty(nb, dtype=np.complex128)
    if _load().orc_spectrum_local(_p(x), x.size, int(block), _p(out)) != 0:
        raise ValueError("series length must be a power of two >= 4 and block must divide N/2")
    return out


def e4m3(v):
    """FP8 E4M3 rounding (nearest, ties to even, saturating at +-448), elementwise."""
    a = np.atleast_1d(np.asarray(v, dtype=np.float64))
    fn = _load().orc_e4m3
    return np.array([fn(float(t)) for t in a.flat]).reshape(a.shape)


def plane_fp8(xhat, zmax: int, m: int, T=None) -> np.ndarray:
    """The FP8 direct-correlation plane (orc_plane_fp8): E4M3 operands with per-1024-bin-tile
    and per-template power-of-two scales, FP64 sums."""
    xhat = np.ascontiguousarray(xhat, dtype=np.complex128)
    if T is None:
        T, _ = templates(zmax, m)
    T = np.ascontiguousarray(T, dtype=np.complex128)
    out = np.empty((zmax + 1, xhat.size), dtype=np.float64)
    if _load().orc_plane_fp8(_p(xhat), xhat.size, int(zmax), int(m), _p(T), _p(out)) != 0:
        raise MemoryError("orc_plane_fp8")
    return out


def plane_fp8_cells(xhat, zmax: int, m: int, T, zi, r) -> np.ndarray:
    """Selected cells of the FP8 direct-correlation plane (orc_plane_fp8_cells)."""
    xhat = np.ascontiguousarray(xhat, dtype=np.complex128)
    T = np.ascontiguousarray(T, dtype=np.complex128)
    zi = np.ascontiguousarray(zi, dtype=np.int32)
    r = np.ascontiguousarray(r, dtype=np.int64)
    out = np.empty(zi.size, dtype=np.float64)
    rc = _load().orc_plane_fp8_cells(_p(xhat), xhat.size, int(zmax), int(m), _p(T), zi.size, _p(zi), _p(r), _p(out))
    if rc == -2:
        raise ValueError("cell index off the plane")
    if rc != 0:
        raise MemoryError("orc_plane_fp8_cells")
    return out


def fresnel(x):
    """(C(x), S(x)) elementwise."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    c = np.empty_like(x)
    s = np.empty_like(x)
    lib = _load()
    cv, sv = ctypes.c_double(), ctypes.c_double()
    for i, v in enumerate(x.flat):
        lib.orc_fresnel(float(v), ctypes.byref(cv), ctypes.byref(sv))
        c.flat[i] = cv.value
        s.flat[i] = sv.value
    return c, s


def _scalar_c(fn, q, z):
    q = np.atleast_1d(np.asarray(q, dtype=np.float64))
    z = np.broadcast_to(np.asarray(z, dtype=np.float64), q.shape)
    out = np.empty(q.shape, dtype=np.complex128)
    v = np.zeros(1, dtype=np.complex128)
    for i in range(q.size):
        fn(float(q.flat[i]), float(z.flat[i]), _p(v))
        out.flat[i] = v[0]
    return out


def response(q, z) -> np.ndarray:
    """I(q, z) = int_0^1 exp(i pi (z u^2 - 2 q u)) du via Fresnel integrals."""
    return _scalar_c(_load().orc_response, q, z)


def response_quad(q, z) -> np.ndarray:
    """I(q, z) by composite Gauss-Legendre quadrature (independent route)."""
    return _scalar_c(_load().orc_response_quad, q, z)


def response_moments_quad(q: float, z: float):
    """(M0, M1, M2), M_p = int_0^1 u^p exp(i pi (z u^2 - 2 q u)) du."""
    a = np.zeros(3, dtype=np.complex128)
    _load().orc_response_moments_quad(float(q), float(z), _p(a[0:]), _p(a[1:]), _p(a[2:]))
    return a[0], a[1], a[2]


def templates(zmax: int, m: int):
    """Unit-norm template bank T[K][m] (K = zmax + 1) and the norms eta[K]."""
    K = zmax + 1
    T = np.empty((K, m), dtype=np.complex128)
    eta = np.empty(K, dtype=np.float64)
    if _load().orc_templates(int(zmax), int(m), _p(T), _p(eta)) != 0:
        raise ValueError("zmax must be even >= 0 and m even >= 2")
    return T, eta


def plane(xhat, zmax: int, m: int, T=None) -> np.ndarray:
    """Full f-z power plane [K][nb] by direct correlation (FP64)."""
    xhat = np.ascontiguousarray(xhat, dtype=np.complex128)
    if T is None:
        T, _ = templates(zmax, m)
    T = np.ascontiguousarray(T, dtype=np.complex128)
    out = np.empty((zmax + 1, xhat.size), dtype=np.float64)
    if _load().orc_plane(_p(xhat), xhat.size, int(zmax), int(m), _p(T), _p(out)) != 0:
        raise ValueError("bad plane arguments")
    return out


def plane_cells(xhat, zmax: int, m: int, T, zi, r) -> np.ndarray:
    """Selected plane cells P(r[c], z_{zi[c]})."""
    xhat = np.ascontiguousarray(xhat, dtype=np.complex128)
    T = np.ascontiguousarray(T, dtype=np.complex128)
    zi = np.ascontiguousarray(zi, dtype=np.int32)
    r = np.ascontiguousarray(r, dtype=np.int64)
    out = np.empty(zi.size, dtype=np.float64)
    if _load().orc_plane_cells(_p(xhat), xhat.size, int(zmax), int(m), _p(T), zi.size,
                               _p(zi), _p(r), _p(out)) != 0:
        raise ValueError("cell index off the plane")
    return out


def _peaks(fn, plane_arr, zmax, max_harm, thr, max_out, pdtype):
    K, nb = plane_arr.shape
    if K != zmax + 1:
        raise ValueError("plane rows must be zmax + 1")
    thr = list(np.atleast_1d(np.asarray(thr, dtype=np.float64)))
    thr = np.array((thr + [thr[-1]] * 5)[:5], dtype=np.float64)   # one threshold per level
    cap = max(int(max_out), 1)
    h = np.empty(cap, np.int32)
    zi = np.empty(cap, np.int32)
    r = np.empty(cap, np.int64)
    p = np.empty(cap, pdtype)
    cnt = ctypes.c_int64(0)
    if fn(_p(plane_arr), nb, int(zmax), int(max_harm), _p(thr), int(max_out), _p(h), _p(zi),
          _p(r), _p(p), ctypes.byref(cnt)) != 0:
        raise ValueError("bad harmonic-sum arguments")
    n = min(cnt.value, int(max_out))
    out = np.empty(n, dtype=[("h", np.int32), ("zi", np.int32), ("r", np.int64), ("power", pdtype)])
    out["h"], out["zi"], out["r"], out["power"] = h[:n], zi[:n], r[:n], p[:n]
    return out, cnt.value


def peaks_f32(plane_f32, zmax: int, max_harm: int, thr, max_out: int = 1 << 20, anchored: bool = False):
    """Harmonic sums + peak list of a float32 plane, in float32 (given-plane mode); anchored:
    the highest-harmonic-anchored sums with rounding."""
    a = np.ascontiguousarray(plane_f32, dtype=np.float32)
    fn = _load().orc_peaks_anch_f32 if anchored else _load().orc_peaks_f32
    return _peaks(fn, a, zmax, max_harm, thr, max_out, np.float32)


def peaks_f64(plane_f64, zmax: int, max_harm: int, thr, max_out: int = 1 << 20, anchored: bool = False):
    """Harmonic sums + peak list of an FP64 plane."""
    a = np.ascontiguousarray(plane_f64, dtype=np.float64)
    fn = _load().orc_peaks_anch_f64 if anchored else _load().orc_peaks_f64
    return _peaks(fn, a, zmax, max_harm, thr, max_out, np.float64)


def interp_power(xhat, m: int, r: float, z: float, k0=None):
    """(P, dP/dr, dP/dz) of the Fourier-interpolated power at fractional (r, z).

    The m-tap window is anchored at bin k0 (default: the nearest bin, floor(r + 1/2))."""
    xhat = np.ascontiguousarray(xhat, dtype=np.complex128)
    v = np.zeros(3, dtype=np.float64)
    if k0 is None:
        _load().orc_interp_power(_p(xhat), xhat.size, int(m), float(r), float(z),
                                 _p(v[0:]), _p(v[1:]), _p(v[2:]))
    else:
        _load().orc_interp_power_at(_p(xhat), xhat.size, int(m), int(k0), float(r), float(z),
                                    _p(v[0:]), _p(v[1:]), _p(v[2:]))
    return float(v[0]), float(v[1]), float(v[2])


def refine(xhat, m: int, rz, steps: int):
    """Gradient-ascent refinement of seeds rz ([n, 2] of (r, z)), every step in FP64.

    Returns (points [n, 2], P [n], evaluations [n])."""
    xhat = np.ascontiguousarray(xhat, dtype=np.complex128)
    rz = np.ascontiguousarray(np.asarray(rz, dtype=np.float64).reshape(-1, 2))
    n = rz.shape[0]
    out = np.zeros((n, 2), dtype=np.float64)
    pw = np.zeros(n, dtype=np.float64)
    ev = np.zeros(n, dtype=np.int32)
    if n:
        _load().orc_refine_many(_p(xhat), xhat.size, int(m), n, _p(rz), int(steps), _p(out), _p(pw), _p(ev))
    return out, pw, ev


def band_max(plane, lo, hi):
    """Band maxima (Sec. 4.3, Table harm_bounds): for each band [lo, hi] of bins (clipped to the
    plane), the largest cell over all template rows and its first position in row-major
    (zi, r) order.  Returns (value, r, zi) arrays; an empty band gives -1 in all three."""
    plane = np.asarray(plane)
    nb = plane.shape[1]
    v, rr, zz = [], [], []
    for l, h in zip(lo, hi):
        l, h = max(0, int(l)), min(nb - 1, int(h))
        if h < l:
            v.append(-1.0); rr.append(-1); zz.append(-1)
            continue
        sub = plane[:, l:h + 1]
        zi, r = np.unravel_index(int(np.argmax(sub)), sub.shape)   # argmax: first maximum, row-major
        v.append(float(sub[zi, r])); rr.append(l + int(r)); zz.append(int(zi))
    return np.array(v), np.array(rr, dtype=np.int64), np.array(zz, dtype=np.int32)


def search(x, zmax: int, m: int, max_harm: int, thr, sigma2: float = 0.0, max_out: int = 1 << 20):
    """The whole oracle path on one series: spectrum, templates, plane, peaks (FP64)."""
    xhat, s2 = spectrum(x, sigma2)
    T, eta = templates(zmax, m)
    pl = plane(xhat, zmax, m, T)
    pk, n = peaks_f64(pl, zmax, max_harm, thr, max_out)
    return {"xhat": xhat, "sigma2": s2, "T": T, "eta": eta, "plane": pl, "peaks": pk, "npeaks": n}
