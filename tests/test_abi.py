"""libfdas C-ABI on the CPU: the library loads, exports every symbol include/fdas.h declares,
validates configurations on the host, derives sizes, and reports errors without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2206_12205_gb300 as fd
from paper_2206_12205_gb300 import fdas as fb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    fd.build.build()
    return fd.load()


def _declared_symbols():
    with open(os.path.join(ROOT, "include", "fdas.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fdas_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = _declared_symbols()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(fb.EXPORTED) == names


def test_version_and_status_strings(lib):
    assert fd.fdas_version() == 106
    for code in range(8):
        assert fd.status_string(code) and fd.status_string(code) != "unknown status"
    assert fd.status_string(99) == "unknown status"


def test_struct_layouts(lib):
    # int64, 5 x int32, float[5], int32, pad, double, int32 norm_block, int32 harm_mode (static_assert'ed in C)
    assert ctypes.sizeof(fb._Config) == 72
    assert fb.PEAK_DTYPE.itemsize == 16


@pytest.mark.parametrize("n,zmax,m,S", [(1 << 16, 16, 64, 1024), (1 << 23, 84, 256, 8192),
                                         (1 << 11, 0, 2, 1024), (1 << 27, 1022, 4096, 8192),
                                         (1 << 12, 8, 512, 1024), (1 << 13, 2, 16, 2048)])
def test_plan_sizes(lib, n, zmax, m, S):
    p = fd.fdas_plan(fd.make_config(n, zmax, m, S, max_harm=16))
    nb, L = n // 2, (S - m + 1) // 32 * 32          # stride rounded down to whole 32-bin runs
    assert p.info.nb == nb and p.info.K == zmax + 1 and p.info.seg_valid == L
    assert p.info.n_seg == -(-nb // L)
    assert p.info.cells == (zmax + 1) * nb and p.info.plane_bytes == 4 * p.info.cells
    assert p.info.workspace_bytes >= 8 * nb * 2 + 8 * p.info.n_seg * S
    fd.fdas_destroy(p)


@pytest.mark.parametrize("kw", [
    dict(n=1 << 16 | 1), dict(n=1 << 10), dict(n=1 << 28), dict(zmax=15), dict(zmax=-2), dict(zmax=1024),
    dict(m=63), dict(m=0), dict(m=513), dict(S=512), dict(S=3000), dict(S=16384), dict(max_harm=3),
    dict(max_harm=32), dict(max_peaks=-1), dict(sigma2=-1.0), dict(sigma2=float("nan")), dict(precision=7),
    dict(thr=(float("nan"),) * 5)])
def test_plan_rejects_invalid(lib, kw):
    a = dict(n=1 << 16, zmax=16, m=64, S=1024, max_harm=1, max_peaks=10, sigma2=0.0, precision=0, thr=(30.0,) * 5)
    a.update(kw)
    cfg = fd.make_config(a["n"], a["zmax"], a["m"], a["S"], precision=a["precision"], max_harm=a["max_harm"],
                         thr=a["thr"], max_peaks=a["max_peaks"], sigma2=a["sigma2"])
    with pytest.raises(fd.FdasError) as ei:
        fd.fdas_plan(cfg)
    assert ei.value.status == fb.FDAS_E_INVALID


def test_null_arguments_rejected(lib):
    assert lib.fdas_plan(None, None, None) == fb.FDAS_E_INVALID
    p = fd.fdas_plan(fd.make_config(1 << 16, 16, 64, 1024))
    for fn, nargs in (("fdas_spectrum", 6), ("fdas_plane", 5), ("fdas_peaks", 6), ("fdas_search", 7),
                      ("fdas_get_templates", 3)):
        assert getattr(lib, fn)(p.handle, *([None] * (nargs - 1))) == fb.FDAS_E_INVALID
        assert getattr(lib, fn)(None, *([None] * (nargs - 1))) == fb.FDAS_E_INVALID
    assert lib.fdas_make_templates(None, None) == fb.FDAS_E_INVALID
    assert lib.fdas_device_status(None, None, 0) == fb.FDAS_E_INVALID
    assert lib.fdas_last_error(None) == b""
    lib.fdas_destroy(None)
    fd.fdas_destroy(p)


def test_calls_before_templates_are_out_of_order(lib):
    p = fd.fdas_plan(fd.make_config(1 << 16, 16, 64, 1024))
    fake = ctypes.c_void_p(1 << 20)        # never dereferenced: the state check comes first
    assert lib.fdas_plane(p.handle, fake, fake, fake, None) == fb.FDAS_E_STATE
    assert lib.fdas_search(p.handle, fake, fake, fake, fake, fake, None) == fb.FDAS_E_STATE
    fd.fdas_destroy(p)


def test_make_templates_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = fd.fdas_plan(fd.make_config(1 << 16, 16, 64, 1024))
    status = lib.fdas_make_templates(p.handle, None)
    assert status in (fb.FDAS_E_CUDA, fb.FDAS_E_NOMEM)
    assert lib.fdas_last_error(p.handle)
    fd.fdas_destroy(p)


def test_binding_refuses_host_tensors(lib):
    import torch
    p = fd.fdas_plan(fd.make_config(1 << 16, 16, 64, 1024))
    with pytest.raises(ValueError):
        fd.fdas_plane(p, torch.zeros(10), torch.zeros(10), torch.zeros(10))
    fd.fdas_destroy(p)


def test_misaligned_pointers_rejected(lib):
    p = fd.fdas_plan(fd.make_config(1 << 16, 16, 64, 1024))
    p_ptr = p.handle
    base = 1 << 20                                # never dereferenced: argument checks come first
    ok = ctypes.c_void_p(base)
    odd = ctypes.c_void_p(base + 4)               # 4-byte aligned only
    assert lib.fdas_plane(p_ptr, ok, ok, odd, None) == fb.FDAS_E_INVALID      # plane needs 16
    assert lib.fdas_plane(p_ptr, odd, ok, ok, None) == fb.FDAS_E_INVALID      # spectrum needs 8
    assert lib.fdas_plane(p_ptr, ok, odd, ok, None) == fb.FDAS_E_INVALID      # workspace needs 256
    assert lib.fdas_plane_static(p_ptr, ok, odd, None) == fb.FDAS_E_INVALID
    assert lib.fdas_search(p_ptr, odd, ok, ok, ok, ok, None) == fb.FDAS_E_INVALID
    fd.fdas_destroy(p)


def test_refine_entry_points_check_arguments(lib):
    """fdas_interp_power / fdas_refine validate on the host before any device work."""
    assert ctypes.sizeof(ctypes.c_double) * 2 == fb.CAND_DTYPE.itemsize == 16
    p = fd.fdas_plan(fd.make_config(1 << 16, 16, 64, 1024))
    h = p.handle
    base = 1 << 20                                # never dereferenced: argument checks come first
    ok = ctypes.c_void_p(base)
    odd = ctypes.c_void_p(base + 4)
    # n = 0 is a no-op even with NULL buffers; negative n, NULL buffers and bad flags are invalid
    assert lib.fdas_interp_power(h, None, None, None, 0, 0, None, None) == fb.FDAS_OK
    assert lib.fdas_refine(h, None, None, 0, 20, None, None, None, None) == fb.FDAS_OK
    assert lib.fdas_interp_power(None, ok, ok, None, 1, 0, ok, None) == fb.FDAS_E_INVALID
    assert lib.fdas_interp_power(h, ok, ok, None, -1, 0, ok, None) == fb.FDAS_E_INVALID
    assert lib.fdas_interp_power(h, ok, ok, None, 1, 2, ok, None) == fb.FDAS_E_INVALID
    assert lib.fdas_interp_power(h, None, ok, None, 1, 0, ok, None) == fb.FDAS_E_INVALID
    assert lib.fdas_interp_power(h, ok, odd, None, 1, 0, ok, None) == fb.FDAS_E_INVALID
    assert lib.fdas_interp_power(h, ok, ok, odd, 1, 0, ok, None) == fb.FDAS_E_INVALID
    assert lib.fdas_refine(None, ok, ok, 1, 20, ok, None, None, None) == fb.FDAS_E_INVALID
    assert lib.fdas_refine(h, ok, ok, 1, -1, ok, None, None, None) == fb.FDAS_E_INVALID
    assert lib.fdas_refine(h, ok, ok, 1, fb.REFINE_MAX_STEPS + 1, ok, None, None, None) == fb.FDAS_E_INVALID
    assert lib.fdas_refine(h, ok, None, 1, 20, ok, None, None, None) == fb.FDAS_E_INVALID
    assert lib.fdas_refine(h, ok, ok, 1, 20, odd, None, None, None) == fb.FDAS_E_INVALID
    assert lib.fdas_refine(h, ok, ok, 1, 20, ok, odd, None, None) == fb.FDAS_E_INVALID
    assert lib.fdas_refine(h, ok, ok, 1, 20, ok, None, ctypes.c_void_p(base + 2), None) == fb.FDAS_E_INVALID
    fd.fdas_destroy(p)


# ------------------------------------------------------------------ direct correlation variant
def test_direct_plan_geometry(lib):
    """FDAS_BF16_DIRECT: a BF16 plane; the taps image (2 ceil(K/8) 8 rows x 2m BF16) and the
    spectrum windows must fit one CTA's shared memory and 2 ceil(K/8) 8 <= 256, m % 8 == 0."""
    ok = fd.fdas_plan(fd.make_config(1 << 23, 84, 256, 8192, precision="bf16_direct", max_harm=16))
    assert ok.info.plane_elem_bytes == 2 and ok.info.K == 85
    assert ok.info.plane_bytes == 2 * 85 * (1 << 22)
    # the packed BF16 spectrum (Nb rounded to 512-bin tiles, plus the taps) fits the workspace
    assert ok.info.workspace_bytes >= 4 * ((1 << 22) + 256)
    fd.fdas_destroy(ok)
    for n, zmax, m in ((1 << 16, 128, 64), (1 << 16, 84, 512), (1 << 16, 16, 36)):
        with pytest.raises(fd.FdasError) as ei:
            fd.fdas_plan(fd.make_config(n, zmax, m, 1024, precision="bf16_direct"))
        assert ei.value.status == fb.FDAS_E_UNSUPPORTED, (n, zmax, m)
    small = fd.fdas_plan(fd.make_config(1 << 11, 0, 8, 1024, precision="bf16_direct"))
    assert small.info.K == 1
    fd.fdas_destroy(small)


def test_fp8_direct_plan_geometry(lib):
    """FDAS_FP8_DIRECT: an FP32 plane; taps % 16 == 0 (a 32-byte MMA K-step is 16 complex E4M3
    pairs) and the taps image (ceil(K/32) groups x 64 rows x 2m bytes) plus the windows within one
    CTA's shared memory, else unsupported."""
    ok = fd.fdas_plan(fd.make_config(1 << 23, 84, 256, 8192, precision="fp8_direct", max_harm=16))
    assert ok.info.plane_elem_bytes == 4 and ok.info.K == 85
    assert ok.info.plane_bytes == 4 * 85 * (1 << 22)
    fd.fdas_destroy(ok)
    wide = fd.fdas_plan(fd.make_config(1 << 16, 1022, 16, 1024, precision="fp8_direct"))
    assert wide.info.K == 1023
    fd.fdas_destroy(wide)
    for n, zmax, m, S in ((1 << 16, 16, 40, 1024), (1 << 16, 16, 8, 1024), (1 << 16, 84, 2048, 8192)):
        with pytest.raises(fd.FdasError) as ei:
            fd.fdas_plan(fd.make_config(n, zmax, m, S, precision="fp8_direct"))
        assert ei.value.status == fb.FDAS_E_UNSUPPORTED, (n, zmax, m)
    small = fd.fdas_plan(fd.make_config(1 << 11, 0, 16, 1024, precision="fp8_direct"))
    assert small.info.K == 1
    fd.fdas_destroy(small)


def test_check_timeout_arguments(lib):
    """The bounded-wait self-check validates on the host: a bound out of range is invalid, and
    it needs the plan's status word (templates made) first."""
    p = fd.fdas_plan(fd.make_config(1 << 16, 16, 64, 1024))
    assert lib.fdas_check_timeout(None, 1000, None) == fb.FDAS_E_INVALID
    assert lib.fdas_check_timeout(p.handle, 0, None) == fb.FDAS_E_INVALID
    assert lib.fdas_check_timeout(p.handle, (1 << 36) + 1, None) == fb.FDAS_E_INVALID
    assert lib.fdas_check_timeout(p.handle, 1000, None) == fb.FDAS_E_STATE
    fd.fdas_destroy(p)


@pytest.mark.parametrize("n,zmax", [(1 << 23, 84), (1 << 12, 0), (1 << 13, 10), (1 << 16, 6), (1 << 27, 200)])
def test_levels_order_is_the_ray_order(lib, n, zmax):
    """The level-2 search order: every (row, 4-chunk block) of level 2's region exactly once
    (rows with |2 z| <= zmax, bins below Nb/2 in 512-bin chunks), sorted by z over the block's
    middle bin, ties by row then block; computed on the host from the plan alone."""
    plan = fd.fdas_plan(fd.make_config(n, zmax, 32, 1024, max_harm=16))
    order = fd.fdas_levels_order(plan)
    nb = n // 2
    zl = zmax // 2
    zl -= zl & 1
    rows = zl + 1
    chunks = ((nb - 1) // 2 + 1 + 511) // 512
    blocks = (chunks + 3) // 4
    assert order.size == rows * blocks
    a, g = (order >> 16).astype(np.int64), (order & 0xFFFF).astype(np.int64)
    assert np.array_equal(np.sort(a * blocks + g), np.arange(rows * blocks))        # a permutation
    z = -zl + 2 * a                                                                # z of the row
    key = z / (4.0 * g + 2.0)                                                      # middle of 4 chunks
    assert np.all(np.diff(key) >= 0)
    tie = np.diff(key) == 0
    code = order.astype(np.int64)
    assert np.all(np.diff(code)[tie] > 0)
    zero = z == 0                                                                  # the z = 0 row: blocks in order
    assert np.array_equal(g[zero], np.arange(blocks))
    fd.fdas_destroy(plan)


def test_levels_order_arguments(lib):
    plan = fd.fdas_plan(fd.make_config(1 << 14, 8, 32, 1024))
    n = ctypes.c_int64(-1)
    assert lib.fdas_levels_order(None, None, 0, ctypes.byref(n)) == fb.FDAS_E_INVALID
    assert lib.fdas_levels_order(plan.handle, None, 0, None) == fb.FDAS_E_INVALID
    assert lib.fdas_levels_order(plan.handle, None, 0, ctypes.byref(n)) == fb.FDAS_OK and n.value > 0
    buf = np.zeros(n.value, dtype=np.uint32)
    assert lib.fdas_levels_order(plan.handle, buf.ctypes.data, n.value - 1, ctypes.byref(n)) == fb.FDAS_E_INVALID
    fd.fdas_destroy(plan)
