"""fdas_plane_static: the plane without a caller workspace, for callers that may not allocate
device memory at call time (code inside CUDA stream capture, real-time pipelines that reserve
all memory at start-up, hosts whose own allocator owns the device).  It must give the same
plane as fdas_plane on consecutive calls that share its static scratch array.

This file is collected last on purpose, so that a run stopping at the first failure has run
every other test before it; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import fdas_synth as synth
import oracle
import paper_2206_12205_gb300 as fd
from paper_2206_12205_gb300 import fdas as fb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fd.build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _floor_err(p, ref):
    return float(np.max(np.abs(p - ref) / np.maximum(ref, 2.0)))


@pytest.mark.parametrize("n,zmax,m,S", [(1 << 16, 16, 64, 1024), (1 << 20, 84, 256, 8192)])
def test_static_plane_matches_workspace_plane_twice(n, zmax, m, S):
    s = fd.Search(fd.make_config(n, zmax, m, S), device="cuda")
    out_static = torch.empty_like(s.plane)
    for call in range(2):                      # two calls in a row share the static scratch
        x = (synth.noise(n, synth.rng_for(70 + call, n.bit_length()))
             + synth.chirp(n, 0.1 + 0.05 * call, n / 11.0 + 100 * call, 4.0 * call)).astype(np.float32)
        xhat = s.spectrum(torch.from_numpy(x).cuda()).clone()
        s.plane_from_spectrum(xhat)
        torch.cuda.synchronize()
        free0, torch0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        # through the C-ABI directly
        st = fd.load().fdas_plane_static(
            s.plan.handle, ctypes.c_void_p(xhat.data_ptr()), ctypes.c_void_p(out_static.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == fb.FDAS_OK, fd.load().fdas_last_error(s.plan.handle)
        torch.cuda.synchronize()
        if call == 1:                          # after the first call (which may load the module): no allocation
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == torch0
        ref = s.plane.cpu().numpy().astype(np.float64)
        got = out_static.cpu().numpy().astype(np.float64)
        assert _floor_err(got, ref) <= 1e-5


def test_static_plane_rejects_oversized_plan():
    # n_seg * S * 8 bytes above the static array: 2^24 samples with 8192-bin segments
    p = fd.fdas_plan(fd.make_config(1 << 24, 4, 256, 8192))
    fd.fdas_make_templates(p)
    assert p.info.n_seg * 8192 * 8 > fb.STATIC_SCRATCH_BYTES
    dummy = torch.empty(1, device="cuda")
    st = fd.load().fdas_plane_static(p.handle, ctypes.c_void_p(dummy.data_ptr()),
                                     ctypes.c_void_p(dummy.data_ptr()), None)
    assert st == fb.FDAS_E_UNSUPPORTED
    assert b"static array holds" in fd.load().fdas_last_error(p.handle)
    fd.fdas_destroy(p)
