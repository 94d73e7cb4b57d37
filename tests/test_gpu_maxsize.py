"""The largest series the interface accepts (N = 2^27, Nb = 2^26 bins) through every precision's
search, checked by properties that hold at any size (the oracle would take minutes here): a
noiseless on-grid tone of amplitude a at bin r0 with the normalisation fixed at sigma2 = N has
P(r0, z = 0) = N a^2 / 2 exactly (the z = 0 template is a delta), it is the plane's largest
cell, nothing beyond four bins of it rises above the rounding floor, and every harmonic level
reports the one peak at (r0, z = 0) with that power (r0 has no divisor h <= 16, so no cell's
harmonic lands on it, and its own harmonics 2 r0, 3 r0, ... hold no power).  Exercises the
64-bit plane indexing, the largest grids and the last segment's ragged tail."""
import numpy as np
import pytest
import torch

import fdas_synth as synth
import paper_2206_12205_gb300 as fd

pytestmark = pytest.mark.gpu

N = 1 << 27
R0 = (1 << 21) + 11                      # inside every level's region (16 r0 < Nb); no divisor 2..16
P0 = 1000.0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fd.build.build()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def tone():
    a = np.sqrt(2.0 * P0 / N)
    x = synth.chirp(N, a, float(R0), 0.0).astype(np.float32)
    return torch.from_numpy(x).cuda()


@pytest.mark.parametrize("precision,m,rtol", [("fp32", 16, 1e-4), ("bf16", 16, 0.015), ("fp16_scaled", 16, 0.002),
                                              ("bf16_direct", 16, 0.015), ("fp8_direct", 16, 0.15)])
def test_max_size_tone(tone, precision, m, rtol):
    zmax = 2
    s = fd.Search(fd.make_config(N, zmax, m, 8192, precision=precision, max_harm=16, thr=(P0 / 2,) * 5,
                                 max_peaks=1024, sigma2=float(N)), device="cuda")
    s.search(tone)
    torch.cuda.synchronize()
    assert fd.fdas_device_status(s.plan) == 0
    plane = s.plane_2d()
    p0 = float(plane[zmax // 2, R0].float())
    assert abs(p0 / P0 - 1.0) <= rtol, (precision, p0)
    # the tone's cell is the plane's maximum; the z = +-2 rows see it within a couple of bins
    # (their templates' response), everything further away stays at the rounding floor
    pf = plane.float().clone()
    assert int(torch.argmax(pf.reshape(-1))) == (zmax // 2) * (N // 2) + R0
    pf[:, R0 - 4:R0 + 5] = 0.0
    assert float(pf.max()) < P0 / 100
    assert bool(torch.isfinite(plane[:, -8:].float()).all())
    pk = s.peak_list()
    assert len(pk) == 5                                     # levels 1, 2, 4, 8, 16
    assert sorted(int(h) for h in pk["harm"]) == [1, 2, 4, 8, 16]
    assert np.all(pk["r"] == R0) and np.all(pk["zi"] == zmax // 2)
    assert np.all(np.abs(pk["power"] / P0 - 1.0) <= rtol + 1e-3)
