"""The level-1 pass fused into the plane kernel (every precision but the split one): inside
fdas_search the plane kernel marks every 512-bin unit of a row that holds a stored value above
min(thr[0], thr[1] / 2); level 1 visits only those units instead of reading the whole plane, and
the level search skips the chunks outside level 4's region whose level-2 sums the marks bound
below thr[1] (the chunk's unit and its second harmonic's two units unmarked).  The peak list
must be the one the full passes give (fdas_peaks on the same plane: no marks, every chunk
searched), record for record -- the full passes are the ones the parity tests pin to the oracle
-- for thresholds from "a handful of units" to "nearly all", every precision with marks, ragged
segment tails and the last bins of the rows."""
import numpy as np
import pytest
import torch

import fdas_synth as synth
import paper_2206_12205_gb300 as fd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fd.build.build()
    torch.cuda.set_device(0)


def _series(n, seed):
    x = synth.noise(n, synth.rng_for(75, seed))
    x += synth.chirp(n, 0.3, n / 9.7, 7.3)
    x += synth.pulse_train(n, n / 53.0, 2.0, 0.08, 40.0, 0.0)
    x += synth.chirp(n, 0.25, n / 2 - 40.5, -3.0)            # power in the last bins of the rows
    return x.astype(np.float32)


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16_scaled", "bf16_direct", "fp8_direct"])
@pytest.mark.parametrize("thr1", [3.0, 12.0, 40.0])
def test_marked_level1_equals_full_pass(precision, thr1):
    n, zmax, m = 1 << 18, 32, 128
    thr = (thr1, thr1 + 8.0, thr1 + 14.0, thr1 + 24.0, thr1 + 40.0)
    s = fd.Search(fd.make_config(n, zmax, m, 8192, precision=precision, max_harm=16, thr=thr, max_peaks=1 << 21),
                  device="cuda")
    fd.fdas_profile_enable(s.plan, True)
    s.search(torch.from_numpy(_series(n, int(thr1))).cuda())
    torch.cuda.synchronize()
    prof = fd.fdas_profile_read(s.plan, reset=True)
    assert prof["level1_fused"] == 1
    fused_n = int(s.npeaks.item())
    fused = s.peak_list().copy()
    s.find_peaks()                                            # the full level-1 pass on the same plane
    torch.cuda.synchronize()
    assert fd.fdas_profile_read(s.plan, reset=True)["level1_fused"] == 0
    full_n = int(s.npeaks.item())
    full = s.peak_list()
    print(f"{precision} thr1={thr1}: {full_n} peaks, level 1: {int(np.sum(full['harm'] == 1))}")
    assert fused_n == full_n and full_n > 0
    assert fused.tobytes() == full.tobytes()
    assert fd.fdas_device_status(s.plan) == 0


def test_marks_cover_the_row_ends():
    """Power only in the last 512-bin unit of every row and in the ragged tail of the last
    segment: its level-1 peaks are found through the marks exactly as by the full pass."""
    n, zmax, m = 1 << 16, 8, 64
    nb = n // 2
    x = (synth.noise(n, synth.rng_for(75, 7)) + synth.chirp(n, 0.4, nb - 3.2, 0.0)).astype(np.float32)
    s = fd.Search(fd.make_config(n, zmax, m, 8192, precision="bf16", max_harm=1, thr=(25.0,) * 5, max_peaks=4096),
                  device="cuda")
    s.search(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    fused = s.peak_list().copy()
    s.find_peaks()
    torch.cuda.synchronize()
    full = s.peak_list()
    assert len(full) > 0 and fused.tobytes() == full.tobytes()
    assert int(full["r"].max()) >= nb - 512
