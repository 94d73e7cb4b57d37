"""Failure detection on the GPU without a fault: a bounded wait that nothing completes runs out,
the kernel records FDAS_DEV_TIMEOUT in the plan's status word and returns, and the context stays
usable -- the next search on the same plan runs and reports a clean status."""
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


def test_bounded_wait_runs_out_and_the_context_survives():
    w = synth.single_chirp_workload()
    s = fd.Search(fd.make_config(w.n, w.zmax, w.taps, w.seg_len, precision="bf16", max_harm=1, thr=(30.0,) * 5,
                                 max_peaks=4096), device="cuda")
    assert fd.fdas_device_status(s.plan) == 0
    fd.fdas.fdas_check_timeout(s.plan, 200_000_000)          # about 0.1 s at 2 GHz
    torch.cuda.synchronize()
    assert fd.fdas_device_status(s.plan) & fd.fdas.FDAS_DEV_TIMEOUT    # read and cleared
    assert fd.fdas_device_status(s.plan) == 0
    s.search(torch.from_numpy(w.series).cuda())
    torch.cuda.synchronize()
    pk = s.peak_list()
    assert len(pk) > 0 and np.all(np.isfinite(pk["power"]))
    assert fd.fdas_device_status(s.plan) == 0
