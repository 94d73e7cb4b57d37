"""GPU parity of the highest-harmonic-anchored harmonic sums (fdas_config.harm_mode = 1) against
the oracle's orc_peaks_anch_f32 on the same plane: bit-exact peak lists (level, row, bin and the
float power), for FP32 and BF16 (quick-cast) planes, every level, ties and the list overflow."""
import numpy as np
import pytest
import torch

import fdas_synth as synth
import oracle
import paper_2206_12205_gb300 as fd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fd.build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _peaks_equal(got, want):
    assert len(got) == len(want)
    for g, w in zip(got, want):
        assert (int(g["harm"]), int(g["zi"]), int(g["r"])) == (int(w["h"]), int(w["zi"]), int(w["r"]))
        assert np.float32(g["power"]).tobytes() == np.float32(w["power"]).tobytes()


@pytest.mark.parametrize("max_harm,precision", [(1, "fp32"), (2, "fp32"), (4, "fp32"), (8, "fp32"), (16, "fp32"),
                                                (16, "bf16")])
def test_anchored_peaks_bit_exact_given_plane(max_harm, precision):
    """The oracle's FP64 plane of a harmonic-rich accelerated signal, rounded once to the plane
    format, searched by both sides with anchored sums: bit-exact lists."""
    n, zmax, m, S = 1 << 16, 32, 64, 1024
    x = synth.noise(n, synth.rng_for(72, max_harm))
    for h in range(1, 6):
        x += synth.chirp(n, 0.08 / h, 1234.0 * h, 6.0 * h)
    x = x.astype(np.float32)
    xr, _ = oracle.spectrum(x)
    pl = oracle.plane(xr, zmax, m).astype(np.float32)
    if precision == "bf16":
        t = torch.from_numpy(pl).to(torch.bfloat16)
        pl = t.float().numpy()
    thr = (12.0, 18.0, 28.0, 45.0, 70.0)
    s = fd.Search(fd.make_config(n, zmax, m, S, precision=precision, max_harm=max_harm, thr=thr, max_peaks=1 << 16,
                                 harm_mode=1), device="cuda")
    if precision == "bf16":
        s.plane.copy_(t.reshape(-1).cuda())
    else:
        s.plane.copy_(torch.from_numpy(pl.ravel()))
    s.find_peaks()
    torch.cuda.synchronize()
    got = s.peak_list()
    want, cnt = oracle.peaks_f32(pl, zmax, max_harm, thr, anchored=True)
    assert int(s.npeaks.item()) == cnt > 0
    _peaks_equal(got, want)
    assert fd.fdas_device_status(s.plan) == 0


def test_anchored_ties_edges_and_overflow():
    n, zmax, m, S = 1 << 14, 6, 16, 1024
    K, nb = zmax + 1, n // 2
    s = fd.Search(fd.make_config(n, zmax, m, S, max_harm=4, thr=(1.0, 1.0, 1.0), max_peaks=6, harm_mode=1),
                  device="cuda")
    pl = np.zeros((K, nb), dtype=np.float32)
    pl[3, 100] = pl[3, 101] = 9.0                     # plateau in a row
    pl[2, 300] = pl[3, 300] = 7.0                     # plateau in a column
    pl[0, 0] = 5.0                                    # corner cell
    pl[K - 1, nb - 1] = 5.0                           # last cell (its lower harmonics at nb/2, nb/4 ...)
    pl[3, 1500] = 6.0                                 # the fundamental of an anchored pair ...
    pl[3, 3000] = 6.0                                 # ... with the 2nd harmonic at 2r (z = 0 row)
    pl[5, 511] = 4.0; pl[5, 512] = 4.0                # a pair across a 512-bin chunk boundary
    s.plane.copy_(torch.from_numpy(pl.ravel()))
    s.find_peaks()
    torch.cuda.synchronize()
    want, cnt = oracle.peaks_f32(pl, zmax, 4, (1.0, 1.0, 1.0), max_out=6, anchored=True)
    assert int(s.npeaks.item()) == cnt and cnt > 6
    _peaks_equal(s.peak_list(), want)
    assert fd.fdas_device_status(s.plan) & fd.fdas.FDAS_DEV_PEAK_OVERFLOW


def test_anchored_search_finds_the_highest_harmonic():
    """A pulse train at (r0, z0) = (1000, 4) searched end to end with anchored sums: the cell
    (4 r0, 4 z0) reads harmonics j = 1, 2, 3 at exactly (j r0, j z0), so the strongest level-4
    peak is there, and its power is the sum of the four harmonics' plane values."""
    n, zmax, m = 1 << 18, 20, 64
    x = synth.noise(n, synth.rng_for(72, 9)) + synth.pulse_train(n, 1000.0, 4.0, 0.1, 60.0, 0.0)
    x = x.astype(np.float32)
    s = fd.Search(fd.make_config(n, zmax, m, 1024, precision="fp32", max_harm=4, thr=(30, 30, 30, 30, 30),
                                 max_peaks=1 << 16, harm_mode=1), device="cuda")
    s.search(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    pk = s.peak_list()
    lev4 = pk[pk["harm"] == 4]
    best = lev4[np.argmax(lev4["power"])]
    zi4 = (16 + zmax) // 2
    assert (int(best["r"]), int(best["zi"])) == (4000, zi4)
    plane = s.plane_2d().cpu().numpy()
    want = np.float32(0.0)
    for r, zi in ((4000, zi4), (2000, (8 + zmax) // 2), (1000, (4 + zmax) // 2), (3000, (12 + zmax) // 2)):
        want = np.float32(want + plane[zi, r])        # the nested order: anchor, j = 1/2, 1/4, 3/4
    assert np.float32(best["power"]) == want
    assert fd.fdas_device_status(s.plan) == 0
