"""GPU parity of the robust local normalisation (fdas_config.norm_block) against the oracle's
orc_spectrum_local: the normalised spectrum itself, the FP32 plane of a whole search built on it,
and what it is for -- a tone above red noise that one global sigma2 buries."""
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


def _red(n, seed, amp_tone=0.0, r0=0.0):
    rng = synth.rng_for(71, seed)
    w = np.fft.rfft(rng.standard_normal(n))
    f = np.arange(w.size, dtype=np.float64)
    f[0] = 1.0
    x = np.fft.irfft(w * f ** -0.5, n)
    if amp_tone:
        x = x + amp_tone * np.cos(2 * np.pi * r0 * np.arange(n) / n)
    return x.astype(np.float32)


@pytest.mark.parametrize("n,block", [(1 << 16, 64), (1 << 18, 1024), (1 << 18, 4096), (1 << 12, 2048)])
def test_local_spectrum_matches_oracle(n, block):
    x = _red(n, n.bit_length(), 0.05, n / 3.7)
    s = fd.Search(fd.make_config(n, 8, 32, 1024, norm_block=block), device="cuda")
    xh = s.spectrum(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    got = xh.cpu().numpy().view(np.complex64).astype(np.complex128)
    ref = oracle.spectrum_local(x, block)
    assert got[0] == 0
    # The FP32 FFT's error is absolute, set by the whole spectrum (the global spectrum test's
    # bound: 2e-6 of the largest raw amplitude); the local normalisation multiplies it by the
    # block's scale, which is large in the quiet blocks of red noise.
    raw, _ = oracle.spectrum(x, sigma2=2.0)                   # sigma2 = 2: scale 1, the raw X
    scale = np.ones(raw.size)
    for b0 in range(0, raw.size, block):
        k = b0 + np.argmax(np.abs(raw[b0:b0 + block]))
        scale[b0:b0 + block] = np.abs(ref[k]) / np.abs(raw[k])
    bound = 2e-6 * np.abs(raw).max() * scale + 2e-5
    err = np.abs(got - ref)
    print(f"local norm n={n} block={block}: max error / bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound)
    # the median of every block maps to 2 ln 2 on the GPU too
    p = np.abs(got) ** 2
    for b0 in range(0, p.size, block):
        v = p[b0 + (1 if b0 == 0 else 0):b0 + block]
        assert abs(np.sort(v)[(v.size - 1) // 2] / (2 * np.log(2.0)) - 1.0) < 1e-5


def test_local_search_plane_matches_oracle():
    """The FP32 plane of a whole search with local normalisation against the oracle's plane on
    its locally normalised spectrum (white noise with a chirp: every block gets its own median
    scale, and the FP32 path's 1e-5 floor-relative plane bound applies; on red noise the FFT's
    absolute error is amplified in quiet blocks, as the spectrum test bounds)."""
    n, zmax, m, block = 1 << 15, 16, 64, 1024
    x = (synth.noise(n, synth.rng_for(71, 40)) + synth.chirp(n, 0.3, 5000.3, 6.2)).astype(np.float32)
    s = fd.Search(fd.make_config(n, zmax, m, 1024, norm_block=block), device="cuda")
    s.search(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    got = s.plane_2d().cpu().numpy().astype(np.float64)
    ref = oracle.plane(oracle.spectrum_local(x, block), zmax, m)
    fr = np.abs(got - ref) / np.maximum(ref, 2.0)
    print(f"local-norm search plane: floor-relative max {fr.max():.2e}")
    assert fr.max() <= 1e-5
    assert fd.fdas_device_status(s.plan) == 0


def test_tone_above_red_noise_is_recovered():
    """A weak tone at a high frequency over 1/f noise: with one global sigma2 (set by the strong
    low-frequency power) its plane peak stays far below the threshold; with the local
    normalisation it is detected at its bin with the power the white-noise case would give."""
    n, zmax, m, thr = 1 << 18, 4, 32, 40.0
    r0 = 100000
    # 1/f noise has mean power n / k at bin k (here 2.6) against a global mean of about
    # 2 (ln(N/2) + 0.58) = 24.7: a tone of bin power 100 n / r0 normalises to ~200 locally and to
    # ~21 globally
    amp = np.sqrt(100.0 * n / r0) / (n / 2)
    x = _red(n, 41, amp, r0)
    found = {}
    for block in (0, 4096):
        s = fd.Search(fd.make_config(n, zmax, m, 1024, norm_block=block, thr=(thr,) * 5, max_peaks=4096), device="cuda")
        s.search(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        pk = s.peak_list()
        found[block] = [p for p in pk if abs(int(p["r"]) - r0) <= 1]
        plane = s.plane_2d().cpu().numpy()
        found[(block, "p")] = float(plane[:, r0 - 1:r0 + 2].max())
    assert not found[0] and found[(0, "p")] < thr
    assert found[4096] and found[(4096, "p")] > 3 * thr
