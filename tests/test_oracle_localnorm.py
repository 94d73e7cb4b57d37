"""Pins of the oracle's robust local normalisation (orc_spectrum_local), against what the
mathematics fixes: the median of an exponential variable is its mean times ln 2; a median does
not move under a few outliers; the normalisation is invariant to the series' scale; and on red
noise it flattens the mean power block by block where one global sigma2 cannot."""
import numpy as np
import pytest

import fdas_synth as synth
import oracle


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _block_stat(xh, block, fn):
    p = np.abs(xh) ** 2
    out = []
    for b0 in range(0, p.size, block):
        v = p[b0:b0 + block]
        out.append(fn(v[1:] if b0 == 0 else v))
    return np.array(out)


def test_block_median_maps_to_2ln2_and_noise_mean_is_2():
    n, block = 1 << 18, 4096
    x = synth.noise(n, synth.rng_for(70, 0)).astype(np.float32)
    xh = oracle.spectrum_local(x, block)
    assert xh[0] == 0
    # the lower median of each block lands on 2 ln 2 (up to rounding of the scale)
    med = _block_stat(xh, block, lambda v: np.sort(v)[(v.size - 1) // 2])
    assert np.allclose(med, 2.0 * np.log(2.0), rtol=1e-12)
    # white noise: the exponential law then gives mean 2 per block (std of a block mean 2/64)
    mean = _block_stat(xh, block, np.mean)
    assert np.all(np.abs(mean - 2.0) < 0.2)
    assert abs(mean.mean() - 2.0) < 0.02


def test_scale_invariance():
    n = 1 << 14
    x = synth.noise(n, synth.rng_for(70, 1)).astype(np.float32)
    a = oracle.spectrum_local(x, 1024)
    b = oracle.spectrum_local((x * np.float32(4.0)).astype(np.float32), 1024)   # exact power-of-two scale
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12)


def test_strong_tone_moves_only_its_own_block_and_barely():
    """A tone with 2^16 times the noise power in one bin: the global sigma2 grows by a large
    factor, every other block is unchanged (up to the float32 rounding of the summed series) and
    its own block's scale moves by less than 1 %."""
    n, block = 1 << 16, 2048
    x = synth.noise(n, synth.rng_for(70, 2))
    r0 = 5 * block + 700
    tone = 2.0 * np.cos(2 * np.pi * r0 * np.arange(n) / n)
    a = oracle.spectrum_local(x.astype(np.float32), block)
    b = oracle.spectrum_local((x + tone).astype(np.float32), block)
    g_a, s2a = oracle.spectrum(x.astype(np.float32))
    g_b, s2b = oracle.spectrum((x + tone).astype(np.float32))
    assert s2b / s2a > 1.5                               # the global estimate is biased by the tone
    nb = n // 2
    for b0 in range(0, nb, block):
        sl = slice(b0, b0 + block)
        if b0 <= r0 < b0 + block:
            # this block's scale: ratio of normalised to raw at a bin away from the tone
            k = b0 + 100
            ra = abs(a[k]) / abs(g_a[k] / np.sqrt(2.0 / s2a))
            rb = abs(b[k]) / abs(g_b[k] / np.sqrt(2.0 / s2b))
            assert abs(rb / ra - 1.0) < 0.01
        else:
            assert np.allclose(np.abs(a[sl][1 if b0 == 0 else 0:]), np.abs(b[sl][1 if b0 == 0 else 0:]), rtol=1e-5)


def test_red_noise_is_flattened():
    """Red (1/f) noise: the power falls by decades across the spectrum.  One global sigma2
    leaves block means spread over orders of magnitude; the local normalisation brings every
    block's mean power to within 15 % of 2 wherever the power changes little across a block --
    all but the lowest block, where the power spans decades inside the block (its median still
    maps to 2 ln 2; only smaller blocks there would flatten it)."""
    n, block = 1 << 18, 4096
    rng = synth.rng_for(70, 3)
    w = np.fft.rfft(rng.standard_normal(n))                  # 1/f power: amplitude f^(-1/2)
    f = np.arange(w.size, dtype=np.float64)
    f[0] = 1.0
    x = np.fft.irfft(w * f ** -0.5, n).astype(np.float32)
    glob, _ = oracle.spectrum(x)
    loc = oracle.spectrum_local(x, block)
    gm = _block_stat(glob, block, np.mean)
    lm = _block_stat(loc, block, np.mean)
    assert gm[1:].max() / gm[1:].min() > 10.0
    assert np.all(np.abs(lm[1:] - 2.0) < 0.3)


def test_one_block_is_a_median_normalisation():
    """block = N/2: a single scale, the global mean replaced by median / ln 2 — for white noise
    within a few per cent of the mean-based normalisation."""
    n = 1 << 16
    x = synth.noise(n, synth.rng_for(70, 4)).astype(np.float32)
    loc = oracle.spectrum_local(x, n // 2)
    glob, _ = oracle.spectrum(x)
    ratio = np.abs(loc[1:]) / np.abs(glob[1:])
    assert np.allclose(ratio, ratio[0], rtol=1e-12)      # one scale for every bin
    assert abs(ratio[0] - 1.0) < 0.03


def test_bad_arguments_rejected():
    x = np.zeros(1 << 12, dtype=np.float32)
    with pytest.raises(ValueError):
        oracle.spectrum_local(x, 3000)
