"""Sensitivity analysis on the GPU: band maxima (the paper's harmonic-band peak selection,
Sec. 4.3, Table harm_bounds) against the oracle on the same plane, and the noise law of
noise-only planes in every precision (Sec. 5.1: chi^2 with 2 degrees of freedom, no skew
between precisions)."""
import numpy as np
import pytest
import scipy.stats
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


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_band_max_matches_oracle(precision):
    n, zmax = 1 << 16, 16
    K, nb = zmax + 1, n // 2
    rng = synth.rng_for(90, 1 if precision == "fp32" else 2)
    pl = synth.noise_plane(K, nb, rng)
    # ties: equal maxima in one band, the earlier cell in row-major (zi, r) order must win
    pl[3, 1000] = pl[7, 900] = pl[3, 1100] = 77.0
    pl[0, 5] = 55.0
    pl[K - 1, nb - 1] = 66.0
    s = fd.Search(fd.make_config(n, zmax, 64, 1024, precision=precision))
    if precision == "bf16":
        t = torch.from_numpy(pl).to(torch.bfloat16)
        want_plane = t.float().numpy()
        s.plane.copy_(t.reshape(-1).cuda())
    else:
        want_plane = pl
        s.plane.copy_(torch.from_numpy(pl.ravel()))
    lo = [0, 800, 4096, 20000, nb - 10, nb + 5, -30, 950]
    hi = [2000, 1200, 4096, 30000, nb + 100, nb + 50, 3, 1099]
    v, r, zi = fd.fdas_band_max(s.plan, s.plane, lo, hi)
    torch.cuda.synchronize()
    wv, wr, wz = oracle.band_max(want_plane, lo, hi)
    assert np.array_equal(v.cpu().numpy().astype(np.float64), wv)
    assert np.array_equal(r.cpu().numpy(), wr)
    assert np.array_equal(zi.cpu().numpy(), wz)
    assert (int(r[1]), int(zi[1])) == (1000, 3)     # the tie: (3, 1000) precedes (3, 1100) and (7, 900)
    assert int(r[5]) == -1 and int(zi[5]) == -1     # a band beyond the plane is empty


@pytest.fixture(scope="module")
def noise_planes():
    n, zmax, m = 1 << 20, 84, 256
    x = synth.noise(n, synth.rng_for(91, 0)).astype(np.float32)
    out = {}
    for prec in ("fp32", "bf16", "bf16_split", "fp16_scaled"):
        s = fd.Search(fd.make_config(n, zmax, m, 8192, precision=prec))
        s.search(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        out[prec] = s.plane.float().cpu().numpy()
    return out


def test_noise_planes_follow_chi2_two_dof(noise_planes):
    """Every precision's noise-only plane: mean 2 and the chi^2_2 law (Kolmogorov-Smirnov on a
    random subsample, which thins the correlation between neighbouring cells)."""
    rng = np.random.default_rng(5)
    for prec, pl in noise_planes.items():
        assert abs(float(pl.mean()) - 2.0) < 0.02, prec
        sample = pl[rng.integers(0, pl.size, 200_000)]
        d = scipy.stats.kstest(sample, scipy.stats.chi2(df=2).cdf).statistic
        print(f"{prec}: mean {pl.mean():.4f}, KS D {d:.5f}")
        assert d < 0.01, (prec, d)


def test_noise_histograms_agree_between_precisions(noise_planes):
    """The reduced-precision noise against FP32's (the paper's Fig. noise_hist bottom panel): the
    two-sample Kolmogorov-Smirnov distance is small, and bin-by-bin count differences stay within
    a few percent wherever a bin holds many cells.  BF16 plane values lie on a grid 2^-8 of their
    size apart (1/16 .. 1/8 at powers 16-30), so rounding moves counts across 0.5-wide bin edges;
    that quantisation, not a change of the law, sets the bin-level bound."""
    rng = np.random.default_rng(6)
    idx = rng.integers(0, noise_planes["fp32"].size, 200_000)
    edges = np.linspace(0.0, 30.0, 61)
    ref, _ = np.histogram(noise_planes["fp32"], bins=edges)
    for prec in ("bf16", "bf16_split", "fp16_scaled"):
        if prec not in noise_planes:
            continue
        d = scipy.stats.ks_2samp(noise_planes[prec].ravel()[idx], noise_planes["fp32"].ravel()[idx]).statistic
        cnt, _ = np.histogram(noise_planes[prec], bins=edges)
        big = ref > 10_000
        rel = np.abs(cnt[big] - ref[big]) / ref[big]
        print(f"{prec}: two-sample KS D {d:.5f}, max relative bin-count difference {rel.max():.4f} over {big.sum()} bins")
        assert d < 0.005
        assert rel.max() < (0.05 if prec == "bf16" else 0.01)


def test_sweep_small_series_against_fp64_oracle():
    """The sweep on small sensitivity series (N = 2^16, one binary pulsar each, SNR 3-40): band
    peaks (Table harm_bounds) of the FP32 plane against those of the oracle's FP64 plane computed
    from the same series (the paper finds no drift and <= 0.0098 % power differences between
    single and double precision), and of the BF16 / split / FP16 planes against FP32 (the
    paper's criterion: same bin or adjacent z bin, powers within 3 %) above the noise canopy."""
    from paper_2206_12205_gb300 import sensitivity as se
    n, zmax, m = 1 << 16, 16, 64
    forms = ("fp32", "bf16", "bf16_split", "fp16_scaled")
    rows = {f: [] for f in forms[1:]}
    fp64_rows = []
    for sidx in range(6):
        w = synth.sensitivity_workload(config_index=92, series_index=sidx, n=n, zmax=zmax, taps=m, seg_len=1024)
        f_bins = w.trains[0].r0
        lo, hi = se.harmonic_bands(f_bins, 6, n // 2)
        x = torch.from_numpy(w.series).cuda()
        peaks = {}
        for form in forms:
            s = fd.Search(fd.make_config(n, zmax, m, 1024, precision=form))
            s.search(x)
            torch.cuda.synchronize()
            peaks[form] = se.band_peaks(s.plan, s.plane_2d(), lo, hi)
        for form in forms[1:]:
            rows[form].append(se.compare(peaks["fp32"], peaks[form]))
        ref = oracle.search(w.series, zmax, m, 1, (1e9,))["plane"]
        v, r, zi = oracle.band_max(ref, lo, hi)
        fp64 = {"power": v, "r": r, "zi": zi, "std": float(ref.std())}
        fp64_rows.append(se.compare(fp64, peaks["fp32"]))
    s64 = se.summarise(fp64_rows)
    print("fp32 vs fp64:", s64)
    assert s64["no_drift_fraction"] >= 0.95 and s64["perc_diff_max_abs"] <= 0.01
    for form, rr in rows.items():
        sm = se.summarise(rr, canopy_hi_snr=8.0)
        print(form, "vs fp32:", sm)
        if "above_canopy_bands" in sm:
            assert sm["above_canopy_recovered_fraction"] >= 0.9
            assert sm["above_canopy_perc_diff_max_abs"] <= 3.0
