"""GPU parity of the BF16 tensor-core path against the FP64 oracle.

The paper's acceptance criterion for reduced precision (abstract; Sec. 5.2-5.3): every peak's
power within 3 % of the reference under Eq. perc_diff, at the same frequency bin and the same
or an adjacent acceleration (z) bin.  Given the same (BF16) plane, the peak list is bit-exact
against the oracle's float mode.

Plane-level bounds follow from the arithmetic: a cell passes through seven BF16 roundings
(spectrum, template, their product, the DFT matrix twice, the inter-stage values, the stored
power), each with relative error at most u = 2^-9 (RMS u/sqrt(3)); amplitude errors add in
quadrature, so the power's relative RMS error is about 2 sqrt(6) u / sqrt(3) + u / sqrt(3)
= 0.57 % (the paper reports sd = 0.6 % for BF16 peak powers).  Tests use: RMS of
|P - P_ref| / max(P_ref, 2) <= 1 %, its 99.9th percentile <= 2.5 % (3.3 sigma ~ 1.9 %), strong
cells (P_ref > 20) within 3 %, and every cell within 3 % of max(P_ref, 2) plus 2 % of the
geometric mean of the cell's and its neighbourhood's peak power (rounding errors of a strong
component spread over the whole transform).
"""
import json
import os

import numpy as np
import pytest
import torch

import fdas_synth as synth
import oracle
import paper_2206_12205_gb300 as fd

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fd.build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _criteria():
    with open(os.path.join(GOLDEN, "paper_criteria.json")) as f:
        return json.load(f)


def perc_diff(b, s):
    """Eq. perc_diff: (b - s) / ((b + s) / 2) x 100."""
    return (b - s) / ((b + s) / 2.0) * 100.0


def _bf16_search(n, zmax, m, **kw):
    return fd.Search(fd.make_config(n, zmax, m, 8192, precision="bf16", **kw), device="cuda")


def _shared_spectrum(x):
    """The oracle's spectrum rounded once to complex64: (device float32 view, same values as complex128)."""
    xr, _ = oracle.spectrum(x)
    c64 = np.ascontiguousarray(xr.astype(np.complex64))
    return torch.from_numpy(c64.view(np.float32)).cuda(), c64.astype(np.complex128)


def _plane_f64(s):
    return s.plane_2d().float().cpu().numpy().astype(np.float64)


def match_peaks(ref, got, thr_by_h, tol_pct, margin=1.03):
    """Paper criterion: each reference peak at least `margin` x its threshold has a peak in
    `got` at the same r and harmonic level, |dzi| <= 1, |perc_diff| <= tol_pct."""
    idx = {}
    for g in got:
        idx.setdefault((int(g["harm"]), int(g["r"])), []).append(g)
    worst = 0.0
    for p in ref:
        h = int(p["h"]) if "h" in p.dtype.names else int(p["harm"])
        if p["power"] < margin * thr_by_h[h]:
            continue
        cands = [g for g in idx.get((h, int(p["r"])), []) if abs(int(g["zi"]) - int(p["zi"])) <= 1]
        assert cands, f"reference peak H={h} r={p['r']} zi={p['zi']} P={p['power']:.2f} not found"
        d = min(abs(perc_diff(float(g["power"]), float(p["power"]))) for g in cands)
        worst = max(worst, d)
        assert d <= tol_pct, f"peak H={h} r={p['r']} zi={p['zi']}: {d:.3f}% > {tol_pct}%"
    return worst


@pytest.mark.parametrize("n,zmax,m", [(1 << 16, 16, 64), (1 << 14, 0, 8), (1 << 18, 84, 256),
                                       (1 << 13, 6, 2048), (1 << 12, 2, 32)])
def test_bf16_plane_matches_oracle(n, zmax, m):
    x = (synth.noise(n, synth.rng_for(60, n.bit_length())) + synth.chirp(n, 0.25, n / 13.3, zmax * 0.6)).astype(np.float32)
    s = _bf16_search(n, zmax, m)
    xdev, xin = _shared_spectrum(x)
    s.plane_from_spectrum(xdev)
    torch.cuda.synchronize()
    got = _plane_f64(s)
    ref = oracle.plane(xin, zmax, m)
    # BF16 operands carry 8 significant bits: a transform's rounding error in amplitude is a
    # few 2^-9 of the largest amplitude in its segment, so a cell's power error is bounded by
    # the local peak power, not by the cell's own power (the paper's 3 % applies to peaks).
    err = np.abs(got - ref)
    seg = 4096 - m + 1
    local = np.maximum.reduceat(np.maximum(ref, 2.0), np.arange(0, ref.shape[1], 64), axis=1)
    local = np.maximum(local, np.roll(local, 1, axis=1))
    local = np.maximum(local, np.roll(local, -1, axis=1))
    bound = 0.03 * np.maximum(ref, 2.0) + 0.02 * np.sqrt(np.maximum(ref, 2.0) * np.repeat(local, 64, axis=1)[:, :ref.shape[1]])
    i, r = np.unravel_index(np.argmax(err / bound), err.shape)
    assert np.all(err <= bound), (f"cell ({i},{r}) P_ref={ref[i, r]:.3f} got={got[i, r]:.3f} local={local[i, r // 64]:.1f}"
                                  f" floor-rel={err[i, r] / max(ref[i, r], 2.0):.4f} seg={seg}")
    fr = err / np.maximum(ref, 2.0)
    assert np.sqrt(np.mean(fr ** 2)) <= 0.01
    assert np.percentile(fr, 99.9) <= 0.025
    strong = ref > 20.0
    if strong.any():
        assert np.abs(perc_diff(got[strong], ref[strong])).max() <= 3.0
    assert np.all(np.isfinite(got))


def test_bf16_single_chirp_peaks_paper_criterion():
    crit = _criteria()
    w = synth.single_chirp_workload()
    thr = (30.0,)
    s = _bf16_search(w.n, w.zmax, w.taps, max_harm=1, thr=thr, max_peaks=4096)
    s.search(torch.from_numpy(w.series).cuda())
    torch.cuda.synchronize()
    ref = oracle.search(w.series, w.zmax, w.taps, 1, thr)
    worst = match_peaks(ref["peaks"], s.peak_list(), {1: 30.0}, crit["bf16_vs_fp32_peak_power_max_percent"])
    got = _plane_f64(s)
    i, r = np.unravel_index(np.argmax(got), got.shape)
    assert (int(r), -w.zmax + 2 * int(i)) == (8000, 6)
    assert worst <= 3.0


def test_bf16_peaks_bit_exact_given_plane():
    """The oracle's FP64 plane rounded once to BF16 (round to nearest even), searched by the BF16
    peak kernel (quick cast on read) and by the oracle's float mode on the widened values."""
    n, zmax, m = 1 << 16, 32, 64
    x = synth.noise(n, synth.rng_for(61, 0))
    for h in range(1, 6):
        x += synth.chirp(n, 0.08 / h, 1234.0 * h, 6.0 * h)
    x = x.astype(np.float32)
    xr, _ = oracle.spectrum(x)
    pl_bf = torch.from_numpy(oracle.plane(xr, zmax, m).astype(np.float32)).to(torch.bfloat16)
    widened = pl_bf.float().numpy()
    thr = (12.0, 18.0, 28.0, 45.0, 70.0)
    s = _bf16_search(n, zmax, m, max_harm=16, thr=thr, max_peaks=1 << 16)
    s.plane.copy_(pl_bf.reshape(-1).cuda())
    s.find_peaks()
    torch.cuda.synchronize()
    want, cnt = oracle.peaks_f32(widened, zmax, 16, thr)
    got = s.peak_list()
    assert int(s.npeaks.item()) == cnt > 0
    assert len(got) == len(want)
    for g, w_ in zip(got, want):
        assert (int(g["harm"]), int(g["zi"]), int(g["r"])) == (int(w_["h"]), int(w_["zi"]), int(w_["r"]))
        assert np.float32(g["power"]).tobytes() == np.float32(w_["power"]).tobytes()
    assert fd.fdas_device_status(s.plan) == 0


@pytest.fixture(scope="module")
def bf16_full():
    w = synth.pulse_train_workload()
    thr = (40.0, 44.0, 51.0, 64.0, 88.0)
    s = _bf16_search(w.n, w.zmax, w.taps, max_harm=16, thr=thr, max_peaks=1 << 16)
    s.search(torch.from_numpy(w.series).cuda())           # end to end: the peak list
    xdev, xh = _shared_spectrum(w.series)
    s.plane_from_spectrum(xdev)                            # shared spectrum: the sampled cells
    torch.cuda.synchronize()
    return w, s, xh, thr


def test_bf16_full_size_sampled_cells(bf16_full):
    w, s, xh, _ = bf16_full
    K, nb = w.K, w.nb
    rng = np.random.default_rng(8)
    zi = rng.integers(0, K, 4000)
    r = rng.integers(0, nb, 4000)
    L = (4096 - w.taps + 1) // 64 * 64
    extra_r = [j * L + t for j in (0, 1, 500, nb // L) for t in (0, 1, L - 1) if j * L + t < nb] + list(range(nb - 4, nb))
    zi = np.concatenate([zi, np.repeat([0, K // 2, K - 1], len(extra_r))])
    r = np.concatenate([r, np.tile(extra_r, 3)])
    for tr in w.trains:
        i0 = int(np.clip(round((tr.z0 + w.zmax) / 2), 0, K - 1))
        zi = np.concatenate([zi, [i0] * 3])
        r = np.concatenate([r, np.clip(np.round(tr.r0) + np.arange(-1, 2), 0, nb - 1).astype(np.int64)])
    T, _ = oracle.templates(w.zmax, w.taps)
    ref = oracle.plane_cells(xh, w.zmax, w.taps, T, zi.astype(np.int32), r.astype(np.int64))
    got = s.plane_2d().reshape(-1)[torch.from_numpy(zi * nb + r).cuda()].float().cpu().numpy().astype(np.float64)
    floor_rel = np.abs(got - ref) / np.maximum(ref, 2.0)
    assert np.sqrt(np.mean(floor_rel ** 2)) <= 0.01
    assert np.percentile(floor_rel, 99.9) <= 0.025 and floor_rel.max() <= 0.05
    strong = ref > 20.0
    assert np.abs(perc_diff(got[strong], ref[strong])).max() <= 3.0
    mean = float(s.plane_2d().float().mean().item())
    assert abs(mean - 2.0) < 0.1


def test_bf16_full_size_peaks_vs_fp32(bf16_full):
    """The paper's comparison at full size: the FP32 path's peaks (themselves within 1e-5 of
    the FP64 oracle) recovered by the BF16 path within 3 % power and +-1 z bin."""
    w, s, _, thr = bf16_full
    s32 = fd.Search(fd.make_config(w.n, w.zmax, w.taps, w.seg_len, precision="fp32", max_harm=16, thr=thr,
                                   max_peaks=1 << 16), device="cuda")
    s32.search(torch.from_numpy(w.series).cuda())
    torch.cuda.synchronize()
    ref = s32.peak_list()
    thr_by_h = {1 << l: thr[l] for l in range(5)}
    worst = match_peaks(ref, s.peak_list(), thr_by_h, 3.0)
    assert worst <= 3.0


# ------------------------------------------------------------------ split-BF16 (accuracy recovery)
@pytest.mark.parametrize("n,zmax,m", [(1 << 16, 16, 64), (1 << 18, 84, 256), (1 << 12, 2, 32)])
def test_split_bf16_plane_matches_oracle(n, zmax, m):
    """Compensated hi+lo BF16 operands (~16 significant bits, three products per MMA step):
    floor-relative plane error ~2^-16 per operand rounding -> bound 5e-4 (FP32 path: 1e-5,
    plain BF16: a few 1e-3)."""
    x = (synth.noise(n, synth.rng_for(62, n.bit_length())) + synth.chirp(n, 0.25, n / 13.3, zmax * 0.6)).astype(np.float32)
    s = fd.Search(fd.make_config(n, zmax, m, 8192, precision="bf16_split"), device="cuda")
    assert s.plan.info.plane_elem_bytes == 4
    xdev, xin = _shared_spectrum(x)
    s.plane_from_spectrum(xdev)
    torch.cuda.synchronize()
    got = s.plane_2d().cpu().numpy().astype(np.float64)
    ref = oracle.plane(xin, zmax, m)
    err = np.abs(got - ref) / np.maximum(ref, 2.0)
    print(f"split-bf16 floor-relative error: max {err.max():.2e} rms {np.sqrt(np.mean(err ** 2)):.2e}")
    assert err.max() <= 5e-4
    assert fd.fdas_device_status(s.plan) == 0


def test_split_bf16_search_peaks():
    w = synth.single_chirp_workload()
    s = fd.Search(fd.make_config(w.n, w.zmax, w.taps, w.seg_len, precision="bf16_split", max_harm=1, thr=(30.0,),
                                 max_peaks=4096), device="cuda")
    s.search(torch.from_numpy(w.series).cuda())
    torch.cuda.synchronize()
    ref = oracle.search(w.series, w.zmax, w.taps, 1, (30.0,))
    worst = match_peaks(ref["peaks"], s.peak_list(), {1: 30.0}, 0.1)
    assert worst <= 0.1


# ------------------------------------------------------------------ FP16 with per-segment scaling (ablation)
@pytest.mark.parametrize("n,zmax,m", [(1 << 16, 16, 64), (1 << 18, 84, 256), (1 << 12, 2, 32)])
def test_fp16_scaled_plane_matches_oracle(n, zmax, m):
    """FP16 operands (10-bit mantissa, u = 2^-11) after a power-of-two scale per segment: the
    same error budget as BF16 (seven operand roundings) with u four times smaller."""
    x = (synth.noise(n, synth.rng_for(63, n.bit_length())) + synth.chirp(n, 0.25, n / 13.3, zmax * 0.6)).astype(np.float32)
    s = fd.Search(fd.make_config(n, zmax, m, 8192, precision="fp16_scaled"), device="cuda")
    assert s.plan.info.plane_elem_bytes == 4
    xdev, xin = _shared_spectrum(x)
    s.plane_from_spectrum(xdev)
    torch.cuda.synchronize()
    got = s.plane_2d().cpu().numpy().astype(np.float64)
    ref = oracle.plane(xin, zmax, m)
    fr = np.abs(got - ref) / np.maximum(ref, 2.0)
    print(f"fp16-scaled floor-relative error: max {fr.max():.2e} rms {np.sqrt(np.mean(fr ** 2)):.2e} "
          f"p99.9 {np.percentile(fr, 99.9):.2e}")
    assert np.all(np.isfinite(got))
    # BF16's bounds scaled by (2^-11 / 2^-9) = 1/4: RMS 0.25 %, 99.9th percentile 0.6 %, any cell 1.5 %
    assert np.sqrt(np.mean(fr ** 2)) <= 0.0025
    assert np.percentile(fr, 99.9) <= 0.006
    assert fr.max() <= 0.015
    assert fd.fdas_device_status(s.plan) == 0
