"""GPU parity: libfdas (through its C-ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (FP32 path):
  - plane:     max_cells |P - P_ref| / max(P_ref, 2) <= 1e-5 (2 = mean noise power; a purely
               relative error is unbounded where P_ref ~ 0);
  - spectrum:  max |Xhat - Xhat_ref| <= 2e-6 * max|Xhat_ref| + 2e-5 (FP32 long FFT, log2 N levels);
  - templates: max |G - G_ref| <= 1e-6 * max|G_ref| (one FP32 rounding of an FP64 value);
  - peaks:     bit-exact (r, zi, H, power) against the oracle's float given-plane mode.
"""
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


def _floor_err(p, ref):
    return float(np.max(np.abs(p - ref) / np.maximum(ref, 2.0)))


def _search(n, zmax, m, S, **kw):
    return fd.Search(fd.make_config(n, zmax, m, S, **kw), device="cuda")


def _to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _xhat_f32(xhat_c128):
    return np.ascontiguousarray(xhat_c128.astype(np.complex64)).view(np.float32)


# ------------------------------------------------------------------ templates (K0)
@pytest.mark.parametrize("zmax,m,S", [(16, 64, 1024), (84, 256, 8192), (0, 2, 1024), (6, 512, 1024)])
def test_templates_match_oracle(zmax, m, S):
    s = _search(1 << 12, zmax, m, S)
    K = zmax + 1
    out = torch.empty(2 * K * S, dtype=torch.float32, device="cuda")
    fd.fdas_get_templates(s.plan, out)
    G = out.cpu().numpy().view(np.complex64).reshape(K, S).astype(np.complex128)
    T, _ = oracle.templates(zmax, m)
    c = np.zeros((K, S), dtype=np.complex128)
    c[:, :m] = T
    ref = np.fft.fft(c, axis=1) / S
    assert np.abs(G - ref).max() <= 1e-6 * np.abs(ref).max()


# ------------------------------------------------------------------ spectrum (K1)
@pytest.mark.parametrize("n", [1 << 11, 1 << 12, 1 << 13, 1 << 16, 1 << 20, 1 << 21, 1 << 24])
def test_spectrum_matches_oracle(n):
    x = (synth.noise(n, synth.rng_for(50, n.bit_length())) + synth.chirp(n, 0.3, n / 7.3, 3.0)).astype(np.float32)
    x[: n // 3] += 5.0                                 # a DC offset and a step: DC must still vanish
    s = _search(n, 8, 32, 1024)
    xh = s.spectrum(_to_dev(x))
    torch.cuda.synchronize()
    got = xh.cpu().numpy().view(np.complex64).astype(np.complex128)
    ref, s2 = oracle.spectrum(x)
    assert got[0] == 0
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max() + 2e-5
    assert abs(s.sigma2.item() - s2) <= 1e-5 * s2


@pytest.mark.parametrize("n", [1 << 26, 1 << 27])
def test_spectrum_long_transform_lengths(n):
    """The four-step passes at transform lengths 8192 x 4096 (N = 2^26) and 8192 x 8192 (N = 2^27),
    where the FP64 oracle takes a minute or more: every bin against an FP64 FFT with the spectrum's
    definition applied (DC zeroed, scale sqrt(2 / sigma2)), and sigma2 against Parseval's identity,
    sum_{k=1}^{N/2-1} |X_k|^2 = (N sum x^2 - X_0^2 - X_{N/2}^2) / 2, which needs no transform."""
    x = (synth.noise(n, synth.rng_for(51, n.bit_length())) + synth.chirp(n, 0.3, n / 7.3, 3.0)).astype(np.float32)
    s = _search(n, 8, 32, 1024)
    xh = s.spectrum(_to_dev(x))
    torch.cuda.synchronize()
    got = xh.cpu().numpy().view(np.complex64).astype(np.complex128)
    xd = x.astype(np.float64)
    nb = n // 2
    x0, xnyq = xd.sum(), xd[0::2].sum() - xd[1::2].sum()
    s2 = (n * np.dot(xd, xd) - x0 * x0 - xnyq * xnyq) / 2.0 / (nb - 1)
    assert abs(s.sigma2.item() - s2) <= 1e-5 * s2
    ref = np.fft.rfft(xd)[:nb]
    ref[0] = 0.0
    ref *= np.sqrt(2.0 / s2)
    assert got[0] == 0
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max() + 2e-5


def test_spectrum_fixed_sigma2():
    n = 1 << 14
    x = synth.chirp(n, 0.1, 2000.0, 0.0).astype(np.float32)
    s = _search(n, 4, 16, 1024, sigma2=float(n))
    got = s.spectrum(_to_dev(x)).cpu().numpy().view(np.complex64)
    ref, _ = oracle.spectrum(x, sigma2=float(n))
    assert s.sigma2.item() == float(n)
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()


@pytest.mark.parametrize("precision", ["fp32", "bf16", "bf16_split", "fp16_scaled", "bf16_direct", "fp8_direct"])
def test_zero_series_gives_zero_plane(precision):
    """A series with no power outside DC: sigma2 = 0, and, as in the oracle, the normalised
    spectrum, the plane and the candidate list are empty (no 0 * inf) on every path."""
    n = 1 << 16
    s = _search(n, 16, 64, 8192, precision=precision, max_harm=16, thr=(0.0,) * 5, max_peaks=64)
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    xh = s.spectrum(x)
    torch.cuda.synchronize()
    assert s.sigma2.item() == 0.0 and not bool(xh.any())
    s.plane.fill_(1.0)
    s.search(x)
    torch.cuda.synchronize()
    assert fd.fdas_device_status(s.plan) == 0
    assert not bool(s.plane.float().any())
    assert int(s.npeaks.item()) == 0


# ------------------------------------------------------------------ plane (K2 + K3)
@pytest.mark.parametrize("n,zmax,m,S", [
    (1 << 16, 16, 64, 1024),      # the plain FP32 workload's shape
    (1 << 12, 0, 2, 1024),        # one template, minimal taps
    (1 << 12, 4, 512, 1024),      # maximal taps: L = S/2 + 1
    (1 << 13, 10, 100, 2048),     # m not a power of two, ragged last segment
    (1 << 14, 20, 128, 4096),
    (1 << 15, 6, 64, 8192),       # several segments of the largest size
    (1 << 11, 2, 8, 8192),        # Nb < S: one zero-padded segment
])
def test_plane_shared_spectrum(n, zmax, m, S):
    """fdas_plane on the oracle's spectrum (rounded to FP32) vs the oracle's FP64 plane of
    that same rounded spectrum."""
    x = (synth.noise(n, synth.rng_for(51, S)) + synth.chirp(n, 0.2, n / 9.1, zmax / 2.0)).astype(np.float32)
    xr, _ = oracle.spectrum(x)
    xr32 = _xhat_f32(xr)
    xin = xr32.view(np.complex64).astype(np.complex128)
    s = _search(n, zmax, m, S)
    s.plane_from_spectrum(_to_dev(xr32))
    torch.cuda.synchronize()
    got = s.plane_2d().cpu().numpy().astype(np.float64)
    ref = oracle.plane(xin, zmax, m)
    assert _floor_err(got, ref) <= 1e-5


def test_single_chirp_end_to_end():
    """The plain FP32 workload end to end (long FFT included): plane within 1e-5 of the FP64
    oracle, the injected signal at (8000, z = +6), peak list above 30."""
    w = synth.single_chirp_workload()
    s = _search(w.n, w.zmax, w.taps, w.seg_len, max_harm=1, thr=(30.0,), max_peaks=1024)
    s.search(_to_dev(w.series))
    torch.cuda.synchronize()
    got = s.plane_2d().cpu().numpy().astype(np.float64)
    ref = oracle.search(w.series, w.zmax, w.taps, 1, (30.0,))
    assert _floor_err(got, ref["plane"]) <= 1e-5
    i, r = np.unravel_index(np.argmax(got), got.shape)
    assert (int(r), -w.zmax + 2 * int(i)) == (8000, 6)
    pk = s.peak_list()
    assert any(p["r"] == 8000 and p["zi"] == 11 for p in pk)
    want = ref["peaks"]
    # the FP64 oracle's peak set equals ours up to cells within 1e-5 of the threshold
    close = lambda v: abs(v - 30.0) <= 1e-4 * 30.0
    a = {(p["zi"], p["r"]) for p in pk if not close(p["power"])}
    b = {(p["zi"], p["r"]) for p in want if not close(p["power"])}
    assert a == b


# ------------------------------------------------------------------ peaks (K4)
def _peaks_equal(got, want):
    assert len(got) == len(want)
    for g, w in zip(got, want):
        assert (int(g["harm"]), int(g["zi"]), int(g["r"])) == (int(w["h"]), int(w["zi"]), int(w["r"]))
        assert np.float32(g["power"]).tobytes() == np.float32(w["power"]).tobytes()


@pytest.mark.parametrize("max_harm", [1, 2, 4, 8, 16])
def test_peaks_bit_exact_given_plane(max_harm):
    """The oracle's FP64 plane of a harmonic-rich accelerated signal, rounded once to float,
    searched by both sides: bit-exact peak lists."""
    n, zmax, m, S = 1 << 16, 32, 64, 1024
    x = synth.noise(n, synth.rng_for(52, max_harm))
    for h in range(1, 6):                             # a harmonic-rich accelerated signal
        x += synth.chirp(n, 0.08 / h, 1234.0 * h, 6.0 * h)
    x = x.astype(np.float32)
    xr, _ = oracle.spectrum(x)
    pl = oracle.plane(xr, zmax, m).astype(np.float32)
    thr = (12.0, 18.0, 28.0, 45.0, 70.0)
    s = _search(n, zmax, m, S, max_harm=max_harm, thr=thr, max_peaks=1 << 16)
    s.plane.copy_(torch.from_numpy(pl.ravel()))
    s.find_peaks()
    torch.cuda.synchronize()
    got = s.peak_list()
    want, cnt = oracle.peaks_f32(pl, zmax, max_harm, thr)
    assert int(s.npeaks.item()) == cnt > 0
    _peaks_equal(got, want)
    assert fd.fdas_device_status(s.plan) == 0


def test_peaks_ties_plateaus_and_overflow():
    n, zmax, m, S = 1 << 14, 4, 16, 1024
    s = _search(n, zmax, m, S, max_harm=2, thr=(1.0, 1.0), max_peaks=5)
    K, nb = zmax + 1, n // 2
    pl = np.zeros((K, nb), dtype=np.float32)
    pl[2, 100] = pl[2, 101] = 9.0                     # plateau in a row
    pl[1, 300] = pl[2, 300] = 7.0                     # plateau in a column
    pl[0, 0] = 5.0                                    # corner cell
    pl[4, nb - 1] = 5.0                               # last cell
    pl[2, 4000:4010] = 3.0                            # a flat run
    pl[3, 1500] = 6.0; pl[4, 3000] = 6.0              # a harmonic pair (z = 2 -> 4, r -> 2r)
    s.plane.copy_(torch.from_numpy(pl.ravel()))
    s.find_peaks()
    torch.cuda.synchronize()
    want, cnt = oracle.peaks_f32(pl, zmax, 2, (1.0, 1.0), max_out=5)
    assert int(s.npeaks.item()) == cnt and cnt > 5
    _peaks_equal(s.peak_list(), want)
    assert fd.fdas_device_status(s.plan) & fd.fdas.FDAS_DEV_PEAK_OVERFLOW
    assert fd.fdas_device_status(s.plan) == 0         # cleared by the previous read


@pytest.mark.parametrize("thr1", [20.0, 14.0, 13.0, 8.0])
def test_peaks_listed_and_full_scan_paths(thr1):
    """The peak list's two output paths: when at most 1024 units (level, row, 512-bin chunk)
    hold peaks, one block orders the listed units and writes the records; beyond that the full
    offset scan does.  Exponential noise planes (mean 2, the normalised plane's noise law) at
    thresholds that put the non-empty unit count on both sides of 1024: bit-exact against the
    oracle either way, with the true count."""
    n, zmax, m, S = 1 << 16, 32, 64, 1024
    K, nb = zmax + 1, n // 2
    rng = np.random.default_rng(9000 + int(thr1))
    pl = rng.exponential(2.0, size=(K, nb)).astype(np.float32)
    thr = (thr1, thr1 * 1.6)
    s = _search(n, zmax, m, S, max_harm=2, thr=thr, max_peaks=1 << 17)
    s.plane.copy_(torch.from_numpy(pl.ravel()))
    s.find_peaks()
    torch.cuda.synchronize()
    want, cnt = oracle.peaks_f32(pl, zmax, 2, thr, max_out=1 << 17)
    units = {(int(w["h"]), int(w["zi"]), int(w["r"]) // 512) for w in want}
    if thr1 >= 14.0:                                   # 51 and 799 non-empty units: the listed path
        assert 0 < len(units) <= 1024
    else:                                              # 1177 and 2654: the full scan
        assert len(units) > 1024
    assert int(s.npeaks.item()) == cnt
    _peaks_equal(s.peak_list(), want)
    assert fd.fdas_device_status(s.plan) == 0


def test_bf16_plane_peaks_quick_cast():
    """The peak kernel widens BF16 planes by bit placement (Sec. 3.1 quick cast): given the
    same values, BF16 and FP32 planes give the same peaks."""
    n, zmax = 1 << 13, 8
    rng = np.random.default_rng(3)
    pl = rng.exponential(2.0, size=(zmax + 1, n // 2)).astype(np.float32)
    bits = pl.view(np.uint32) & np.uint32(0xFFFF0000)
    pl_bf = bits.view(np.float32)                     # values exactly representable in BF16
    s = _search(n, zmax, 16, 1024, max_harm=4, thr=(9.0, 14.0, 22.0), max_peaks=1 << 14)
    s.plane.copy_(torch.from_numpy(pl_bf.ravel()))
    s.find_peaks()
    torch.cuda.synchronize()
    want, _ = oracle.peaks_f32(pl_bf, zmax, 4, (9.0, 14.0, 22.0))
    _peaks_equal(s.peak_list(), want)


# ------------------------------------------------------------------ full size, sampled
FULL_THR = (40.0, 44.0, 51.0, 64.0, 88.0)   # about one noise peak per harmonic level


@pytest.fixture(scope="module")
def pulse_train_case():
    """The benchmark series: the oracle's spectrum (FP64, and rounded once to complex64 for the
    shared-spectrum plane) and a search plan in the benchmark's configuration."""
    w = synth.pulse_train_workload()
    s = _search(w.n, w.zmax, w.taps, w.seg_len, max_harm=16, thr=FULL_THR, max_peaks=1 << 16)
    xr, s2 = oracle.spectrum(w.series)
    xr32 = _xhat_f32(xr)
    return w, s, xr, s2, xr32


def test_full_size_spectrum(pulse_train_case):
    w, s, xr, s2, _ = pulse_train_case
    xh = s.spectrum(_to_dev(w.series))
    torch.cuda.synchronize()
    got = xh.cpu().numpy().view(np.complex64).astype(np.complex128)
    assert np.abs(got - xr).max() <= 2e-6 * np.abs(xr).max() + 2e-5
    assert abs(s.sigma2.item() - s2) <= 1e-5 * s2


@pytest.mark.parametrize("seg_len", [8192, 2048])
def test_full_size_plane_sampled(pulse_train_case, seg_len):
    """N = 2^23, 85 templates, 256 taps, with the workload's 8192-bin segments and with the
    2048-bin segments the benchmark's FP32 path runs (its launch configuration): sampled cells
    (random, segment edges, the ragged tail, each train's fundamental) against the oracle
    evaluated cell by cell on the same spectrum."""
    w, s, xr, _, xr32 = pulse_train_case
    if seg_len != w.seg_len:
        s = _search(w.n, w.zmax, w.taps, seg_len, max_harm=16, thr=FULL_THR, max_peaks=1 << 16)
    xh = xr32.view(np.complex64).astype(np.complex128)
    s.plane_from_spectrum(_to_dev(xr32))
    torch.cuda.synchronize()
    K, nb, L = w.K, w.nb, s.plan.info.seg_valid
    rng = np.random.default_rng(7)
    zi = list(rng.integers(0, K, 3000))
    r = list(rng.integers(0, nb, 3000))
    for j in (0, 1, 2, 100, nb // L - 1, nb // L):    # segment starts and ends
        for t in (0, 1, L - 2, L - 1):
            rr = j * L + t
            if 0 <= rr < nb:
                zi += [0, K // 2, K - 1]
                r += [rr] * 3
    for rr in range(nb - 5, nb):                      # the ragged tail
        zi += [0, K - 1]
        r += [rr] * 2
    for tr in w.trains:
        i0 = int(np.clip(round((tr.z0 + w.zmax) / 2), 0, K - 1))
        for dr in range(-2, 3):
            zi.append(i0)
            r.append(int(np.clip(round(tr.r0) + dr, 0, nb - 1)))
    zi = np.array(zi)
    r = np.array(r)
    T, _ = oracle.templates(w.zmax, w.taps)
    ref = oracle.plane_cells(xh, w.zmax, w.taps, T, zi, r)
    plane = s.plane_2d()
    idx = torch.from_numpy(zi * nb + r).cuda()
    got = plane.reshape(-1)[idx].cpu().numpy().astype(np.float64)
    assert _floor_err(got, ref) <= 1e-5
    # the whole-plane noise law: mean power 2 (chi^2, 2 dof) away from injected signals
    assert abs(float(plane.double().mean().item()) - 2.0) < 0.1
    # end to end from the series (the FP32 long FFT included) against the oracle's FP64 spectrum
    s.search(_to_dev(w.series))
    torch.cuda.synchronize()
    got_e2e = plane.reshape(-1)[idx].cpu().numpy().astype(np.float64)
    ref_e2e = oracle.plane_cells(xr, w.zmax, w.taps, T, zi, r)
    e2e = _floor_err(got_e2e, ref_e2e)
    print(f"full size end to end: floor-relative plane error {e2e:.2e}")
    assert e2e <= 1e-5


def _planted_plane(K, nb, zmax, rng, families):
    """Exponential noise cells plus `families` harmonic families: fundamental power A at a random
    (i, r) and A/h at (h r, i_h) (z_{i_h} = h z_i) wherever that cell is on the plane."""
    pl = synth.noise_plane(K, nb, rng)
    for f in range(families):
        # every other family drifts slowly enough (|z| <= 4) and sits low enough in frequency
        # (r < nb/16) to reach the 16-harmonic level
        i = int(rng.integers(0, K)) if f % 2 else zmax // 2 + int(rng.integers(-2, 3))
        r = int(rng.integers(1, nb // 2 if f % 2 else nb // 16))
        A = float(rng.uniform(25.0, 90.0))
        z = -zmax + 2 * i
        for h in range(1, 17):
            ih = (h * z + zmax) // 2
            if abs(h * z) > zmax or h * r >= nb:
                break
            pl[ih, h * r] += np.float32(A / h)
    return pl


def test_full_size_peaks_bit_exact(pulse_train_case):
    """16-harmonic peak search over a full-size plane (85 x 2^22 cells) of exponential noise with
    planted harmonic families, given to both sides: bit-exact peak lists at every level."""
    w, s, _, _, _ = pulse_train_case
    pl = _planted_plane(w.K, w.nb, w.zmax, synth.rng_for(53, 0), 400)
    s.plane.copy_(torch.from_numpy(pl.ravel()))
    s.find_peaks()
    torch.cuda.synchronize()
    got = s.peak_list()
    want, cnt = oracle.peaks_f32(pl, w.zmax, 16, FULL_THR)
    assert int(s.npeaks.item()) == cnt
    assert len({int(p["h"]) for p in want}) == 5          # every harmonic level has peaks
    _peaks_equal(got, want)
