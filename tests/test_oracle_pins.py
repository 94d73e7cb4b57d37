"""Pins of the FP64 oracle to things other than itself: brute force on tiny inputs,
closed forms, special cases that reduce to textbook or library routines, invariants and the
values the paper prints.  CPU only.

Each test names the part of the oracle it pins; the sensitivity tests at the end show that
plausible mistakes (a conjugated template, a flipped FFT sign, an index shifted by one)
break at least one pin.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.special
import scipy.stats

import fdas_synth as synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- FFT and spectrum
@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 64, 256, 1024])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_brute_force_dft(oracle_mod, n, sign):
    rng = np.random.default_rng(n)
    a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    j = np.arange(n)
    # explicit O(n^2) sum, phases reduced exactly with integer arithmetic
    ph = (np.outer(j, j) % n) / n
    ref = (np.exp(sign * 2j * np.pi * ph) * a[None, :]).sum(axis=1)
    got = oracle_mod.fft(a, sign)
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_fft_parseval_and_numpy(oracle_mod):
    n = 1 << 14
    rng = np.random.default_rng(7)
    a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    A = oracle_mod.fft(a, -1)
    assert abs(np.vdot(A, A).real / n - np.vdot(a, a).real) <= 1e-10 * np.vdot(a, a).real
    assert np.abs(A - np.fft.fft(a)).max() <= 1e-10


def test_spectrum_definition_small(oracle_mod):
    n = 256
    x = np.random.default_rng(3).standard_normal(n).astype(np.float32)
    xhat, s2 = oracle_mod.spectrum(x)
    j = np.arange(n)
    k = np.arange(n // 2)
    X = (x.astype(np.float64)[None, :] * np.exp(-2j * np.pi * ((np.outer(k, j) % n) / n))).sum(1)
    X[0] = 0.0
    sig2 = np.mean(np.abs(X[1:]) ** 2)
    assert abs(s2 - sig2) <= 1e-12 * sig2
    assert np.abs(xhat - X * math.sqrt(2.0 / sig2)).max() <= 1e-12 * np.abs(xhat).max()
    # by construction the normalised non-DC powers average exactly 2
    assert abs(np.mean(np.abs(xhat[1:]) ** 2) - 2.0) <= 1e-12
    # Parseval for a real series: sum x^2 = (|X0|^2 + 2 sum_{1..n/2-1} |Xk|^2 + |X_{n/2}|^2) / n
    Xf = np.fft.fft(x.astype(np.float64))
    lhs = float(np.dot(x.astype(np.float64), x.astype(np.float64)))
    rhs = (abs(Xf[0]) ** 2 + 2 * np.sum(np.abs(Xf[1:n // 2]) ** 2) + abs(Xf[n // 2]) ** 2) / n
    assert abs(lhs - rhs) <= 1e-9 * lhs


def test_spectrum_fixed_sigma2(oracle_mod):
    x = synth.chirp(1024, 1.0, 100.0, 0.0).astype(np.float32)
    xhat, s2 = oracle_mod.spectrum(x, sigma2=1024.0)
    assert s2 == 1024.0
    # a unit cosine at bin 100: X_100 = n/2
    assert abs(abs(xhat[100]) - 512.0 * math.sqrt(2.0 / 1024.0)) <= 1e-3


def test_spectrum_without_power_outside_dc(oracle_mod):
    """A zero or constant series has X_k = 0 for every k >= 1 (the DFT of a constant is a delta
    at DC), so sigma2 = 0; the normalisation then gives the zero spectrum, a zero plane and no
    candidates (no 0 * inf).  A constant's DFT is exactly zero off DC in FP64 butterflies."""
    n, zmax, m = 1024, 6, 32
    for c in (0.0, 3.25, -7.0):
        x = np.full(n, c, dtype=np.float32)
        xhat, s2 = oracle_mod.spectrum(x)
        assert s2 == 0.0 and not np.any(xhat)
        pl = oracle_mod.plane(xhat, zmax, m)
        assert pl.shape == (zmax + 1, n // 2) and not np.any(pl)
        rec, cnt = oracle_mod.peaks_f64(pl, zmax, 16, (0.0,) * 5)
        assert cnt == 0 and len(rec) == 0
    # a fixed sigma2 still applies; the local variant's zero-median blocks agree
    xhat, s2 = oracle_mod.spectrum(np.zeros(n, dtype=np.float32), sigma2=5.0)
    assert s2 == 5.0 and not np.any(xhat)
    assert not np.any(oracle_mod.spectrum_local(np.full(n, 2.0, dtype=np.float32), 64))
    # the smallest non-zero case is normalised as usual: one tone's bin carries all the power
    x = synth.chirp(n, 1.0, 37.0, 0.0).astype(np.float32)
    xhat, s2 = oracle_mod.spectrum(x)
    assert abs(np.sum(np.abs(xhat[1:]) ** 2) - 2.0 * (n // 2 - 1)) <= 1e-9 * n


# ---------------------------------------------------------------- Fresnel and response
def test_fresnel_matches_scipy(oracle_mod):
    x = np.concatenate([np.linspace(-12.0, 12.0, 4801), np.linspace(12.0, 600.0, 2001),
                        [1.6 - 1e-12, 1.6, 1.6 + 1e-12, 1e-9, -1e-9, 0.0]])
    c, s = oracle_mod.fresnel(x)
    S, C = scipy.special.fresnel(x)          # scipy returns (S, C)
    assert np.abs(c - C).max() <= 2e-15
    assert np.abs(s - S).max() <= 2e-15
    c_inf, s_inf = oracle_mod.fresnel([1e6])
    assert abs(c_inf[0] - 0.5) < 1e-6 and abs(s_inf[0] - 0.5) < 1e-6


def _numpy_quadrature(q, z, nodes=24):
    """Independent check of I(q, z) = int_0^1 exp(i pi (z u^2 - 2 q u)) du written in the
    test itself: composite Gauss-Legendre from numpy's nodes."""
    xs, ws = np.polynomial.legendre.leggauss(nodes)
    panels = int(math.ceil(abs(z) + abs(q))) + 8
    edges = np.arange(panels) / panels
    u = (edges[:, None] + (xs[None, :] + 1.0) * 0.5 / panels).ravel()
    w = np.tile(ws * 0.5 / panels, panels)
    return np.sum(w * np.exp(1j * np.pi * (z * u * u - 2.0 * q * u)))


@pytest.mark.parametrize("z", [2.0, 6.2, 16.0, 84.0, -84.0, -6.2, 0.5, 0.01, 0.0005, 190.0])
def test_response_matches_quadrature(oracle_mod, z):
    qs = np.concatenate([np.arange(-128, 129, 1.0), [0.3, -17.25, 100.5]])
    got = oracle_mod.response(qs, z)
    ref = np.array([_numpy_quadrature(q, z) for q in qs])
    tol = 1e-11 if abs(z) >= 1.0 else 1e-9
    assert np.abs(got - ref).max() <= tol
    # and the oracle's own quadrature route agrees with its Fresnel route
    assert np.abs(got - oracle_mod.response_quad(qs, z)).max() <= tol


def test_response_z0_is_delta_and_sinc(oracle_mod):
    q = np.arange(-40, 41, dtype=np.float64)
    v = oracle_mod.response(q, 0.0)
    expect = (q == 0).astype(np.complex128)
    assert np.abs(v - expect).max() == 0.0
    h = oracle_mod.response(np.array([0.5, -0.5, 1.5]), 0.0)
    # exp(-i pi q) sin(pi q)/(pi q)
    ref = np.exp(-1j * np.pi * np.array([0.5, -0.5, 1.5])) * np.sinc(np.array([0.5, -0.5, 1.5]))
    assert np.abs(h - ref).max() <= 1e-15


def test_response_symmetry_and_continuity(oracle_mod):
    q = np.linspace(-60.0, 60.0, 241)
    for z in (2.0, 7.3, 50.0):
        assert np.abs(oracle_mod.response(q, -z) - np.conj(oracle_mod.response(-q, z))).max() <= 1e-14
    # continuity across the z = 0 branch and the small-|z| quadrature branch
    for qq in (0.0, 3.0, 10.5):
        a = oracle_mod.response(np.array([qq]), 1e-7)[0]
        b = oracle_mod.response(np.array([qq]), 0.0)[0]
        assert abs(a - b) <= 1e-5
        c = oracle_mod.response(np.array([qq]), 0.999e-3)[0]
        d = oracle_mod.response(np.array([qq]), 1.001e-3)[0]
        assert abs(c - d) <= 1e-5


@pytest.mark.parametrize("z", [0.0, 2.0, 16.0, 84.0])
def test_response_unit_energy(oracle_mod, z):
    """Parseval of the continuous unit-amplitude chirp: sum over all integer q of |I|^2 = 1."""
    q = np.arange(-4096, 4097, dtype=np.float64)
    e = np.sum(np.abs(oracle_mod.response(q, z)) ** 2)
    assert abs(e - 1.0) <= 2e-4


def test_templates_unit_norm_and_delta(oracle_mod):
    T, eta = oracle_mod.templates(16, 64)
    assert T.shape == (17, 64)
    assert np.abs(np.sum(np.abs(T) ** 2, axis=1) - 1.0).max() <= 1e-13
    assert np.all(eta <= 1.0 + 1e-12) and np.all(eta > 0.999)
    row0 = T[8]                       # z = 0
    assert np.abs(row0 - (np.arange(64) == 32)).max() == 0.0
    # conjugate symmetry of the unnormalised bank: I(q, -z) = conj(I(-q, z)) where both
    # taps exist (the norms differ: the window q = -m/2 .. m/2-1 is not symmetric)
    for i in range(17):
        a = T[i, 1:] * math.sqrt(eta[i])                      # q = -31 .. 31
        b = np.conj(T[16 - i, 1:][::-1]) * math.sqrt(eta[16 - i])
        assert np.abs(a - b).max() <= 1e-14


def test_templates_reject_bad_args(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.templates(15, 64)
    with pytest.raises(ValueError):
        oracle_mod.templates(16, 63)


# ---------------------------------------------------------------- correlation / plane
def test_plane_matches_brute_force(oracle_mod):
    rng = np.random.default_rng(11)
    nb, zmax, m = 40, 4, 8
    xhat = rng.standard_normal(nb) + 1j * rng.standard_normal(nb)
    T = rng.standard_normal((zmax + 1, m)) + 1j * rng.standard_normal((zmax + 1, m))
    got = oracle_mod.plane(xhat, zmax, m, T)
    ref = np.zeros((zmax + 1, nb))
    for i in range(zmax + 1):
        for r in range(nb):
            acc = 0j
            for t in range(m):
                k = r + t - m // 2
                if 0 <= k < nb:
                    acc += xhat[k] * np.conj(T[i, t])
            ref[i, r] = abs(acc) ** 2
    assert np.abs(got - ref).max() <= 1e-12 * ref.max()
    cells = oracle_mod.plane_cells(xhat, zmax, m, T, [0, 2, 4, 4], [0, 17, 39, 5])
    assert np.abs(cells - ref[[0, 2, 4, 4], [0, 17, 39, 5]]).max() <= 1e-12 * ref.max()
    with pytest.raises(ValueError):
        oracle_mod.plane_cells(xhat, zmax, m, T, [5], [0])


def test_plane_z0_row_is_power_spectrum(oracle_mod):
    x = synth.noise(4096, np.random.default_rng(5)).astype(np.float32)
    xhat, _ = oracle_mod.spectrum(x)
    pl = oracle_mod.plane(xhat, 8, 32)
    assert np.abs(pl[4] - np.abs(xhat) ** 2).max() <= 1e-12 * pl[4].max()


@pytest.mark.parametrize("r0,z0", [(8000, 6), (3000, -10), (3000, 0), (12000, 16)])
def test_closed_form_peak_power(oracle_mod, r0, z0):
    """Noiseless on-grid constant-fdot sinusoid of amplitude a: with sigma^2 fixed to N (unit
    noise), P(r0, z0) = 2 (N a / 2)^2 eta / sigma^2 = N a^2 eta / 2, up to O(z/N) and the
    negative-frequency leakage; and the plane maximum sits on the injected cell."""
    n, a, zmax, m = 1 << 16, 0.05, 16, 64
    x = synth.chirp(n, a, r0, z0).astype(np.float32)
    xhat, _ = oracle_mod.spectrum(x, sigma2=float(n))
    T, eta = oracle_mod.templates(zmax, m)
    pl = oracle_mod.plane(xhat, zmax, m, T)
    i0 = (z0 + zmax) // 2
    expect = n * a * a * eta[i0] / 2.0
    assert abs(pl[i0, r0] - expect) <= 2e-5 * expect
    i, r = np.unravel_index(np.argmax(pl), pl.shape)
    assert (i, r) == (i0, r0)


def test_single_chirp_off_grid_peak(oracle_mod):
    """The plain FP32 workload's injected signal (r = 8000.3, z = 6.2), noiseless with
    sigma^2 = N: scalloping leaves 46.85 of the on-grid 81.92 at the nearest cell
    (8000, z = 6)."""
    w = synth.single_chirp_workload(with_noise=False)
    xhat, _ = oracle_mod.spectrum(w.series, sigma2=float(w.n))
    pl = oracle_mod.plane(xhat, w.zmax, w.taps)
    i, r = np.unravel_index(np.argmax(pl), pl.shape)
    assert (r, -w.zmax + 2 * i) == (8000, 6)
    assert abs(pl[i, r] - 46.8466) <= 1e-3


def test_noise_law_chi2_2dof(oracle_mod):
    """Noise-only planes follow chi^2 with 2 dof (paper Sec. 5.1): mean 2, exponential law.
    Cells 128 bins apart (more than the 64 taps) are independent."""
    x = synth.noise(1 << 16, synth.rng_for(9, 0)).astype(np.float32)
    xhat, _ = oracle_mod.spectrum(x)
    pl = oracle_mod.plane(xhat, 16, 64)
    assert abs(pl[:, 64:-64].mean() - 2.0) <= 0.03
    sample = pl[::4, 64:-64:128].ravel()
    p = scipy.stats.kstest(sample, "expon", args=(0.0, 2.0)).pvalue
    assert p > 1e-3


# ---------------------------------------------------------------- harmonic sum and peaks
def _brute_peaks(pl, zmax, max_harm, thr, dtype):
    K, nb = pl.shape
    pl = pl.astype(dtype)
    out = []
    lev = 0
    H = 1
    while H <= max_harm:
        def ok(i, r):
            return 0 <= i < K and abs(H * (-zmax + 2 * i)) <= zmax and 0 <= r and H * r < nb

        def S(i, r):
            z = -zmax + 2 * i
            s = dtype(0.0)
            for h in range(1, H + 1):
                s = dtype(s + pl[(h * z + zmax) // 2, h * r])
            return s
        for i in range(K):
            for r in range(nb):
                if not ok(i, r):
                    continue
                s = S(i, r)
                if not s > dtype(thr[lev]):
                    continue
                peak = True
                for di in (-1, 0, 1):
                    for dr in (-1, 0, 1):
                        if (di, dr) == (0, 0) or not ok(i + di, r + dr):
                            continue
                        sn = S(i + di, r + dr)
                        earlier = di < 0 or (di == 0 and dr < 0)
                        if (earlier and not s > sn) or (not earlier and not s >= sn):
                            peak = False
                if peak:
                    out.append((H, i, r, s))
        lev += 1
        H *= 2
    return out


@pytest.mark.parametrize("max_harm", [1, 2, 4, 8, 16])
def test_peaks_match_brute_force(oracle_mod, max_harm):
    rng = np.random.default_rng(max_harm)
    zmax, nb = 8, 97
    pl = rng.exponential(2.0, size=(zmax + 1, nb))
    thr = [4.0, 7.0, 12.0, 20.0, 35.0]
    for fn, dt in ((oracle_mod.peaks_f64, np.float64), (oracle_mod.peaks_f32, np.float32)):
        got, n = fn(pl, zmax, max_harm, thr)
        ref = _brute_peaks(pl, zmax, max_harm, thr, dt)
        assert n == len(ref) == len(got)
        assert [tuple(g)[:3] for g in got] == [t[:3] for t in ref]
        assert all(g["power"] == t[3] for g, t in zip(got, ref))


def test_peaks_tie_rule_and_overflow(oracle_mod):
    pl = np.zeros((3, 10))
    pl[1, 4] = pl[1, 5] = 9.0            # a plateau of two equal cells in one row
    pl[0, 8] = pl[2, 8] = 5.0            # two equal cells in a column, one row apart
    got, n = oracle_mod.peaks_f64(pl, 2, 1, [1.0])
    assert [(g["zi"], g["r"]) for g in got] == [(0, 8), (1, 4), (2, 8)]
    # overflow: true count reported, only max_out written
    got, n = oracle_mod.peaks_f64(pl, 2, 1, [1.0], max_out=2)
    assert n == 3 and len(got) == 2


# ---------------------------------------------------------------- refinement
def test_interp_power_on_grid_and_gradient(oracle_mod):
    n, a = 1 << 14, 0.1
    x = synth.chirp(n, a, 2000.0, 8.0).astype(np.float32)
    xhat, _ = oracle_mod.spectrum(x, sigma2=float(n))
    m = 64
    # on-grid value equals the plane cell with unnormalised templates: P = N a^2 eta^2 / 2
    P, dr, dz = oracle_mod.interp_power(xhat, m, 2000.0, 8.0)
    eta = np.sum(np.abs(oracle_mod.response(np.arange(-32, 32) * 1.0, 8.0)) ** 2)
    assert abs(P - n * a * a * eta * eta / 2) <= 1e-4 * P
    # the injected point is a maximum: gradient ~ 0 relative to the curvature scale
    assert abs(dr) <= 1e-2 * P and abs(dz) <= 1e-2 * P
    # central finite differences, h = 1e-3, away from the window switch at half-integers
    for (r, z) in ((1999.8, 7.1), (2000.2, 9.3), (2000.05, 7.9)):
        P0, gr, gz = oracle_mod.interp_power(xhat, m, r, z)
        h = 1e-3
        fr = (oracle_mod.interp_power(xhat, m, r + h, z)[0] - oracle_mod.interp_power(xhat, m, r - h, z)[0]) / (2 * h)
        fz = (oracle_mod.interp_power(xhat, m, r, z + h)[0] - oracle_mod.interp_power(xhat, m, r, z - h)[0]) / (2 * h)
        # central differences are O(h^2): 1e-5 of the gradient scale at h = 1e-3
        scale = max(1.0, abs(P0), abs(fr), abs(fz))
        assert abs(gr - fr) <= 1e-5 * scale
        assert abs(gz - fz) <= 1e-5 * scale
        # and the error shrinks as h^2 (h = 1e-4 is 100x closer)
        h = 1e-4
        fr4 = (oracle_mod.interp_power(xhat, m, r + h, z)[0] - oracle_mod.interp_power(xhat, m, r - h, z)[0]) / (2 * h)
        assert abs(gr - fr4) <= 1e-7 * scale + 1e-8


def test_interp_power_anchored_window_against_fresnel_sum(oracle_mod):
    """P with the window anchored at an explicit bin equals |sum_k Xhat_k conj(I(k - r, z))|^2
    summed over that window with I from the Fresnel closed form (an independent route from the
    quadrature moments); moving the anchor by one bin drops the lowest tap and adds one above."""
    n, m = 1 << 14, 32
    rng = synth.rng_for(60, 1)
    x = (synth.noise(n, rng) + synth.chirp(n, 0.1, 3000.37, -5.3)).astype(np.float32)
    xhat, _ = oracle_mod.spectrum(x, sigma2=float(n))
    r, z = 3000.37, -5.3
    for k0 in (2999, 3000, 3001):
        k = np.arange(k0 - m // 2, k0 + m // 2)
        A = np.sum(xhat[k] * np.conj(oracle_mod.response(k - r, z)))
        P = oracle_mod.interp_power(xhat, m, r, z, k0)[0]
        assert abs(P - abs(A) ** 2) <= 1e-11 * abs(A) ** 2
    # the default anchor is the nearest bin
    assert oracle_mod.interp_power(xhat, m, r, z) == oracle_mod.interp_power(xhat, m, r, z, 3000)
    # an anchored window is smooth across the half-integer where the nearest bin changes
    k0, h = 3000, 1e-3
    for rr in (3000.5, 3000.9):
        P0, gr, _ = oracle_mod.interp_power(xhat, m, rr, z, k0)
        fr = (oracle_mod.interp_power(xhat, m, rr + h, z, k0)[0] - oracle_mod.interp_power(xhat, m, rr - h, z, k0)[0]) / (2 * h)
        assert abs(gr - fr) <= 1e-5 * max(1.0, abs(P0), abs(fr))


def _refine_err(oracle_mod, m, r0, z0, seeds, n=1 << 16, a=0.05):
    x = synth.chirp(n, a, r0, z0)
    xhat, _ = oracle_mod.spectrum(x, sigma2=float(n))
    pts, P, ev = oracle_mod.refine(xhat, m, seeds, 21)
    out = []
    for s, p, pp in zip(seeds, pts, P):
        k0 = math.floor(s[0] + 0.5)
        k = np.arange(k0 - m // 2, k0 + m // 2)
        eta = np.sum(np.abs(oracle_mod.response(k - r0, z0)) ** 2)
        Pseed = oracle_mod.interp_power(xhat, m, s[0], s[1], k0)[0]
        out.append((p[0] - r0, p[1] - z0, pp / (n * a * a * eta * eta / 2) - 1.0, pp - Pseed))
    return np.array(out)


def test_refine_recovers_noiseless_chirp(oracle_mod):
    """The ascent ends at the injected (r0, z0) of a noiseless constant-fdot sinusoid, from seeds
    up to half a bin away (the nearest integer bins and off-grid points), with the closed-form
    peak power N a^2 eta^2 / 2 (sigma2 = N, eta = window energy of the response at the truth).
    What remains is the bias of the m-tap window (it falls as 1/m)."""
    for (r0, z0) in ((8000.3, 6.2), (12000.71, -13.4), (5000.5, 0.4)):
        seeds = np.array([(round(r0), round(z0)), (r0 + 0.45, z0 - 0.45), (r0 - 0.4, z0 + 0.5)])
        e = _refine_err(oracle_mod, 256, r0, z0, seeds)
        assert np.all(np.abs(e[:, 0]) <= 1.5e-3), e
        assert np.all(np.abs(e[:, 1]) <= 1e-3), e
        assert np.all(np.abs(e[:, 2]) <= 1e-4), e
        assert np.all(e[:, 3] >= 0.0)                     # the ascent never lowers P
        # one maximum, whatever the seed
        assert np.ptp(e[:, 0]) <= 1e-5 and np.ptp(e[:, 1]) <= 1e-5
    # the window bias shrinks as the window grows (long sinc tails at z ~ 0)
    seeds = np.array([(5000.0, 0.0)])
    e64 = _refine_err(oracle_mod, 64, 5000.5, 0.4, seeds)
    e256 = _refine_err(oracle_mod, 256, 5000.5, 0.4, seeds)
    assert abs(e256[0, 0]) < 0.5 * abs(e64[0, 0])


# ---------------------------------------------------------------- paper's printed numbers
def test_template_bf16_conversion_stats_match_paper(oracle_mod):
    """Table template_stats (Sec. 3.3): FP32 -> BF16 template conversion error under Eq.
    perc_diff.  Our FP32 frequency-domain templates, rounded to BF16 (round to nearest
    even), reproduce the paper's spread: mean ~ 0, sd ~ 0.153%, |extremes| <= 2^-8."""
    with open(os.path.join(GOLDEN, "template_stats.json")) as f:
        ref = json.load(f)
    zmax, m, S = 84, 256, 8192
    T, _ = oracle_mod.templates(zmax, m)
    c = np.zeros((zmax + 1, S), dtype=np.complex128)
    c[:, :m] = T
    G = (oracle_mod.fft(c.ravel()[:S], -1),)  # one row through the oracle FFT as a check
    G = np.fft.fft(c, axis=1) / S
    assert np.abs(G[0] - oracle_mod.fft(c[0], -1) / S).max() <= 1e-15
    for comp, key in ((G.real, "real"), (G.imag, "imag")):
        s = comp.astype(np.float32)
        bits = s.view(np.uint32).astype(np.uint64)
        rounded = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16
        b = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
        s64 = s.astype(np.float64)
        keep = s64 != 0
        d = (b[keep] - s64[keep]) / ((b[keep] + s64[keep]) / 2.0) * 100.0
        paper = ref[key]
        assert abs(d.mean()) <= 0.01
        assert abs(d.std() - paper["sd"]) <= 0.2 * paper["sd"]
        assert d.max() <= 100.0 * 2.0 ** -8 + 1e-9 and d.min() >= -100.0 * 2.0 ** -8 - 1e-9
        assert d.max() >= 0.9 * paper["max"] and d.min() <= 0.9 * paper["min"]


# ---------------------------------------------------------------- pin sensitivity
def test_pins_catch_planted_mistakes(oracle_mod):
    """Plant plausible mistakes into oracle intermediates (on the CPU) and check that the
    closed-form and brute-force pins fail on each of them."""
    n, a, zmax, m, r0, z0 = 1 << 14, 0.05, 16, 64, 3000, 10
    x = synth.chirp(n, a, r0, z0).astype(np.float32)
    xhat, _ = oracle_mod.spectrum(x, sigma2=float(n))
    T, eta = oracle_mod.templates(zmax, m)
    i0 = (z0 + zmax) // 2
    expect = n * a * a * eta[i0] / 2.0

    def peak_ok(xh, TT):
        pl = oracle_mod.plane(xh, zmax, m, TT)
        return abs(pl[i0, r0] - expect) <= 2e-5 * expect

    assert peak_ok(xhat, T)
    assert not peak_ok(xhat, np.conj(T))                       # conjugated template
    assert not peak_ok(np.conj(xhat), T)                       # FFT sign flipped
    assert not peak_ok(xhat, np.roll(T, 1, axis=1))            # tap index shifted by one
    assert not peak_ok(xhat, T[::-1])                          # z axis reversed
    assert not peak_ok(xhat, T[:, ::-1])                       # taps reversed


# ---------------------------------------------------------------- band maxima (harmonic-band analysis)
def test_band_max_against_brute_force(oracle_mod):
    """Band maxima vs an explicit loop over rows then bins (the first of equal maxima wins)."""
    rng = np.random.default_rng(12)
    pl = rng.integers(0, 6, size=(5, 40)).astype(np.float32)        # many ties
    lo = [0, 3, 17, 39, 35, 50, -4]
    hi = [39, 9, 17, 39, 60, 70, 2]
    v, r, zi = oracle_mod.band_max(pl, lo, hi)
    for b, (l, h) in enumerate(zip(lo, hi)):
        l, h = max(0, l), min(39, h)
        if h < l:
            assert (v[b], r[b], zi[b]) == (-1.0, -1, -1)
            continue
        best = (-1.0, -1, -1)
        for i in range(pl.shape[0]):
            for k in range(l, h + 1):
                if pl[i, k] > best[0]:
                    best = (float(pl[i, k]), k, i)
        assert (v[b], r[b], zi[b]) == best
