"""Pins of the oracle's FP8 E4M3 rounding and FP8 direct-correlation plane (the FP8 ablation):
against torch's float8_e4m3fn conversion (an independent implementation of the format), hand
values of the format, and the exact plane the quantised plane must approach as operands grow
exact."""
import numpy as np
import pytest

import fdas_synth as synth
import oracle


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def test_e4m3_hand_values():
    cases = {0.0: 0.0, 1.0: 1.0, 1.0625: 1.0, 1.1875: 1.25, -1.1875: -1.25, 448.0: 448.0, 460.0: 448.0,
             470.0: 448.0, 1e6: 448.0, 2.0 ** -6: 2.0 ** -6, 2.0 ** -9: 2.0 ** -9, 2.0 ** -10: 0.0,
             3 * 2.0 ** -10: 2.0 ** -8, 0.3: 0.3125, 17.0: 16.0, 19.0: 20.0}
    for v, want in cases.items():
        assert oracle.e4m3(v)[0] == want, (v, oracle.e4m3(v)[0], want)


def test_e4m3_matches_torch():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8_e4m3fn")
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.standard_normal(20000) * 50, rng.standard_normal(5000) * 0.01,
                        rng.uniform(-448, 448, 5000)])
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.float8_e4m3fn).double().numpy()
    got = oracle.e4m3(v.astype(np.float32).astype(np.float64))
    assert np.array_equal(got, ref)


def test_fp8_plane_against_exact_plane():
    """The FP8 plane scatters around the exact plane by the E4M3 operand error (3 mantissa bits,
    u = 2^-4): noise cells within tens of per cent, the strong signal's peak within a few per
    cent; and a plane whose operands are exact in E4M3 reproduces the exact plane."""
    n, zmax, m = 1 << 13, 4, 16
    x = (synth.noise(n, synth.rng_for(73, 0)) + synth.chirp(n, 0.3, 700.0, 2.0)).astype(np.float32)
    xh, _ = oracle.spectrum(x)
    xh = xh.astype(np.complex64).astype(np.complex128)
    ex = oracle.plane(xh, zmax, m)
    q = oracle.plane_fp8(xh, zmax, m)
    fr = np.abs(q - ex) / np.maximum(ex, 2.0)
    assert np.sqrt(np.mean(fr ** 2)) < 0.15
    i, r = np.unravel_index(np.argmax(ex), ex.shape)
    assert abs(q[i, r] / ex[i, r] - 1.0) < 0.05
    # zmax = 0: one template, a delta (T(0) = 1, exact); a spectrum of small integers is exact in
    # E4M3 at any power-of-two scale that keeps them in range: the FP8 plane is then |Xhat|^2
    rng = np.random.default_rng(6)
    xi = (rng.integers(-7, 8, 4096) + 1j * rng.integers(-7, 8, 4096)).astype(np.complex128)
    xi[0] = 0
    p8 = oracle.plane_fp8(xi, 0, 8)
    assert np.allclose(p8[0], np.abs(xi) ** 2, rtol=0, atol=1e-9)


def test_fp8_cells_are_the_planes_cells():
    """The sampled-cell form (used at sizes the full plane would take hours for) agrees bit for
    bit with the full FP8 plane, tile edges and the last bins included."""
    n, zmax, m = 1 << 13, 6, 32
    x = (synth.noise(n, synth.rng_for(73, 1)) + synth.chirp(n, 0.2, 1500.0, 3.0)).astype(np.float32)
    xh, _ = oracle.spectrum(x)
    T, _ = oracle.templates(zmax, m)
    full = oracle.plane_fp8(xh, zmax, m, T)
    r = np.array([0, 1, 1023, 1024, 1025, 2047, 3000, n // 2 - 1] * 3, dtype=np.int64)
    zi = np.repeat(np.array([0, 3, zmax], dtype=np.int32), 8)
    got = oracle.plane_fp8_cells(xh, zmax, m, T, zi, r)
    assert np.array_equal(got, full[zi, r])
    with pytest.raises(ValueError):
        oracle.plane_fp8_cells(xh, zmax, m, T, np.array([zmax + 1], np.int32), np.array([0]))
