"""Host-side arithmetic of the sensitivity analysis (no GPU): harmonic band bounds (Table
harm_bounds), Eq. perc_diff, and the per-band comparison and summary."""
import numpy as np
import pytest

from paper_2206_12205_gb300 import sensitivity as se


def test_harmonic_bands_follow_the_table():
    f = 1000.4
    lo, hi = se.harmonic_bands(f, 5, 10 ** 6)
    # fundamental [0, 1.5 f]; harmonic n ((n + 0.5) f, (n + 1.5) f], upper bound included
    assert (lo[0], hi[0]) == (0, 1500)
    for n in range(1, 5):
        assert lo[n] == int(np.floor((n + 0.5) * f)) + 1 and hi[n] == int(np.floor((n + 1.5) * f))
        assert lo[n] == hi[n - 1] + 1                       # contiguous, no shared bin
    # integer edges: the upper bound belongs to the lower band
    lo, hi = se.harmonic_bands(1000.0, 3, 10 ** 6)
    assert hi == [1500, 2500, 3500] and lo == [0, 1501, 2501]
    # bands are clipped to the plane
    lo, hi = se.harmonic_bands(1000.0, 4, 3000)
    assert hi[-1] == 2999 and hi[2] == 2999


def test_perc_diff_is_the_paper_equation():
    assert se.perc_diff(101.0, 99.0) == pytest.approx(2.0)
    assert se.perc_diff(5.0, 5.0) == 0.0
    assert se.perc_diff(99.0, 101.0) == pytest.approx(-2.0)


def test_compare_and_summarise():
    ref = {"power": np.array([100.0, 50.0, 10.0, 7.0]), "r": np.array([10, 20, 30, -1]),
           "zi": np.array([5, 5, 5, -1]), "std": 2.0}
    oth = {"power": np.array([101.0, 50.0, 10.5, 7.0]), "r": np.array([10, 20, 31, 40]),
           "zi": np.array([6, 7, 5, 3]), "std": 2.0}
    c = se.compare(ref, oth)
    assert list(c["valid"]) == [True, True, True, False]           # an empty reference band is skipped
    assert list(c["recovered"]) == [True, False, False, False]     # same r and |dz| <= 1
    assert list(c["dr"][:3]) == [0, 0, 1] and list(c["dz"][:3]) == [1, 2, 0]
    s = se.summarise([c], canopy_hi_snr=10.0)
    assert s["bands"] == 3 and s["recovered_fraction"] == pytest.approx(1 / 3)
    assert s["perc_diff_max_abs"] == pytest.approx(se.perc_diff(10.5, 10.0))
    assert s["no_drift_fraction"] == 0.0 and s["drift_le1_fraction"] == pytest.approx(2 / 3)
    # above the canopy (SNR > 10): the first two bands
    assert s["above_canopy_bands"] == 2 and s["above_canopy_recovered_fraction"] == 0.5
