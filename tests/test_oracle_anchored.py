"""Pins of the oracle's highest-harmonic-anchored harmonic sums (orc_peaks_anch_*), against facts
that do not depend on its code: a plane that is a pure function of the grid coordinates has sums
computable by hand; harmonics of an exact lattice land where they must; the nesting identity
(level 2L contains level L's terms exactly); level 1 equals the fundamental-anchored level 1."""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _round_half_up(num, den):
    """floor(num / den + 1/2) for integers, written from the definition of rounding."""
    return np.floor(np.asarray(num, dtype=np.float64) / den + 0.5).astype(np.int64)


def test_single_bright_cell_is_summed_by_the_cells_that_round_onto_it():
    """A plane that is 0 except P = 1 at one cell (r*, i*): S_H(r, i) counts the harmonics
    j/H (nested set) whose rounded coordinates hit (r*, i*); peaks of level H appear exactly at
    the cells where that count is maximal, found here by brute force over every cell."""
    zmax, nb = 8, 512
    K = zmax + 1
    pl = np.zeros((K, nb))
    rs, is_ = 300, 6                                  # z* = 4
    pl[is_, rs] = 1.0
    for H in (2, 4, 8):
        # brute force: S_H(r, i) = number of (level L <= H, odd j < L or the anchor) terms on (rs, is_)
        S = np.zeros((K, nb))
        for i in range(K):
            z = -zmax + 2 * i
            for r in range(nb):
                s = 1.0 if (r == rs and i == is_) else 0.0
                L = 2
                while L <= H:
                    for j in range(1, L, 2):
                        rj = _round_half_up(j * r, L)
                        zj = j * z / L
                        ij = _round_half_up(zj + zmax, 2)     # nearest grid row of j z / L
                        if rj == rs and ij == is_:
                            s += 1.0
                    L *= 2
                S[i, r] = s
        pk, n = oracle.peaks_f64(pl, zmax, H, [0.5] * 5, anchored=True)
        got = pk[pk["h"] == H]
        want = np.argwhere(S >= 0.5)
        # every cell with a positive sum either is a peak or has a neighbour beating it
        assert len(got) >= 1
        for g in got:
            assert S[g["zi"], g["r"]] == g["power"]
        assert max(S.max(), 0) == got["power"].max()


def test_exact_lattice_harmonics():
    """Lattice plane P(r, i) = r + 1000 i (integers, exact in FP64): S_2(r, i) = P(r, i) +
    P(round(r/2), row of z/2) in closed form, checked over every cell against peaks' powers
    (all cells are peaks of level 2 at the plane's top-right corner only, so compare sums through
    a threshold that selects one cell)."""
    zmax, nb = 6, 64
    K = zmax + 1
    r = np.arange(nb)
    pl = (r[None, :] + 1000.0 * np.arange(K)[:, None]).astype(np.float64)
    # the maximum of S_2 is at the last cell: (r = nb - 1, i = K - 1)
    z = zmax
    r2 = int(_round_half_up(nb - 1, 2))
    i2 = int(_round_half_up(z / 2 + zmax, 2))
    want = pl[K - 1, nb - 1] + pl[i2, r2]
    pk, n = oracle.peaks_f64(pl, zmax, 2, [0.0, want - 0.5, 0, 0, 0], anchored=True)
    lev2 = pk[pk["h"] == 2]
    assert len(lev2) == 1 and lev2["r"][0] == nb - 1 and lev2["zi"][0] == K - 1
    assert lev2["power"][0] == want


def test_nesting_and_level_one():
    """S_2L = S_L + the odd-j terms: on a random plane the level-2L sum at a cell minus the
    level-L sum equals the brute-force odd-j terms; level 1 equals the fundamental-anchored
    level 1 exactly (same peaks)."""
    rng = np.random.default_rng(3)
    zmax, nb = 10, 256
    K = zmax + 1
    pl = rng.exponential(2.0, size=(K, nb))
    a1, _ = oracle.peaks_f64(pl, zmax, 1, [6.0] * 5, anchored=True)
    e1, _ = oracle.peaks_f64(pl, zmax, 1, [6.0] * 5, anchored=False)
    assert np.array_equal(a1["r"], e1["r"]) and np.array_equal(a1["zi"], e1["zi"])
    assert np.array_equal(a1["power"], e1["power"])
    # one peak at a known cell with a huge value: its S_H reported at every level equals the
    # brute-force nested sum
    i0, r0 = 7, 200
    pl[i0, r0] = 1e6
    pk, _ = oracle.peaks_f64(pl, zmax, 16, [1e5] * 5, anchored=True)
    z0 = -zmax + 2 * i0
    for H in (1, 2, 4, 8, 16):
        rec = pk[(pk["h"] == H) & (pk["r"] == r0) & (pk["zi"] == i0)]
        assert len(rec) == 1
        s = pl[i0, r0]
        L = 2
        while L <= H:
            for j in range(1, L, 2):
                s += pl[int(_round_half_up(z0 * j / L + zmax, 2)), int(_round_half_up(j * r0, L))]
            L *= 2
        assert rec["power"][0] == s


def test_float_mode_matches_double_on_exact_plane():
    """On a plane of small integers every float sum is exact: the float (given-plane) mode
    returns the same peaks and powers as FP64."""
    rng = np.random.default_rng(4)
    zmax, nb = 12, 1024
    pl = rng.integers(0, 8, size=(zmax + 1, nb)).astype(np.float64)
    a, na = oracle.peaks_f64(pl, zmax, 16, [20, 30, 50, 90, 160], anchored=True)
    b, nb_ = oracle.peaks_f32(pl.astype(np.float32), zmax, 16, [20, 30, 50, 90, 160], anchored=True)
    assert na == nb_
    assert np.array_equal(a["r"], b["r"]) and np.array_equal(a["zi"], b["zi"]) and np.array_equal(a["h"], b["h"])
    assert np.array_equal(a["power"], b["power"].astype(np.float64))
