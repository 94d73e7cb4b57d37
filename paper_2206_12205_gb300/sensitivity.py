"""Precision sensitivity analysis (Sec. 4.3 and 5 of arXiv:2206.12205): harmonic-band peak
selection on f-z planes, and the comparison of reduced-precision planes with the FP32 one.

With the pulsar's fundamental f known, the plane is split along frequency into bands
(Table harm_bounds: the fundamental [0, 1.5 f], harmonic n [(n + 0.5) f, (n + 1.5) f]) and the
highest cell of each band (fdas_band_max, on the device) is taken as that harmonic.  Between a
form and FP32, a band's peak is "recovered" when it sits in the same frequency bin and the same
or an adjacent z bin; its power is compared as SNR = P / std(plane) (Sec. 5.2) with Eq. perc_diff.
The noise canopy (Sec. 5.3.1) is the range of the highest cell of noise-only bands.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence

import numpy as np

from . import fdas as _f


def harmonic_bands(f_bins: float, n_bands: int, nb: int):
    """Bin bounds [lo, hi] of the fundamental band and harmonics 1 .. n_bands - 1 of a
    fundamental f_bins (frequency in bins, f T), per Table harm_bounds: the fundamental spans
    [0, 1.5 f] and harmonic n spans ((n + 0.5) f, (n + 1.5) f] (upper bound included, lower
    excluded), so neighbouring bands never share a bin."""
    lo, hi = [], []
    for n in range(n_bands):
        b = (n + 1.5) * f_bins
        lo.append(0 if n == 0 else int(math.floor((n + 0.5) * f_bins)) + 1)
        hi.append(min(nb - 1, int(math.floor(b))))
    return lo, hi


def perc_diff(b, s):
    """Eq. perc_diff: (b - s) / ((b + s) / 2) x 100."""
    b = np.asarray(b, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    return (b - s) / ((b + s) / 2.0) * 100.0


def band_peaks(plan, plane, lo: Sequence[int], hi: Sequence[int]) -> Dict[str, np.ndarray]:
    """Band maxima of a device plane plus its standard deviation (for SNR = P / std)."""
    v, r, zi = _f.fdas_band_max(plan, plane, lo, hi)
    std = float(plane.float().std().item())
    return {"power": v.cpu().numpy().astype(np.float64), "r": r.cpu().numpy(), "zi": zi.cpu().numpy(),
            "std": std}


def compare(ref: Dict[str, np.ndarray], other: Dict[str, np.ndarray]) -> Dict[str, np.ndarray]:
    """Per band: recovered (same r, |dzi| <= 1), SNR perc_diff, frequency and z bin drift."""
    ok = (ref["r"] >= 0) & (other["r"] >= 0)
    dr = other["r"] - ref["r"]
    dz = other["zi"] - ref["zi"]
    snr_ref = ref["power"] / ref["std"]
    snr_oth = other["power"] / other["std"]
    return {"valid": ok, "recovered": ok & (dr == 0) & (np.abs(dz) <= 1), "perc_diff": perc_diff(snr_oth, snr_ref),
            "dr": dr, "dz": dz, "snr_ref": snr_ref}


def summarise(rows: List[Dict[str, np.ndarray]], canopy_hi_snr: float = None) -> Dict[str, float]:
    """Aggregate per-band comparisons: recovered fraction, perc_diff spread, drift fractions; the
    same restricted to peaks above the noise canopy when its upper bound is given."""
    cat = {k: np.concatenate([r[k] for r in rows]) for k in rows[0]}
    v = cat["valid"]
    out = {"bands": int(v.sum()), "recovered_fraction": float(cat["recovered"][v].mean()),
           "perc_diff_sd": float(np.std(cat["perc_diff"][v])), "perc_diff_max_abs": float(np.abs(cat["perc_diff"][v]).max()),
           "no_drift_fraction": float(((cat["dr"] == 0) & (cat["dz"] == 0))[v].mean()),
           "drift_le1_fraction": float(((np.abs(cat["dr"]) <= 1) & (np.abs(cat["dz"]) <= 1))[v].mean())}
    if canopy_hi_snr is not None:
        a = v & (cat["snr_ref"] > canopy_hi_snr)
        if a.any():
            out.update({"above_canopy_bands": int(a.sum()),
                        "above_canopy_recovered_fraction": float(cat["recovered"][a].mean()),
                        "above_canopy_perc_diff_max_abs": float(np.abs(cat["perc_diff"][a]).max())})
    return out


def noise_canopy(plan, plane, widths_bins: Sequence[float], rng: np.random.Generator):
    """Sec. 5.3.1: for each width (1.5 f of a pulsar, in bins), the highest cell of a random band of
    that width in a noise-only plane, in SNR units; returns (min, max) over the widths."""
    nb = plan.info.nb
    lo, hi = [], []
    for w in widths_bins:
        w = max(1, int(round(w)))
        a = int(rng.integers(0, max(1, nb - w)))
        lo.append(a)
        hi.append(min(nb - 1, a + w - 1))
    p = band_peaks(plan, plane, lo, hi)
    snr = p["power"] / p["std"]
    return float(snr.min()), float(snr.max())
