"""Many series (dispersion-measure trials) in one call: the libfdas batch API with torch buffers,
and the rule that shards a batch over several GPUs.

A batch runs every series through the spectrum, plane and peak kernels back to back in one
CUDA graph (fdas_batch_search).  Across GPUs the series are independent, so a batch is split
by cost with no data exchange during the search; only the peak lists are gathered afterwards.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np

from . import fdas as _f


def series_cost(n_samples: int, zmax: int) -> int:
    """Plane cells of a series, K * Nb: what the plane and peak kernels' time scales with."""
    return (zmax + 1) * (n_samples // 2)


def shard_series(costs: Sequence[int], world: int) -> List[List[int]]:
    """Split series over `world` ranks: largest cost first, each to the least loaded rank (the
    lowest rank on ties).  Deterministic, so every rank computes the same split on its own.
    Returns each rank's series indices in increasing order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-int(costs[k]), k)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += int(costs[i])
    return [sorted(p) for p in parts]


class BatchSearch:
    """A planned batch with its device buffers (torch-owned): workspace, peak regions, counts."""

    def __init__(self, cfgs: Sequence[dict], device="cuda", autotune_cache: Optional[str] = None,
                 autotune: bool = False, stream=None, lanes: Optional[int] = None):
        import torch
        self.device = torch.device(device)
        self.batch = _f.fdas_batch_plan(cfgs)
        if lanes is not None:
            _f.fdas_batch_set_lanes(self.batch, lanes)
        if autotune:
            _f.fdas_batch_autotune(self.batch, autotune_cache, stream)
        _f.fdas_batch_make_templates(self.batch, stream)
        b = self.batch
        self.workspace = torch.empty(b.workspace_bytes, dtype=torch.uint8, device=self.device)
        self.peaks = torch.zeros(max(16, 16 * b.total_peaks), dtype=torch.uint8, device=self.device)
        self.npeaks = torch.zeros(b.n_series, dtype=torch.int32, device=self.device)

    @property
    def sample_offsets(self) -> List[int]:
        return [s.sample_offset for s in self.batch.series]

    def search(self, series_packed, stream=None):
        _f.fdas_batch_search(self.batch, series_packed, self.workspace, self.peaks, self.npeaks, stream)

    def peak_lists(self) -> List[np.ndarray]:
        """Each series' records (up to its capacity), in (H, zi, r) order."""
        counts = self.npeaks.cpu().numpy()
        raw = self.peaks.cpu().numpy()
        out = []
        for s, n in zip(self.batch.series, counts):
            n = min(int(n), s.cfg["max_peaks"])
            a = raw[16 * s.peak_offset: 16 * (s.peak_offset + n)]
            out.append(a.view(_f.PEAK_DTYPE).copy())
        return out
