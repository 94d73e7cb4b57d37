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


def gather_peak_lists(mine: Sequence[int], lists: Sequence[np.ndarray], n_series: int, dist, dst: int = 0):
    """After a sharded search: each rank holds the peak lists of its own series `mine` (in that
    order, as its sub-batch numbered them).  Their `series` fields (where present) are set to the
    series' index in the whole batch and the lists gathered on rank `dst`, which receives one list
    per series of the whole batch (other ranks receive None).  Only these lists travel between
    ranks; the search itself exchanges nothing."""
    if len(mine) != len(lists):
        raise ValueError("one peak list per series of the rank's share")
    local = []
    for s, a in zip(mine, lists):
        a = np.array(a, copy=True)
        if a.dtype.names and "series" in a.dtype.names:
            a["series"] = int(s)
        local.append((int(s), a))
    world = dist.get_world_size()
    parts = [None] * world if dist.get_rank() == dst else None
    dist.gather_object(local, parts, dst=dst)
    if dist.get_rank() != dst:
        return None
    out: List[Optional[np.ndarray]] = [None] * n_series
    for part in parts:
        for s, a in part:
            if out[s] is not None:
                raise RuntimeError(f"series {s} searched by two ranks")
            out[s] = a
    missing = [s for s, a in enumerate(out) if a is None]
    if missing:
        raise RuntimeError(f"series {missing[:8]} searched by no rank")
    return out


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
