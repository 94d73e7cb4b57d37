"""Batched search, host side (no GPU): planning, layout and validation of the batch C-ABI, and
the multi-GPU sharding rule with its gather of per-series peak lists over gloo (world size 2)."""
import ctypes
import json
import os
import socket

import numpy as np
import pytest

import fdas_synth as synth
import paper_2206_12205_gb300 as fd
from paper_2206_12205_gb300 import batch as fb
from paper_2206_12205_gb300 import fdas as fbind


@pytest.fixture(scope="module")
def lib():
    fd.build.build()
    return fd.load()


def _cfgs(shapes, precision="fp32", seg=1024):
    return [fd.make_config(n, z, synth.taps_for_zmax(z), seg, precision=precision, max_harm=4,
                           thr=(20.0, 24.0, 30.0), max_peaks=100 + 7 * i) for i, (n, z) in enumerate(shapes)]


def _align(x):
    return (x + 255) // 256 * 256


def test_batch_plan_layout(lib):
    shapes = [(1 << 14, 4), (1 << 16, 16), (1 << 14, 4), (1 << 15, 10), (1 << 16, 16), (1 << 13, 0)]
    cfgs = _cfgs(shapes)
    b = fd.fdas_batch_plan(cfgs)
    assert b.n_series == len(shapes)
    assert b.total_samples == sum(n for n, _ in shapes)
    assert b.total_peaks == sum(c["max_peaks"] for c in cfgs)
    assert b.total_cells == sum((z + 1) * (n // 2) for n, z in shapes)
    so = np.cumsum([0] + [n for n, _ in shapes])[:-1]
    po = np.cumsum([0] + [c["max_peaks"] for c in cfgs])[:-1]
    assert [s.sample_offset for s in b.series] == list(so)
    assert [s.peak_offset for s in b.series] == list(po)
    # series with the same shape share a group (one template bank)
    g = [s.group for s in b.series]
    assert g[0] == g[2] and g[1] == g[4] and len(set(g)) == 4
    # the workspace holds the largest series' scratch and the largest plane
    plans = [fd.fdas_plan(c) for c in cfgs]
    ws = max(p.info.workspace_bytes for p in plans)
    pl = max(p.info.plane_bytes for p in plans)
    assert b.workspace_bytes == _align(ws) + _align(pl)
    for s, c, p in zip(b.series, cfgs, plans):
        assert s.info == p.info
        assert s.cfg["n_samples"] == c["n_samples"] and s.cfg["zmax"] == c["zmax"] and s.cfg["taps"] == c["taps"]
        assert s.cfg["max_peaks"] == c["max_peaks"]
    fd.fdas_batch_destroy(b)
    fd.fdas_batch_destroy(b)                     # a second destroy is a no-op


def test_batch_lanes_layout(lib):
    """fdas_batch_set_lanes (host only): the workspace is lanes x (largest scratch + largest
    plane); out-of-range lane counts are rejected and leave the batch as it was."""
    cfgs = _cfgs([(1 << 14, 4), (1 << 16, 16), (1 << 15, 10), (1 << 13, 0), (1 << 16, 16)])
    b = fd.fdas_batch_plan(cfgs)
    one = b.workspace_bytes
    for lanes in (1, 2, 3, 8):
        assert fd.fdas_batch_set_lanes(b, lanes) == lanes * one
        assert b.workspace_bytes == lanes * one
    for bad in (0, -1, 9):
        with pytest.raises(fd.FdasError) as ei:
            fd.fdas_batch_set_lanes(b, bad)
        assert ei.value.status == fbind.FDAS_E_INVALID
    assert b.workspace_bytes == 8 * one
    assert lib.fdas_batch_set_lanes(None, 2, None) == fbind.FDAS_E_INVALID
    fd.fdas_batch_destroy(b)


def test_batch_plan_rejects(lib):
    with pytest.raises(fd.FdasError):
        fd.fdas_batch_plan([])
    bad = _cfgs([(1 << 14, 4), (1 << 14, 4)])
    bad[1]["zmax"] = 5                           # odd zmax
    with pytest.raises(fd.FdasError) as ei:
        fd.fdas_batch_plan(bad)
    assert ei.value.status == fbind.FDAS_E_INVALID
    assert lib.fdas_batch_plan(None, 1, None, None) == fbind.FDAS_E_INVALID


def test_batch_calls_out_of_order(lib):
    b = fd.fdas_batch_plan(_cfgs([(1 << 14, 4), (1 << 15, 10)]))
    fake = ctypes.c_void_p(1 << 20)              # never dereferenced: the state check comes first
    assert lib.fdas_batch_search(b.handle, fake, fake, fake, fake, None) == fbind.FDAS_E_STATE
    assert lib.fdas_batch_search(b.handle, None, fake, fake, fake, None) == fbind.FDAS_E_INVALID
    assert lib.fdas_batch_search(b.handle, fake, ctypes.c_void_p((1 << 20) + 64), fake, fake, None) == \
        fbind.FDAS_E_INVALID                     # workspace must be 256-byte aligned
    assert lib.fdas_batch_get_info(None, None, None, None, None, None) == fbind.FDAS_E_INVALID
    assert lib.fdas_batch_series_info(b.handle, 2, None, None, None, None, None) == fbind.FDAS_E_INVALID
    assert lib.fdas_batch_last_error(None) == b""
    lib.fdas_batch_destroy(None)
    fd.fdas_batch_destroy(b)


def test_batch_device_calls_without_gpu_fail_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    b = fd.fdas_batch_plan(_cfgs([(1 << 14, 4)]))
    assert lib.fdas_batch_make_templates(b.handle, None) in (fbind.FDAS_E_CUDA, fbind.FDAS_E_NOMEM)
    assert lib.fdas_batch_autotune(b.handle, None, None) in (fbind.FDAS_E_CUDA, fbind.FDAS_E_NOMEM)
    fd.fdas_batch_destroy(b)


# ------------------------------------------------------------------ sharding over GPUs
def _batch_costs(n_series=256):
    shapes = synth._batch_shapes(2, n_series, synth.BATCH_N, synth.BATCH_ZMAX)
    return [fb.series_cost(n, z) for n, z in shapes]


def test_shard_series_rule():
    costs = _batch_costs()
    for world in (1, 2, 3, 4, 8):
        parts = fb.shard_series(costs, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))                 # every series exactly once
        loads = [sum(costs[i] for i in p) for p in parts]
        # largest-first greedy: no rank exceeds the mean by more than the largest series
        assert max(loads) <= sum(costs) / world + max(costs)
        assert fb.shard_series(costs, world) == parts          # deterministic
    assert fb.shard_series([3, 3, 3], 2) == [[0, 2], [1]]      # ties go to the lowest rank
    with pytest.raises(ValueError):
        fb.shard_series(costs, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _gloo_rank(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = _batch_costs()
        mine = fb.shard_series(costs, world)[rank]
        # what a rank's search returns: (series, peak records) for its own series only
        records = [(s, [(s, 1, 3, 40.0 + s)]) for s in mine]
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        gathered = [None] * world if rank == 0 else None
        dist.gather_object(records, gathered, dst=0)
        if rank == 0:
            merged = sorted((s, r) for part in gathered for s, r in part)
            with open(out_path, "w") as f:
                json.dump({"parts": parts, "series": [s for s, _ in merged],
                           "loads": [sum(costs[i] for i in p) for p in parts]}, f)
    finally:
        dist.destroy_process_group()


def test_shard_and_gather_two_gloo_ranks(tmp_path):
    """Two CPU ranks: each derives the same split on its own (no exchange before the search);
    after the search only the per-series peak lists travel, gathered on rank 0."""
    import torch.multiprocessing as tmp
    out = str(tmp_path / "gather.json")
    tmp.spawn(_gloo_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    with open(out) as f:
        res = json.load(f)
    costs = _batch_costs()
    assert res["parts"] == fb.shard_series(costs, 2)
    assert res["series"] == list(range(len(costs)))
    assert abs(res["loads"][0] - res["loads"][1]) <= max(costs)


# ------------------------------------------------------------------ sharded search, gathered lists
SHARD_KW = dict(config_index=85, n_series=7, n_choices=(1 << 12, 1 << 13), zmax_choices=(4, 8), snr=(20.0, 40.0))
SHARD_THR = (14.0, 18.0, 22.0)


def _oracle_lists(wl):
    """Each series' peak list from the FP64 oracle's whole search (the stand-in for a rank's batch
    search on a machine without a GPU), with the series field a rank's sub-batch would give it."""
    import oracle
    out = []
    for k, w in enumerate(wl.series):
        x = wl.packed[int(wl.offsets[k]): int(wl.offsets[k]) + w.n]
        pk = oracle.search(x, w.zmax, w.taps, 4, SHARD_THR)["peaks"]
        a = np.zeros(len(pk), dtype=fbind.PEAK_DTYPE)
        a["series"] = k
        a["r"], a["zi"], a["harm"], a["power"] = pk["r"], pk["zi"], pk["h"], pk["power"]
        out.append(a)
    return out


def _shard_rank(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shapes = synth._batch_shapes(SHARD_KW["config_index"], SHARD_KW["n_series"], SHARD_KW["n_choices"],
                                     SHARD_KW["zmax_choices"])
        mine = fb.shard_series([fb.series_cost(n, z) for n, z in shapes], world)[rank]
        wl = synth.batch_workload(series=mine, **SHARD_KW)       # only this rank's series
        lists = fb.gather_peak_lists(mine, _oracle_lists(wl), SHARD_KW["n_series"], dist)
        if rank == 0:
            np.savez(out_path, *lists)
        else:
            assert lists is None
    finally:
        dist.destroy_process_group()


def test_sharded_search_gathers_the_single_rank_lists(tmp_path):
    """Two gloo ranks each search only their share of a batch (split by shard_series, inputs
    synthesised per rank) and gather the per-series lists on rank 0: the result equals one
    process searching the whole batch, list for list, with each record's series field the
    series' index in the whole batch."""
    import oracle
    import torch.multiprocessing as tmp
    oracle.build()
    out = str(tmp_path / "lists.npz")
    tmp.spawn(_shard_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    whole = _oracle_lists(synth.batch_workload(**SHARD_KW))
    assert len(got.files) == len(whole) == SHARD_KW["n_series"]
    assert sum(len(a) for a in whole) > 0
    for s, want in enumerate(whole):
        g = got[f"arr_{s}"]
        assert np.all(g["series"] == s)
        want = want.copy()
        want["series"] = s
        assert g.tobytes() == want.tobytes()


def test_gather_rejects_overlapping_shares():
    class FakeDist:                                   # one process standing in for rank 0 of two
        def get_world_size(self):
            return 2

        def get_rank(self):
            return 0

        def gather_object(self, obj, parts, dst=0):
            parts[0] = obj
            parts[1] = obj                            # the other rank searched the same series

    a = np.zeros(1, dtype=fbind.PEAK_DTYPE)
    with pytest.raises(RuntimeError):
        fb.gather_peak_lists([0], [a], 2, FakeDist())
