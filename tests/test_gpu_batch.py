"""Batched search on the GPU (fdas_batch_*): every series of a batch against the same series
searched alone (the same kernels on the same input: bit-exact peak lists), FP32 series against
the FP64 oracle's own search, the captured graph relaunched and re-captured, and the autotuner
with its JSON cache."""
import json

import numpy as np
import pytest
import torch

import fdas_synth as synth
import oracle
import paper_2206_12205_gb300 as fd
from paper_2206_12205_gb300 import batch as fb

pytestmark = pytest.mark.gpu

THR = (18.0, 24.0, 30.0, 40.0, 56.0)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fd.build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _small_batch(n_series=10, seed=80):
    return synth.batch_workload(config_index=seed, n_series=n_series, n_choices=(1 << 14, 1 << 15, 1 << 16),
                                zmax_choices=(4, 10, 16), snr=(20.0, 40.0))


def _cfgs(wl, precision, seg=1024):
    return [fd.make_config(w.n, w.zmax, w.taps, seg, precision=precision, max_harm=16, thr=THR, max_peaks=4096)
            for w in wl.series]


def _peaks_equal(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert (int(x["harm"]), int(x["zi"]), int(x["r"])) == (int(y["harm"]), int(y["zi"]), int(y["r"]))
        assert np.float32(x["power"]).tobytes() == np.float32(y["power"]).tobytes()


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16_scaled", "bf16_direct", "fp8_direct"])
def test_batch_equals_series_searched_alone(precision):
    wl = _small_batch()
    cfgs = _cfgs(wl, precision)
    bs = fb.BatchSearch(cfgs)
    dev = torch.from_numpy(wl.packed).cuda()
    bs.search(dev)
    torch.cuda.synchronize()
    lists = bs.peak_lists()
    total = 0
    for i, (w, cfg) in enumerate(zip(wl.series, cfgs)):
        s = fd.Search(cfg)
        x = dev[int(wl.offsets[i]): int(wl.offsets[i]) + w.n]
        s.search(x)
        torch.cuda.synchronize()
        want = s.peak_list()
        got = lists[i]
        assert np.all(got["series"] == i)
        _peaks_equal(got, want)
        total += len(got)
    assert total > 0
    assert fd.fdas_batch_device_status(bs.batch) == 0


@pytest.mark.parametrize("precision,lanes", [("fp32", 3), ("bf16", 2), ("bf16", 4)])
def test_batch_lanes_give_the_same_lists(precision, lanes):
    """Concurrent lanes (the graph's parallel branches, each with its own workspace and plane
    buffer) change only the schedule: every series' list is the one-lane list, record for record,
    and the lanes' workspaces do not overlap (a series would otherwise read another's plane)."""
    wl = _small_batch(n_series=11, seed=84)
    cfgs = _cfgs(wl, precision)
    dev = torch.from_numpy(wl.packed).cuda()
    one = fb.BatchSearch(cfgs)
    one.search(dev)
    many = fb.BatchSearch(cfgs, lanes=lanes)
    assert many.batch.workspace_bytes == lanes * one.batch.workspace_bytes
    for _ in range(2):                                  # capture, then relaunch
        many.npeaks.zero_()
        many.search(dev)
        torch.cuda.synchronize()
        for x, y in zip(one.peak_lists(), many.peak_lists()):
            _peaks_equal(x, y)
    assert sum(len(x) for x in one.peak_lists()) > 0
    assert fd.fdas_batch_device_status(many.batch) == 0


def test_batch_zero_series_reports_nothing():
    """A series of zeros inside a batch (sigma2 = 0) yields an empty list and leaves every other
    series' list unchanged."""
    wl = _small_batch(n_series=6, seed=81)
    bs = fb.BatchSearch(_cfgs(wl, "bf16"))
    dev = torch.from_numpy(wl.packed).cuda()
    bs.search(dev)
    torch.cuda.synchronize()
    before = [a.copy() for a in bs.peak_lists()]
    z = 3
    dev[int(wl.offsets[z]): int(wl.offsets[z]) + wl.series[z].n] = 0.0
    bs.search(dev)
    torch.cuda.synchronize()
    after = bs.peak_lists()
    assert len(before[z]) > 0 and len(after[z]) == 0
    for i in range(len(wl.series)):
        if i != z:
            _peaks_equal(after[i], before[i])
    assert fd.fdas_batch_device_status(bs.batch) == 0


def test_batch_fp32_against_oracle():
    """FP32 batch series against the oracle's FP64 search of the same series: the same peaks
    (level, row, bin), powers within the FP32 plane tolerance (1e-5 of max(P, 2) per summed term),
    cells within that tolerance of a threshold excepted."""
    wl = _small_batch(n_series=6, seed=81)
    cfgs = _cfgs(wl, "fp32")
    bs = fb.BatchSearch(cfgs)
    bs.search(torch.from_numpy(wl.packed).cuda())
    torch.cuda.synchronize()
    lists = bs.peak_lists()
    for i, w in enumerate(wl.series):
        if w.n > (1 << 15):
            continue                                   # the oracle's direct correlation: small series only
        x = wl.packed[wl.offsets[i]: wl.offsets[i] + w.n]
        ref = oracle.search(x, w.zmax, w.taps, 16, THR)
        thr_of = {1 << l: THR[l] for l in range(5)}

        def key(p, hname):
            return (int(p[hname]), int(p["zi"]), int(p["r"]))

        def near_thr(p, hname):
            h = int(p[hname])
            return abs(float(p["power"]) - thr_of[h]) <= 1e-5 * h * max(thr_of[h], 2.0)
        got = {key(p, "harm"): float(p["power"]) for p in lists[i] if not near_thr(p, "harm")}
        want = {key(p, "h"): float(p["power"]) for p in ref["peaks"] if not near_thr(p, "h")}
        assert got.keys() == want.keys(), (i, set(got) ^ set(want))
        for k, v in want.items():
            assert abs(got[k] - v) <= 1e-5 * k[0] * max(v, 2.0)


def test_batch_graph_reuse_and_recapture():
    wl = _small_batch(n_series=5, seed=82)
    bs = fb.BatchSearch(_cfgs(wl, "bf16"))
    a = torch.from_numpy(wl.packed).cuda()
    bs.search(a)
    torch.cuda.synchronize()
    first = [p.copy() for p in bs.peak_lists()]
    bs.npeaks.zero_()
    bs.peaks.zero_()
    bs.search(a)                                       # the same buffers: graph relaunched
    torch.cuda.synchronize()
    for x, y in zip(first, bs.peak_lists()):
        _peaks_equal(x, y)
    b = a.clone()                                      # another input buffer: captured again
    bs.npeaks.zero_()
    bs.search(b)
    torch.cuda.synchronize()
    for x, y in zip(first, bs.peak_lists()):
        _peaks_equal(x, y)


def test_batch_autotune_cache(tmp_path):
    wl = _small_batch(n_series=6, seed=83)
    cfgs = _cfgs(wl, "fp32")
    cache = str(tmp_path / "tune.json")
    b1 = fd.fdas_batch_plan(cfgs)
    fd.fdas_batch_autotune(b1, cache)
    with open(cache) as f:
        entries = json.load(f)["entries"]
    groups = {s.group for s in b1.series}
    per_group = {k: e for k, e in entries.items() if not k.startswith("batch:")}
    per_batch = {k: e for k, e in entries.items() if k.startswith("batch:")}
    assert len(per_group) == len(groups) and len(per_batch) == 1
    for e in per_group.values():
        assert e["seg_len"] in (1024, 2048, 4096, 8192) and e["zb"] in (1, 2, 4, 8, 16) and e["ms"] > 0
    (eb,) = per_batch.values()
    assert 1 <= eb["lanes"] <= 4 and eb["ms"] > 0
    assert b1.workspace_bytes % eb["lanes"] == 0        # lanes x one lane's scratch and plane
    chosen = [s.cfg["seg_len"] for s in b1.series]
    # a second batch reads the cache: the same choices, no new timing
    b2 = fd.fdas_batch_plan(cfgs)
    fd.fdas_batch_autotune(b2, cache)
    assert [s.cfg["seg_len"] for s in b2.series] == chosen
    with open(cache) as f:
        assert json.load(f)["entries"] == entries
    # the tuned batch still finds what the untuned one finds (the plane does not depend on S)
    bs = fb.BatchSearch(cfgs, autotune=True, autotune_cache=cache)
    ref = fb.BatchSearch(cfgs)
    dev = torch.from_numpy(wl.packed).cuda()
    bs.search(dev)
    ref.search(dev)
    torch.cuda.synchronize()
    for x, y in zip(bs.peak_lists(), ref.peak_lists()):
        assert len(x) == len(y)
        assert [(int(p["harm"]), int(p["zi"]), int(p["r"])) for p in x] == \
               [(int(p["harm"]), int(p["zi"]), int(p["r"])) for p in y]
        assert np.allclose(x["power"], y["power"], rtol=1e-5, atol=0)
    fd.fdas_batch_destroy(b1)
    fd.fdas_batch_destroy(b2)
