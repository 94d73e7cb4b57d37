"""bench.py's host-side pieces on the CPU: the algorithmic byte count of the harmonic sums
against a cell-by-cell count, the per-source-hash validity of committed DRAM traffic figures, and
the parsing of the clock samples (rejection reasons) taken during the timed region."""
import hashlib
import json
import types

import bench


def _w(nb, zmax):
    return types.SimpleNamespace(nb=nb, zmax=zmax, K=zmax + 1)


def test_gathers_counts_every_new_harmonic_term():
    """Level H adds harmonics H/2+1 .. H for each cell (r, z) with |H z| <= zmax and H r < Nb;
    counted cell by cell on small planes (odd and even zmax / H, Nb a power of two)."""
    for nb, zmax in ((1024, 84), (512, 20), (256, 6), (2048, 0)):
        for levels in (range(1, 2), range(1, 5), range(2, 4)):
            want = 0
            for l in levels:
                H = 1 << l
                for i in range(zmax + 1):
                    z = -zmax + 2 * i
                    if abs(H * z) > zmax:
                        continue
                    want += sum(H // 2 for r in range(nb) if H * r < nb)
            assert bench._gathers(_w(nb, zmax), levels) == want, (nb, zmax, list(levels))


def test_traffic_valid_only_for_the_hashed_source(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    sha = hashlib.sha1(src.read_bytes()).hexdigest()[:16]
    table = tmp_path / "traffic.json"
    table.write_text(json.dumps({"k:bf16:w": {"bytes": 1234, "src": "kernel.cu", "sha": sha}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_peaks_file", lambda: str(table))
    assert bench._traffic("k", "bf16", "w") == 1234
    assert bench._traffic("k", "fp32", "w") is None                 # no capture for that path
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench._traffic("k", "bf16", "w") is None                 # source changed since the capture


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_parsed(tmp_path):
    path = tmp_path / "clocks.csv"
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    path.write_text("\n".join(rows) + "\n")
    s = bench.ClockSampler(0)
    s.path = str(path)
    s.proc = _Done()
    s.fh = open(tmp_path / "unused", "w")
    out = s.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    path.write_text("0, 1500, 2070, 700.0, 0x8, Active, Not Active, Not Active, Not Active\n")
    s.proc = _Done()
    s.fh = open(tmp_path / "unused", "w")
    assert s.stop()["reasons"] == ["hw_slowdown"]
