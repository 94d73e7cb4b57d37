"""Seeded synthetic inputs shaped like the paper's FDAS workloads.

This module is the only code shared by the CUDA path's tests, the benchmark and the CPU
oracle, and it holds none of the method's arithmetic: it only draws time series (Gaussian
noise plus injected accelerated signals), so that both sides see the same float32 input.

The paper's inputs (SIGPROC ``fake`` filterbanks and a GMRT observation) are not available;
these generators stand in for them.  Seeds follow ``20220624 + 1000 * config + series``
and every draw uses numpy's PCG64.

Signal model: phase in cycles phi(u) = phi0 + r0 u + z0 u^2 / 2 over u = t / T in [0, 1),
so r0 is the start frequency in Fourier bins and z0 = fdot T^2 the drift in bins over the
observation (Eq. fdotz: acceleration = z c / (f T^2)).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 20220624
C_LIGHT = 299_792_458.0


def seed_for(config_index: int, series_index: int = 0) -> int:
    return SEED_BASE + 1000 * int(config_index) + int(series_index)


def rng_for(config_index: int, series_index: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed_for(config_index, series_index)))


def noise(n: int, rng: np.random.Generator) -> np.ndarray:
    """Unit-variance white Gaussian noise, float64 (the caller casts once at the end)."""
    return rng.standard_normal(n)


def chirp(n: int, amp: float, r0: float, z0: float, phase: float = 0.0) -> np.ndarray:
    """amp * cos(2 pi (r0 u + z0 u^2 / 2) + phase), u = j / n, float64."""
    u = np.arange(n, dtype=np.float64) / n
    cyc = r0 * u + 0.5 * z0 * u * u
    cyc -= np.floor(cyc)
    return amp * np.cos(2.0 * np.pi * cyc + phase)


def pulse_train(n: int, r0: float, z0: float, duty: float, snr: float, phase0: float) -> np.ndarray:
    """Gaussian pulses (FWHM = duty x period) on the phase phi(u) = phase0 + r0 u + z0 u^2/2,
    mean removed and scaled so that sqrt(sum s_j^2) = snr in units of the noise sigma."""
    u = np.arange(n, dtype=np.float64) / n
    cyc = phase0 + r0 * u + 0.5 * z0 * u * u
    d = cyc - np.round(cyc)
    w = duty / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    s = np.exp(-0.5 * (d / w) ** 2)
    s -= s.mean()
    return s * (snr / math.sqrt(float(np.dot(s, s))))


def accel_to_z(accel: float, f: float, tobs: float) -> float:
    """Eq. fdotz inverted: z = a f T^2 / c."""
    return accel * f * tobs * tobs / C_LIGHT


def z_to_accel(z: float, f: float, tobs: float) -> float:
    """Eq. fdotz: a = z c / (f T^2)."""
    return z * C_LIGHT / (f * tobs * tobs)


@dataclasses.dataclass
class Train:
    period_s: float
    r0: float
    z0: float
    duty: float
    snr: float
    phase0: float


@dataclasses.dataclass
class Workload:
    """One series of a workload: its float32 samples and what was injected."""
    name: str
    n: int
    tsamp: float
    zmax: int
    taps: int
    seg_len: int
    series: np.ndarray
    trains: list
    max_harm: int = 1
    thr: tuple = (30.0, 30.0, 30.0, 30.0, 30.0)

    @property
    def nb(self) -> int:
        return self.n // 2

    @property
    def K(self) -> int:
        return self.zmax + 1


def single_chirp_workload(seed_config: int = 0, n: int = 1 << 16, amp: float = 0.05,
                          r0: float = 8000.3, z0: float = 6.2, zmax: int = 16, taps: int = 64,
                          seg_len: int = 1024, with_noise: bool = True) -> Workload:
    """Plain FP32 FDAS case: N = 2^16 N(0,1) samples plus one sinusoid of amplitude 0.05 at
    bin 8000.3 with z = +6.2; 17 templates (zmax 16), 64 taps, 1024-bin segments."""
    x = chirp(n, amp, r0, z0)
    if with_noise:
        x = x + noise(n, rng_for(seed_config, 0))
    return Workload("single_chirp_n65536_z16_m64_s1024", n, 1.0 / n, zmax, taps, seg_len,
                    x.astype(np.float32), [Train(0.0, r0, z0, 0.0, 0.0, 0.0)])


def draw_trains(rng: np.random.Generator, count: int, n: int, tsamp: float,
                zlim: float = 80.0, duty: float = 0.05, snr=(5.0, 30.0),
                period=(1e-3, 20e-3)) -> list:
    tobs = n * tsamp
    out = []
    for _ in range(count):
        p = math.exp(rng.uniform(math.log(period[0]), math.log(period[1])))
        out.append(Train(p, tobs / p, float(rng.uniform(-zlim, zlim)), duty,
                         float(rng.uniform(snr[0], snr[1])), float(rng.uniform(0.0, 1.0))))
    return out


def pulse_train_workload(config_index: int = 1, n: int = 1 << 23, tsamp: float = 64e-6,
                         n_trains: int = 8, zmax: int = 84, taps: int = 256,
                         seg_len: int = 8192, series_index: int = 0, zlim: float = 80.0,
                         duty: float = 0.05, snr=(5.0, 30.0)) -> Workload:
    """Precision case: N = 2^23 Gaussian-noise samples at 64 us with 8 injected pulse trains
    (period log-uniform 1-20 ms, 5% duty Gaussian pulses, z uniform in [-80, 80], per-train
    SNR 5-30); 85 templates (zmax 84), 256 taps, 8192-bin segments."""
    rng = rng_for(config_index, series_index)
    x = noise(n, rng)
    trains = draw_trains(rng, n_trains, n, tsamp, zlim=zlim, duty=duty, snr=snr)
    for t in trains:
        x += pulse_train(n, t.r0, t.z0, t.duty, t.snr, t.phase0)
    name = f"pulse_trains_n{n}_z{zmax}_m{taps}_s{seg_len}"
    return Workload(name, n, tsamp, zmax, taps, seg_len, x.astype(np.float32), trains)


def harmonic_shares(duty: float, h_max: int = 4096) -> np.ndarray:
    """Fraction of a Gaussian pulse train's power in each harmonic h = 1..h_max.

    The periodic Gaussian of width w (in cycles, FWHM = duty) has Fourier coefficients
    c_h ~ exp(-2 pi^2 h^2 w^2); with the mean removed, harmonic h carries c_h^2 / sum_h' c_h'^2
    of sum_j s_j^2 (Parseval).  Index 0 of the result is harmonic 1."""
    w = duty / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    h = np.arange(1, h_max + 1, dtype=np.float64)
    c2 = np.exp(-4.0 * math.pi ** 2 * h * h * w * w)
    return c2 / c2.sum()


@dataclasses.dataclass
class RefineWorkload:
    """Candidates seeded near the injected harmonics of a pulse-train series."""
    series: Workload
    truths: np.ndarray        # [T, 3]: r, z (start bin, drift in bins) and expected noiseless power
    seeds: np.ndarray         # [n_cand, 2]: r, z
    truth_index: np.ndarray   # [n_cand]: row of truths each seed belongs to


def refine_workload(config_index: int = 3, n: int = 1 << 23, tsamp: float = 64e-6, n_trains: int = 8,
                    zmax: int = 84, taps: int = 256, seg_len: int = 8192, n_cand: int = 100_000,
                    p_min: float = 30.0, series_index: int = 0) -> RefineWorkload:
    """Differentiation case: a series like the precision case (N = 2^23 at 64 us, 8 pulse trains,
    z in [-80, 80], SNR 5-30, 5% duty), and n_cand candidates seeded within half a bin in r and in z
    (uniform offsets) of the trains' harmonics (h r0, h z0).  Harmonics qualify when their
    expected noiseless power snr^2 * share_h is at least p_min, |h z0| <= zmax and the m-tap window
    stays inside the spectrum.  The first len(truths) seeds are the nearest integer bins of each
    truth; the rest pick a truth uniformly at random."""
    w = pulse_train_workload(config_index, n, tsamp, n_trains, zmax, taps, seg_len, series_index)
    nb = n // 2
    rows = []
    for t in w.trains:
        share = harmonic_shares(t.duty)
        for h in range(1, share.size + 1):
            p = t.snr ** 2 * share[h - 1]
            if p < p_min:
                break
            r, z = h * t.r0, h * t.z0
            if abs(z) <= zmax and taps <= r < nb - taps:
                rows.append((r, z, p))
    truths = np.array(rows, dtype=np.float64).reshape(-1, 3)
    rng = rng_for(config_index, 1000 + series_index)
    if truths.shape[0] == 0:
        return RefineWorkload(w, truths, np.zeros((0, 2)), np.zeros(0, dtype=np.int64))
    idx = rng.integers(0, truths.shape[0], n_cand)
    seeds = truths[idx, :2] + rng.uniform(-0.5, 0.5, (n_cand, 2))
    k = min(n_cand, truths.shape[0])
    idx[:k] = np.arange(k)
    seeds[:k] = np.round(truths[:k, :2])
    return RefineWorkload(w, truths, seeds, idx)


def noise_plane(K: int, nb: int, rng: np.random.Generator) -> np.ndarray:
    """A stand-in f-z plane for peak-search tests: K x nb independent exponential cells of mean 2
    (the chi^2, 2 dof law of noise-only plane cells), float32.  Callers plant signals on top."""
    return rng.exponential(2.0, size=(K, nb)).astype(np.float32)


BATCH_N = (1 << 21, 1 << 22, 1 << 23)
BATCH_ZMAX = (20, 50, 84)


def taps_for_zmax(zmax: int) -> int:
    """Smallest power-of-two tap count with m/2 >= zmax + 12 (the response of the largest drift
    plus its tails fits the window)."""
    m = 2
    while m // 2 < zmax + 12:
        m *= 2
    return m


@dataclasses.dataclass
class BatchWorkload:
    """Many dispersion-trial series of uneven length and zmax, packed back to back."""
    series: list              # Workload per series (series arrays not kept: see `packed`)
    packed: np.ndarray        # float32, all series concatenated
    offsets: np.ndarray       # int64 start of each series in `packed`

    @property
    def total_cells(self) -> int:
        return int(sum(w.K * w.nb for w in self.series))


def _batch_shapes(config_index, n_series, n_choices, zmax_choices):
    shapes = []
    for s in range(n_series):
        rng = rng_for(config_index, s)
        n = int(rng.choice(np.array(n_choices)))
        zmax = int(rng.choice(np.array(zmax_choices)))
        shapes.append((n, zmax))
    return shapes


def _batch_series(config_index, s, n_choices, zmax_choices, tsamp, max_trains, duty, snr, out):
    """Series s of a batch into `out` (float32, its length); returns its trains."""
    rng = rng_for(config_index, s)
    n = int(rng.choice(np.array(n_choices)))                 # the shape draws of _batch_shapes
    zmax = int(rng.choice(np.array(zmax_choices)))
    assert out.shape[0] == n
    out[:] = rng.standard_normal(n, dtype=np.float32)
    k = int(rng.integers(0, max_trains + 1))
    trains = draw_trains(rng, k, n, tsamp, zlim=0.95 * zmax, duty=duty, snr=snr)
    for t in trains:
        out += pulse_train(n, t.r0, t.z0, t.duty, t.snr, t.phase0).astype(np.float32)
    return trains


def _batch_worker(args):
    from multiprocessing import shared_memory
    shm_name, total, jobs = args
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        packed = np.ndarray((total,), dtype=np.float32, buffer=shm.buf)
        res = []
        for (config_index, s, nc, zc, tsamp, max_trains, duty, snr, off, n) in jobs:
            res.append((s, _batch_series(config_index, s, nc, zc, tsamp, max_trains, duty, snr,
                                         packed[off:off + n])))
        del packed
        return res
    finally:
        shm.close()


def batch_workload(config_index: int = 2, n_series: int = 256, tsamp: float = 64e-6, n_choices=BATCH_N,
                   zmax_choices=BATCH_ZMAX, max_trains: int = 2, duty: float = 0.05, snr=(5.0, 30.0),
                   seg_len: int = 8192, workers: int = 1, series=None) -> BatchWorkload:
    """Batching case: n_series series, each with N drawn from {2^21, 2^22, 2^23}, zmax from
    {20, 50, 84} (K = zmax + 1, taps from taps_for_zmax), 0 .. max_trains injected pulse trains
    (periods 1-20 ms, z uniform within 95% of the series' zmax, 5% duty, SNR 5-30), unit
    Gaussian noise, float32.  Series s draws from the generator seeded (config_index, s), so the
    result does not depend on `workers` (processes started with spawn, filling shared memory).
    `series` (optional): only these series indices of the n_series, packed in that order (one
    rank's share of a batch split over GPUs); each is the same as in the whole batch."""
    all_shapes = _batch_shapes(config_index, n_series, n_choices, zmax_choices)
    index = list(range(n_series)) if series is None else [int(s) for s in series]
    shapes = [all_shapes[s] for s in index]
    offsets = np.zeros(len(index), dtype=np.int64)
    o = 0
    for k, (n, _) in enumerate(shapes):
        offsets[k] = o
        o += n
    total = o
    jobs = [(config_index, s, tuple(n_choices), tuple(zmax_choices), tsamp, max_trains, duty, snr, int(offsets[k]), n)
            for k, (s, (n, zmax)) in enumerate(zip(index, shapes))]
    trains = {}
    if workers <= 1:
        packed = np.empty(total, dtype=np.float32)
        for j in jobs:
            trains[j[1]] = _batch_series(*j[:8], packed[j[8]:j[8] + j[9]])
    else:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        from multiprocessing import shared_memory
        shm = shared_memory.SharedMemory(create=True, size=4 * total)
        try:
            chunks = [(shm.name, total, jobs[w::workers]) for w in range(workers)]
            with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
                for res in ex.map(_batch_worker, chunks):
                    for s, tr in res:
                        trains[s] = tr
            packed = np.ndarray((total,), dtype=np.float32, buffer=shm.buf).copy()
        finally:
            shm.close()
            shm.unlink()
    meta = []
    for s, (n, zmax) in zip(index, shapes):
        m = taps_for_zmax(zmax)
        meta.append(Workload(f"batch{config_index}_s{s}_n{n}_z{zmax}_m{m}", n, tsamp, zmax, m, seg_len,
                             np.empty(0, dtype=np.float32), trains[s]))
    return BatchWorkload(meta, packed, offsets)


def sensitivity_workload(config_index: int = 4, series_index: int = 0, n: int = 1 << 23, tsamp: float = 64e-6,
                         period=(1e-3, 20e-3), accel=(-200.0, 200.0), duty=(0.02, 0.10), snr=(3.0, 40.0),
                         zmax: int = 84, taps: int = 256, seg_len: int = 8192) -> Workload:
    """Sensitivity case: one binary pulsar per series (period log-uniform 1-20 ms, line-of-sight
    acceleration uniform in +-200 m/s^2, so z = a f T^2 / c can exceed zmax; duty cycle 2-10 %;
    SNR 3-40) in unit Gaussian noise, N = 2^23 at 64 us, 85 templates.  The one train's r0 is its
    fundamental frequency in bins, f = r0 / T."""
    rng = rng_for(config_index, series_index)
    tobs = n * tsamp
    p = math.exp(rng.uniform(math.log(period[0]), math.log(period[1])))
    f = 1.0 / p
    z = accel_to_z(float(rng.uniform(accel[0], accel[1])), f, tobs)
    d = float(rng.uniform(duty[0], duty[1]))
    t = Train(p, tobs / p, z, d, float(rng.uniform(snr[0], snr[1])), float(rng.uniform(0.0, 1.0)))
    x = rng.standard_normal(n, dtype=np.float32)
    x += pulse_train(n, t.r0, t.z0, t.duty, t.snr, t.phase0).astype(np.float32)
    return Workload(f"sensitivity{config_index}_s{series_index}_n{n}", n, tsamp, zmax, taps, seg_len, x, [t])
