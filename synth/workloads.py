"""Synthetic OVRO-LWA-like workloads (inputs only).

Random numbers come from NumPy's Philox counter-based bit generator
(Salmon et al. 2011, Philox-4x64-10), keyed per sub-stream by SplitMix64
(Steele, Lea & Flood 2014) so that any (config, coarse channel, time block)
slice can be regenerated on its own.  Noise-only voltages are drawn with
integer arithmetic only (inverse-CDF thresholds on 32-bit uniforms), so the
bytes are identical on every host.

Array model (the paper's Section 2.1 and the OVRO-LWA description in Section 1):
352 dual-polarisation antennas, ~24 kHz complex coarse channels from the
F-engine, 4+4-bit two's-complement samples.  The sky model for a tone is a
plane wave from direction (l, m): antenna a sees
``A exp(i phi(t)) exp(-2 pi i nu (x_a l + y_a m) / c)``, so visibilities carry
``exp(-2 pi i (u l + v m))`` and an ``exp(+...)`` imaging transform peaks at
(l, m).
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

C_LIGHT = 299_792_458.0          # m/s
F_COARSE_HZ = 24_000.0           # coarse-channel width and complex sample rate
NU0_HZ = 60.0e6                  # sky frequency of coarse channel 0 (inside 50-86 MHz)
SIGMA_LEVELS = 2.0               # Gaussian noise per component, in 4-bit levels

_MASK64 = (1 << 64) - 1

# P(N(0, 2^2) < k + 1/2) * 2^32, rounded, for k = -7..6: the boundaries of the
# 15 levels of a Gaussian (sigma = 2) rounded half away from zero and clipped
# to [-7, 7].  tests/test_synth.py re-derives them from scipy.special.ndtr.
NOISE_THRESHOLDS_U32 = np.array(
    [2478304, 12797986, 52503710, 172052769, 453762323, 973357067,
     1723543207, 2571424089, 3321610229, 3841204973, 4122914527,
     4242463586, 4282169310, 4292488992], dtype=np.uint32)


def splitmix64(x: int) -> int:
    """One SplitMix64 output for state ``x`` (Steele, Lea & Flood 2014)."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def substream(seed: int, *tags: int) -> np.random.Generator:
    """Independent Philox generator for (seed, tag, tag, ...)."""
    k = splitmix64(seed & _MASK64)
    for t in tags:
        k = splitmix64(k ^ (int(t) & _MASK64))
    k2 = splitmix64(k ^ 0x5851F42D4C957F2D)
    return np.random.Generator(np.random.Philox(key=(k2 << 64) | k))


@dataclass
class Tone:
    """A narrowband plane-wave emitter injected before 4-bit quantisation."""
    coarse: int          # coarse channel index
    fine: int            # fine channel (post-fftshift index) it is centred in at t = 0
    row: int             # sky pixel it is centred on (for the config's default image)
    col: int
    amp: float           # amplitude per component, in 4-bit levels (pre-quantisation)
    phase: float = 0.0   # radians
    drift_hz_s: float = 0.0
    snr_target: float = 0.0


@dataclass
class Burst:
    """Broadband radio-frequency interference: a point source of complex white
    noise (all fine channels) switched on for a fraction of a second."""
    coarse: int
    t0_s: float
    dur_s: float
    row: int
    col: int
    amp: float           # rms amplitude per component, 4-bit levels


@dataclass
class Config:
    name: str
    n_ant: int
    n_coarse: int
    nfft: List[int]
    n_time: int
    image_size: int
    seed: int
    core_ant: int = 0                 # antennas in the core disk (rest in the annulus)
    core_radius_m: float = 200.0
    outer_radius_m: float = 1500.0
    cell_dircos: float = 0.0          # 0 -> all-sky default 2 / image_size
    tones: List[Tone] = field(default_factory=list)
    carriers: List[Tone] = field(default_factory=list)   # stationary CW tones at the horizon (RFI)
    bursts: List[Burst] = field(default_factory=list)

    @property
    def n_input(self) -> int:
        return 2 * self.n_ant

    @property
    def n_spec(self) -> List[int]:
        return [self.n_time // n for n in self.nfft]

    @property
    def cell(self) -> float:
        return self.cell_dircos if self.cell_dircos > 0 else 2.0 / self.image_size

    @property
    def n_chan_total(self) -> int:
        return int(sum(self.nfft))

    def describe(self) -> dict:
        d = dataclasses.asdict(self)
        d["tones"] = len(self.tones)
        d["carriers"] = len(self.carriers)
        d["bursts"] = len(self.bursts)
        return d


def coarse_centre_hz(c: int) -> float:
    """Sky frequency at the centre of coarse channel ``c``."""
    return NU0_HZ + c * F_COARSE_HZ


def fine_freqs_hz(nfft: Sequence[int]) -> np.ndarray:
    """Sky frequency of every fine channel, coarse-major, fftshifted order.

    Fine channel k' of an N-point upchannelizer in coarse channel c sits at
    nu_c + (k' - N/2) * f_c / N.
    """
    out = []
    for c, n in enumerate(nfft):
        k = np.arange(n, dtype=np.float64)
        out.append(coarse_centre_hz(c) + (k - n / 2) * (F_COARSE_HZ / n))
    return np.concatenate(out)


def antenna_positions(cfg: Config) -> np.ndarray:
    """ENU positions [n_ant][3] in metres, uniform in area, planar (z = 0)."""
    g = substream(cfg.seed, 1)
    n_core = cfg.core_ant if cfg.core_ant > 0 else cfg.n_ant
    n_out = cfg.n_ant - n_core
    r = np.empty(cfg.n_ant)
    r[:n_core] = np.sqrt(g.uniform(0.0, cfg.core_radius_m ** 2, n_core))
    if n_out:
        r[n_core:] = np.sqrt(g.uniform(cfg.core_radius_m ** 2, cfg.outer_radius_m ** 2, n_out))
    th = g.uniform(0.0, 2 * np.pi, cfg.n_ant)
    pos = np.zeros((cfg.n_ant, 3))
    pos[:, 0] = r * np.cos(th)
    pos[:, 1] = r * np.sin(th)
    return pos


def pack_nibbles(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """F-engine byte format: real part in the high nibble, imaginary in the low
    nibble, each 4-bit two's complement."""
    r = np.asarray(re, dtype=np.int8).view(np.uint8)
    i = np.asarray(im, dtype=np.int8).view(np.uint8)
    return ((r & np.uint8(0xF)) << np.uint8(4)) | (i & np.uint8(0xF))


def _noise_levels(g: np.random.Generator, n: int) -> np.ndarray:
    """n quantised Gaussian levels from n 32-bit uniforms (two per raw draw)."""
    raw = g.bit_generator.random_raw((n + 1) // 2)
    u = raw.astype("<u8", copy=False).view("<u4")[:n]
    lev = np.searchsorted(NOISE_THRESHOLDS_U32, u, side="right")
    return lev.astype(np.int8) - np.int8(7)


def _quantise(x: np.ndarray) -> np.ndarray:
    """Round half away from zero, clip to [-7, 7]."""
    q = np.sign(x) * np.floor(np.abs(x) + 0.5)
    return np.clip(q, -7, 7).astype(np.int8)


def pfb_prototype(nfft: int, n_taps: int) -> np.ndarray:
    """A P-tap polyphase-filter-bank prototype for N fine channels: a sinc one
    fine channel wide under a Hann taper, P N coefficients, FP32.  An input for
    the PFB upchannelizer option (any real P N coefficients are valid)."""
    m = np.arange(nfft * n_taps, dtype=np.float64) + 0.5
    t = m / nfft - n_taps / 2.0
    taper = 0.5 - 0.5 * np.cos(2.0 * np.pi * m / (nfft * n_taps))
    return (np.sinc(t) * taper).astype(np.float32)


def pixel_dircos(row: int, col: int, image_size: int, cell: float):
    return (col - image_size // 2) * cell, (row - image_size // 2) * cell


def generate(cfg: Config, coarse: Optional[Sequence[int]] = None,
             time_block: int = 1 << 15) -> np.ndarray:
    """4+4-bit voltages, uint8 [n_coarse][n_time][n_input], input = 2*ant + pol.

    Noise-only coarse channels use the integer-only quantised-Gaussian draw.
    Coarse channels with tones draw continuous Gaussian noise, add the tones,
    then quantise (round half away from zero, clip [-7, 7]).
    """
    coarse = list(range(cfg.n_coarse)) if coarse is None else list(coarse)
    pos = antenna_positions(cfg)
    out = np.empty((len(coarse), cfg.n_time, cfg.n_input), dtype=np.uint8)
    for ci, c in enumerate(coarse):
        tones = [t for t in cfg.tones + cfg.carriers if t.coarse == c]
        bursts = [b for b in cfg.bursts if b.coarse == c]
        for t0 in range(0, cfg.n_time, time_block):
            nt = min(time_block, cfg.n_time - t0)
            g = substream(cfg.seed, 2, c, t0 // time_block)
            if not tones and not bursts:
                re = _noise_levels(g, nt * cfg.n_input)
                im = _noise_levels(g, nt * cfg.n_input)
                out[ci, t0:t0 + nt] = pack_nibbles(re, im).reshape(nt, cfg.n_input)
                continue
            xr = g.standard_normal((nt, cfg.n_input)) * SIGMA_LEVELS
            xi = g.standard_normal((nt, cfg.n_input)) * SIGMA_LEVELS
            tt = (t0 + np.arange(nt, dtype=np.float64)) / F_COARSE_HZ
            n = cfg.nfft[c]
            # every source is rank one in (time, input): a time series times a
            # per-antenna geometric phasor, so the block is one complex product
            et, ga = [], []
            for tone in tones:
                f0 = (tone.fine - n / 2) * (F_COARSE_HZ / n)          # baseband Hz
                nu = coarse_centre_hz(c) + f0
                l0, m0 = pixel_dircos(tone.row, tone.col, cfg.image_size, cfg.cell)
                geo = -2 * np.pi * nu * (pos[:, 0] * l0 + pos[:, 1] * m0) / C_LIGHT
                ph_t = 2 * np.pi * (f0 * tt + 0.5 * tone.drift_hz_s * tt * tt) + tone.phase
                et.append(tone.amp * np.exp(1j * ph_t))
                ga.append(np.exp(1j * np.repeat(geo, 2)))
            for bi, burst in enumerate(bursts):
                on = (tt >= burst.t0_s) & (tt < burst.t0_s + burst.dur_s)
                if not on.any():
                    continue
                gb = substream(cfg.seed, 5, c, bi, t0 // time_block)
                sig = np.zeros(nt, dtype=np.complex128)
                k = int(on.sum())
                sig[on] = (gb.standard_normal(k) + 1j * gb.standard_normal(k)) * burst.amp
                l0, m0 = pixel_dircos(burst.row, burst.col, cfg.image_size, cfg.cell)
                geo = -2 * np.pi * coarse_centre_hz(c) * (pos[:, 0] * l0 + pos[:, 1] * m0) / C_LIGHT
                et.append(sig)
                ga.append(np.exp(1j * np.repeat(geo, 2)))
            if et:
                inj = np.stack(et, axis=1) @ np.stack(ga, axis=0)        # [nt][n_input]
                xr += inj.real
                xi += inj.imag
            out[ci, t0:t0 + nt] = pack_nibbles(_quantise(xr), _quantise(xi))
    return out


def tone_amplitude(snr: float, nfft: int, n_spec: int, n_bl: int) -> float:
    """Amplitude whose image-plane SNR is about ``snr`` (radiometer estimate).

    Per fine channel a tone of amplitude A gives N A^2 signal power against
    2 sigma^2 noise power per sample; averaging K spectra over n_bl baselines
    and two polarisations gives SNR ~ (N A^2 / 2 sigma^2) sqrt(2 K n_bl).
    """
    return math.sqrt(snr * 2 * SIGMA_LEVELS ** 2 / (nfft * math.sqrt(2 * n_spec * n_bl)))


def _seeded_tones(cfg: Config, n: int, snr_lo: float, snr_hi: float,
                  drift_hi: float, r2_max: float = 0.6) -> List[Tone]:
    g = substream(cfg.seed, 3)
    tones = []
    n_bl = cfg.n_ant * (cfg.n_ant - 1) // 2
    N = cfg.image_size
    while len(tones) < n:
        c = int(g.integers(0, cfg.n_coarse))
        nf = cfg.nfft[c]
        fine = int(g.integers(nf // 8, nf - nf // 8))
        row = int(g.integers(0, N))
        col = int(g.integers(0, N))
        l0, m0 = pixel_dircos(row, col, N, cfg.cell)
        if l0 * l0 + m0 * m0 > r2_max:
            continue
        snr = float(g.uniform(snr_lo, snr_hi))
        amp = tone_amplitude(snr, nf, cfg.n_time // nf, n_bl)
        tones.append(Tone(c, fine, row, col, amp, float(g.uniform(0, 2 * np.pi)),
                          float(g.uniform(0.0, drift_hi)) if drift_hi > 0 else 0.0, snr))
    return tones


def _add_rfi(cfg: Config, n_carriers: int, n_bursts: int):
    """Stationary CW carriers just above the horizon and broadband bursts."""
    g = substream(cfg.seed, 6)
    N = cfg.image_size
    n_bl = cfg.n_ant * (cfg.n_ant - 1) // 2
    while len(cfg.carriers) < n_carriers:
        row, col = int(g.integers(0, N)), int(g.integers(0, N))
        l0, m0 = pixel_dircos(row, col, N, cfg.cell)
        if not (0.95 <= l0 * l0 + m0 * m0 < 1.0):
            continue
        c = int(g.integers(0, cfg.n_coarse))
        nf = cfg.nfft[c]
        snr = float(g.uniform(8.0, 30.0))
        cfg.carriers.append(Tone(c, int(g.integers(nf // 8, nf - nf // 8)), row, col,
                                 tone_amplitude(snr, nf, cfg.n_time // nf, n_bl),
                                 float(g.uniform(0, 2 * np.pi)), 0.0, snr))
    T = cfg.n_time / F_COARSE_HZ
    while len(cfg.bursts) < n_bursts:
        row, col = int(g.integers(0, N)), int(g.integers(0, N))
        l0, m0 = pixel_dircos(row, col, N, cfg.cell)
        if l0 * l0 + m0 * m0 > 0.8:
            continue
        dur = float(g.uniform(0.2, 1.0))
        cfg.bursts.append(Burst(int(g.integers(0, cfg.n_coarse)), float(g.uniform(0, T - dur)), dur, row, col,
                                float(g.uniform(0.6, 1.5))))


SEED_BASE = 20240406


def make_config(name: str, **over) -> Config:
    """The five workloads, by what they are.

    tiny      16 antennas in a 200 m disk, 2 coarse x 256-pt, K = 64, 64^2 images, 1 tone
    full      352 antennas (251 in a 200 m core, 101 in a 200 m-1.5 km annulus),
              1 coarse x 8192-pt, 10 s (K = 29), 256^2 images, noise only
    batched   352 antennas, 32 coarse channels with N in {1024, 4096, 16384} by seed,
              10 s, 256^2 images, 20 tones SNR 5-30, drift 0-0.5 Hz/s
    precision 352 antennas, 4 coarse x 4096-pt (K = 58), 1024^2 grids
    scorer    352 antennas, 8 coarse x 8192-pt, 256^2, tones SNR 4-20, drift 0-1 Hz/s
    """
    idx = {"tiny": 0, "full": 1, "batched": 2, "precision": 3, "scorer": 4, "scorer_train": 5}[name]
    seed = SEED_BASE + idx
    if name == "tiny":
        cfg = Config(name, 16, 2, [256, 256], 64 * 256, 64, seed)
    elif name == "full":
        cfg = Config(name, 352, 1, [8192], 240_000, 256, seed, core_ant=251)
    elif name == "batched":
        g = substream(seed, 4)
        nf = [int(x) for x in g.choice([1024, 4096, 16384], size=32)]
        cfg = Config(name, 352, 32, nf, 240_000, 256, seed, core_ant=251)
    elif name == "precision":
        cfg = Config(name, 352, 4, [4096] * 4, 240_000, 1024, seed, core_ant=251)
    elif name == "scorer":
        cfg = Config(name, 352, 8, [8192] * 8, 240_000, 256, seed, core_ant=251)
    else:
        # a compact 64-antenna array whose baselines all fit the 128^2 all-sky grid
        cfg = Config(name, 64, 2, [2048, 2048], 240_000, 128, seed, core_radius_m=70.0)
    n_tones = over.pop("n_tones", None)
    for k, v in over.items():
        setattr(cfg, k, v)
    if name == "tiny":
        cfg.tones = _seeded_tones(cfg, 1 if n_tones is None else n_tones, 30.0, 30.0, 0.0, 0.3)
    elif name == "batched":
        cfg.tones = _seeded_tones(cfg, 20 if n_tones is None else n_tones, 5.0, 30.0, 0.5)
    elif name == "scorer":
        cfg.tones = _seeded_tones(cfg, 64 if n_tones is None else n_tones, 4.0, 20.0, 1.0)
        _add_rfi(cfg, 16, 16)
    elif name == "scorer_train":
        cfg.tones = _seeded_tones(cfg, 24 if n_tones is None else n_tones, 4.0, 20.0, 1.0)
        _add_rfi(cfg, 8, 6)
    elif n_tones:
        cfg.tones = _seeded_tones(cfg, n_tones, 10.0, 30.0, 0.0)
    return cfg


CONFIGS = ("tiny", "full", "batched", "precision", "scorer", "scorer_train")


def _generate_one(args):
    cfg, c = args
    return generate(cfg, coarse=[c])[0]


def generate_parallel(cfg: Config, workers: Optional[int] = None) -> np.ndarray:
    """generate(cfg) with the coarse channels drawn in parallel (spawned
    processes; every slice comes from its own counter-based substreams, so the
    bytes are those of generate)."""
    import multiprocessing as mp
    import os
    workers = workers or min(cfg.n_coarse, os.cpu_count() or 1)
    if workers <= 1 or cfg.n_coarse == 1:
        return generate(cfg)
    out = np.empty((cfg.n_coarse, cfg.n_time, cfg.n_input), dtype=np.uint8)
    with mp.get_context("spawn").Pool(workers) as pool:
        for c, v in enumerate(pool.imap(_generate_one, [(cfg, c) for c in range(cfg.n_coarse)])):
            out[c] = v
    return out
