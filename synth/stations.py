"""Station data generator: geometry, noise, dispersed pulses (inputs only).

Input recipe (stated again in the design notes):
  * stations uniform in a disk of 1 km radius (the paper's ~2 km dense core),
    local ENU metres, z = 0;
  * pointing azimuth 180 deg, elevation 45 deg; beams are the points of a
    hexagonal grid of 0.06 deg spacing in the tangent plane nearest to it;
  * noise: per (seed, block, pol, subband) slab, Philox bits -> 16-bit index ->
    table of rounded Gaussian quantiles (sigma given, clipped to the dtype);
  * pulses: a real delta of amplitude a at baseband sample n0, dispersed by the
    ionosphere (group delay A / nu^2) and analysed by a forward 1024-point,
    16-tap Kaiser-sinc PPF; every station sees it with its plane-wave phase
    from the pulse direction.  Amplitude from a nominal SNR (see ``pulse_amplitude``).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.special import ndtri

__all__ = [
    "station_groups",
    "Workload", "TINY", "FULLBAND", "PRECISION", "SERVING", "STRESS", "WORKLOADS",
    "station_positions", "pointing_enu", "hex_beam_directions", "gaussian_table",
    "noise_slab", "analysis_filter", "forward_ppf", "dispersed_pulse",
    "pulse_amplitude", "pulse_subbands", "Pulse", "make_geometry", "make_block",
    "SAMPLE_RATE_HZ", "FFT_LEN", "device_noise_block", "pulse_contributions",
]

SAMPLE_RATE_HZ = 200e6
FFT_LEN = 1024
N_TAPS = 16
_NU0 = SAMPLE_RATE_HZ / 2          # sky frequency of bin 0 (second Nyquist zone)
_C = 299792458.0
_KAPPA = 40.308                    # m^3 s^-2
_TECU = 1e16


@dataclass(frozen=True)
class Workload:
    """One synthetic workload: shapes, dtype, noise level, pulses, seed."""
    name: str
    stations: int
    pols: int
    subbands: int
    first_bin: int
    beams: int
    tec_trials: tuple
    block_len: int
    dtype: str
    noise_sigma: float
    n_pulses: int = 0
    snr_range: tuple = (10.0, 10.0)
    pulse_tec_range: tuple = (10.0, 10.0)
    precision: str = "fp32"
    seed: int = 1

    @property
    def n_streams(self) -> int:
        return self.beams * len(self.tec_trials) * self.pols

    @property
    def input_bytes(self) -> int:
        return (self.pols * self.subbands * self.block_len * self.stations * 2
                * (1 if self.dtype == "int8" else 2))


# 6 stations, 16 subbands from 130 MHz, 1 beam, 4096 frames, int16 sigma 8,
# one pulse at TEC 10 and SNR 10, plain FP32 path.
TINY = Workload("tiny-6st-16sb-1bm-4096fr-int16-fp32", 6, 2, 16, 154, 1, (10.0,),
                4096, "int16", 8.0, 1, (10.0, 10.0), (10.0, 10.0), "fp32", 1)
# 24 stations, 244 subbands 110-157.6 MHz, 1 beam, 65536 frames, int16 sigma 16,
# 20 pulses TEC U(5,30) SNR U(4,20), one trial at 17.5 TECU, plain FP32 path.
FULLBAND = Workload("fullband-24st-244sb-1bm-65536fr-int16-fp32", 24, 2, 244, 52, 1,
                    (17.5,), 65536, "int16", 16.0, 20, (4.0, 20.0), (5.0, 30.0),
                    "fp32", 2)
# 48 stations, 488 subbands, 50 beams (0.5 deg disk), 65536 frames, int8 sigma 4,
# FP16 tensor-core beamformer; no pulses.
PRECISION = Workload("precision-48st-488sb-50bm-65536fr-int8-fp16", 48, 2, 488, 12, 50,
                     (20.0,), 65536, "int8", 4.0, 0, (10.0, 10.0), (10.0, 10.0),
                     "fp16", 3)
# Serving loop: same station stream as PRECISION, requests vary per block.
SERVING = Workload("serving-48st-488sb-65536fr-int8", 48, 2, 488, 12, 50,
                   (5.0, 15.0, 25.0, 35.0), 65536, "int8", 4.0, 0, (10.0, 10.0),
                   (5.0, 40.0), "fp16", 4)
# Stress: 200 beams x 8 trials, 262144 frames, 200 pulses.
STRESS = Workload("stress-48st-488sb-200bm-8tec-262144fr-int8", 48, 2, 488, 12, 200,
                  (5.0, 10.0, 15.0, 20.0, 25.0, 30.0, 35.0, 40.0), 262144, "int8", 4.0,
                  200, (5.0, 20.0), (5.0, 40.0), "fp16", 5)
WORKLOADS = {w.name: w for w in (TINY, FULLBAND, PRECISION, SERVING, STRESS)}


# ----------------------------------------------------------------------------
# Geometry
# ----------------------------------------------------------------------------

def _rng(*key: int) -> np.random.Generator:
    k = np.array([int(v) & 0xFFFFFFFFFFFFFFFF for v in key] + [0] * (2 - len(key)),
                 dtype=np.uint64)
    if k.size > 2:
        # fold extra words into the second key word
        acc = int(k[1])
        for v in k[2:]:
            acc = (acc * 0x9E3779B97F4A7C15 + int(v)) & 0xFFFFFFFFFFFFFFFF
        k = np.array([k[0], acc], dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=k))


def station_positions(n: int, seed: int, radius_m: float = 1000.0) -> np.ndarray:
    """n station positions uniform in a disk (ENU metres, z = 0), [n, 3]."""
    rng = _rng(seed, 0x57A7)
    r = radius_m * np.sqrt(rng.random(n))
    phi = 2 * np.pi * rng.random(n)
    return np.stack([r * np.cos(phi), r * np.sin(phi), np.zeros(n)], axis=1)


def pointing_enu(az_deg: float = 180.0, el_deg: float = 45.0) -> np.ndarray:
    """Unit vector toward azimuth/elevation in ENU (azimuth from north to east)."""
    az, el = np.radians(az_deg), np.radians(el_deg)
    return np.array([np.sin(az) * np.cos(el), np.cos(az) * np.cos(el), np.sin(el)])


def hex_beam_directions(n_beams: int, spacing_deg: float = 0.06,
                        az_deg: float = 180.0, el_deg: float = 45.0) -> np.ndarray:
    """n_beams unit vectors on a hexagonal grid around the pointing, [n, 3].

    Grid points (l, m) = spacing * (i + j/2, j sqrt(3)/2) in the tangent plane;
    the n nearest to the centre are kept (ties broken by position angle).
    """
    s0 = pointing_enu(az_deg, el_deg)
    e1 = np.cross([0.0, 0.0, 1.0], s0)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(s0, e1)
    r = int(np.ceil(np.sqrt(n_beams))) + 2
    pts = []
    for j in range(-r, r + 1):
        for i in range(-r, r + 1):
            l = i + 0.5 * j
            m = j * np.sqrt(3) / 2
            pts.append((l * l + m * m, np.arctan2(m, l) % (2 * np.pi), l, m))
    pts.sort()
    sp = np.radians(spacing_deg)
    out = []
    for _, _, l, m in pts[:n_beams]:
        v = s0 + sp * l * e1 + sp * m * e2
        out.append(v / np.linalg.norm(v))
    return np.array(out)


def station_groups(station_enu: np.ndarray, n_groups: int, iters: int = 50) -> np.ndarray:
    """Compact disjoint station groups for two-stage beamforming, [S] group index.

    Lloyd's k-means on the ENU positions, started from the farthest-point
    sequence beginning at the station nearest the array centre (deterministic);
    ties go to the lower group index.  Input geometry only: the pipeline and the
    oracle take any grouping.
    """
    r = np.asarray(station_enu, dtype=np.float64)
    first = int(np.argmin(np.linalg.norm(r - r.mean(axis=0), axis=1)))
    seeds = [first]
    dist = np.linalg.norm(r - r[first], axis=1)
    while len(seeds) < n_groups:
        nxt = int(np.argmax(dist))
        seeds.append(nxt)
        dist = np.minimum(dist, np.linalg.norm(r - r[nxt], axis=1))
    centres = r[seeds].copy()
    grp = np.zeros(r.shape[0], dtype=np.int32)
    for _ in range(iters):
        d2 = ((r[:, None, :] - centres[None, :, :]) ** 2).sum(axis=2)
        new = np.argmin(d2, axis=1).astype(np.int32)
        for g in range(n_groups):
            if not np.any(new == g):          # keep every group populated
                new[int(np.argmin(d2[:, g]))] = g
        if np.array_equal(new, grp) and _ > 0:
            break
        grp = new
        centres = np.stack([r[grp == g].mean(axis=0) for g in range(n_groups)])
    return grp


def make_geometry(w: Workload):
    """(station_enu [S,3], beam_dir [B,3], tec [Tr]) of a workload."""
    if w.beams == 1:
        beams = pointing_enu()[None, :]
    else:
        beams = hex_beam_directions(w.beams)
    return station_positions(w.stations, w.seed), beams, np.array(w.tec_trials, dtype=np.float64)


# ----------------------------------------------------------------------------
# Noise
# ----------------------------------------------------------------------------

def gaussian_quantiles(sigma: float) -> np.ndarray:
    """65536 Gaussian quantiles sigma * Phi^-1((i + 1/2) / 65536) (continuous)."""
    q = (np.arange(65536, dtype=np.float64) + 0.5) / 65536.0
    return sigma * ndtri(q)


def gaussian_table(sigma: float, dtype: str) -> np.ndarray:
    """The quantiles rounded and clipped to the sample type (noise-only samples)."""
    info = np.iinfo(np.dtype(dtype))
    return np.clip(np.rint(gaussian_quantiles(sigma)), info.min, info.max).astype(dtype)


_TABLES: dict = {}


def _noise_index(seed, block, pol, k, frames, stations):
    rng = _rng(seed, block, pol, k)
    return np.frombuffer(rng.bytes(frames * stations * 2 * 2), dtype=np.uint16)


def noise_slab(seed: int, block: int, pol: int, k: int, frames: int, stations: int,
               sigma: float, dtype: str) -> np.ndarray:
    """Integer noise of one (pol, subband) slab, [frames, stations, 2]."""
    key = (sigma, dtype)
    if key not in _TABLES:
        _TABLES[key] = gaussian_table(sigma, dtype)
    idx = _noise_index(seed, block, pol, k, frames, stations)
    return _TABLES[key][idx].reshape(frames, stations, 2)


def noisy_slab(seed: int, block: int, pol: int, k: int, frames: int, stations: int,
               sigma: float, dtype: str, adds) -> np.ndarray:
    """One slab of continuous Gaussian noise plus signal, rounded and clipped
    to the sample type (the station's quantiser).  adds: list of (m_lo, m_hi,
    complex [m_hi - m_lo, stations]) signal contributions of this subband.
    Without signal it equals ``noise_slab``."""
    key = ("q", sigma)
    if key not in _TABLES:
        _TABLES[key] = gaussian_quantiles(sigma)
    idx = _noise_index(seed, block, pol, k, frames, stations)
    v = _TABLES[key][idx].reshape(frames, stations, 2)
    for (m_lo, m_hi, c) in adds:
        v[m_lo:m_hi, :, 0] += c.real
        v[m_lo:m_hi, :, 1] += c.imag
    info = np.iinfo(np.dtype(dtype))
    return np.clip(np.rint(v), info.min, info.max).astype(dtype)


# ----------------------------------------------------------------------------
# Pulses (the station's analysis filter bank is the generator's, not the pipeline's)
# ----------------------------------------------------------------------------

def analysis_filter(m: int = FFT_LEN, taps: int = N_TAPS, beta: float = 9.0) -> np.ndarray:
    """Station PPF prototype: numpy's Kaiser window times numpy's sinc, sum 1."""
    L = m * taps
    n = np.arange(L, dtype=np.float64)
    h = np.sinc((n - (L - 1) / 2.0) / m) * np.kaiser(L, beta)
    return h / h.sum()


def forward_ppf(x: np.ndarray, n_start: int, m_lo: int, m_hi: int, bins: np.ndarray,
                h: np.ndarray) -> np.ndarray:
    """Forward PPF of a real series x (x[i] is sample n_start + i, zero elsewhere).

    Frame m covers samples [(m-15) M, (m+1) M):
        v_m[p] = sum_t h[t M + p] x[(m - 15 + t) M + p],
        X_m[k] = sum_p v_m[p] exp(-2 pi i k p / M).
    Returns complex [m_hi - m_lo, len(bins)].
    """
    Mm = FFT_LEN
    taps = h.size // Mm
    out = np.zeros((m_hi - m_lo, bins.size), dtype=np.complex128)
    hh = h.reshape(taps, Mm)
    for i, m in enumerate(range(m_lo, m_hi)):
        n0 = (m - (taps - 1)) * Mm
        seg = np.zeros(taps * Mm)
        a, b = max(n0, n_start), min(n0 + taps * Mm, n_start + x.size)
        if a >= b:
            continue
        seg[a - n0:b - n0] = x[a - n_start:b - n_start]
        v = (hh * seg.reshape(taps, Mm)).sum(axis=0)
        out[i] = np.fft.fft(v)[bins]
    return out


def dispersed_pulse(n_len: int, n0_local: int, amp: float, tec_tecu: float) -> np.ndarray:
    """Real baseband series: delta a at n0_local, dispersed by exp(+2 pi i A / nu)."""
    f = np.fft.rfftfreq(n_len, d=1.0 / SAMPLE_RATE_HZ)
    nu = _NU0 + f
    a_hz = _KAPPA * tec_tecu * _TECU / _C
    spec = amp * np.exp(-2j * np.pi * f * n0_local / SAMPLE_RATE_HZ)
    spec = spec * np.exp(2j * np.pi * a_hz / nu)
    spec[0] = 0.0
    spec[-1] = 0.0
    return np.fft.irfft(spec, n_len)


def pulse_amplitude(snr: float, w: Workload, h: np.ndarray | None = None) -> float:
    """Delta amplitude a for a nominal SNR.

    Nominal SNR := peak envelope of the undispersed, coherently beamformed pulse
    band-limited to the K selected subbands (S * 2 a K / M) divided by the
    noise standard deviation of the synthesized series,
    sigma_y^2 = 4 K S sigma^2 M sum(h^2) (sigma the per-component station noise).
    """
    if h is None:
        h = analysis_filter()
    sig_y = np.sqrt(4.0 * w.subbands * w.stations * w.noise_sigma ** 2
                    * FFT_LEN * float(np.sum(h * h)))
    return snr * sig_y * FFT_LEN / (2.0 * w.subbands * w.stations)


@dataclass
class Pulse:
    n0: int            # global baseband sample of the undispersed delta
    amp: float
    tec: float
    snr: float
    beam: int          # beam index whose direction the pulse comes from
    frames: tuple = field(default=(0, 0))


def pulse_subbands(p: Pulse, w: Workload, h: np.ndarray, block: int):
    """Subband frames of one pulse inside block ``block``: (m_lo, m_hi, X [n, K])."""
    n_len = 1 << 16
    start = p.n0 - n_len // 2
    x = dispersed_pulse(n_len, n_len // 2, p.amp, p.tec)
    bins = np.arange(w.first_bin, w.first_bin + w.subbands)
    g_lo = (start // FFT_LEN)
    g_hi = (start + n_len) // FFT_LEN + N_TAPS
    b0 = block * w.block_len
    m_lo = max(g_lo, b0)
    m_hi = min(g_hi, b0 + w.block_len)
    if m_lo >= m_hi:
        return m_lo, m_lo, np.zeros((0, w.subbands), np.complex128)
    return m_lo - b0, m_hi - b0, forward_ppf(x, start, m_lo, m_hi, bins, h)


def _draw_pulses(w: Workload, block: int):
    rng = _rng(w.seed, block, 0x9015E)
    pulses = []
    margin = 32
    for i in range(w.n_pulses):
        m = int(rng.integers(margin, w.block_len - margin))
        frame = block * w.block_len + m
        n0 = (frame - (N_TAPS - 1)) * FFT_LEN + int(rng.integers(0, FFT_LEN))
        snr = float(rng.uniform(*w.snr_range))
        tec = float(rng.uniform(*w.pulse_tec_range))
        beam = int(rng.integers(0, w.beams))
        pulses.append(Pulse(n0, pulse_amplitude(snr, w), tec, snr, beam))
    return pulses


def pulse_contributions(w: Workload, block: int, station_enu, beam_dir):
    """The injected pulses of a block and their station subband contributions:
    list of (m_lo, m_hi, complex [K, m_hi - m_lo, S]) to add before rounding."""
    plist = _draw_pulses(w, block)
    h = analysis_filter()
    nu = _NU0 + np.arange(w.first_bin, w.first_bin + w.subbands) * (SAMPLE_RATE_HZ / FFT_LEN)
    out = []
    for p in plist:
        m_lo, m_hi, xs = pulse_subbands(p, w, h, block)
        p.frames = (m_lo, m_hi)
        if m_hi <= m_lo:
            continue
        tau = station_enu @ beam_dir[p.beam] / _C
        phase = np.exp(2j * np.pi * nu[:, None] * tau[None, :])
        out.append((m_lo, m_hi, xs.T[:, :, None] * phase[:, None, :]))
    return plist, out


def make_block(w: Workload, block: int = 0, station_enu=None, beam_dir=None,
               noise: bool = True, pulses: bool = True):
    """Station block [P, K, F, S, 2] of w.dtype plus the list of injected pulses.

    Pulses are added to the continuous noise before the rounding to integers,
    as a station quantises signal and noise together (a pulse weaker than half a
    quantisation step per station still survives, dithered by the noise)."""
    if station_enu is None or beam_dir is None:
        station_enu, beam_dir, _ = make_geometry(w)
    P, K, F, S = w.pols, w.subbands, w.block_len, w.stations
    plist, contrib = (pulse_contributions(w, block, station_enu, beam_dir) if pulses
                      else ([], []))
    x = np.zeros((P, K, F, S, 2), dtype=w.dtype)
    info = np.iinfo(np.dtype(w.dtype))
    for pol in range(P):
        for k in range(K):
            adds = [(m_lo, m_hi, c[k]) for (m_lo, m_hi, c) in contrib]
            if noise:
                x[pol, k] = noisy_slab(w.seed, block, pol, k, F, S, w.noise_sigma, w.dtype, adds)
            elif adds:
                v = np.zeros((F, S, 2))
                for (m_lo, m_hi, c) in adds:
                    v[m_lo:m_hi, :, 0] += c.real
                    v[m_lo:m_hi, :, 1] += c.imag
                x[pol, k] = np.clip(np.rint(v), info.min, info.max).astype(w.dtype)
    return x, plist


def device_noise_block(w: Workload, seed: int, device, contrib=None):
    """Seeded noise block [P, K, F, S, 2] generated directly in device memory
    (PyTorch's generator indexing the same Gaussian quantiles); signal
    contributions (``pulse_contributions``) are added before rounding.  For
    timing runs at full size, where host generation would dominate."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    table = torch.from_numpy(gaussian_quantiles(w.noise_sigma).astype(np.float32)).to(device)
    dt = torch.int8 if w.dtype == "int8" else torch.int16
    info = np.iinfo(np.dtype(w.dtype))
    x = torch.empty((w.pols, w.subbands, w.block_len, w.stations, 2), dtype=dt, device=device)
    adds = []
    for (m_lo, m_hi, c) in contrib or []:
        adds.append((m_lo, m_hi, torch.from_numpy(
            np.stack([c.real, c.imag], axis=-1).astype(np.float32)).to(device)))
    for pol in range(w.pols):
        for k in range(w.subbands):
            idx = torch.randint(0, 65536, (w.block_len, w.stations, 2), generator=g,
                                device=device, dtype=torch.int32)
            v = table[idx]
            for (m_lo, m_hi, a) in adds:
                v[m_lo:m_hi] += a[k]
            x[pol, k] = torch.clamp(torch.round(v), info.min, info.max).to(dt)
    return x
