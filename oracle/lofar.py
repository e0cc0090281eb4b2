"""FP64 oracle of the lunar nanosecond-pulse hot path (arXiv:1612.06592).

TEST INFRASTRUCTURE ONLY -- see the package docstring.  Every function below
cites the passage of the paper it follows (section and paragraph), and where
the paper is silent it states the reading taken.  Nothing here is blocked,
fused or reordered for speed; every step is its plain definition in float64.

Notation (the paper's and the pipeline's):
  S stations, P polarisations, K selected subbands (contiguous, starting at
  bin ``first_bin`` of the 512 bins of a 1024-point polyphase filter bank),
  B beams, Tr STEC trials, F frames per block, M = 1024, 16 taps, fs = 200 MHz.
  A *stream* is one (beam, STEC trial, polarisation); its index is
  j = (b * Tr + t) * P + pol.

Parity pins for everything here live in ``tests/test_oracle_pins.py``.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "FS_HZ", "M", "NBINS", "TAPS", "NU0_HZ", "C_LIGHT", "KAPPA", "TECU",
    "sky_frequencies", "geometric_weights", "dispersion_coefficient_hz",
    "dedispersion_cycles", "dedispersion_weights", "beamform",
    "bessel_i0", "prototype_filter", "synthesis_filter", "fft_radix2",
    "windowed_sums", "ippf", "parseval_power", "update_sigma2", "find_triggers",
    "LSMR_ITERS", "LSMR_WINDOW", "LSMR_OVERLAP", "lsmr", "lsmr_phase_taps", "lsmr_invert",
    "lsmr_noise_power",
    "Pipeline", "stream_window", "brute_force_stream",
    "INT16_MAX", "group_centres", "prebeam_weights", "prebeam", "transport_int16",
    "FINE_TAPS", "FINE_DELAY", "FINE_BETA", "FINE_GRID", "fine_dedispersion_taps",
    "fine_dedisperse", "fullrate_dedisperse",
    "FULLRATE_TAPS", "FULLRATE_DELAY", "FULLRATE_FLAT", "FULLRATE_GRID", "fullrate_max_delay",
    "fullrate_taps", "fullrate_filter",
]

# Sec. 2: antennas are sampled every 5 ns  ->  fs = 200 MHz.
FS_HZ = 200e6
# Sec. 2: the PPF lowers the time resolution from 5 ns to "about 5 us"; a
# 1024-point filter bank gives 1024 / 200 MHz = 5.12 us frames and 512 bins.
M = 1024
NBINS = M // 2
# Synthesis filter length in frames (16 taps, Kaiser-windowed sinc, beta = 9).
TAPS = 16
# Reading (paper silent): the HBA band 110-240 MHz is sampled in the second
# Nyquist zone, spectrum already un-flipped, so bin b has sky frequency
# fs/2 + b * fs / M.
NU0_HZ = FS_HZ / 2
C_LIGHT = 299792458.0
# Dispersion constant e^2 / (8 pi^2 eps0 m_e) in m^3 s^-2 (pinned against
# CODATA in the tests) and one TEC unit in electrons per m^2.
KAPPA = 40.308
TECU = 1e16


# --------------------------------------------------------------------------
# Frequencies and phase weights (Sec. 3)
# --------------------------------------------------------------------------

def sky_frequencies(first_bin: int, n_subbands: int) -> np.ndarray:
    """Sky frequency [Hz] of each selected subband (Sec. 2, sampling and PPF).

    Reading: bin b sits at fs/2 + b * fs/M (second Nyquist zone, un-flipped).
    """
    b = np.arange(first_bin, first_bin + n_subbands, dtype=np.float64)
    return NU0_HZ + b * (FS_HZ / M)


def geometric_weights(nu_hz: np.ndarray, station_enu_m: np.ndarray,
                      beam_dir: np.ndarray) -> np.ndarray:
    """Tied-array beam weights w[k, b, s] (Sec. 3, first paragraph).

    The paper: each station signal is summed "with a complex weight given by
    the station position and the beam direction".  Reading: a plane wave from
    unit direction s_b reaches station s (ENU position r_s) earlier by
    tau = r_s . s_b / c than the array origin, which multiplies that station's
    subband value by exp(+2 pi i nu tau); the weight undoes it:
        w[k, b, s] = exp(-2 pi i nu_k (r_s . s_b) / c).
    """
    nu = np.asarray(nu_hz, dtype=np.float64)
    r = np.asarray(station_enu_m, dtype=np.float64)          # [S, 3]
    d = np.asarray(beam_dir, dtype=np.float64)               # [B, 3]
    tau = (d @ r.T) / C_LIGHT                                 # [B, S] seconds
    cycles = nu[:, None, None] * tau[None, :, :]              # [K, B, S]
    return np.exp(-2j * np.pi * cycles)


def dispersion_coefficient_hz(tec_tecu) -> np.ndarray:
    """A = kappa * STEC / c in Hz; the ionospheric group delay is A / nu^2.

    Sec. 1 and Sec. 3: the signal is dispersed in the ionosphere and the
    correction depends on the slant electron content (STEC); the paper gives
    no formula, the standard cold-plasma one is used.
    """
    return KAPPA * np.asarray(tec_tecu, dtype=np.float64) * TECU / C_LIGHT


def dedispersion_cycles(nu_hz, tec_tecu, nu_ref_hz: float) -> np.ndarray:
    """De-dispersion phase in cycles, [K, Tr] (Sec. 3, third paragraph).

    The ionosphere multiplies the spectrum by H(nu) = exp(+2 pi i A / nu)
    (group delay A / nu^2).  Reading of the paper's "complex weight depending
    on the current electron content": remove that phase relative to the
    reference frequency nu_ref, keeping the pulse at the delay it has at nu_ref:
        phi(nu) = A * (1/nu - 2/nu_ref + nu / nu_ref^2)   [cycles].
    Written out exactly in this expanded form; the tests pin it against the
    factored form A (nu - nu_ref)^2 / (nu nu_ref^2) in 40-digit arithmetic.
    """
    nu = np.asarray(nu_hz, dtype=np.float64)[:, None]
    a = dispersion_coefficient_hz(tec_tecu)[None, :]
    return a * (1.0 / nu - 2.0 / nu_ref_hz + nu / (nu_ref_hz * nu_ref_hz))


def dedispersion_weights(nu_hz, tec_tecu, nu_ref_hz: float) -> np.ndarray:
    """D[k, t] = exp(-2 pi i phi(nu_k, STEC_t)) (Sec. 3, third paragraph)."""
    return np.exp(-2j * np.pi * dedispersion_cycles(nu_hz, tec_tecu, nu_ref_hz))


def beamform(x: np.ndarray, w: np.ndarray, d: np.ndarray) -> np.ndarray:
    """Beamformed, de-dispersed subband data (Sec. 3, first and third paragraphs).

    x: complex [P, K, F, S] station subband samples.
    w: complex [K, B, S] beam weights.   d: complex [K, Tr] de-dispersion.
    Returns complex [B, Tr, P, K, F] with
        beam[b, t, p, k, m] = d[k, t] * sum_s w[k, b, s] * x[p, k, m, s]
    evaluated as a direct sum over stations.
    """
    x = np.asarray(x, dtype=np.complex128)
    P, K, F, S = x.shape
    B = w.shape[1]
    Tr = d.shape[1]
    acc = np.zeros((B, P, K, F), dtype=np.complex128)
    for s in range(S):
        # acc[b, p, k, m] += w[k, b, s] * x[p, k, m, s]
        acc += w[:, :, s].T[:, None, :, None] * x[None, :, :, :, s]
    out = acc[:, None, :, :, :] * d.T[None, :, None, :, None]
    assert out.shape == (B, Tr, P, K, F)
    return out


# --------------------------------------------------------------------------
# Fine-resolution de-dispersion in the channel domain (Sec. 3, third paragraph)
# --------------------------------------------------------------------------
#
# The paper de-disperses by multiplying the spectrum at full resolution.  The
# per-subband weight D[k, t] above applies that phase at each subband centre
# only; what is left inside subband k is
#     psi(nu_k + dnu) = phi(nu_k + dnu) - phi(nu_k)      [cycles],
# mostly a delay A (1/nu_ref^2 - 1/nu_k^2) (a fraction of a frame) and a tiny
# chirp.  A subband's frame series carries the band nu_k + dnu, |dnu| < dnu_sb/2,
# at the frame rate (bin centres are whole cycles per frame), so the rest of
# the phase is a filter along frames with frequency response
#     R(f) = exp(-2 pi i (psi(f * dnu_sb) + f * FINE_DELAY)),  f in [-1/2, 1/2),
# f the frame-rate frequency, dnu_sb = fs / M.  Readings: the taps are R's
# inverse DTFT by the midpoint rule on FINE_GRID points, kept for q in
# [0, FINE_TAPS), times a Kaiser window (beta FINE_BETA) centred on the
# subband's first-order group delay c_k = FINE_DELAY + A dnu_sb (1/nu_ref^2 -
# 1/nu_k^2) frames with the largest half-width that fits the taps on both
# sides, min(c_k, FINE_TAPS - 1 - c_k) (a window or a support off that centre
# pulls the delay toward its own centre); the extra common delay of
# FINE_DELAY frames makes
# the filter causal (a pulse appears FINE_DELAY * M samples later).  The noise
# level stays the raw beams' (the filter passes power unchanged in band).

FINE_TAPS = 17
FINE_DELAY = 8
FINE_BETA = 4.0
FINE_GRID = 1024


def fine_dedispersion_taps(nu_hz, tec_tecu, nu_ref_hz: float, taps: int = FINE_TAPS,
                           delay: int = FINE_DELAY, beta: float = FINE_BETA,
                           grid: int = FINE_GRID) -> np.ndarray:
    """Channel-domain de-dispersion taps r[k, t, q], complex [K, Tr, taps]
    (readings above): r[q] = w_k[q] (1/grid) sum_j R(f_j) exp(+2 pi i f_j q),
    f_j = (j + 1/2)/grid - 1/2, psi = phi(nu_k + f dnu_sb) - phi(nu_k) from
    ``dedispersion_cycles``."""
    nu = np.asarray(nu_hz, dtype=np.float64)
    tec = np.asarray(tec_tecu, dtype=np.float64)
    f = (np.arange(grid) + 0.5) / grid - 0.5
    dnu = f * (FS_HZ / M)
    q = np.arange(taps)
    basis = np.exp(2j * np.pi * np.outer(f, q)) / grid                 # [grid, taps]
    a = dispersion_coefficient_hz(tec)                                   # [Tr]
    out = np.zeros((nu.size, tec.size, taps), dtype=np.complex128)
    for k in range(nu.size):
        centre = dedispersion_cycles(nu[k:k + 1], tec, nu_ref_hz)[0]    # [Tr]
        full = dedispersion_cycles(nu[k] + dnu, tec, nu_ref_hz)         # [grid, Tr]
        resp = np.exp(-2j * np.pi * (full - centre[None, :] + f[:, None] * delay))
        c = delay + a * (FS_HZ / M) * (1.0 / nu_ref_hz ** 2 - 1.0 / nu[k] ** 2)   # [Tr]
        hw = np.minimum(c, taps - 1 - c)                                 # [Tr]
        x = np.clip(1.0 - ((q[None, :] - c[:, None]) / hw[:, None]) ** 2, 0.0, None)
        win = bessel_i0(beta * np.sqrt(x)) / bessel_i0(beta)             # [Tr, taps]
        out[k] = (resp.T @ basis) * win
    return out


def fine_dedisperse(frames_ext: np.ndarray, r_k: np.ndarray) -> np.ndarray:
    """One stream's channel-domain de-dispersion filter along frames.

    frames_ext: complex [taps - 1 + F, K], the stream's beam frames (already
    multiplied by D[k, t]) with the taps - 1 frames before the block first;
    r_k: complex [K, taps], the taps of the stream's trial.  Returns [F, K]:
        out[m, k] = sum_q r_k[k, q] frames_ext[taps - 1 + m - q, k].
    """
    frames_ext = np.asarray(frames_ext, dtype=np.complex128)
    taps = r_k.shape[1]
    F = frames_ext.shape[0] - (taps - 1)
    out = np.zeros((F, frames_ext.shape[1]), dtype=np.complex128)
    for q in range(taps):
        out += r_k[None, :, q] * frames_ext[taps - 1 - q: taps - 1 - q + F]
    return out


def fullrate_dedisperse(u: np.ndarray, tec_tecu: float, nu_ref_hz: float) -> np.ndarray:
    """De-dispersion of a recovered 200 MHz analytic series at full resolution
    (Sec. 3, third paragraph, in the paper's order: after the PPF inversion).

    The series' frequency f (cycles per sample, the band lies in f >= 0) is the
    sky frequency nu = fs/2 + f fs; its spectrum is multiplied by
    exp(-2 pi i phi(nu)) with phi from ``dedispersion_cycles`` (zero phase for
    f < 0, where an analytic series has no content).  The whole series is one
    discrete Fourier transform (a library FFT as a step): circular, so the
    series must extend past the dispersion span on both sides.  Reference for
    the loss table of the de-dispersion chains; no GPU path computes it."""
    u = np.asarray(u, dtype=np.complex128)
    f = np.fft.fftfreq(u.size)
    phi = np.zeros(u.size)
    pos = f >= 0
    phi[pos] = dedispersion_cycles(NU0_HZ + f[pos] * FS_HZ, [tec_tecu], nu_ref_hz)[:, 0]
    return np.fft.ifft(np.fft.fft(u) * np.exp(-2j * np.pi * phi))


# Full-rate de-dispersion as a streaming filter (Sec. 3, third paragraph, on a
# continuous stream).  Readings (the paper gives only "FFT, multiply, inverse
# FFT" of the time series):
#   * it follows the inversion, on the 200 MHz analytic series, and carries the
#     whole STEC phase (no per-subband phase is applied before the inversion);
#   * the whole-series transform becomes a linear filter of FULLRATE_TAPS taps:
#     the response of ``fullrate_dedisperse`` (exp(-2 pi i phi(nu)) for f >= 0,
#     1 for f < 0) sampled on FULLRATE_GRID frequencies and inverted, taken over
#     the delays -FULLRATE_DELAY .. FULLRATE_TAPS - 1 - FULLRATE_DELAY, times a
#     Tukey window (1 within FULLRATE_FLAT / 2 of zero delay, a half-cosine
#     down to 0 at the ends), then delayed by FULLRATE_DELAY samples so that it
#     is causal: a pulse appears FULLRATE_DELAY samples (one frame) later;
#   * the series is filtered continuously across blocks (the last
#     FULLRATE_TAPS - 1 samples of a block are the next block's history; zero
#     before the stream start);
#   * the noise level and threshold are the unfiltered series' (the response
#     has unit modulus).
# The window holds the response's group delays when they lie within
# FULLRATE_FLAT / 2 of zero delay over the whole 100-200 MHz band (checked by
# ``fullrate_max_delay``).

FULLRATE_TAPS = 2048
FULLRATE_DELAY = 1024
FULLRATE_FLAT = 1536
FULLRATE_GRID = 8192


def fullrate_max_delay(tec_tecu, nu_ref_hz: float) -> np.ndarray:
    """Largest |group delay| of the full-rate response over 100-200 MHz, in
    samples, [Tr]: A |1/nu^2 - 1/nu_ref^2| fs at the band ends (the delay
    A (1/nu^2 - 1/nu_ref^2) is monotonic in nu)."""
    a = dispersion_coefficient_hz(tec_tecu)
    ends = np.array([NU0_HZ, FS_HZ])
    d = np.abs(a[:, None] * (1.0 / ends[None, :] ** 2 - 1.0 / nu_ref_hz ** 2)) * FS_HZ
    return d.max(axis=1)


def fullrate_taps(tec_tecu, nu_ref_hz: float, taps: int = FULLRATE_TAPS,
                  delay: int = FULLRATE_DELAY, flat: int = FULLRATE_FLAT,
                  grid: int = FULLRATE_GRID) -> np.ndarray:
    """Causal taps h[t, l], complex [Tr, taps] (readings above):
    h[l] = w(l - delay) (1/grid) sum_j H_j exp(+2 pi i j (l - delay) / grid),
    H_j = exp(-2 pi i phi(fs/2 + f_j fs)) for f_j = j / grid < 1/2, else 1, and
    w(d) = 1 for |d| <= flat/2, (1 + cos(pi (|d| - flat/2) / ((taps - flat)/2))) / 2
    beyond.  The inverse transform is this module's own FFT."""
    tec = np.atleast_1d(np.asarray(tec_tecu, dtype=np.float64))
    j = np.arange(grid)
    pos = j < grid // 2
    d = np.arange(taps) - delay
    half, ramp = flat / 2.0, (taps - flat) / 2.0
    win = np.where(np.abs(d) <= half, 1.0,
                   0.5 * (1.0 + np.cos(np.pi * np.clip(np.abs(d) - half, 0.0, ramp) / ramp)))
    out = np.zeros((tec.size, taps), dtype=np.complex128)
    for t in range(tec.size):
        phi = np.zeros(grid)
        phi[pos] = dedispersion_cycles(NU0_HZ + (j[pos] / grid) * FS_HZ, tec[t:t + 1],
                                       nu_ref_hz)[:, 0]
        h = fft_radix2(np.exp(-2j * np.pi * phi), +1) / grid     # h[n], n mod grid
        out[t] = win * h[d % grid]
    return out


def fullrate_filter(u_ext: np.ndarray, h: np.ndarray) -> np.ndarray:
    """One stream's full-rate filter: u_ext complex [taps - 1 + n], the stream's
    series with the taps - 1 samples before the block first; h complex [taps].
    Returns v [n], v[o] = sum_l h[l] u_ext[taps - 1 + o - l] (a library
    convolution as the step)."""
    return np.convolve(np.asarray(u_ext, dtype=np.complex128), h, mode="valid")


# --------------------------------------------------------------------------
# Two-stage beamforming (Sec. 4, network paragraph)
# --------------------------------------------------------------------------
#
# The paper: fewer than ten stations' worth of 16-bit data fit through the link
# to the processing cluster, so preliminary beams are first formed from subsets
# of stations by the correlator's regular beamformer, sent on, and combined into
# the final beams there.  Readings (the paper gives no more than that):
#   * the subsets are disjoint station groups; a station in no group is unused;
#   * each group forms one preliminary beam, toward a direction of its own
#     (normally the pointing centre), phased to the group's phase centre r_g =
#     the mean position of its stations, so the preliminary beam is a "station"
#     at r_g for the final stage;
#   * it travels as complex int16 like station data: round half to even of
#     scale * value, saturated to [-32767, 32767];
#   * the final stage is the ordinary beamformer of this module with the group
#     centres as station positions.

INT16_MAX = 32767


def group_centres(station_enu: np.ndarray, group_of_station: np.ndarray,
                  n_groups: int) -> np.ndarray:
    """Phase centre of each station group: the mean ENU position of its
    stations, [G, 3] (reading above).  Every group must have a station."""
    r = np.asarray(station_enu, dtype=np.float64)
    grp = np.asarray(group_of_station)
    out = np.zeros((n_groups, 3))
    for g in range(n_groups):
        members = np.flatnonzero(grp == g)
        if members.size == 0:
            raise ValueError(f"group {g} has no station")
        out[g] = r[members].sum(axis=0) / members.size
    return out


def prebeam_weights(nu_hz: np.ndarray, station_enu: np.ndarray, group_of_station: np.ndarray,
                    group_dir: np.ndarray) -> np.ndarray:
    """Preliminary-beam weights w1[k, g, s] (Sec. 4 network paragraph, Sec. 3 first
    paragraph): the tied-array weight of station s toward the group's direction
    s_g, relative to the group's phase centre r_g, for the stations of group g,
    and zero for the others:
        w1[k, g, s] = exp(-2 pi i nu_k ((r_s - r_g) . s_g) / c)  if s in g.
    """
    nu = np.asarray(nu_hz, dtype=np.float64)
    r = np.asarray(station_enu, dtype=np.float64)
    grp = np.asarray(group_of_station)
    d = np.asarray(group_dir, dtype=np.float64)
    G = d.shape[0]
    centres = group_centres(r, grp, G)
    w1 = np.zeros((nu.size, G, r.shape[0]), dtype=np.complex128)
    for s in range(r.shape[0]):
        g = int(grp[s])
        if g < 0:
            continue
        cycles = nu * ((r[s] - centres[g]) @ d[g]) / C_LIGHT
        w1[:, g, s] = np.exp(-2j * np.pi * cycles)
    return w1


def prebeam(x: np.ndarray, w1: np.ndarray) -> np.ndarray:
    """Preliminary beams pb[p, k, m, g] = sum_s w1[k, g, s] x[p, k, m, s] as a
    direct sum over stations (complex128).  x: complex [P, K, F, S]."""
    x = np.asarray(x, dtype=np.complex128)
    P, K, F, S = x.shape
    G = w1.shape[1]
    out = np.zeros((P, K, F, G), dtype=np.complex128)
    for s in range(S):
        out += w1[None, :, None, :, s] * x[:, :, :, s, None]
    return out


def transport_int16(v: np.ndarray, scale: float) -> np.ndarray:
    """Complex value -> the int16 transport code [..., 2] (re, im): round half to
    even of scale * value, saturated to [-INT16_MAX, INT16_MAX] (reading)."""
    v = np.asarray(v, dtype=np.complex128) * scale
    out = np.stack([np.rint(v.real), np.rint(v.imag)], axis=-1)
    return np.clip(out, -INT16_MAX, INT16_MAX).astype(np.int16)


# --------------------------------------------------------------------------
# Prototype filter (inverse PPF, Sec. 3 second paragraph; 16-tap synthesis)
# --------------------------------------------------------------------------

def bessel_i0(x) -> np.ndarray:
    """Modified Bessel function I0 by its power series sum_k ((x/2)^k / k!)^2."""
    x = np.asarray(x, dtype=np.float64)
    term = np.ones_like(x)
    total = np.ones_like(x)
    q = (x / 2.0) ** 2
    for k in range(1, 200):
        term = term * q / (k * k)
        total = total + term
        if np.all(term <= 1e-18 * total):
            break
    return total


def prototype_filter(m: int = M, taps: int = TAPS, beta: float = 9.0) -> np.ndarray:
    """Kaiser-windowed sinc prototype h[n], n < L = m * taps, sum(h) = 1.

    h[n] = sinc((n - (L-1)/2) / m) * I0(beta sqrt(1 - (2n/(L-1) - 1)^2)) / I0(beta),
    sinc(x) = sin(pi x) / (pi x).  Reading of "cutoff one subband": the sinc
    has its zeros every m samples, i.e. -6 dB at +-half a subband.
    """
    L = m * taps
    n = np.arange(L, dtype=np.float64)
    xs = (n - (L - 1) / 2.0) / m
    sinc = np.empty_like(xs)
    nz = xs != 0.0
    sinc[nz] = np.sin(np.pi * xs[nz]) / (np.pi * xs[nz])
    sinc[~nz] = 1.0
    arg = 1.0 - (2.0 * n / (L - 1) - 1.0) ** 2
    window = bessel_i0(beta * np.sqrt(np.maximum(arg, 0.0))) / bessel_i0(beta)
    h = sinc * window
    return h / np.sum(h)


def synthesis_filter(m: int = M, taps: int = TAPS, beta: float = 9.0) -> np.ndarray:
    """Synthesis filter g = m^2 h: unit round-trip gain for subband-centred tones."""
    return (m * m) * prototype_filter(m, taps, beta)


# --------------------------------------------------------------------------
# FFT (radix-2 Cooley-Tukey, the algorithm the paper's FLOP count assumes)
# --------------------------------------------------------------------------

def _bit_reverse_indices(n: int) -> np.ndarray:
    bits = n.bit_length() - 1
    idx = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def fft_radix2(x, sign: int) -> np.ndarray:
    """Unnormalised DFT along the last axis: X[k] = sum_n x[n] exp(sign 2 pi i k n / N).

    Iterative radix-2 decimation in time (Sec. 3 counts 5 N log2 N FLOP for
    it).  sign = -1 is the forward transform, sign = +1 the inverse without
    the 1/N.
    """
    a = np.asarray(x, dtype=np.complex128)
    n = a.shape[-1]
    if n & (n - 1) or n == 0:
        raise ValueError("length must be a power of two")
    a = a[..., _bit_reverse_indices(n)]
    lead = a.shape[:-1]
    span = 1
    while span < n:
        tw = np.exp(sign * 2j * np.pi * np.arange(span) / (2 * span))
        a = a.reshape(lead + (n // (2 * span), 2, span))
        even = a[..., 0, :]
        odd = a[..., 1, :] * tw
        a = np.stack([even + odd, even - odd], axis=-2).reshape(lead + (n,))
        span *= 2
    return a


# --------------------------------------------------------------------------
# Inverse polyphase filter bank (Sec. 2 and Sec. 3 second paragraph)
# --------------------------------------------------------------------------

def windowed_sums(frames: np.ndarray, first_bin: int) -> np.ndarray:
    """The inverse-FFT step of the PPF inversion (Sec. 3, second paragraph),
    complex [..., n, M] from subband frames [..., n, K]: per frame, 2 * beam in
    the selected bins (all other bins, DC and Nyquist zero), 1024-point inverse
    DFT with 1/M:  z_m[p] = (1/M) sum_k 2 c_m[k] exp(+2 pi i k p / M).  Its real
    part is the PPF branch signal of frame m, the imaginary part its Hilbert pair."""
    frames = np.asarray(frames, dtype=np.complex128)
    K = frames.shape[-1]
    if first_bin < 1 or first_bin + K > NBINS:
        raise ValueError("selected bins must avoid DC and Nyquist")
    c = np.zeros(frames.shape[:-1] + (M,), dtype=np.complex128)
    c[..., first_bin:first_bin + K] = 2.0 * frames
    return fft_radix2(c, +1) / M


def ippf(frames_ext: np.ndarray, first_bin: int, g: np.ndarray) -> np.ndarray:
    """Synthesis of the 200 MHz analytic time series from subband frames.

    frames_ext: complex [..., F + 15, K]: 15 history frames, then F new ones.
    Returns u: complex [..., F, M], u[i, p] is sample n = (m - 15) M + p of the
    output, m the frame of new row i.

    Step 1 (the paper's inverse FFT): per frame, place 2 * beam in the
    selected bins (all other bins, DC and Nyquist zero) and take the 1024-point
    inverse DFT with 1/M: z_m[p] = (1/M) sum_k 2 c_m[k] exp(+2 pi i k p / M);
    its real part is the PPF branch signal, the imaginary part its Hilbert pair.
    Step 2 (replaces the paper's sparse LSMR solve by the FIR synthesis):
        u_m[p] = sum_{t=0}^{15} g[t M + p] * z_{m-t}[p].
    """
    frames_ext = np.asarray(frames_ext, dtype=np.complex128)
    nfr = frames_ext.shape[-2]
    taps = g.shape[0] // M
    F = nfr - (taps - 1)
    if F < 0:
        raise ValueError("need at least taps-1 history frames")
    z = windowed_sums(frames_ext, first_bin)
    u = np.zeros(frames_ext.shape[:-2] + (F, M), dtype=np.complex128)
    for t in range(taps):
        u += g[t * M:(t + 1) * M] * z[..., taps - 1 - t:taps - 1 - t + F, :]
    return u


# --------------------------------------------------------------------------
# PPF inversion by LSMR (Sec. 3, second paragraph)
# --------------------------------------------------------------------------
#
# The paper inverts the filter bank by the inverse FFT (``windowed_sums``) and
# then solves the sparse system H x = y with about 25 LSMR iterations.  H is the
# PPF's window: y_m[p] = sum_{t<16} h[t M + p] x[(m - 15 + t) M + p], so it
# splits into one banded Toeplitz system per phase p along the frames, with
# taps a_p[t] = h[t M + p] (the prototype, sum h = 1).  Readings:
#   * the analytic series is solved for (y = the complex windowed sums), one
#     system per stream and phase;
#   * a block is solved window by window: window w takes the equations of
#     frames [wW - 16, wW + W) (W = LSMR_WINDOW; the 16 frames before the block
#     are the previous block's) over the unknowns x_p[q], q in [wW - 31, wW + W),
#     and keeps q in [wW - 16, wW + W - 16): the unknowns all 16 of whose
#     equations lie in the window.  Windows tile q in [-16, F - 16): the output
#     of a block lags its frames by 16 frames (sample n = (m - 16) M + p);
#   * LSMR_ITERS iterations from x = 0, no damping (Fong and Saunders 2011).

LSMR_ITERS = 25
LSMR_WINDOW = 256
LSMR_OVERLAP = 16


def lsmr(matvec, rmatvec, b: np.ndarray, n: int, iters: int) -> np.ndarray:
    """LSMR for min ||A x - b|| (Fong and Saunders 2011, their Algorithm 1 in
    its order and notation): Golub-Kahan bidiagonalisation started from b,
    two plane rotations per step, iters steps from x = 0, no damping.
    matvec(v) = A v, rmatvec(u) = A^H u."""
    b = np.asarray(b, dtype=np.complex128)
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return np.zeros(n, dtype=np.complex128)
    u = b / beta
    v = rmatvec(u)
    alpha = np.linalg.norm(v)
    if alpha == 0.0:
        return np.zeros(n, dtype=np.complex128)
    v = v / alpha
    alphabar, zetabar = alpha, alpha * beta
    rho, rhobar, cbar, sbar = 1.0, 1.0, 1.0, 0.0
    h = v.copy()
    hbar = np.zeros(n, dtype=np.complex128)
    x = np.zeros(n, dtype=np.complex128)
    for _ in range(iters):
        # continue the bidiagonalisation
        u = matvec(v) - alpha * u
        beta = np.linalg.norm(u)
        if beta > 0:
            u = u / beta
        v = rmatvec(u) - beta * v
        alpha = np.linalg.norm(v)
        if alpha > 0:
            v = v / alpha
        # rotation P_k
        rho_old = rho
        rho = math.hypot(alphabar, beta)
        c, s = alphabar / rho, beta / rho
        theta = s * alpha
        alphabar = c * alpha
        # rotation Pbar_k
        rhobar_old = rhobar
        thetabar = sbar * rho
        rhobar = math.hypot(cbar * rho, theta)
        cbar, sbar = cbar * rho / rhobar, theta / rhobar
        zeta = cbar * zetabar
        zetabar = -sbar * zetabar
        # update h, hbar, x
        hbar = h - (thetabar * rho / (rho_old * rhobar_old)) * hbar
        x = x + (zeta / (rho * rhobar)) * hbar
        h = v - (theta / rho) * h
    return x


def lsmr_phase_taps(h: np.ndarray) -> np.ndarray:
    """a[p, t] = h[t M + p], the window taps of each phase, [M, taps]."""
    taps = h.shape[0] // M
    return np.asarray(h, dtype=np.float64).reshape(taps, M).T.copy()


def lsmr_invert(frames_ext: np.ndarray, first_bin: int, h: np.ndarray,
                iters: int = LSMR_ITERS, window: int = LSMR_WINDOW) -> np.ndarray:
    """PPF inversion of one stream's block by windowed LSMR (readings above).

    frames_ext: complex [16 + F, K], the 16 frames before the block first
    (zero before the stream start); F a multiple of ``window``.  Returns the
    analytic series x [F, M]: row i is x[(i - 16) M + p] relative to the block's
    first frame, i.e. sample n = (m - 16) M + p of the stream for frame m.
    """
    ov = LSMR_OVERLAP
    nfr = frames_ext.shape[0]
    F = nfr - ov
    if F % window:
        raise ValueError("block length must be a multiple of the window")
    z = windowed_sums(frames_ext, first_bin)                  # [16 + F, M]
    a = lsmr_phase_taps(h)                                    # [M, 16]
    taps = a.shape[1]
    rows = window + ov                                        # equations per window
    cols = rows + taps - 1                                    # unknowns per window
    out = np.zeros((F, M), dtype=np.complex128)
    for w0 in range(0, F, window):
        for p in range(M):
            ap = a[p]

            def matvec(x, ap=ap):
                return sum(ap[t] * x[t:t + rows] for t in range(taps))

            def rmatvec(u, ap=ap):
                r = np.zeros(cols, dtype=np.complex128)
                for t in range(taps):
                    r[t:t + rows] += ap[t] * u
                return r

            # equation e is frame w0 - 16 + e (row w0 + e of z); unknown j is
            # q = w0 - 31 + j; the kept q in [w0 - 16, w0 + W - 16) are j in [15, 15 + W)
            x = lsmr(matvec, rmatvec, z[w0:w0 + rows, p], cols, iters)
            out[w0:w0 + window, p] = x[taps - 1:taps - 1 + window]
    return out


def lsmr_noise_power(xhat: np.ndarray) -> np.ndarray:
    """Noise level of one block of the LSMR series, per phase (reading):
    Pi_p = mean over the block's rows of |x[i, p]|^2 / 2, [M].  The solver's
    noise gain differs from phase to phase (ill-conditioned phase systems
    amplify it, by up to ~4x in power), so a single level per stream would
    over-trigger on the noisy phases; per phase, |x| follows the Rayleigh law.
    The levels feed the same running update as the FIR path
    (``update_sigma2``), and a sample triggers iff |x| > k_sigma sigma_p."""
    x = np.asarray(xhat)
    return np.mean(x.real ** 2 + x.imag ** 2, axis=0) / 2.0


# --------------------------------------------------------------------------
# Noise level and trigger (Sec. 1 and Sec. 2: trigger on the pulse amplitude)
# --------------------------------------------------------------------------

def parseval_power(frames_new: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Block estimate of the output mean square <y^2> per stream.

    frames_new: complex [..., F, K] beam frames of this block.
    Reading (paper silent on the noise estimate): with independent bins of
    power P_k, the analytic output has E|u|^2 = 4 sum(g^2) sum_k P_k / M^3 and
    y = Re u half of that, so
        Pi = (2 sum(g^2) / M^3) * (1/F) * sum_{m,k} |beam_m[k]|^2.
    """
    f = np.asarray(frames_new, dtype=np.complex128)
    F = f.shape[-2]
    g2 = float(np.sum(np.asarray(g, dtype=np.float64) ** 2))
    power = np.sum(np.abs(f) ** 2, axis=(-2, -1)) / F
    return (2.0 * g2 / float(M) ** 3) * power


def update_sigma2(prev_sigma2, block_power, alpha: float, first_block: bool):
    """Running noise variance: s2_0 = Pi_0, s2_j = (1 - alpha) s2_{j-1} + alpha Pi_j."""
    if first_block:
        return np.asarray(block_power, dtype=np.float64).copy()
    return (1.0 - alpha) * np.asarray(prev_sigma2) + alpha * np.asarray(block_power)


def find_triggers(env: np.ndarray, theta: float, n_first: int):
    """Samples with envelope strictly above theta and n >= 0.

    env: [N] envelope of one stream, env[i] at sample n_first + i.
    Returns (n, env) arrays.  The envelope of Gaussian noise is Rayleigh with
    scale sigma_y, so theta = k sigma_y gives a rate exp(-k^2/2) per sample.
    """
    env = np.asarray(env)
    n = n_first + np.arange(env.shape[0], dtype=np.int64)
    hit = (env > theta) & (n >= 0)
    return n[hit], env[hit]


# --------------------------------------------------------------------------
# Block pipeline with state carried across blocks
# --------------------------------------------------------------------------

def _as_complex(x: np.ndarray) -> np.ndarray:
    """Integer station samples [..., 2] (re, im) -> complex128 [...]."""
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return x.astype(np.complex128)
    return x[..., 0].astype(np.float64) + 1j * x[..., 1].astype(np.float64)


@dataclass
class Pipeline:
    """The whole hot path, block after block, in float64.

    State carried between blocks: the last 15 beam frames of every stream
    (synthesis history; frames before the stream start are zero), the running
    noise variance and the block counter.
    """
    stations: int
    pols: int
    subbands: int
    beams: int
    tec_trials: int
    block_len: int
    first_bin: int
    station_enu: np.ndarray
    beam_dir: np.ndarray
    tec: np.ndarray
    nu_ref_hz: float | None = None
    k_sigma: float = 6.0
    sigma_alpha: float = 0.25
    beta: float = 9.0
    keep_timeseries: bool = True
    fine_dedispersion: bool = False
    fullrate_dedispersion: bool = False
    # state
    block_index: int = 0
    history: np.ndarray | None = field(default=None, repr=False)
    fine_history: np.ndarray | None = field(default=None, repr=False)
    fullrate_history: np.ndarray | None = field(default=None, repr=False)
    sigma2: np.ndarray | None = None

    def __post_init__(self):
        self.nu = sky_frequencies(self.first_bin, self.subbands)
        if self.nu_ref_hz is None:
            self.nu_ref_hz = 0.5 * (self.nu[0] + self.nu[-1])
        self.w = geometric_weights(self.nu, self.station_enu, self.beam_dir)
        self.d = dedispersion_weights(self.nu, np.asarray(self.tec), self.nu_ref_hz)
        self.g = synthesis_filter(M, TAPS, self.beta)
        J = self.beams * self.tec_trials * self.pols
        self.history = np.zeros((J, TAPS - 1, self.subbands), dtype=np.complex128)
        if self.fullrate_dedispersion:
            # the whole STEC phase is applied at full rate, none per subband
            self.d = np.ones_like(self.d)
            self.fullrate_h = fullrate_taps(np.asarray(self.tec), self.nu_ref_hz)
            self.fullrate_history = np.zeros((J, FULLRATE_TAPS - 1), dtype=np.complex128)
        if self.fine_dedispersion:
            self.fine_taps = fine_dedispersion_taps(self.nu, np.asarray(self.tec), self.nu_ref_hz)
            self.fine_history = np.zeros((J, FINE_TAPS - 1, self.subbands), dtype=np.complex128)

    @property
    def n_streams(self) -> int:
        return self.beams * self.tec_trials * self.pols

    def stream_index(self, b: int, t: int, p: int) -> int:
        return (b * self.tec_trials + t) * self.pols + p

    def process_block(self, x):
        """x: station block [P, K, F, S, 2] integers (or complex [P, K, F, S]).

        Returns dict with beams [J, F, K] (after the fine de-dispersion filter
        when it is on), sigma [J], theta [J], n_first,
        (full-rate mode: y, env and the triggers are those of the filtered
        series v; u is the synthesis output before the filter)
        y/env [J, F*M] (if keep_timeseries) and triggers: list of
        (n, beam, tec, pol, env, sigma) sorted by (beam, tec, pol, n).
        """
        xc = _as_complex(x)
        P, K, F, S = xc.shape
        assert (P, K, F, S) == (self.pols, self.subbands, self.block_len, self.stations)
        bm = beamform(xc, self.w, self.d)                 # [B, Tr, P, K, F]
        J = self.n_streams
        frames = bm.reshape(J, K, F).transpose(0, 2, 1)   # [J, F, K]
        pi = parseval_power(frames, self.g)
        self.sigma2 = update_sigma2(self.sigma2, pi, self.sigma_alpha,
                                    self.block_index == 0)
        if self.fine_dedispersion:
            fine = np.empty_like(frames)
            for j in range(J):
                t = (j // self.pols) % self.tec_trials
                fext = np.concatenate([self.fine_history[j], frames[j]], axis=0)
                fine[j] = fine_dedisperse(fext, self.fine_taps[:, t, :])
                self.fine_history[j] = fext[-(FINE_TAPS - 1):]
            frames = fine
        sigma = np.sqrt(self.sigma2)
        theta = self.k_sigma * sigma
        n_first = (self.block_index * F - (TAPS - 1)) * M
        y = np.zeros((J, F * M)) if self.keep_timeseries else None
        env_all = np.zeros((J, F * M)) if self.keep_timeseries else None
        trig = []
        new_history = np.empty_like(self.history)
        for j in range(J):
            ext = np.concatenate([self.history[j], frames[j]], axis=0)
            u = ippf(ext, self.first_bin, self.g).reshape(F * M)
            if self.fullrate_dedispersion:
                t = (j // self.pols) % self.tec_trials
                uext = np.concatenate([self.fullrate_history[j], u])
                self.fullrate_history[j] = uext[-(FULLRATE_TAPS - 1):]
                u = fullrate_filter(uext, self.fullrate_h[t])
            env = np.abs(u)
            if self.keep_timeseries:
                y[j] = u.real
                env_all[j] = env
            n_hit, e_hit = find_triggers(env, theta[j], n_first)
            b, rem = divmod(j, self.tec_trials * self.pols)
            t, p = divmod(rem, self.pols)
            for n, e in zip(n_hit.tolist(), e_hit.tolist()):
                trig.append((n, b, t, p, e, float(sigma[j])))
            new_history[j] = ext[-(TAPS - 1):]
        self.history = new_history
        self.block_index += 1
        trig.sort(key=lambda r: (r[1], r[2], r[3], r[0]))
        return {"beams": frames, "block_power": pi, "sigma": sigma,
                "theta": theta, "n_first": n_first, "y": y, "env": env_all,
                "triggers": trig}


def stream_window(x, w_bs: np.ndarray, d_kt: np.ndarray, pol: int,
                  first_bin: int, g: np.ndarray, m0: int, m1: int):
    """Output u of one stream for block frames [m0, m1), first block of a stream.

    x: station block [P, K, F, S, 2] (or complex).  w_bs: complex [K, S] the
    weights of the stream's beam; d_kt: complex [K] its de-dispersion column.
    Frames before the block start are zero (stream start).  Evaluates the same
    definitions as ``Pipeline`` on only the frames the window needs, so large
    blocks can be checked at sampled places.  Returns u [m1 - m0, M] whose row
    i is frame m0 + i, i.e. samples (m0 + i - 15) M + p.
    """
    xa = np.asarray(x)
    lo = max(0, m0 - (TAPS - 1))
    xc = _as_complex(xa[pol, :, lo:m1])                       # [K, n, S]
    beam = np.einsum("ks,kns->kn", w_bs, xc) * d_kt[:, None]  # [K, n]
    ext = np.zeros((m1 - m0 + TAPS - 1, w_bs.shape[0]), dtype=np.complex128)
    ext[(lo - (m0 - (TAPS - 1))):] = beam.T
    return ippf(ext, first_bin, g)


def brute_force_stream(frames_ext: np.ndarray, first_bin: int, g: np.ndarray) -> np.ndarray:
    """The synthesis written as one explicit double sum, for tiny inputs only.

    u_m[p] = sum_t g[tM+p] (1/M) sum_k 2 c_{m-t}[k] exp(2 pi i (first_bin+k) p / M)
    with no FFT and no vectorised reshapes: a check on ``ippf``.
    """
    frames_ext = np.asarray(frames_ext, dtype=np.complex128)
    nfr, K = frames_ext.shape
    taps = g.shape[0] // M
    F = nfr - (taps - 1)
    u = np.zeros((F, M), dtype=np.complex128)
    for i in range(F):
        m = i + taps - 1
        for p in range(M):
            acc = 0j
            for t in range(taps):
                row = frames_ext[m - t]
                zsum = 0j
                for k in range(K):
                    zsum += 2.0 * row[k] * complex(
                        math.cos(2 * math.pi * (first_bin + k) * p / M),
                        math.sin(2 * math.pi * (first_bin + k) * p / M))
                acc += g[t * M + p] * zsum / M
            u[i, p] = acc
    return u
