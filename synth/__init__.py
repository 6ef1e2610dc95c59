"""Seeded synthetic LOFAR-shaped inputs for the FX correlator hot path.

This module only *makes inputs*: station samples, prototype filter taps,
subband centre frequencies, station delays, bandpass weights and gains. It
holds none of the correlator's arithmetic (no FIR, no FFT, no delay
correction, no correlation), so both the FP64 oracle and the CUDA path can
take their inputs from here without sharing any of the method.

Signal model (the reading taken for the paper's station data, Sec. "LOFAR" and
Sec. "Signal processing with GPU kernels"): each station delivers complex
baseband samples of one 195.3125 kHz subband (sample period 5.12 us),
quantised to complex int16 (16-bit mode) or complex int8 (8-bit mode).
A sample is Gaussian noise plus point-source tones. Station n sees a tone of
sky frequency f_sky = f_subband + f_bb delayed by tau_n, so its baseband
sample at time t is  A * exp(2*pi*i*f_bb*t) * exp(-2*pi*i*f_sky*tau_n).
Tones sit on channel centres (f_bb = m * fs / C), which makes the delay
correction exact and lets the tests predict the output in closed form.

Layouts (all row-major):
  raw    [SB][N][L][P][2]  int16 or int8, L = (S + T - 1) * C, last axis re, im
  taps   [T * C]           float64, tap k of channel c at index k * C + c
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SAMPLE_RATE_HZ = 195312.5          # one LOFAR subband, complex sampled
BASE_SEED = 180104834              # seeds are BASE_SEED + workload index

CI16, CI8, CI4 = 0, 1, 2           # sample formats (match include/fx.h)
FORMAT_MAX = {CI16: 32767, CI8: 127, CI4: 7}
FORMAT_DTYPE = {CI16: np.int16, CI8: np.int8, CI4: np.uint8}
FORMAT_LAST = {CI16: 2, CI8: 2, CI4: 1}   # trailing axis: (re, im), or one packed byte


def pack_ci4(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """Complex 4-bit samples, one byte each: real part in the high nibble,
    imaginary part in the low nibble, two's complement."""
    r = np.asarray(re).astype(np.int64) & 15
    i = np.asarray(im).astype(np.int64) & 15
    return ((r << 4) | i).astype(np.uint8)


def kaiser_sinc_taps(n_taps: int, n_channels: int, beta: float = 9.0) -> np.ndarray:
    """Prototype low-pass filter of length L = T*C: sinc with cutoff 1/C times a
    Kaiser window, normalised to unit sum. The paper gives no filter; this is
    the conventional PPF prototype. Both sides receive the same array, so the
    parity of the method does not depend on the window."""
    L = n_taps * n_channels
    n = np.arange(L, dtype=np.float64)
    x = (n - (L - 1) / 2.0) / n_channels
    arg = np.clip(1.0 - (2.0 * n / (L - 1) - 1.0) ** 2, 0.0, None)
    w = np.i0(beta * np.sqrt(arg)) / np.i0(beta)
    h = np.sinc(x) * w
    return h / h.sum()


def subband_centres(n_subbands: int, centre_hz: float = 150e6,
                    fs: float = SAMPLE_RATE_HZ) -> np.ndarray:
    """Centre sky frequency of each subband: contiguous subbands of width fs
    around centre_hz (subband n_subbands//2 sits on centre_hz)."""
    sb = np.arange(n_subbands, dtype=np.float64)
    return centre_hz + (sb - n_subbands // 2) * fs


def bandpass_ripple(rng: np.random.Generator, n_stations: int, n_channels: int,
                    depth: float = 0.05) -> np.ndarray:
    """Per-station multiplicative ripple across channels, 1 + depth*sin(...):
    stands in for the station filter-bank ripple the paper's bandpass
    correction removes. Shape [N][C] float64."""
    k = np.arange(n_channels, dtype=np.float64)[None, :]
    cycles = rng.uniform(1.0, 3.0, size=(n_stations, 1))
    phase = rng.uniform(0.0, 2 * np.pi, size=(n_stations, 1))
    return 1.0 + depth * np.sin(2 * np.pi * cycles * k / n_channels + phase)


@dataclass
class Tone:
    """A point source on output channel `channel` with per-station delays
    (seconds). Polarisation p gets amplitude amp*(1 - 0.25 p) and an extra
    phase p*pi/3, so XY and YX differ and a swapped pol index is visible."""
    amp: float
    channel: int
    delays: np.ndarray                      # [N] seconds
    ripple: np.ndarray | None = None        # [N][C] amplitude ripple or None


@dataclass
class Block:
    """One integration block of synthetic station data plus its metadata."""
    fmt: int
    n_subbands: int
    n_stations: int
    n_pols: int
    n_channels: int
    n_taps: int
    n_spectra: int
    raw: np.ndarray                         # [SB][N][L][P][2] int16/int8
    taps: np.ndarray                        # [T*C] float64
    centres: np.ndarray                     # [SB] float64 Hz
    tones: list = field(default_factory=list)
    sample_rate: float = SAMPLE_RATE_HZ


def tone_samples(tone: Tone, n_channels: int, f_sub: float, n_stations: int,
                 n_pols: int, n_samples: int, fs: float = SAMPLE_RATE_HZ) -> np.ndarray:
    """Complex128 tone samples [N][L][P] for one subband. The baseband phase
    2*pi*m*t/C is formed from the exact integer (m*t mod C) so it carries no
    rounding error at any t."""
    C = n_channels
    m = tone.channel - C // 2                       # baseband channel offset
    t = np.arange(n_samples, dtype=np.int64)
    bb_phase = 2 * np.pi * ((m * t) % C).astype(np.float64) / C          # [L]
    f_sky = f_sub + m * fs / C
    dl_phase = -2 * np.pi * f_sky * np.asarray(tone.delays, np.float64)  # [N]
    out = np.empty((n_stations, n_samples, n_pols), np.complex128)
    for n in range(n_stations):
        a = tone.amp * (1.0 if tone.ripple is None else tone.ripple[n, tone.channel])
        base = np.exp(1j * (bb_phase + dl_phase[n]))
        for p in range(n_pols):
            out[n, :, p] = a * (1.0 - 0.25 * p) * base * np.exp(1j * p * np.pi / 3)
    return out


def quantise(z: np.ndarray, fmt: int) -> np.ndarray:
    """Round half to even and clip to the format's range; returns [..., 2]
    (int16/int8) or [..., 1] packed bytes (int4)."""
    lim = FORMAT_MAX[fmt]
    re = np.clip(np.rint(z.real), -lim, lim)
    im = np.clip(np.rint(z.imag), -lim, lim)
    if fmt == CI4:
        return pack_ci4(re, im)[..., None]
    return np.stack([re, im], axis=-1).astype(FORMAT_DTYPE[fmt])


def make_block(seed: int, fmt: int, n_subbands: int, n_stations: int, n_channels: int,
               n_spectra: int, n_taps: int = 16, n_pols: int = 2, sigma: float = 100.0,
               tones: list | None = None, centre_hz: float = 150e6,
               beta: float = 9.0) -> Block:
    """Noise N(0, sigma^2) per real component plus the given tones, quantised.
    Deterministic in `seed` (numpy PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    C, T, S = n_channels, n_taps, n_spectra
    L = (S + T - 1) * C
    centres = subband_centres(n_subbands, centre_hz)
    raw = np.empty((n_subbands, n_stations, L, n_pols, FORMAT_LAST[fmt]), FORMAT_DTYPE[fmt])
    for sb in range(n_subbands):
        z = (rng.standard_normal((n_stations, L, n_pols))
             + 1j * rng.standard_normal((n_stations, L, n_pols))) * sigma
        for tone in tones or []:
            z = z + tone_samples(tone, C, centres[sb], n_stations, n_pols, L)
        raw[sb] = quantise(z, fmt)
    return Block(fmt, n_subbands, n_stations, n_pols, C, T, S, raw,
                 kaiser_sinc_taps(T, C, beta), centres, list(tones or []))


def random_gains(rng: np.random.Generator, n_stations: int, n_pols: int = 2,
                 amp_lo: float = 0.8, amp_hi: float = 1.2) -> np.ndarray:
    """Complex per-(station, pol) gains, amplitude U(lo, hi), phase U(0, 2pi).
    Returned as float64 [N][P][2] (re, im)."""
    amp = rng.uniform(amp_lo, amp_hi, size=(n_stations, n_pols))
    ph = rng.uniform(0, 2 * np.pi, size=(n_stations, n_pols))
    return np.stack([amp * np.cos(ph), amp * np.sin(ph)], axis=-1)


def noise(seed: int, shape, sigma: float = 1.0) -> np.ndarray:
    """Plain seeded Gaussian noise of any shape (float64)."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(shape) * sigma


def channelised_noise(seed: int, n_subbands: int, n_stations: int, n_pols: int,
                      n_channels: int, n_spectra: int, sigma: float = 1.0) -> np.ndarray:
    """Already-channelised complex samples [SB][N][P][S][C][2] float64 (the
    differentiation workload starts from channelised data)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (n_subbands, n_stations, n_pols, n_spectra, n_channels, 2)
    return rng.standard_normal(shape) * sigma


# ---------------------------------------------------------------------------
# Device-side generation for full-size workloads (tens of GB): the same signal
# model drawn with torch's counter-based CUDA generator. Only used where the
# numpy path would take minutes; never mixed with numpy data in one comparison.
# ---------------------------------------------------------------------------

def make_raw_torch(seed: int, fmt: int, n_subbands: int, n_stations: int, n_channels: int,
                   n_spectra: int, n_taps: int = 16, n_pols: int = 2, sigma: float = 100.0,
                   tones: list | None = None, centre_hz: float = 150e6, device="cuda",
                   out=None):
    """Returns a torch int16/int8 tensor [SB][N][L][P][2] on `device`, made one
    subband at a time so the float scratch stays small. Same signal model as
    make_block (noise + channel-centred tones with per-station delays)."""
    import torch
    C, T, S, N, P = n_channels, n_taps, n_spectra, n_stations, n_pols
    L = (S + T - 1) * C
    dt = {CI16: torch.int16, CI8: torch.int8, CI4: torch.uint8}[fmt]
    lim = FORMAT_MAX[fmt]
    if out is None:
        out = torch.empty((n_subbands, N, L, P, FORMAT_LAST[fmt]), dtype=dt, device=device)
    g = torch.Generator(device=device)
    centres = subband_centres(n_subbands, centre_hz)
    t = torch.arange(L, device=device, dtype=torch.int64)
    pol_ph = torch.tensor([p * math.pi / 3 for p in range(P)], device=device, dtype=torch.float64)
    pol_amp = torch.tensor([1.0 - 0.25 * p for p in range(P)], device=device, dtype=torch.float64)
    prepared = []
    for tone in tones or []:
        m = tone.channel - C // 2
        bb = (2 * math.pi * ((m * t) % C).to(torch.float64) / C)                 # [L]
        amp = torch.full((N,), float(tone.amp), dtype=torch.float64, device=device)
        if tone.ripple is not None:
            amp = amp * torch.as_tensor(np.asarray(tone.ripple)[:, tone.channel], device=device)
        delays = torch.as_tensor(np.asarray(tone.delays, np.float64), device=device)
        prepared.append((m, bb, amp, delays))
    for sb in range(n_subbands):
        g.manual_seed(seed * 1000003 + sb)
        z = torch.randn((N, L, P, 2), generator=g, device=device, dtype=torch.float32) * sigma
        for m, bb, amp, delays in prepared:
            f_sky = centres[sb] + m * SAMPLE_RATE_HZ / C
            ph0 = -2 * math.pi * f_sky * delays                                    # [N]
            ph = (bb[None, :, None] + ph0[:, None, None] + pol_ph[None, None, :])  # [N][L][P]
            a = (amp[:, None, None] * pol_amp[None, None, :])
            z[..., 0] += (a * torch.cos(ph)).to(torch.float32)
            z[..., 1] += (a * torch.sin(ph)).to(torch.float32)
            del ph
        q = torch.clamp(torch.round(z), -lim, lim)
        if fmt == CI4:
            qi = q.to(torch.int32) & 15
            out[sb] = ((qi[..., 0] << 4) | qi[..., 1]).to(torch.uint8)[..., None]
        else:
            out[sb] = q.to(dt)
    return out
