"""Torch-tensor convenience layer over the C ABI (include/fx.h).

`Correlator` owns one fx_handle and calls the same entry points with device
pointers taken from torch tensors. It checks dtypes, devices, contiguity and
byte sizes before every call (the C side trusts the sizes implied by the
handle), allocates outputs when none are given, and launches on torch's
current CUDA stream. It does no arithmetic of its own.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi
from ._abi import FX_CI4, FX_CI8, FX_CI16, FX_F16, FX_F16_SPLIT, FX_F32, FX_TF32_SPLIT, check

SAMPLE_RATE_HZ = 195312.5


def f32_unblock(corr, n_spectra: int):
    """View of the FP32 corrected layout [SB][C][S16/16][N][16][2][2] (the
    spectrum-blocked order the X-stage reads; torch tensor or numpy array) in
    natural order [SB][C][S][N][2][2] (spectra S .. S16-1 dropped). A reshape,
    no arithmetic."""
    SB, C, NB, N = corr.shape[:4]
    if isinstance(corr, torch.Tensor):
        y = corr.permute(0, 1, 2, 4, 3, 5, 6).reshape(SB, C, NB * 16, N, 2, 2)
    else:
        y = np.ascontiguousarray(corr.transpose(0, 1, 2, 4, 3, 5, 6)).reshape(SB, C, NB * 16, N, 2, 2)
    return y[:, :, :n_spectra]


def f32_block(y):
    """[SB][C][S][N][2][2] (natural order; torch tensor or numpy array) ->
    the FP32 corrected layout [SB][C][S16/16][N][16][2][2], zero-padded to a
    multiple of 16 spectra. A reshape, no arithmetic."""
    SB, C, S, N = y.shape[:4]
    S16 = (S + 15) // 16 * 16
    if isinstance(y, torch.Tensor):
        z = torch.zeros((SB, C, S16, N, 2, 2), dtype=y.dtype, device=y.device)
        z[:, :, :S] = y
        return z.reshape(SB, C, S16 // 16, 16, N, 2, 2).permute(0, 1, 2, 4, 3, 5, 6).contiguous()
    z = np.zeros((SB, C, S16, N, 2, 2), dtype=y.dtype)
    z[:, :, :S] = y
    return np.ascontiguousarray(z.reshape(SB, C, S16 // 16, 16, N, 2, 2).transpose(0, 1, 2, 4, 3, 5, 6))


def _stream_ptr(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Correlator:
    """One FX correlator configuration (stations, subbands, channels, taps,
    spectra per block, sample format, X-stage precision)."""

    def __init__(self, n_stations: int, n_subbands: int, n_channels: int, n_spectra: int,
                 taps, centres, n_taps: int = 16, fmt: int = FX_CI16, precision: int = FX_F32,
                 sample_rate_hz: float = SAMPLE_RATE_HZ, operand_scale: float = 0.0, device=None,
                 host_chunk_subbands: int = 0, streaming: bool = False, max_coarse_shift: int = 0,
                 max_beams: int = 0, xf32_form: str = "auto", extra_flags: int = 0,
                 chunk_subbands: int = 0, chunk_spectra: int = 0):
        self.lib = _abi.load()
        if device is not None:
            torch.cuda.set_device(device)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.N, self.SB, self.C, self.S, self.T = n_stations, n_subbands, n_channels, n_spectra, n_taps
        self.fmt, self.precision = fmt, precision
        self.operand_scale = operand_scale if operand_scale else 1.0
        taps = np.ascontiguousarray(np.asarray(taps, dtype=np.float32).reshape(-1))
        centres = np.ascontiguousarray(np.asarray(centres, dtype=np.float64).reshape(-1))
        if taps.size != n_taps * n_channels:
            raise ValueError("taps must have n_taps * n_channels entries")
        if centres.size != n_subbands:
            raise ValueError("centres must have n_subbands entries")
        self._taps, self._centres = taps, centres
        p = _abi.fx_params()
        p.n_stations, p.n_pols, p.n_subbands = n_stations, 2, n_subbands
        p.n_channels, p.n_taps, p.n_spectra = n_channels, n_taps, n_spectra
        p.format, p.precision = fmt, precision
        p.sample_rate_hz = sample_rate_hz
        p.h_subband_centre_hz = centres.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        p.h_taps = taps.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        p.operand_scale = operand_scale
        # FP32 X-stage form: "auto" (4x4 tiles from 16 stations up), "2x4" tiles, or
        # "3mult" (2x4 tiles with the three-multiplication complex product)
        form = {"auto": 0, "2x4": _abi.FX_FLAG_XF32_SMALL_TILES, "3mult": _abi.FX_FLAG_XF32_THREE_MULT}[xf32_form]
        p.flags = (_abi.FX_FLAG_STREAMING if streaming else 0) | form | extra_flags
        p.host_chunk_subbands = host_chunk_subbands
        p.max_coarse_shift = max_coarse_shift
        p.max_beams = max_beams
        p.chunk_subbands, p.chunk_spectra = chunk_subbands, chunk_spectra
        h = ctypes.c_void_p()
        check(self.lib.fx_create(ctypes.byref(p), ctypes.byref(h)), "fx_create")
        self.handle = h
        sz = _abi.fx_sizes()
        check(self.lib.fx_query_sizes(h, ctypes.byref(sz)), "fx_query_sizes")
        self.sizes = sz
        self.I, self.I_pad, self.S_pad, self.B = sz.n_inputs, sz.n_inputs_pad, sz.n_spectra_pad, sz.n_baselines
        self.planes = sz.corr_planes

    # -- shapes -----------------------------------------------------------
    def raw_shape(self):
        # int16/int8: trailing (re, im); int4: one packed byte per complex sample
        return (self.SB, self.N, (self.S + self.T - 1) * self.C, 2, 1 if self.fmt == FX_CI4 else 2)

    def raw_dtype(self):
        return {FX_CI16: torch.int16, FX_CI8: torch.int8, FX_CI4: torch.uint8}[self.fmt]

    def new_shape(self):
        # streaming: the S*C new samples of one block per (subband, station, pol)
        return (self.SB, self.N, self.S * self.C, 2, 1 if self.fmt == FX_CI4 else 2)

    def chan_shape(self):
        return (self.SB, self.N, 2, self.S, self.C, 2)

    def corr_shape(self):
        if self.precision == FX_F32:   # spectrum-blocked; f32_unblock gives [SB][C][S][N][2][2]
            return (self.SB, self.C, (self.S + 15) // 16, self.N, 16, 2, 2)
        return (self.SB, self.C, self.planes, self.I_pad, self.S_pad)

    def corr_dtype(self):
        return {FX_F32: torch.float32, FX_F16: torch.float16, FX_F16_SPLIT: torch.float16,
                FX_TF32_SPLIT: torch.float32}.get(
            self.precision, torch.bfloat16)

    def vis_shape(self):
        return (self.SB, self.C, self.B, 4, 2)

    # -- checks -----------------------------------------------------------
    def _dev(self, t: torch.Tensor, name: str, dtype, nbytes: int):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if t.device != self.device:
            raise ValueError(f"{name} must be on {self.device} (got {t.device})")
        if t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype} (got {t.dtype})")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() * t.element_size() != nbytes:
            raise ValueError(f"{name} has {t.numel() * t.element_size()} bytes, expected {nbytes}")
        return ctypes.c_void_p(t.data_ptr())

    def _host(self, t, name, dtype, nbytes, optional=False):
        if t is None and optional:
            return None
        if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
            raise TypeError(f"{name} must be a CPU torch tensor")
        if t.dtype != dtype or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous {dtype} tensor")
        if t.numel() * t.element_size() != nbytes:
            raise ValueError(f"{name} has {t.numel() * t.element_size()} bytes, expected {nbytes}")
        return ctypes.c_void_p(t.data_ptr())

    def process_host(self, raw, delay_begin, delay_end, bandpass=None, gains=None, out=None, stream=None):
        """fx_process_host: host raw block in, host visibilities out (page-locked
        CPU tensors for overlap), pipelined over subband chunks. Returns `out`
        after synchronising `stream`."""
        rdt = self.raw_dtype()
        if out is None:
            out = torch.empty(self.vis_shape(), dtype=torch.float32, pin_memory=True)
        N, C = self.N, self.C
        s = torch.cuda.current_stream() if stream is None else stream
        check(self.lib.fx_process_host(
            self.handle, self._host(raw, "raw", rdt, self.sizes.raw_bytes),
            self._host(delay_begin, "delay_begin", torch.float64, 8 * N),
            self._host(delay_end, "delay_end", torch.float64, 8 * N),
            self._host(bandpass, "bandpass", torch.float32, 4 * N * C, optional=True),
            self._host(gains, "gains", torch.float32, 16 * N, optional=True),
            self._host(out, "vis", torch.float32, self.sizes.vis_bytes), ctypes.c_void_p(s.cuda_stream)),
            "fx_process_host")
        s.synchronize()
        return out

    def _opt(self, t, name, dtype, nbytes):
        return None if t is None else self._dev(t, name, dtype, nbytes)

    # -- entry points -----------------------------------------------------
    def channelize(self, raw: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        rdt = self.raw_dtype()
        if out is None:
            out = torch.empty(self.chan_shape(), dtype=torch.float32, device=self.device)
        check(self.lib.fx_channelize(self.handle, self._dev(raw, "raw", rdt, self.sizes.raw_bytes),
                                     self._dev(out, "chan", torch.float32, self.sizes.chan_bytes),
                                     _stream_ptr(stream)), "fx_channelize")
        return out

    def correct(self, chan, delay_begin, delay_end, bandpass=None, gains=None, out=None, stream=None):
        if out is None:
            out = torch.empty(self.corr_shape(), dtype=self.corr_dtype(), device=self.device)
        N, C = self.N, self.C
        check(self.lib.fx_correct(
            self.handle, self._dev(chan, "chan", torch.float32, self.sizes.chan_bytes),
            self._dev(delay_begin, "delay_begin", torch.float64, 8 * N),
            self._dev(delay_end, "delay_end", torch.float64, 8 * N),
            self._opt(bandpass, "bandpass", torch.float32, 4 * N * C),
            self._opt(gains, "gains", torch.float32, 16 * N),
            self._dev(out, "corr", self.corr_dtype(), self.sizes.corr_bytes),
            _stream_ptr(stream)), "fx_correct")
        return out

    def channelize_correct(self, raw, delay_begin, delay_end, bandpass=None, gains=None, out=None,
                           stream=None):
        """fx_channelize + fx_correct in one pass (no channelised intermediate)."""
        rdt = self.raw_dtype()
        if out is None:
            out = torch.empty(self.corr_shape(), dtype=self.corr_dtype(), device=self.device)
        N, C = self.N, self.C
        check(self.lib.fx_channelize_correct(
            self.handle, self._dev(raw, "raw", rdt, self.sizes.raw_bytes),
            self._dev(delay_begin, "delay_begin", torch.float64, 8 * N),
            self._dev(delay_end, "delay_end", torch.float64, 8 * N),
            self._opt(bandpass, "bandpass", torch.float32, 4 * N * C),
            self._opt(gains, "gains", torch.float32, 16 * N),
            self._dev(out, "corr", self.corr_dtype(), self.sizes.corr_bytes),
            _stream_ptr(stream)), "fx_channelize_correct")
        return out

    def channelize_correlate(self, raw, delay_begin, delay_end, bandpass=None, gains=None, out=None, stream=None):
        """fx_channelize_correlate: raw samples to visibilities piece by piece
        (chunk_subbands x chunk_spectra), the corrected block never whole in HBM."""
        if out is None:
            out = torch.empty(self.vis_shape(), dtype=torch.float32, device=self.device)
        N, C = self.N, self.C
        check(self.lib.fx_channelize_correlate(
            self.handle, self._dev(raw, "raw", self.raw_dtype(), self.sizes.raw_bytes),
            self._dev(delay_begin, "delay_begin", torch.float64, 8 * N),
            self._dev(delay_end, "delay_end", torch.float64, 8 * N),
            self._opt(bandpass, "bandpass", torch.float32, 4 * N * C),
            self._opt(gains, "gains", torch.float32, 16 * N),
            self._dev(out, "vis", torch.float32, self.sizes.vis_bytes), _stream_ptr(stream)),
            "fx_channelize_correlate")
        return out

    def correlate(self, corr, out=None, stream=None):
        if out is None:
            out = torch.empty(self.vis_shape(), dtype=torch.float32, device=self.device)
        check(self.lib.fx_correlate(self.handle,
                                    self._dev(corr, "corr", self.corr_dtype(), self.sizes.corr_bytes),
                                    self._dev(out, "vis", torch.float32, self.sizes.vis_bytes),
                                    _stream_ptr(stream)), "fx_correlate")
        return out

    # -- streaming form ---------------------------------------------------------
    def stream_block(self, new, delay_begin, delay_end, coarse_shift=None, bandpass=None, gains=None,
                     flags=None, corr=None, vis=None, counts=None, want_vis=True, stream=None):
        """fx_stream_block: one block of a continuous stream (history kept in
        the handle). Returns (corr, vis or None, counts or None); counts are
        produced when `flags` is given or `counts` is passed."""
        N, C, S = self.N, self.C, self.S
        new_bytes = int(np.prod(self.new_shape())) * (2 if self.fmt == FX_CI16 else 1)
        if corr is None:
            corr = torch.empty(self.corr_shape(), dtype=self.corr_dtype(), device=self.device)
        if vis is None and want_vis:
            vis = torch.empty(self.vis_shape(), dtype=torch.float32, device=self.device)
        if counts is None and flags is not None:
            counts = torch.empty(self.B, dtype=torch.float32, device=self.device)
        check(self.lib.fx_stream_block(
            self.handle, self._dev(new, "new", self.raw_dtype(), new_bytes),
            self._opt(coarse_shift, "coarse_shift", torch.int32, 4 * N),
            self._dev(delay_begin, "delay_begin", torch.float64, 8 * N),
            self._dev(delay_end, "delay_end", torch.float64, 8 * N),
            self._opt(bandpass, "bandpass", torch.float32, 4 * N * C),
            self._opt(gains, "gains", torch.float32, 16 * N),
            self._opt(flags, "flags", torch.float32, 4 * N * S),
            self._dev(corr, "corr", self.corr_dtype(), self.sizes.corr_bytes),
            self._opt(vis, "vis", torch.float32, self.sizes.vis_bytes),
            self._opt(counts, "counts", torch.float32, 4 * self.B), _stream_ptr(stream)), "fx_stream_block")
        return corr, vis, counts

    # -- coherent beamformer ----------------------------------------------------
    def beam_shape(self, n_beams, output=0, tint=1):
        SB, C, S = self.SB, self.C, self.S
        return {0: (SB, n_beams, C, S, 4), 1: (SB, n_beams, C, S // tint),
                2: (SB, n_beams, C, S // tint, 4)}[output]

    def beamform(self, corr, beam_delays, station_weights=None, output=0, tint=1, out=None, stream=None):
        """fx_beamform: coherent beams from the corrected FP16/BF16 block.
        beam_delays [n_beams][N] float64 (seconds), station_weights [N] float32."""
        nb = int(beam_delays.shape[0])
        if out is None:
            out = torch.empty(self.beam_shape(nb, output, tint), dtype=torch.float32, device=self.device)
        check(self.lib.fx_beamform(
            self.handle, self._dev(corr, "corr", self.corr_dtype(), self.sizes.corr_bytes), nb,
            self._dev(beam_delays, "beam_delays", torch.float64, 8 * nb * self.N),
            self._opt(station_weights, "station_weights", torch.float32, 4 * self.N), output, tint,
            self._dev(out, "out", torch.float32, 4 * int(np.prod(self.beam_shape(nb, output, tint)))),
            _stream_ptr(stream)), "fx_beamform")
        return out

    def beamform_incoherent(self, corr, station_weights=None, output=1, tint=1, out=None, stream=None):
        """fx_beamform_incoherent: Stokes I (output 1) or IQUV (2) per station,
        weighted sum over stations, summed over tint spectra."""
        shape = (self.SB, self.C, self.S // tint) if output == 1 else (self.SB, self.C, self.S // tint, 4)
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=self.device)
        check(self.lib.fx_beamform_incoherent(
            self.handle, self._dev(corr, "corr", self.corr_dtype(), self.sizes.corr_bytes),
            self._opt(station_weights, "station_weights", torch.float32, 4 * self.N), output, tint,
            self._dev(out, "out", torch.float32, 4 * int(np.prod(shape))), _stream_ptr(stream)),
            "fx_beamform_incoherent")
        return out

    def poll_status(self):
        """fx_poll_status: (status, code) of the device-side error word (synchronises)."""
        code = ctypes.c_int(0)
        rc = self.lib.fx_poll_status(self.handle, ctypes.byref(code))
        return rc, code.value

    def stream_reset(self, stream=None):
        check(self.lib.fx_stream_reset(self.handle, _stream_ptr(stream)), "fx_stream_reset")

    # -- differentiation form -------------------------------------------------
    def raw_vis(self, chan, bandpass=None, stream=None):
        """R: correlation of the bandpass-corrected data with unit gains and zero
        delays (fx_correct + fx_correlate); input of fx_apply_gains and of the
        adjoint."""
        zero = torch.zeros(self.N, dtype=torch.float64, device=self.device)
        return self.correlate(self.correct(chan, zero, zero, bandpass=bandpass, stream=stream), stream=stream)

    def apply_gains(self, raw_vis, gains, delays, out=None, stream=None):
        if out is None:
            out = torch.empty(self.vis_shape(), dtype=torch.float32, device=self.device)
        vb = self.sizes.vis_bytes
        check(self.lib.fx_apply_gains(self.handle, self._dev(raw_vis, "raw_vis", torch.float32, vb),
                                      self._opt(gains, "gains", torch.float32, 16 * self.N),
                                      self._dev(delays, "delays", torch.float64, 8 * self.N),
                                      self._dev(out, "vis", torch.float32, vb), _stream_ptr(stream)),
              "fx_apply_gains")
        return out

    def backward(self, raw_vis, gains, delays, grad_vis, stream=None):
        """(dL/d gains [N][2][2] float32, dL/d delays [N] float64) from
        grad_vis = (dL/dRe V, dL/dIm V) in the vis layout."""
        gg = torch.empty((self.N, 2, 2), dtype=torch.float32, device=self.device)
        gt = torch.empty(self.N, dtype=torch.float64, device=self.device)
        vb = self.sizes.vis_bytes
        check(self.lib.fx_correct_correlate_backward(
            self.handle, self._dev(raw_vis, "raw_vis", torch.float32, vb),
            self._opt(gains, "gains", torch.float32, 16 * self.N),
            self._dev(delays, "delays", torch.float64, 8 * self.N),
            self._dev(grad_vis, "grad_vis", torch.float32, vb),
            self._dev(gg, "grad_gains", torch.float32, 16 * self.N),
            self._dev(gt, "grad_delays", torch.float64, 8 * self.N), _stream_ptr(stream)),
            "fx_correct_correlate_backward")
        return gg, gt

    def backward_interp(self, chan, gains, delay_begin, delay_end, grad_vis, bandpass=None, stream=None,
                        work_corr=None, work_vis=None):
        """(dL/d gains [N][2][2] float32, dL/d delay_begin [N], dL/d delay_end [N]
        float64) for delays moving linearly over the block, from the channelised
        block and grad_vis = (dL/dRe V, dL/dIm V) (fx_correct_correlate_backward_interp;
        the work buffers are allocated here when not given)."""
        gg = torch.empty((self.N, 2, 2), dtype=torch.float32, device=self.device)
        gb = torch.empty(self.N, dtype=torch.float64, device=self.device)
        ge = torch.empty(self.N, dtype=torch.float64, device=self.device)
        if work_corr is None:
            work_corr = torch.empty(self.corr_shape(), dtype=self.corr_dtype(), device=self.device)
        if work_vis is None:
            work_vis = torch.empty((2,) + self.vis_shape(), dtype=torch.float32, device=self.device)
        vb = self.sizes.vis_bytes
        check(self.lib.fx_correct_correlate_backward_interp(
            self.handle, self._dev(chan, "chan", torch.float32, self.sizes.chan_bytes),
            self._dev(delay_begin, "delay_begin", torch.float64, 8 * self.N),
            self._dev(delay_end, "delay_end", torch.float64, 8 * self.N),
            self._opt(bandpass, "bandpass", torch.float32, 4 * self.N * self.C),
            self._opt(gains, "gains", torch.float32, 16 * self.N),
            self._dev(grad_vis, "grad_vis", torch.float32, vb),
            self._dev(work_corr, "work_corr", self.corr_dtype(), self.sizes.corr_bytes),
            self._dev(work_vis, "work_vis", torch.float32, 2 * vb),
            self._dev(gg, "grad_gains", torch.float32, 16 * self.N),
            self._dev(gb, "grad_delay_begin", torch.float64, 8 * self.N),
            self._dev(ge, "grad_delay_end", torch.float64, 8 * self.N), _stream_ptr(stream)),
            "fx_correct_correlate_backward_interp")
        return gg, gb, ge

    def close(self):
        if getattr(self, "handle", None):
            self.lib.fx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
