"""FP64 CPU oracle for the FX correlator hot path (ctypes binding to fx_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
bench.py's CPU-baseline leg, never by the product package. It shares no code
with the CUDA path. Each wrapper takes and returns numpy arrays in the layouts
documented in fx_oracle.c (complex values as a trailing axis of 2 float64).

Parity status: every function here is pinned by tests/test_oracle_pins.py
against closed forms, library routines (numpy.fft, numpy.einsum), invariants
or finite differences; none is "parity unpinned". tests/test_oracle_mutants.py
plants mistakes in a copy of fx_oracle.c and checks that a pin catches each.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "fx_oracle.c")
LIBRARY = os.path.join(_HERE, "libfxoracle.so")


def compile_oracle(src: str, out: str) -> str:
    """gcc -O2 with OpenMP and IEEE semantics (no fast-math)."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIBRARY) or os.path.getmtime(LIBRARY) < os.path.getmtime(SOURCE):
        compile_oracle(SOURCE, LIBRARY)
    return LIBRARY


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """The oracle's entry points, bound to one compiled copy of fx_oracle.c."""

    def __init__(self, path: str):
        L = ctypes.CDLL(path)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.fxo_channelize.argtypes = [I, P, I, I, I, I, I, I, P, P]
        L.fxo_correct.argtypes = [P, I, I, I, I, I, D, P, P, P, P, P, P, P]
        L.fxo_baseline_counts.argtypes = [P, I, I, P]
        L.fxo_baseline_counts.restype = I
        L.fxo_correlate.argtypes = [P, I, I, I, I, I, P]
        L.fxo_fx.argtypes = [I, P, I, I, I, I, I, I, P, D, P, P, P, P, P, P]
        L.fxo_vjp.argtypes = [P, I, I, I, I, I, D, P, P, P, P, P, P, P]
        L.fxo_vjp_interp.argtypes = [P, I, I, I, I, I, D, P, P, P, P, P, P, P, P, P]
        L.fxo_beamform.argtypes = [P, I, I, I, I, I, D, P, I, P, P, I, I, P]
        L.fxo_beamform_incoherent.argtypes = [P, I, I, I, I, I, P, I, I, P]
        for f in (L.fxo_channelize, L.fxo_correct, L.fxo_correlate, L.fxo_fx, L.fxo_vjp, L.fxo_vjp_interp,
                  L.fxo_beamform, L.fxo_beamform_incoherent, L.fxo_threads):
            f.restype = I
        self._L = L

    @staticmethod
    def _check(rc, name):
        if rc != 0:
            raise RuntimeError(f"oracle {name} failed with {rc}")

    def threads(self) -> int:
        return self._L.fxo_threads()

    def channelize(self, fmt, raw, n_taps, n_channels, n_spectra, taps):
        """raw [SB][N][L][P][2] int16/int8 -> chan [SB][N][P][S][C][2] float64."""
        raw = np.ascontiguousarray(raw)
        SB, N, L, P, _ = raw.shape
        assert L == (n_spectra + n_taps - 1) * n_channels
        out = np.empty((SB, N, P, n_spectra, n_channels, 2))
        self._check(self._L.fxo_channelize(fmt, _ptr(raw), SB, N, P, n_channels, n_taps,
                                           n_spectra, _ptr(_f64(taps)), _ptr(out)), "channelize")
        return out

    def correct(self, chan, fs, centres, tau_begin, tau_end, bandpass=None, gains=None, flags=None):
        """chan [SB][N][P][S][C][2] -> corr [SB][C][S][N][P][2]; flags [N][S] weights."""
        chan = _f64(chan)
        SB, N, P, S, C, _ = chan.shape
        out = np.empty((SB, C, S, N, P, 2))
        self._check(self._L.fxo_correct(_ptr(chan), SB, N, P, C, S, fs, _ptr(_f64(centres)),
                                        _ptr(_f64(tau_begin)), _ptr(_f64(tau_end)),
                                        _ptr(_f64(bandpass)), _ptr(_f64(gains)), _ptr(_f64(flags)),
                                        _ptr(out)),
                    "correct")
        return out

    def baseline_counts(self, flags, N, S):
        """counts [B]: spectra valid for both stations of each baseline."""
        out = np.empty(N * (N + 1) // 2)
        self._check(self._L.fxo_baseline_counts(_ptr(_f64(flags)), N, S, _ptr(out)), "baseline_counts")
        return out

    def correlate(self, corr):
        """corr [SB][C][S][N][P][2] -> vis [SB][C][B][4][2]."""
        corr = _f64(corr)
        SB, C, S, N, P, _ = corr.shape
        out = np.empty((SB, C, N * (N + 1) // 2, 4, 2))
        self._check(self._L.fxo_correlate(_ptr(corr), SB, N, P, C, S, _ptr(out)), "correlate")
        return out

    def fx(self, fmt, raw, n_taps, n_channels, n_spectra, taps, fs, centres, tau_begin,
           tau_end, bandpass=None, gains=None):
        """Whole chain, raw samples -> vis [SB][C][B][4][2]."""
        raw = np.ascontiguousarray(raw)
        SB, N, L, P, _ = raw.shape
        out = np.empty((SB, n_channels, N * (N + 1) // 2, 4, 2))
        self._check(self._L.fxo_fx(fmt, _ptr(raw), SB, N, P, n_channels, n_taps, n_spectra,
                                   _ptr(_f64(taps)), fs, _ptr(_f64(centres)),
                                   _ptr(_f64(tau_begin)), _ptr(_f64(tau_end)),
                                   _ptr(_f64(bandpass)), _ptr(_f64(gains)), _ptr(out)), "fx")
        return out

    def vjp(self, chan, fs, centres, tau, grad_vis, bandpass=None, gains=None):
        """Gradient of a real loss through correct+correlate (constant delays).
        grad_vis holds dL/dRe(V), dL/dIm(V). Returns (grad_gains [N][P][2], grad_tau [N])."""
        chan = _f64(chan)
        SB, N, P, S, C, _ = chan.shape
        gg = np.empty((N, P, 2))
        gt = np.empty(N)
        self._check(self._L.fxo_vjp(_ptr(chan), SB, N, P, C, S, fs, _ptr(_f64(centres)),
                                    _ptr(_f64(tau)), _ptr(_f64(bandpass)), _ptr(_f64(gains)),
                                    _ptr(_f64(grad_vis)), _ptr(gg), _ptr(gt)), "vjp")
        return gg, gt

    def vjp_interp(self, chan, fs, centres, tau_begin, tau_end, grad_vis, bandpass=None, gains=None):
        """Gradient of a real loss through correct+correlate with delays moving
        linearly from tau_begin to tau_end over the block. Returns (grad_gains
        [N][P][2], grad_tau_begin [N], grad_tau_end [N])."""
        chan = _f64(chan)
        SB, N, P, S, C, _ = chan.shape
        gg = np.empty((N, P, 2))
        gb = np.empty(N)
        ge = np.empty(N)
        self._check(self._L.fxo_vjp_interp(_ptr(chan), SB, N, P, C, S, fs, _ptr(_f64(centres)),
                                           _ptr(_f64(tau_begin)), _ptr(_f64(tau_end)), _ptr(_f64(bandpass)),
                                           _ptr(_f64(gains)), _ptr(_f64(grad_vis)), _ptr(gg), _ptr(gb),
                                           _ptr(ge)), "vjp_interp")
        return gg, gb, ge

    def beamform(self, corr, fs, centres, delays, weights=None, mode=0, tint=1):
        """Coherent beams from corr [SB][C][S][N][P][2]; delays [NB][N] seconds,
        weights [N] real. mode 0: voltages [SB][NB][C][S][4]; 1: Stokes I
        [SB][NB][C][S/tint]; 2: Stokes IQUV [SB][NB][C][S/tint][4]."""
        corr = _f64(corr)
        SB, C, S, N, P, _ = corr.shape
        delays = _f64(delays).reshape(-1, N)
        NB = delays.shape[0]
        shape = {0: (SB, NB, C, S, 4), 1: (SB, NB, C, S // tint), 2: (SB, NB, C, S // tint, 4)}[mode]
        out = np.empty(shape)
        self._check(self._L.fxo_beamform(_ptr(corr), SB, N, P, C, S, fs, _ptr(_f64(centres)), NB,
                                         _ptr(delays), _ptr(_f64(weights)), mode, tint, _ptr(out)),
                    "beamform")
        return out

    def beamform_incoherent(self, corr, weights=None, mode=1, tint=1):
        """Incoherent beam from corr [SB][C][S][N][P][2]: mode 1 Stokes I
        [SB][C][S/tint]; mode 2 Stokes IQUV [SB][C][S/tint][4]."""
        corr = _f64(corr)
        SB, C, S, N, P, _ = corr.shape
        out = np.empty((SB, C, S // tint) if mode == 1 else (SB, C, S // tint, 4))
        self._check(self._L.fxo_beamform_incoherent(_ptr(corr), SB, N, P, C, S, _ptr(_f64(weights)), mode, tint,
                                                    _ptr(out)), "beamform_incoherent")
        return out


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def threads():
    return default().threads()


def channelize(*a, **k):
    return default().channelize(*a, **k)


def correct(*a, **k):
    return default().correct(*a, **k)


def baseline_counts(*a, **k):
    return default().baseline_counts(*a, **k)


def correlate(*a, **k):
    return default().correlate(*a, **k)


def fx(*a, **k):
    return default().fx(*a, **k)


def vjp(*a, **k):
    return default().vjp(*a, **k)


def vjp_interp(*a, **k):
    return default().vjp_interp(*a, **k)


def beamform(*a, **k):
    return default().beamform(*a, **k)


def beamform_incoherent(*a, **k):
    return default().beamform_incoherent(*a, **k)
