"""ctypes binding of include/fx.h: the same entry points, argument marshalling
only. Every step of the hot path runs in libfx_gb300.so; if the library is
missing or cannot load, import fails loudly (there is no fallback)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfx_gb300.so")

FX_OK, FX_ERR_INVALID, FX_ERR_CUDA, FX_ERR_NOMEM, FX_ERR_TIMEOUT, FX_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5
FX_CI16, FX_CI8, FX_CI4 = 0, 1, 2
FX_F32, FX_F16, FX_BF16, FX_F16_SPLIT, FX_TF32_SPLIT = 0, 1, 2, 3, 4

STATUS_NAMES = {0: "FX_OK", -1: "FX_ERR_INVALID", -2: "FX_ERR_CUDA", -3: "FX_ERR_NOMEM",
                -4: "FX_ERR_TIMEOUT", -5: "FX_ERR_UNSUPPORTED"}


class FxError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class fx_params(ctypes.Structure):
    _fields_ = [("n_stations", ctypes.c_int), ("n_pols", ctypes.c_int),
                ("n_subbands", ctypes.c_int), ("n_channels", ctypes.c_int),
                ("n_taps", ctypes.c_int), ("n_spectra", ctypes.c_int),
                ("format", ctypes.c_int), ("precision", ctypes.c_int),
                ("sample_rate_hz", ctypes.c_double),
                ("h_subband_centre_hz", ctypes.POINTER(ctypes.c_double)),
                ("h_taps", ctypes.POINTER(ctypes.c_float)),
                ("operand_scale", ctypes.c_float), ("flags", ctypes.c_uint),
                ("host_chunk_subbands", ctypes.c_int), ("max_coarse_shift", ctypes.c_int),
                ("chunk_subbands", ctypes.c_int), ("chunk_spectra", ctypes.c_int),
                ("max_beams", ctypes.c_int)]


class fx_sizes(ctypes.Structure):
    _fields_ = [("raw_bytes", ctypes.c_size_t), ("chan_bytes", ctypes.c_size_t),
                ("corr_bytes", ctypes.c_size_t), ("vis_bytes", ctypes.c_size_t),
                ("n_inputs", ctypes.c_int), ("n_inputs_pad", ctypes.c_int),
                ("n_spectra_pad", ctypes.c_int), ("n_baselines", ctypes.c_int),
                ("corr_planes", ctypes.c_int)]


# name -> (restype, argtypes); mirrors include/fx.h
P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
SIGNATURES = {
    "fx_create": (I, [ctypes.POINTER(fx_params), ctypes.POINTER(P)]),
    "fx_destroy": (None, [P]),
    "fx_last_error": (ctypes.c_char_p, []),
    "fx_query_sizes": (I, [P, ctypes.POINTER(fx_sizes)]),
    "fx_channelize": (I, [P, P, P, P]),
    "fx_correct": (I, [P, P, P, P, P, P, P, P]),
    "fx_correlate": (I, [P, P, P, P]),
    "fx_channelize_correct": (I, [P, P, P, P, P, P, P, P]),
    "fx_process_host": (I, [P, P, P, P, P, P, P, P]),
    "fx_stream_block": (I, [P, P, P, P, P, P, P, P, P, P, P, P]),
    "fx_stream_reset": (I, [P, P]),
    "fx_beamform": (I, [P, P, I, P, P, I, I, P, P]),
    "fx_ffma_probe": (I, [I, I, P, P]),
    "fx_channelize_correlate": (I, [P, P, P, P, P, P, P, P]),
    "fx_beamform_incoherent": (I, [P, P, P, I, I, P, P]),
    "fx_poll_status": (I, [P, ctypes.POINTER(ctypes.c_int)]),
    "fx_apply_gains": (I, [P, P, P, P, P, P]),
    "fx_batch_create": (I, [P, I, I, ctypes.c_float, ctypes.POINTER(P)]),
    "fx_batch_autotune": (I, [P, I, P]),
    "fx_correlate_batched": (I, [P, P]),
    "fx_batch_describe": (ctypes.c_char_p, [P]),
    "fx_batch_poll_status": (I, [P, ctypes.POINTER(ctypes.c_int)]),
    "fx_batch_destroy": (None, [P]),
    "fx_correct_correlate_backward": (I, [P, P, P, P, P, P, P, P]),
    "fx_correct_correlate_backward_interp": (I, [P, P, P, P, P, P, P, P, P, P, P, P, P]),
    "fx_correct_f32_noalloc": (I, [I, I, I, I, D, P, P, P, P, P, P, P, P]),
}
FX_NOALLOC_MAX_PHASES = 1 << 20
FX_FLAG_TEST_NO_LOADS = 0x80000000
FX_FLAG_STREAMING = 0x1
FX_FLAG_XF32_SMALL_TILES = 0x2
FX_FLAG_XF32_THREE_MULT = 0x4
FX_BEAM_VOLTAGES, FX_BEAM_STOKES_I, FX_BEAM_STOKES_IQUV = 0, 1, 2

_lib = None


def load(path: str = LIB_PATH):
    """Load the compiled library (build it first with __graft_entry__.build()
    or python -m paper_1801_04834_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built; run paper_1801_04834_gb300/build.py "
                          "(the hot path has no fallback)")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def last_error() -> str:
    return load().fx_last_error().decode()


def check(status: int, where: str):
    if status != FX_OK:
        raise FxError(status, where, last_error())


class fx_job(ctypes.Structure):
    _fields_ = [("n_stations", ctypes.c_int), ("n_subbands", ctypes.c_int),
                ("n_channels", ctypes.c_int), ("n_spectra", ctypes.c_int),
                ("d_corr", ctypes.c_void_p), ("d_vis", ctypes.c_void_p)]
