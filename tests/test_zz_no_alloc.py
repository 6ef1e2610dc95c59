"""The allocation-free correction entry point (fx_correct_f32_noalloc) against
the handle-based fx_correct and against the FP64 oracle's correction, through
the C ABI.

fx_correct_f32_noalloc exists for callers that may not allocate device memory
(a fixed memory budget owned by the host program, a plugin host that forbids
the CUDA allocator, a real-time thread that cannot afford an allocation's
device-wide synchronisation). It keeps its phase table in a fixed device array
inside the library instead of a handle's workspace. This file is collected
last so that a run stopping at the first failure has already run every other
test; it passes alone in a fresh process and after the other tests (the first
call on the device does the one-time address lookup either way).
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE_HZ


def _dev(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _noalloc(lib, N, SB, C, S, centres, tb, te, bp, g, chan, out):
    return lib.fx_correct_f32_noalloc(N, SB, C, S, FS, _p(centres), _p(tb), _p(te), _p(bp), _p(g),
                                      _p(chan), _p(out), None)


@pytest.mark.parametrize("N,SB,C,S", [(6, 3, 64, 37), (500, 1, 16, 20)])
def test_noalloc_matches_fx_correct_on_two_calls(N, SB, C, S):
    """Two calls in a row with different inputs, each equal to fx_correct
    (same kernels, so within 2e-6) and to the oracle's correction (FP32
    rotation of an FP64-formed phase: 2e-6 normwise). 500 stations is above
    any shared-memory limit the correction could have per station."""
    import paper_1801_04834_gb300 as fxg
    from paper_1801_04834_gb300 import _abi
    lib = _abi.load()
    centres = synth.subband_centres(SB)
    blk = synth.Block(0, SB, N, 2, C, 16, S, None, synth.kaiser_sinc_taps(16, C), centres)
    c = fxg.Correlator(N, SB, C, S, taps=blk.taps, centres=centres)
    d_centres = _dev(centres, torch.float64)
    out = torch.empty(c.corr_shape(), dtype=torch.float32, device="cuda")
    for call in range(2):                       # two calls in a row, different inputs
        rng = np.random.default_rng(100 + call)
        chan_h = synth.channelised_noise(200 + call, SB, N, 2, C, S, sigma=300.0)
        chan = _dev(chan_h)
        tb = rng.uniform(-5e-6, 5e-6, N)
        te = tb + rng.uniform(-2e-8, 2e-8, N)
        bp_h = rng.uniform(0.7, 1.3, (N, C)) if call == 0 else None
        bp = None if bp_h is None else _dev(bp_h)
        g_h = synth.random_gains(rng, N)
        g = _dev(g_h)
        d_tb, d_te = _dev(tb, torch.float64), _dev(te, torch.float64)
        ref = c.correct(chan, d_tb, d_te, bandpass=bp, gains=g)
        out.fill_(float("nan"))
        rc = _noalloc(lib, N, SB, C, S, d_centres, d_tb, d_te, bp, g, chan, out)
        assert rc == 0, _abi.last_error()
        torch.cuda.synchronize()
        rel = (torch.linalg.vector_norm((out - ref).double()) / torch.linalg.vector_norm(ref.double())).item()
        assert rel < 2e-6, f"call {call}: relative difference {rel}"
        oref = oracle.correct(chan_h, FS, centres, tb, te, bandpass=bp_h, gains=g_h)
        got = fxg.f32_unblock(out, S).cpu().numpy().astype(np.float64)
        orel = np.linalg.norm(got - oref) / np.linalg.norm(oref)
        assert orel < 2e-6, f"call {call}: relative error against the oracle {orel}"
    c.close()


def test_noalloc_rejects_oversize_and_bad_args():
    from paper_1801_04834_gb300 import _abi
    lib = _abi.load()
    t = torch.zeros(16, dtype=torch.float64, device="cuda")
    # 65 subbands x 64 stations x 256 channels = 1064960 > 2^20 entries
    rc = lib.fx_correct_f32_noalloc(64, 65, 256, 8, FS, _p(t), _p(t), _p(t), None, None, _p(t), _p(t), None)
    assert rc == _abi.FX_ERR_INVALID
    assert "exceeds" in _abi.last_error()
    rc = lib.fx_correct_f32_noalloc(4, 1, 32, 8, FS, _p(t), _p(t), _p(t), None, None, _p(t), _p(t), None)
    assert rc == _abi.FX_ERR_UNSUPPORTED
    rc = lib.fx_correct_f32_noalloc(4, 1, 64, 8, FS, None, _p(t), _p(t), None, None, _p(t), _p(t), None)
    assert rc == _abi.FX_ERR_INVALID
    # more spectra than the correction's grid covers: rejected before any launch
    rc = lib.fx_correct_f32_noalloc(1, 1, 16, 4194241, FS, _p(t), _p(t), _p(t), None, None, _p(t), _p(t), None)
    assert rc == _abi.FX_ERR_INVALID
    assert "out of range" in _abi.last_error()
