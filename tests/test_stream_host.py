"""Host-side pins of the streaming reading used by the GPU streaming test.

The per-block windows the oracle is given must (a) tile one long block: with
zero coarse shifts, the spectra of block k of the stream are spectra
[k*S, (k+1)*S) of the channelisation of the whole stream with (T-1)*C zeros
before it (the FIR history carried across blocks); and (b) apply a coarse
shift of d samples as a stream delayed by d samples (d zeros prepended).
"""
import numpy as np

import oracle
import synth
from test_gpu_stream import make_stream, window


def test_windows_tile_the_stream():
    fmt, SB, N, C, S, T, K = synth.CI16, 1, 2, 16, 5, 4, 3
    stream = make_stream(3, fmt, SB, N, K * S * C)
    taps = synth.kaiser_sinc_taps(T, C)
    whole = np.concatenate([np.zeros((SB, N, (T - 1) * C, 2, 2), np.int16), stream], axis=2)
    ref = oracle.channelize(fmt, whole, T, C, K * S, taps)
    zero = np.zeros(N, np.int64)
    for k in range(K):
        got = oracle.channelize(fmt, window(stream, k, S, C, T, zero), T, C, S, taps)
        assert np.array_equal(got, ref[:, :, :, k * S:(k + 1) * S])


def test_coarse_shift_is_a_delayed_stream():
    fmt, SB, N, C, S, T, K = synth.CI8, 2, 3, 16, 4, 4, 3
    stream = make_stream(5, fmt, SB, N, K * S * C)
    shifts = np.array([0, 5, 21])
    for k in range(K):
        w = window(stream, k, S, C, T, shifts)
        for n, d in enumerate(shifts):
            delayed = np.concatenate([np.zeros((SB, d, 2, 2), np.int8), stream[:, n]], axis=1)[:, :K * S * C]
            solo = window(delayed[:, None], k, S, C, T, [0])
            assert np.array_equal(w[:, n], solo[:, 0])
