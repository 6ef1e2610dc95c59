"""The FP32 corrected layout (spectrum-blocked, include/fx.h) and its host-side
reshape helpers: block/unblock round trip, zero padding, and the element
offset formula written in the header, checked element by element."""
import numpy as np
import pytest
import torch

import paper_1801_04834_gb300.api as api


@pytest.mark.parametrize("SB,C,S,N", [(2, 16, 37, 3), (1, 64, 16, 5), (3, 4, 1, 2), (1, 8, 48, 1)])
def test_block_roundtrip_and_padding(SB, C, S, N):
    rng = np.random.default_rng(S * 7 + N)
    y = rng.standard_normal((SB, C, S, N, 2, 2)).astype(np.float32)
    b = api.f32_block(y)
    S16 = (S + 15) // 16 * 16
    assert b.shape == (SB, C, S16 // 16, N, 16, 2, 2)
    assert np.array_equal(api.f32_unblock(b, S), y)
    # padding spectra are zero
    full = api.f32_unblock(b, S16)
    assert np.all(full[:, :, S:] == 0)
    # torch path agrees with the numpy path
    bt = api.f32_block(torch.from_numpy(y))
    assert np.array_equal(bt.numpy(), b)
    assert np.array_equal(api.f32_unblock(bt, S).numpy(), y)


def test_header_offset_formula():
    """Flat float2 offset of (sb, k, s, n, p) =
    (((sb*C + k)*S16/16 + s/16)*N + n)*16*P + (s%16)*P + p."""
    SB, C, S, N, P = 2, 8, 35, 3, 2
    rng = np.random.default_rng(1)
    y = rng.standard_normal((SB, C, S, N, P, 2)).astype(np.float32)
    flat = api.f32_block(y).reshape(-1, 2)
    S16 = (S + 15) // 16 * 16
    for sb in range(SB):
        for k in range(C):
            for s in range(S):
                for n in range(N):
                    for p in range(P):
                        off = (((sb * C + k) * (S16 // 16) + s // 16) * N + n) * 16 * P + (s % 16) * P + p
                        assert np.array_equal(flat[off], y[sb, k, s, n, p]), (sb, k, s, n, p)
