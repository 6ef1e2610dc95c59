"""fx_channelize_correlate: the F-stage and X-stage run piece by piece
(chunk_subbands x chunk_spectra) through two L2-sized operand buffers, the
X-stage adding each piece into the visibilities. Against the unchunked calls
(fx_channelize_correct + fx_correlate) the operands are identical and only
the order of the FP32 sums over time differs, so FP32 agrees to ~1e-7
normwise (bound 1e-6) and the tensor-core forms agree to their accumulation
rounding (bound 1e-5 normwise); against the FP64 oracle the path bounds hold.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import baseline_max_rel, make_corr, per_subband_rel, tone_block

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE_HZ


@pytest.mark.parametrize("precision,bound", [(0, 1e-5), (1, 5e-3), (2, 2e-2)])
@pytest.mark.parametrize("fmt,SB,N,C,S,G,TC", [(synth.CI16, 3, 8, 64, 256, 2, 64),
                                              (synth.CI8, 2, 20, 256, 128, 1, 128),
                                              (synth.CI16, 4, 5, 16, 192, 4, 64)])
def test_chunked_matches_unchunked_and_oracle(precision, bound, fmt, SB, N, C, S, G, TC):
    blk, tau, rip = tone_block(40 + N + C, fmt, SB, N, C, S, ripple=True,
                               sigma=100.0 if fmt == synth.CI16 else 20.0)
    rng = np.random.default_rng(S)
    te = tau + rng.uniform(-2e-8, 2e-8, N)
    g = synth.random_gains(rng, N)
    kw = dict(precision=precision, operand_scale=2.0 ** -6 if precision else 0.0)
    c = make_corr(blk, chunk_subbands=G, chunk_spectra=TC, **kw)
    raw = torch.from_numpy(blk.raw).cuda()
    tb_d, te_d = torch.from_numpy(tau).cuda(), torch.from_numpy(te).cuda()
    bp = torch.from_numpy((1.0 / rip).astype(np.float32)).cuda()
    gd = torch.from_numpy(g.astype(np.float32)).cuda()
    vis = torch.full(c.vis_shape(), float("nan"), device="cuda")
    c.channelize_correlate(raw, tb_d, te_d, bandpass=bp, gains=gd, out=vis)
    ref_gpu = c.correlate(c.channelize_correct(raw, tb_d, te_d, bandpass=bp, gains=gd))
    torch.cuda.synchronize()
    a, b = vis.double(), ref_gpu.double()
    assert torch.isfinite(a).all()
    rel = (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()
    assert rel < (1e-6 if precision == 0 else 1e-5), rel
    chan = oracle.channelize(fmt, blk.raw, 16, C, S, blk.taps)
    ref = oracle.correlate(oracle.correct(chan, FS, blk.centres, tau, te, 1.0 / rip, g))
    got = vis.cpu().numpy().astype(np.float64)
    e = per_subband_rel(got, ref)
    assert np.all(e < bound), e
    # per baseline, max |dV_ij| / sqrt(|V_ii| |V_jj|): 5e-5 FP32, 1e-3 FP16, 1e-2 BF16 operands
    assert baseline_max_rel(got, ref, N) < {0: 5e-5, 1: 1e-3, 2: 1e-2}[precision]
    c.close()


def test_chunked_needs_chunk_buffers():
    blk, tau, _ = tone_block(1, synth.CI16, 1, 4, 16, 64)
    c = make_corr(blk)
    t = torch.from_numpy(tau).cuda()
    with pytest.raises(RuntimeError):
        c.channelize_correlate(torch.from_numpy(blk.raw).cuda(), t, t)
    c.close()
    with pytest.raises(RuntimeError):
        make_corr(blk, chunk_subbands=1, chunk_spectra=48)     # not a multiple of 64
