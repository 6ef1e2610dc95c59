"""fx_process_host (host memory in and out, copies overlapped with compute
over subband chunks) against the device-resident path and the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import per_subband_rel, tone_block

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE_HZ


@pytest.mark.parametrize("precision,bound", [(0, 1e-5), (1, 5e-3), (4, 1e-5)])
@pytest.mark.parametrize("chunk", [2, 5, 7])
def test_process_host_matches_device_path(precision, bound, chunk):
    import paper_1801_04834_gb300 as fxg
    SB, N, C, S = 5, 8, 64, 100
    blk, tau, rip = tone_block(41, synth.CI16, SB, N, C, S, ripple=True)
    g = synth.random_gains(np.random.default_rng(2), N)
    c = fxg.Correlator(N, SB, C, S, taps=blk.taps, centres=blk.centres, precision=precision,
                       host_chunk_subbands=chunk)
    h_raw = torch.from_numpy(blk.raw).pin_memory()
    h_tb = torch.from_numpy(tau.copy())
    h_te = torch.from_numpy(tau + 5e-9)
    h_bp = torch.from_numpy((1.0 / rip).astype(np.float32))
    h_g = torch.from_numpy(g.astype(np.float32))
    vis_h = c.process_host(h_raw, h_tb, h_te, bandpass=h_bp, gains=h_g)
    # device-resident path
    dv = lambda t, dt=None: t.to("cuda") if dt is None else t.to("cuda", dt)
    vis_d = c.correlate(c.channelize_correct(dv(h_raw), dv(h_tb), dv(h_te), bandpass=dv(h_bp),
                                             gains=dv(h_g))).cpu()
    rel = (torch.linalg.vector_norm((vis_h - vis_d).double()) / torch.linalg.vector_norm(vis_d.double())).item()
    assert rel < 1e-6, rel
    ref = oracle.fx(blk.fmt, blk.raw, 16, C, S, blk.taps, FS, blk.centres, tau, tau + 5e-9,
                    bandpass=1.0 / rip, gains=g)
    assert np.all(per_subband_rel(vis_h.numpy().astype(np.float64), ref) < bound)
    # a second call on the same handle reuses the pipeline buffers
    vis_h2 = c.process_host(h_raw, h_tb, h_te, bandpass=h_bp, gains=h_g)
    assert torch.equal(vis_h, vis_h2)
    c.close()


def test_process_host_requires_pipeline():
    import paper_1801_04834_gb300 as fxg
    blk, tau, _ = tone_block(1, synth.CI16, 1, 4, 16, 20)
    c = fxg.Correlator(4, 1, 16, 20, taps=blk.taps, centres=blk.centres)
    with pytest.raises(fxg.FxError):
        c.process_host(torch.from_numpy(blk.raw), torch.from_numpy(tau), torch.from_numpy(tau))
