"""CUDA-graph capture of the production step, and the bounded-wait failure
path of the tensor-core beamformer, the TF32-split X-stage and the F-stage's
raw-row waits.

Failure detection is tested without a GPU fault: with FX_FLAG_TEST_NO_LOADS
the kernels' TMA producer issues no loads, so the consumers' mbarrier waits
run out (about a millisecond), the kernel records the role in the status word,
drains, frees its tensor memory and exits; fx_poll_status then reports
FX_ERR_TIMEOUT, and the context stays usable.
"""
import numpy as np
import pytest
import torch

import synth
from test_gpu_parity import make_corr, tone_block

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1, 4])
def test_step_replays_from_a_cuda_graph(precision):
    """fx_channelize_correct + fx_correlate captured once in a CUDA graph and
    replayed give exactly the eagerly computed visibilities (the calls do no
    host work or allocation)."""
    blk, tau, rip = tone_block(12, synth.CI16, 2, 9, 64, 70, ripple=True)
    c = make_corr(blk, precision=precision)
    raw = torch.from_numpy(blk.raw).cuda()
    t = torch.from_numpy(tau).cuda()
    bp = torch.from_numpy((1.0 / rip).astype(np.float32)).cuda()
    corr = torch.empty(c.corr_shape(), dtype=c.corr_dtype(), device="cuda")
    vis = torch.empty(c.vis_shape(), dtype=torch.float32, device="cuda")
    c.channelize_correct(raw, t, t, bandpass=bp, out=corr)
    c.correlate(corr, vis)
    torch.cuda.synchronize()
    eager = vis.clone()
    vis.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            c.channelize_correct(raw, t, t, bandpass=bp, out=corr)
            c.correlate(corr, vis)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        vis.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(vis, eager)
    c.close()


def _normal_call_works():
    blk, tau, _ = tone_block(3, synth.CI16, 1, 4, 16, 32)
    c = make_corr(blk, precision=0)
    t = torch.from_numpy(tau).cuda()
    v = c.correlate(c.channelize_correct(torch.from_numpy(blk.raw).cuda(), t, t))
    torch.cuda.synchronize()
    assert torch.isfinite(v).all()
    c.close()


def test_beamformer_failure_detection_timeout():
    import paper_1801_04834_gb300 as fxg
    blk = synth.make_block(1, synth.CI16, 1, 8, 64, 128)
    c = make_corr(blk, precision=1, max_beams=64, extra_flags=fxg._abi.FX_FLAG_TEST_NO_LOADS)
    corr = torch.zeros(c.corr_shape(), dtype=c.corr_dtype(), device="cuda")
    out = c.beamform(corr, torch.zeros((5, 8), dtype=torch.float64, device="cuda"), output=1, tint=4)
    rc, code = c.poll_status()
    assert rc == fxg._abi.FX_ERR_TIMEOUT and code in (1, 2, 3), (rc, code)
    assert c.poll_status() == (0, 0)                    # cleared
    c.close()
    del out
    _normal_call_works()


def test_tf32_failure_detection_timeout():
    import paper_1801_04834_gb300 as fxg
    blk = synth.make_block(1, synth.CI16, 1, 8, 16, 64)
    c = make_corr(blk, precision=4, extra_flags=fxg._abi.FX_FLAG_TEST_NO_LOADS)
    corr = torch.zeros(c.corr_shape(), dtype=c.corr_dtype(), device="cuda")
    c.correlate(corr)
    rc, code = c.poll_status()
    assert rc == fxg._abi.FX_ERR_TIMEOUT and code in (1, 2, 3, 4), (rc, code)
    assert c.poll_status() == (0, 0)
    c.close()
    _normal_call_works()


@pytest.mark.parametrize("C,precision,call", [(64, 4, "channelize_correct"), (64, 0, "channelize_correct"),
                                              (256, 1, "channelize_correct"), (64, 0, "channelize")])
def test_fstage_failure_detection_timeout(C, precision, call):
    """The F-stage kernels wait for each round's raw rows (moved by bulk copies)
    with a bounded wait. With FX_FLAG_TEST_NO_LOADS no copy is issued, every
    wait runs out (about a millisecond each), the kernel records role 6 and
    finishes on stale rows without hanging; fx_poll_status reports
    FX_ERR_TIMEOUT with code 6, clears it, and the context stays usable."""
    import paper_1801_04834_gb300 as fxg
    blk = synth.make_block(2, synth.CI16, 1, 2, C, 32)
    c = make_corr(blk, precision=precision, extra_flags=fxg._abi.FX_FLAG_TEST_NO_LOADS)
    raw = torch.from_numpy(blk.raw).cuda()
    t = torch.zeros(2, dtype=torch.float64, device="cuda")
    if call == "channelize":
        c.channelize(raw)
    else:
        c.channelize_correct(raw, t, t)
    rc, code = c.poll_status()
    assert rc == fxg._abi.FX_ERR_TIMEOUT and code == 6, (rc, code)
    assert c.poll_status() == (0, 0)
    c.close()
    _normal_call_works()
