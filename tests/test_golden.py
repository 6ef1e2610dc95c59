"""Golden fixtures (tests/golden/): figures printed in the paper that the
sample formats must reproduce, and the oracle's visibilities for one tiny
seeded block (written by tests/golden/make_golden.py, which calls only the
oracle), so that an unintended change of the oracle or of the seeded inputs
fails here."""
import json
import os

import numpy as np
import pytest

import synth

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def test_paper_input_rates():
    """The raw formats reproduce the paper's input bandwidths: 64 (80) antenna
    fields x 2 pols x 244 subbands of complex 16-bit samples at the subband
    rate is ~192 (~240) Gbps, and 488 subbands of 8-bit samples give the same
    rate (the paper trades bits for subbands one for one)."""
    p = load("paper_numbers.json")
    fs = synth.SAMPLE_RATE_HZ
    assert abs(fs / 1e3 - p["subband_width_khz"]["value"]) / p["subband_width_khz"]["value"] < 0.005
    bytes_per_complex = {synth.CI16: 2 * np.dtype(np.int16).itemsize, synth.CI8: 2 * np.dtype(np.int8).itemsize}
    for fields, key in ((64, "input_gbps_64_fields"), (80, "input_gbps_80_fields")):
        r16 = fields * 2 * p["subbands_16bit"]["value"] * fs * bytes_per_complex[synth.CI16] * 8 / 1e9
        r8 = fields * 2 * p["subbands_8bit"]["value"] * fs * bytes_per_complex[synth.CI8] * 8 / 1e9
        assert r16 == pytest.approx(r8)
        assert abs(r16 - p[key]["value"]) / p[key]["value"] < 0.03, (fields, r16)
    # one complex sample every 1/fs: the coarse-delay step
    assert 1e6 / fs == pytest.approx(p["coarse_delay_step_us"]["value"], rel=1e-3)


def test_oracle_matches_golden():
    import oracle  # noqa: F401
    from golden.make_golden import compute
    g = load("fx_tiny.json")
    _, _, vis = compute(g["case"])
    ref = np.array(g["vis"])
    assert vis.shape == ref.shape
    assert np.allclose(vis, ref, rtol=0, atol=1e-8 * np.abs(ref).max())


@pytest.mark.gpu
def test_gpu_path_matches_golden():
    """The GPU path (fused F-stage + FFMA X-stage) on the golden block, held
    to the FP32 path's bound."""
    import torch
    from golden.make_golden import compute
    from test_gpu_parity import make_corr, per_subband_rel
    g = load("fx_tiny.json")
    blk, tau, _ = compute(g["case"])
    c = make_corr(blk, precision=0)
    t = torch.from_numpy(tau).cuda()
    vis = c.correlate(c.channelize_correct(torch.from_numpy(blk.raw).cuda(), t, t)).cpu().numpy()
    e = per_subband_rel(vis.astype(np.float64), np.array(g["vis"]))
    assert np.all(e < 1e-5), e
