"""Batching form: many uneven correlation jobs in one persistent tensor-core
launch (fx_correlate_batched), against one fx_correlate launch per job and
against the FP64 oracle, through the C ABI; plus the autotuner, CUDA-graph
capture and the split (any station count) tile plan.

Job shapes follow the batching workload: station counts seeded uniform in
24..96, channels in {16, 64, 256}, integration lengths seeded uniform (the
full-size test uses 256..3072 spectra), complex int16 noise plus one point
source per job, FP16 operands with FP32 accumulation.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import baseline_max_rel

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE_HZ


def fxg():
    import paper_1801_04834_gb300 as m
    return m


def job_shapes(seed, n_jobs, s_lo, s_hi):
    rng = np.random.default_rng(seed)
    N = rng.integers(24, 97, n_jobs)
    C = rng.choice([16, 64, 256], n_jobs)
    S = rng.integers(s_lo, s_hi + 1, n_jobs)
    return [(int(n), int(c), int(s)) for n, c, s in zip(N, C, S)]


def prepare_jobs(shapes, seed, precision=1):
    """Per job: raw samples on the device (seeded), channelise + correct with
    its own handle (FP16 planar operands), and the single-launch visibilities."""
    m = fxg()
    out = []
    for k, (N, C, S) in enumerate(shapes):
        rng = np.random.default_rng(seed + k)
        tau = rng.uniform(-5e-6, 5e-6, N)
        tone = synth.Tone(amp=50.0, channel=int(rng.integers(1, C)), delays=tau)
        centres = synth.subband_centres(1, centre_hz=120e6 + 0.2e6 * k)
        raw = synth.make_raw_torch(seed + k, synth.CI16, 1, N, C, S, tones=[tone], centre_hz=120e6 + 0.2e6 * k)
        c = m.Correlator(N, 1, C, S, taps=synth.kaiser_sinc_taps(16, C), centres=centres, precision=precision)
        d = torch.from_numpy(tau).cuda()
        corr = c.correct(c.channelize(raw), d, d)
        vis1 = c.correlate(corr)
        out.append(dict(N=N, C=C, S=S, c=c, corr=corr, vis1=vis1, raw=raw, tau=tau, centres=centres))
    torch.cuda.synchronize()
    return out


def make_batch(jobs, precision=1):
    m = fxg()
    from paper_1801_04834_gb300 import _abi
    lib = _abi.load()
    arr = (_abi.fx_job * len(jobs))()
    for k, j in enumerate(jobs):
        j["visb"] = torch.full_like(j["vis1"], float("nan"))
        arr[k].n_stations, arr[k].n_subbands, arr[k].n_channels, arr[k].n_spectra = j["N"], 1, j["C"], j["S"]
        arr[k].d_corr = j["corr"].data_ptr()
        arr[k].d_vis = j["visb"].data_ptr()
    b = ctypes.c_void_p()
    _abi.check(lib.fx_batch_create(arr, len(jobs), precision, 0.0, ctypes.byref(b)), "fx_batch_create")
    return lib, b


def stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def check_equal_single(jobs, exact):
    for k, j in enumerate(jobs):
        a, b = j["visb"].double(), j["vis1"].double()
        if exact:
            assert torch.equal(j["visb"], j["vis1"]), f"job {k} differs from its single launch"
        else:
            rel = (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()
            assert rel < 1e-6, f"job {k}: {rel}"


def test_batched_matches_single_launches_and_oracle():
    from paper_1801_04834_gb300 import _abi
    shapes = job_shapes(31, 12, 40, 300)
    jobs = prepare_jobs(shapes, 500)
    lib, b = make_batch(jobs)
    _abi.check(lib.fx_correlate_batched(b, stream()), "fx_correlate_batched")
    torch.cuda.synchronize()
    desc = lib.fx_batch_describe(b).decode()
    # the default plan uses the same tiles as the single-job launch: bit-identical
    check_equal_single(jobs, exact="wide" in desc)
    # two sampled jobs against the FP64 oracle of the whole chain
    for k in (0, 5):
        j = jobs[k]
        raw = j["raw"].cpu().numpy()
        ref = oracle.fx(synth.CI16, raw, 16, j["C"], j["S"], synth.kaiser_sinc_taps(16, j["C"]), FS,
                        j["centres"], j["tau"], j["tau"])
        got = j["visb"].cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel < 5e-3, (k, rel)
        # per baseline, max |dV_ij| / sqrt(|V_ii| |V_jj|): FP16 operand rounding (2^-11)
        # averaged over the job's spectra, at its worst entry
        assert baseline_max_rel(got, ref, j["N"]) < 1e-3, k
    code = ctypes.c_int()
    assert lib.fx_batch_poll_status(b, ctypes.byref(code)) == 0
    lib.fx_batch_destroy(b)


def test_autotune_and_graph_capture():
    from paper_1801_04834_gb300 import _abi
    shapes = job_shapes(32, 10, 64, 400)
    jobs = prepare_jobs(shapes, 700)
    lib, b = make_batch(jobs)
    _abi.check(lib.fx_batch_autotune(b, 2, stream()), "fx_batch_autotune")
    desc = lib.fx_batch_describe(b).decode()
    print("autotuned plan:", desc)
    for j in jobs:
        j["visb"].fill_(float("nan"))
    # capture the batched launch in a CUDA graph and replay it twice
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        rc = lib.fx_correlate_batched(b, ctypes.c_void_p(s.cuda_stream))
    assert rc == 0, _abi.last_error()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    check_equal_single(jobs, exact="wide" in desc)
    lib.fx_batch_destroy(b)


@pytest.mark.parametrize("precision", [1, 3])
def test_split_tiles_large_station_count(precision):
    """Station counts above what one 256-column tile holds (I_pad > 256) take
    the split tile plan; results match the oracle correlation of the same
    operands (operand-exact check, FP32 accumulation order only)."""
    from test_gpu_tc import planar
    m = fxg()
    N, C, S, SB = 150, 16, 70, 1
    corr64 = synth.noise(77 + precision, (SB, C, S, N, 2, 2), sigma=30.0)
    c = m.Correlator(N, SB, C, S, taps=synth.kaiser_sinc_taps(16, C), centres=synth.subband_centres(SB),
                     precision=precision)
    ops, held = planar(corr64, c.I_pad, c.S_pad, "split" if precision == 3 else "f16")
    ref = oracle.correlate(held)
    got = c.correlate(ops.cuda().contiguous()).cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel < 2e-5, rel


def test_batch_full_size_shapes():
    """48 jobs of the batching workload at full size (256..3072 spectra):
    one batched launch equals 48 single launches."""
    from paper_1801_04834_gb300 import _abi
    shapes = job_shapes(synth.BASE_SEED + 3, 48, 256, 3072)
    jobs = prepare_jobs(shapes, 900)
    lib, b = make_batch(jobs)
    _abi.check(lib.fx_correlate_batched(b, stream()), "fx_correlate_batched")
    torch.cuda.synchronize()
    check_equal_single(jobs, exact="wide" in lib.fx_batch_describe(b).decode())
    lib.fx_batch_destroy(b)
