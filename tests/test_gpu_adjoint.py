"""Differentiation form on the GPU vs the FP64 oracle, through the C ABI.

Gradients of L = sum w |V - M|^2 with respect to complex per-(station, pol)
gains and per-station delays. The oracle's analytic gradient (fxo_vjp) is
itself pinned by central finite differences (tests/oracle_pins.py); here the
GPU adjoint must match it within the stated gradient bound, 1e-4 normwise
relative. The loss gradient fed to both sides, G = 2 w (V - M), is formed
from the oracle's V, never from the GPU's output.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle_pins import cplx

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE_HZ


def fxg():
    import paper_1801_04834_gb300 as m
    return m


def problem(seed, SB, N, C, S):
    """Channelised noise (rounded to FP32 so both sides see identical values),
    true gains (|g| in 0.8..1.2, random phase) and delays (+-50 ns), a model
    M = V(true) + noise, evaluated at gains/delays perturbed off the truth."""
    rng = np.random.default_rng(seed)
    chan = synth.channelised_noise(seed, SB, N, 2, C, S).astype(np.float32).astype(np.float64)
    centres = synth.subband_centres(SB)
    g_true = synth.random_gains(rng, N)
    t_true = rng.uniform(-50e-9, 50e-9, N)
    bp = rng.uniform(0.8, 1.2, (N, C))
    V_true = cplx(oracle.correlate(oracle.correct(chan, FS, centres, t_true, t_true, bandpass=bp, gains=g_true)))
    M = V_true + 0.05 * np.abs(V_true).mean() * (rng.standard_normal(V_true.shape) + 1j * rng.standard_normal(V_true.shape))
    w = rng.uniform(0.5, 1.5, V_true.shape)
    g = (g_true * (1 + 0.05 * rng.standard_normal(g_true.shape))).astype(np.float32).astype(np.float64)
    t = t_true + rng.uniform(-1e-9, 1e-9, N)
    return chan, centres, g, t, bp.astype(np.float32).astype(np.float64), M, w


def oracle_grad(chan, centres, g, t, bp, M, w, mask=None):
    V = cplx(oracle.correlate(oracle.correct(chan, FS, centres, t, t, bandpass=bp, gains=g)))
    G = 2 * w * (V - M)
    if mask is not None:
        G = G * mask
    Gr = np.stack([G.real, G.imag], -1)
    gg, gt = oracle.vjp(chan, FS, centres, t, Gr, bandpass=bp, gains=g)
    return V, Gr, gg, gt


def dev(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def make(SB, N, C, S, centres):
    return fxg().Correlator(N, SB, C, S, taps=synth.kaiser_sinc_taps(16, C), centres=centres)


@pytest.mark.parametrize("SB,N,C,S", [(2, 12, 16, 40), (1, 76, 64, 24), (2, 5, 256, 9)])
def test_adjoint_vs_oracle(SB, N, C, S):
    chan, centres, g, t, bp, M, w = problem(17 + N, SB, N, C, S)
    V, Gr, gg_ref, gt_ref = oracle_grad(chan, centres, g, t, bp, M, w)
    c = make(SB, N, C, S, centres)
    R = c.raw_vis(dev(chan), bandpass=dev(bp))
    # forward from R matches the hot-path oracle forward
    Vg = c.apply_gains(R, dev(g), dev(t, torch.float64)).cpu().numpy().astype(np.float64)
    assert relerr(cplx(Vg), V) < 1e-5
    gg, gt = c.backward(R, dev(g), dev(t, torch.float64), dev(Gr))
    gg, gt = gg.cpu().numpy().astype(np.float64), gt.cpu().numpy()
    assert relerr(gg, gg_ref) < 1e-4, relerr(gg, gg_ref)
    assert relerr(gt, gt_ref) < 1e-4, relerr(gt, gt_ref)
    # deterministic
    gg2, gt2 = c.backward(R, dev(g), dev(t, torch.float64), dev(Gr))
    assert np.array_equal(gg2.cpu().numpy().astype(np.float64), gg) and np.array_equal(gt2.cpu().numpy(), gt)


@pytest.mark.parametrize("recompute", [True, False])
def test_autograd_function(recompute):
    from paper_1801_04834_gb300.autograd import apply_gains, correct_correlate
    SB, N, C, S = 2, 10, 16, 32
    chan, centres, g, t, bp, M, w = problem(5, SB, N, C, S)
    _, _, gg_ref, gt_ref = oracle_grad(chan, centres, g, t, bp, M, w)
    c = make(SB, N, C, S, centres)
    gains = dev(g).requires_grad_(True)
    delays = dev(t, torch.float64).requires_grad_(True)
    Mt, wt = dev(np.stack([M.real, M.imag], -1), torch.float64), dev(w, torch.float64)
    V = correct_correlate(c, dev(chan), gains, delays, bandpass=dev(bp), recompute=recompute)
    L = (wt * ((V.double() - Mt) ** 2).sum(-1)).sum()
    L.backward()
    assert relerr(gains.grad.cpu().numpy(), gg_ref) < 1e-4
    assert relerr(delays.grad.cpu().numpy(), gt_ref) < 1e-4
    # the R-based forward gives the same gradients
    gains2 = dev(g).requires_grad_(True)
    delays2 = dev(t, torch.float64).requires_grad_(True)
    R = c.raw_vis(dev(chan), bandpass=dev(bp))
    V2 = apply_gains(c, R, gains2, delays2)
    L2 = (wt * ((V2.double() - Mt) ** 2).sum(-1)).sum()
    L2.backward()
    assert relerr(gains2.grad.cpu().numpy(), gg_ref) < 1e-4
    assert relerr(delays2.grad.cpu().numpy(), gt_ref) < 1e-4


def test_gradient_finite_difference_gpu():
    """Central differences of the GPU loss (FP32 forward, FP64 loss) agree with
    the GPU adjoint to the precision an FP32 forward allows."""
    SB, N, C, S = 1, 6, 16, 48
    chan, centres, g, t, bp, M, w = problem(9, SB, N, C, S)
    c = make(SB, N, C, S, centres)
    dchan, dbp = dev(chan), dev(bp)
    Mt, wt = dev(np.stack([M.real, M.imag], -1), torch.float64), dev(w, torch.float64)

    def loss(gg, tt):
        V = c.correlate(c.correct(dchan, tt, tt, bandpass=dbp, gains=gg)).double()
        return float((wt * ((V - Mt) ** 2).sum(-1)).sum())

    R = c.raw_vis(dchan, bandpass=dbp)
    V = c.apply_gains(R, dev(g), dev(t, torch.float64)).double()
    G = (2 * wt[..., None] * (V - Mt)).float().contiguous()
    gg, gt = c.backward(R, dev(g), dev(t, torch.float64), G)
    h = 1e-2
    for idx in [(0, 0, 0), (3, 1, 1), (5, 0, 1)]:
        gp, gm = g.copy(), g.copy()
        gp[idx] += h
        gm[idx] -= h
        fd = (loss(dev(gp), dev(t, torch.float64)) - loss(dev(gm), dev(t, torch.float64))) / (2 * h)
        assert abs(fd - float(gg[idx])) <= 2e-3 * abs(fd) + 1e-3 * float(gg.abs().max())
    ht = 1e-11
    for n in [0, 4]:
        tp, tm = t.copy(), t.copy()
        tp[n] += ht
        tm[n] -= ht
        fd = (loss(dev(g), dev(tp, torch.float64)) - loss(dev(g), dev(tm, torch.float64))) / (2 * ht)
        assert abs(fd - float(gt[n])) <= 2e-3 * abs(fd) + 1e-3 * float(gt.abs().max())


def test_adjoint_full_size_sampled():
    """Differentiation workload at full size (76 stations x 2 pols, 32
    subbands, 64 channels, 768 spectra, 0.96 GB channelised) in one launch;
    the loss gradient is restricted to two sampled subbands, which the oracle
    computes in full."""
    SB, N, C, S = 32, 76, 64, 768
    rng = np.random.default_rng(4)
    centres = synth.subband_centres(SB)
    g_full = synth.random_gains(rng, N).astype(np.float32).astype(np.float64)
    t = rng.uniform(-50e-9, 50e-9, N)
    bp = rng.uniform(0.8, 1.2, (N, C)).astype(np.float32).astype(np.float64)
    c = make(SB, N, C, S, centres)
    chan_t = torch.empty(c.chan_shape(), dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(synth.BASE_SEED + 4)
    chan_t.normal_(generator=gen)
    R = c.raw_vis(chan_t, bandpass=dev(bp))
    sampled = [3, 27]
    B = N * (N + 1) // 2
    Gfull = torch.zeros(c.vis_shape(), dtype=torch.float32, device="cuda")
    grng = np.random.default_rng(6)
    G_s = grng.standard_normal((len(sampled), C, B, 4, 2))
    for k, sb in enumerate(sampled):
        Gfull[sb] = dev(G_s[k])
    gg, gt = c.backward(R, dev(g_full), dev(t, torch.float64), Gfull)
    chan_s = chan_t[sampled].cpu().numpy().astype(np.float64)
    gg_ref, gt_ref = oracle.vjp(chan_s, FS, centres[sampled], t, G_s, bandpass=bp, gains=g_full)
    assert relerr(gg.cpu().numpy().astype(np.float64), gg_ref) < 1e-4
    assert relerr(gt.cpu().numpy(), gt_ref) < 1e-4


@pytest.mark.parametrize("precision", [0, 4])
@pytest.mark.parametrize("SB,N,C,S", [(2, 12, 16, 40), (1, 76, 64, 24), (2, 5, 256, 9)])
def test_adjoint_moving_delays_vs_oracle(SB, N, C, S, precision):
    """Delays moving linearly over the block (begin != end):
    fx_correct_correlate_backward_interp against the oracle's sample-by-sample
    chain rule (fxo_vjp_interp, itself pinned by finite differences in both
    delay ends), 1e-4 normwise for the gains and each delay end; the FP32
    (CUDA-core) and TF32-split (tensor-core) X-stages both form K and M1."""
    chan, centres, g, tb, bp, M, w = problem(31 + N, SB, N, C, S)
    rng = np.random.default_rng(N)
    te = tb + rng.uniform(-20e-9, 20e-9, N)
    V = cplx(oracle.correlate(oracle.correct(chan, FS, centres, tb, te, bandpass=bp, gains=g)))
    G = 2 * w * (V - M)
    Gr = np.stack([G.real, G.imag], -1)
    gg_ref, gb_ref, ge_ref = oracle.vjp_interp(chan, FS, centres, tb, te, Gr, bandpass=bp, gains=g)
    c = fxg().Correlator(N, SB, C, S, taps=synth.kaiser_sinc_taps(16, C), centres=centres, precision=precision)
    gg, gb, ge = c.backward_interp(dev(chan), dev(g), dev(tb, torch.float64), dev(te, torch.float64), dev(Gr),
                                   bandpass=dev(bp))
    gg, gb, ge = gg.cpu().numpy().astype(np.float64), gb.cpu().numpy(), ge.cpu().numpy()
    assert relerr(gg, gg_ref) < 1e-4, relerr(gg, gg_ref)
    assert relerr(gb, gb_ref) < 1e-4, relerr(gb, gb_ref)
    assert relerr(ge, ge_ref) < 1e-4, relerr(ge, ge_ref)
    c.close()


def test_adjoint_moving_delays_autograd_and_constant_limit():
    """torch.autograd through correct_correlate(..., delays_end=...): the
    gradients reach gains and both delay ends and equal the oracle's; at equal
    ends the two delay gradients add up to the constant-delay adjoint's."""
    SB, N, C, S = 1, 8, 16, 48
    chan, centres, g, tb, bp, M, w = problem(41, SB, N, C, S)
    rng = np.random.default_rng(3)
    te = tb + rng.uniform(-20e-9, 20e-9, N)
    c = make(SB, N, C, S, centres)
    from paper_1801_04834_gb300 import autograd as ag
    gt_ = dev(g).requires_grad_(True)
    tb_ = dev(tb, torch.float64).requires_grad_(True)
    te_ = dev(te, torch.float64).requires_grad_(True)
    Mt, wt = dev(np.stack([M.real, M.imag], -1)), dev(w)
    vis = ag.correct_correlate(c, dev(chan), gt_, tb_, bandpass=dev(bp), delays_end=te_)
    loss = (wt * ((vis - Mt) ** 2).sum(-1)).sum()
    loss.backward()
    V = cplx(oracle.correlate(oracle.correct(chan, FS, centres, tb, te, bandpass=bp, gains=g)))
    G = 2 * w * (V - M)
    gg_ref, gb_ref, ge_ref = oracle.vjp_interp(chan, FS, centres, tb, te, np.stack([G.real, G.imag], -1),
                                                bandpass=bp, gains=g)
    assert relerr(gt_.grad.cpu().numpy().astype(np.float64), gg_ref) < 1e-4
    assert relerr(tb_.grad.cpu().numpy(), gb_ref) < 1e-4
    assert relerr(te_.grad.cpu().numpy(), ge_ref) < 1e-4
    # equal ends: begin + end gradients = the constant-delay adjoint's delay gradient
    V1, Gr1, gg0, gt0 = oracle_grad(chan, centres, g, tb, bp, M, w)
    gg1, gb1, ge1 = c.backward_interp(dev(chan), dev(g), dev(tb, torch.float64), dev(tb, torch.float64), dev(Gr1),
                                      bandpass=dev(bp))
    assert relerr(gg1.cpu().numpy().astype(np.float64), gg0) < 1e-4
    assert relerr((gb1 + ge1).cpu().numpy(), gt0) < 1e-4
    c.close()
