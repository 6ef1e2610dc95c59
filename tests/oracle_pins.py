"""Pins for the FP64 oracle: checks against what the mathematics fixes, not
against the oracle itself. Each pin takes an `oracle.Oracle` and raises
AssertionError when the oracle disagrees. They are run on the real oracle
(test_oracle_pins.py) and on copies with planted mistakes
(test_oracle_mutants.py), where at least one pin must fail.

What pins what:
  fir_delta          FIR tap order and indexing, DFT sign and channel order
                     (a unit impulse reproduces the taps, closed form)
  tone               FIR + DFT: a channel-centred tone lands in its channel
                     with amplitude A*sum(h); leakage = DFT of the folded taps
  dft_vs_numpy       naive DFT + reordering vs numpy.fft + fftshift
  point_source       delay correction: closed-form phase -2 pi f_k (tau_i - tau_j)
                     before, zero after; amplitude S A_p A_q (sum h)^2
  bandpass           bandpass weights undo a per-station ripple exactly
  delay_ramp         linear delay interpolation over the block: a tone whose
                     delay drifts linearly is left with a phase constant in time
  correlate_einsum   correlation vs numpy.einsum of Y Y^H
  hermitian          autos: XX, YY real and >= 0, YX = conj(XY)
  linearity          sums over two halves of the block add up to the whole
  gradient_fd        vjp vs central finite differences of the loss
  gradient_truth     zero loss and zero gradient at the true parameters
  gradient_interp    vjp_interp (delays moving over the block) vs finite
                     differences in the gains and both delay ends; at equal
                     ends it agrees with vjp
  ci4_decode         4-bit nibble decoding (hand-decoded bytes, int16 equivalence)
  flags              lost-data weights and per-baseline valid-spectrum counts
  beam_point_source  beam steered at a plane wave sums in phase (closed form);
                     phase-centre beam gives the closed-form array factor
  beam_station_sum   zero delays = numpy station sum; one-hot weight = that
                     station rotated by exp(+2 pi i f_k delay)
  stokes             Stokes closed forms for Y = X, X = iY, Y = 0; integration
                     = sum of per-spectrum values; I^2 >= Q^2 + U^2 + V^2
  incoherent         incoherent beam: powers add (closed form against the
                     coherent beam), per-station Stokes closed forms, linear
                     in the weights, one station = its zero-delay coherent beam
"""
from __future__ import annotations

import numpy as np

import synth

FS = synth.SAMPLE_RATE_HZ


def cplx(a):
    return a[..., 0] + 1j * a[..., 1]


def bidx(i, j):
    return j * (j + 1) // 2 + i


def _random_taps(rng, T, C):
    return rng.uniform(-1.0, 1.0, size=T * C)


def pin_fir_delta(o):
    """A unit impulse at sample s0*C + c0 gives u_s[c0] = A h[(s0 - s) C + c0]
    for 0 <= s0 - s < T and nothing else; its DFT is u * exp(-2 pi i c0 m / C)."""
    rng = np.random.default_rng(1)
    C, T, S = 8, 4, 10
    L = (S + T - 1) * C
    taps = _random_taps(rng, T, C)
    A = 1000
    for s0, c0, p0, comp in [(3, 0, 0, 0), (7, 5, 1, 0), (12, 3, 0, 1), (0, 7, 1, 1)]:
        raw = np.zeros((1, 1, L, 2, 2), np.int16)
        raw[0, 0, s0 * C + c0, p0, comp] = A
        chan = cplx(o.channelize(synth.CI16, raw, T, C, S, taps))[0, 0]   # [P][S][C]
        amp = A * (1j if comp else 1.0)
        exp = np.zeros((S, C), complex)
        for s in range(S):
            k = s0 - s
            if 0 <= k < T:
                u = amp * taps[k * C + c0]
                for kout in range(C):
                    m = (kout - C // 2) % C
                    exp[s, kout] = u * np.exp(-2j * np.pi * c0 * m / C)
        assert np.allclose(chan[p0], exp, rtol=0, atol=1e-9), "delta response"
        assert np.all(chan[1 - p0] == 0), "other polarisation untouched"


def pin_tone(o):
    """Tone exp(i(2 pi m t / C + th)): X_s[k] = A e^{i th} sum_c H_c e^{-2 pi i c (k'-m)/C}
    with H_c = sum_k h[kC + c] and k' = k - C/2; exactly A e^{i th} sum(h) in
    channel m + C/2. Quantisation error bound: sum|h| * 0.5 * sqrt(2)."""
    rng = np.random.default_rng(2)
    C, T, S = 16, 4, 6
    L = (S + T - 1) * C
    taps = synth.kaiser_sinc_taps(T, C) * (1 + 0.1 * rng.uniform(-1, 1, T * C))
    H = taps.reshape(T, C).sum(0)
    A, th = 8000.0, 0.7
    bound = 0.5 * np.sqrt(2) * np.abs(taps).sum() + 1e-9
    for m in (-3, 0, 5, -8):
        t = np.arange(L)
        z = A * np.exp(1j * (2 * np.pi * ((m * t) % C) / C + th))
        raw = np.zeros((1, 1, L, 2, 2), np.int16)
        raw[0, 0, :, 0] = synth.quantise(z, synth.CI16)
        chan = cplx(o.channelize(synth.CI16, raw, T, C, S, taps))[0, 0, 0]    # [S][C]
        FH = np.fft.fft(H)
        exp = np.empty(C, complex)
        for k in range(C):
            mp = (k - C // 2) % C
            exp[k] = A * np.exp(1j * th) * FH[(mp - m) % C]
        assert np.max(np.abs(chan - exp[None, :])) <= bound, "tone response"
        assert abs(chan[0, m + C // 2] - A * np.exp(1j * th) * taps.sum()) <= bound


def pin_dft_vs_numpy(o):
    """Naive DFT + reordering equals numpy.fft.fft + fftshift of the FIR output."""
    rng = np.random.default_rng(3)
    for C, T, S, fmt in [(16, 16, 5, synth.CI16), (64, 4, 3, synth.CI8), (4, 2, 7, synth.CI16)]:
        L = (S + T - 1) * C
        lim = synth.FORMAT_MAX[fmt]
        raw = rng.integers(-lim, lim + 1, size=(1, 2, L, 2, 2)).astype(synth.FORMAT_DTYPE[fmt])
        taps = _random_taps(rng, T, C)
        chan = cplx(o.channelize(fmt, raw, T, C, S, taps))          # [1][N][P][S][C]
        x = cplx(raw.astype(np.float64))[0]                          # [N][L][P]
        h = taps.reshape(T, C)
        for n in range(2):
            for p in range(2):
                xr = x[n, :, p].reshape(S + T - 1, C)
                u = sum(h[k][None, :] * xr[k:k + S] for k in range(T))
                X = np.fft.fftshift(np.fft.fft(u, axis=-1), axes=-1)
                assert np.allclose(chan[0, n, p], X, rtol=1e-12, atol=1e-9), "DFT vs numpy"


def _point_source_setup(seed, N=4, C=16, T=4, S=12, SB=2, A=4000.0, ripple=None):
    rng = np.random.default_rng(seed)
    tau = rng.uniform(-5e-6, 5e-6, N)
    k0 = 11
    tone = synth.Tone(amp=A, channel=k0, delays=tau, ripple=ripple)
    blk = synth.make_block(seed, synth.CI16, SB, N, C, S, n_taps=T, sigma=0.0, tones=[tone])
    return blk, tau, k0


def pin_point_source(o):
    """Before correction V_ij^pq(k0) = S A_p A_q (sum h)^2 e^{i(p-q)pi/3}
    e^{-2 pi i f_k0 (tau_i - tau_j)}; after correction the delay phase is gone."""
    blk, tau, k0 = _point_source_setup(4)
    A, N, S, C = 4000.0, blk.n_stations, blk.n_spectra, blk.n_channels
    chan = o.channelize(blk.fmt, blk.raw, blk.n_taps, C, S, blk.taps)
    zero = np.zeros(N)
    v0 = cplx(o.correlate(o.correct(chan, FS, blk.centres, zero, zero)))
    v1 = cplx(o.correlate(o.correct(chan, FS, blk.centres, tau, tau)))
    sh = blk.taps.sum()
    for sb in range(blk.n_subbands):
        f = blk.centres[sb] + (k0 - C // 2) * FS / C
        for j in range(N):
            for i in range(j + 1):
                for p in range(2):
                    for q in range(2):
                        amp = S * A * A * (1 - .25 * p) * (1 - .25 * q) * sh * sh
                        pol = np.exp(1j * (p - q) * np.pi / 3)
                        e0 = amp * pol * np.exp(-2j * np.pi * f * (tau[i] - tau[j]))
                        e1 = amp * pol
                        got0 = v0[sb, k0, bidx(i, j), 2 * p + q]
                        got1 = v1[sb, k0, bidx(i, j), 2 * p + q]
                        assert abs(got0 - e0) <= 2e-3 * abs(e0), "uncorrected phase"
                        assert abs(got1 - e1) <= 2e-3 * abs(e1), "corrected phase"


def pin_bandpass(o):
    """A tone scaled by ripple r[n][k] comes back to amplitude A_p sum(h) per
    station once corrected with bandpass weights 1/r."""
    rng = np.random.default_rng(5)
    N, C = 4, 16
    ripple = synth.bandpass_ripple(rng, N, C, depth=0.2)
    blk, tau, k0 = _point_source_setup(5, N=N, C=C, ripple=ripple)
    A = 4000.0
    chan = o.channelize(blk.fmt, blk.raw, blk.n_taps, C, blk.n_spectra, blk.taps)
    corr = cplx(o.correct(chan, FS, blk.centres, tau, tau, bandpass=1.0 / ripple))
    sh = blk.taps.sum()
    for p in range(2):
        exp = A * (1 - .25 * p) * sh * np.exp(1j * p * np.pi / 3)
        got = corr[:, k0, :, :, p]
        assert np.max(np.abs(got - exp)) <= 1e-3 * abs(exp), "bandpass restores amplitude"
    # gains multiply in: a gain of 2i on (station 1, pol 0) scales that sample by 2i
    g = np.zeros((N, 2, 2)); g[..., 0] = 1.0; g[1, 0] = (0.0, 2.0)
    corr_g = cplx(o.correct(chan, FS, blk.centres, tau, tau, bandpass=1.0 / ripple, gains=g))
    assert np.allclose(corr_g[:, :, :, 1, 0], 2j * corr[:, :, :, 1, 0], rtol=1e-12, atol=1e-9)
    assert np.allclose(corr_g[:, :, :, 0, :], corr[:, :, :, 0, :], rtol=1e-12, atol=1e-9)


def pin_delay_ramp(o):
    """A tone whose delay drifts linearly, tau(t) = tb + (te - tb) t / (S C), is
    corrected with tau_begin = tb, tau_end = te. The residual phase must be the
    same for every spectrum (only the fixed offset of the FIR window centre is
    left), which fixes the interpolation tau(s) = tb + (te - tb) s / S."""
    C, T, S, N = 16, 4, 16, 2
    L = (S + T - 1) * C
    k0 = 9
    m = k0 - C // 2
    centres = np.array([150e6])
    f = centres[0] + m * FS / C
    tb = np.array([1.3e-6, -2.2e-6])
    te = tb + np.array([3.0e-9, -1.7e-8])          # several turns of phase over the block
    A = 12000.0
    t = np.arange(L)
    raw = np.zeros((1, N, L, 2, 2), np.int16)
    for n in range(N):
        tau_t = tb[n] + (te[n] - tb[n]) * t / (S * C)
        z = A * np.exp(1j * 2 * np.pi * ((m * t) % C) / C) * np.exp(-2j * np.pi * f * tau_t)
        for p in range(2):
            raw[0, n, :, p] = synth.quantise(z, synth.CI16)
    taps = synth.kaiser_sinc_taps(T, C)
    chan = o.channelize(synth.CI16, raw, T, C, S, taps)
    corr = cplx(o.correct(chan, FS, centres, tb, te))
    for n in range(N):
        ph = np.unwrap(np.angle(corr[0, k0, :, n, 0]))
        assert np.ptp(ph) < 2e-2, f"residual phase drifts over the block ({np.ptp(ph)})"


def pin_correlate_einsum(o):
    """Correlation equals numpy.einsum Y Y^H on the station-pair triangle."""
    rng = np.random.default_rng(6)
    SB, C, S, N = 2, 3, 9, 5
    corr = rng.standard_normal((SB, C, S, N, 2, 2))
    vis = cplx(o.correlate(corr))
    Y = cplx(corr).reshape(SB, C, S, N * 2)
    full = np.einsum("aksi,aksj->akij", Y, np.conj(Y))
    for j in range(N):
        for i in range(j + 1):
            for p in range(2):
                for q in range(2):
                    assert np.allclose(vis[:, :, bidx(i, j), 2 * p + q],
                                       full[:, :, 2 * i + p, 2 * j + q], rtol=1e-12, atol=1e-12)


def pin_hermitian(o):
    """Autocorrelations: XX and YY real and non-negative, YX = conj(XY)."""
    rng = np.random.default_rng(7)
    SB, C, S, N = 1, 4, 7, 6
    corr = rng.standard_normal((SB, C, S, N, 2, 2))
    vis = cplx(o.correlate(corr))
    for i in range(N):
        v = vis[:, :, bidx(i, i)]
        assert np.all(np.abs(v[..., 0].imag) < 1e-12) and np.all(v[..., 0].real >= 0)
        assert np.all(np.abs(v[..., 3].imag) < 1e-12) and np.all(v[..., 3].real >= 0)
        assert np.allclose(v[..., 2], np.conj(v[..., 1]), rtol=1e-12, atol=1e-12)


def pin_linearity(o):
    """Integration is a sum over time: two halves add up to the whole block."""
    rng = np.random.default_rng(8)
    corr = rng.standard_normal((1, 3, 10, 4, 2, 2))
    v = o.correlate(corr)
    va = o.correlate(np.ascontiguousarray(corr[:, :, :4]))
    vb = o.correlate(np.ascontiguousarray(corr[:, :, 4:]))
    assert np.allclose(v, va + vb, rtol=1e-12, atol=1e-12)


def _grad_problem(seed, SB=2, N=3, C=4, S=8):
    rng = np.random.default_rng(seed)
    chan = synth.channelised_noise(seed, SB, N, 2, C, S)
    centres = synth.subband_centres(SB)
    gains = synth.random_gains(rng, N)
    tau = rng.uniform(-50e-9, 50e-9, N)
    bandpass = rng.uniform(0.8, 1.2, (N, C))
    B = N * (N + 1) // 2
    w = rng.uniform(0.5, 1.5, (SB, C, B, 4))
    M = rng.standard_normal((SB, C, B, 4)) + 1j * rng.standard_normal((SB, C, B, 4))
    return chan, centres, gains, tau, bandpass, w, M


def _loss(o, chan, centres, gains, tau, bandpass, w, M):
    V = cplx(o.correlate(o.correct(chan, FS, centres, tau, tau, bandpass=bandpass, gains=gains)))
    return float(np.sum(w * np.abs(V - M) ** 2)), V


def pin_gradient_fd(o):
    """vjp against central finite differences of L = sum w |V - M|^2
    (step 1e-3 on gain components, 1e-3 ns on delays)."""
    chan, centres, gains, tau, bandpass, w, M = _grad_problem(9)
    L0, V = _loss(o, chan, centres, gains, tau, bandpass, w, M)
    G = 2 * w * (V - M)
    gg, gt = o.vjp(chan, FS, centres, tau, np.stack([G.real, G.imag], -1),
                   bandpass=bandpass, gains=gains)
    h = 1e-3
    fd_g = np.zeros_like(gains)
    for idx in np.ndindex(gains.shape):
        gp, gm = gains.copy(), gains.copy()
        gp[idx] += h
        gm[idx] -= h
        fd_g[idx] = (_loss(o, chan, centres, gp, tau, bandpass, w, M)[0]
                     - _loss(o, chan, centres, gm, tau, bandpass, w, M)[0]) / (2 * h)
    ht = 1e-12
    fd_t = np.zeros_like(tau)
    for n in range(len(tau)):
        tp, tm = tau.copy(), tau.copy()
        tp[n] += ht
        tm[n] -= ht
        fd_t[n] = (_loss(o, chan, centres, gains, tp, bandpass, w, M)[0]
                   - _loss(o, chan, centres, gains, tm, bandpass, w, M)[0]) / (2 * ht)
    assert np.linalg.norm(gg - fd_g) <= 1e-5 * np.linalg.norm(fd_g), "gain gradient vs FD"
    assert np.linalg.norm(gt - fd_t) <= 1e-4 * np.linalg.norm(fd_t), "delay gradient vs FD"


def pin_gradient_truth(o):
    """With M = V(true) the loss is zero and so is its gradient."""
    chan, centres, gains, tau, bandpass, w, _ = _grad_problem(10)
    _, V = _loss(o, chan, centres, gains, tau, bandpass, w, 0.0)
    gg, gt = o.vjp(chan, FS, centres, tau, np.zeros(V.shape + (2,)), bandpass=bandpass,
                   gains=gains)
    assert np.all(gg == 0) and np.all(gt == 0)
    L, _ = _loss(o, chan, centres, gains, tau, bandpass, w, V)
    assert L == 0.0
    # non-trivial check of the same point: moving the gains makes L > 0
    L2, _ = _loss(o, chan, centres, gains * 1.01, tau, bandpass, w, V)
    assert L2 > 0


def _loss_interp(o, chan, centres, gains, tb, te, bandpass, w, M):
    V = cplx(o.correlate(o.correct(chan, FS, centres, tb, te, bandpass=bandpass, gains=gains)))
    return float(np.sum(w * np.abs(V - M) ** 2)), V


def pin_gradient_interp(o):
    """vjp_interp (delays moving linearly over the block) against central
    finite differences of L = sum w |V - M|^2 in the gains and in both delay
    ends, and, at equal ends, against vjp: the same gain gradient, and the two
    delay gradients add up to the constant-delay one (moving both ends
    together moves the whole delay)."""
    chan, centres, gains, tb, bandpass, w, M = _grad_problem(12)
    rng = np.random.default_rng(13)
    te = tb + rng.uniform(-30e-9, 30e-9, len(tb))
    L0, V = _loss_interp(o, chan, centres, gains, tb, te, bandpass, w, M)
    G = 2 * w * (V - M)
    Gv = np.stack([G.real, G.imag], -1)
    gg, gb, ge = o.vjp_interp(chan, FS, centres, tb, te, Gv, bandpass=bandpass, gains=gains)
    h = 1e-3
    fd_g = np.zeros_like(gains)
    for idx in np.ndindex(gains.shape):
        gp, gm = gains.copy(), gains.copy()
        gp[idx] += h
        gm[idx] -= h
        fd_g[idx] = (_loss_interp(o, chan, centres, gp, tb, te, bandpass, w, M)[0]
                     - _loss_interp(o, chan, centres, gm, tb, te, bandpass, w, M)[0]) / (2 * h)
    ht = 1e-12
    fd_b, fd_e = np.zeros_like(tb), np.zeros_like(te)
    for n in range(len(tb)):
        for arr, out, which in ((tb, fd_b, 0), (te, fd_e, 1)):
            ap, am = arr.copy(), arr.copy()
            ap[n] += ht
            am[n] -= ht
            args_p = (ap, te) if which == 0 else (tb, ap)
            args_m = (am, te) if which == 0 else (tb, am)
            out[n] = (_loss_interp(o, chan, centres, gains, *args_p, bandpass, w, M)[0]
                      - _loss_interp(o, chan, centres, gains, *args_m, bandpass, w, M)[0]) / (2 * ht)
    assert np.linalg.norm(gg - fd_g) <= 1e-5 * np.linalg.norm(fd_g), "gain gradient vs FD"
    assert np.linalg.norm(gb - fd_b) <= 1e-4 * np.linalg.norm(fd_b), "begin-delay gradient vs FD"
    assert np.linalg.norm(ge - fd_e) <= 1e-4 * np.linalg.norm(fd_e), "end-delay gradient vs FD"
    # equal ends: consistent with the constant-delay gradient
    _, V1 = _loss_interp(o, chan, centres, gains, tb, tb, bandpass, w, M)
    G1 = 2 * w * (V1 - M)
    G1v = np.stack([G1.real, G1.imag], -1)
    gg1, gb1, ge1 = o.vjp_interp(chan, FS, centres, tb, tb, G1v, bandpass=bandpass, gains=gains)
    gg0, gt0 = o.vjp(chan, FS, centres, tb, G1v, bandpass=bandpass, gains=gains)
    assert np.allclose(gg1, gg0, rtol=1e-9, atol=1e-9 * np.abs(gg0).max()), "gains at constant delay"
    assert np.allclose(gb1 + ge1, gt0, rtol=1e-9, atol=1e-9 * np.abs(gt0).max()), "delays at constant delay"


def pin_fx_chain(o):
    """The whole-chain entry equals its three steps run one after another."""
    blk, tau, _ = _point_source_setup(11, N=3, C=8, S=5, SB=1)
    chan = o.channelize(blk.fmt, blk.raw, blk.n_taps, 8, 5, blk.taps)
    v = o.correlate(o.correct(chan, FS, blk.centres, tau, tau * 1.5))
    v2 = o.fx(blk.fmt, blk.raw, blk.n_taps, 8, 5, blk.taps, FS, blk.centres, tau, tau * 1.5)
    assert np.array_equal(v, v2)


def pin_ci4_decode(o):
    """int4 samples: hand-decoded bytes through an impulse (0x9A = -7 - 6i,
    0x7F = 7 - i, 0x80 = -8, 0x05 = 5i, 0xFF = -1 - i), and random 4-bit values
    give exactly the channelisation of the same values stored as int16."""
    rng = np.random.default_rng(12)
    C, T, S = 16, 4, 6
    L = (S + T - 1) * C
    taps = _random_taps(rng, T, C)
    for byte, val in [(0x9A, -7 - 6j), (0x7F, 7 - 1j), (0x80, -8 + 0j), (0x05, 5j), (0xFF, -1 - 1j)]:
        s0, c0 = 5, 3
        raw = np.zeros((1, 1, L, 2, 1), np.uint8)
        raw[0, 0, s0 * C + c0, 1, 0] = byte
        chan = cplx(o.channelize(synth.CI4, raw, T, C, S, taps))[0, 0, 1]      # pol 1
        for s in range(S):
            k = s0 - s
            exp = val * taps[k * C + c0] if 0 <= k < T else 0.0
            m = (0 - C // 2) % C            # output channel 0 holds DFT bin -C/2
            got = chan[s, 0] * np.exp(2j * np.pi * c0 * m / C)
            assert abs(got - exp) < 1e-12, (hex(byte), s)
    re = rng.integers(-7, 8, size=(2, 3, L, 2))
    im = rng.integers(-7, 8, size=(2, 3, L, 2))
    raw4 = synth.pack_ci4(re, im)[..., None]
    raw16 = np.stack([re, im], -1).astype(np.int16)
    a = o.channelize(synth.CI4, raw4, T, C, S, taps)
    b = o.channelize(synth.CI16, raw16, T, C, S, taps)
    assert np.array_equal(a, b), "int4 and int16 encodings of the same samples"


def pin_flags(o):
    """Lost-data weights: a station flagged for the whole block leaves exactly
    zero on all its baselines; flagging the second part of the block for every
    station gives the correlation of the first part alone (constant delays);
    counts are S for unflagged baselines and the overlap of valid spectra."""
    rng = np.random.default_rng(13)
    SB, N, C, S, S1 = 2, 4, 8, 10, 6
    chan = synth.noise(14, (SB, N, 2, S, C, 2))
    centres = synth.subband_centres(SB)
    tau = rng.uniform(-5e-6, 5e-6, N)
    w = np.ones((N, S))
    w[2] = 0.0
    v = cplx(o.correlate(o.correct(chan, FS, centres, tau, tau, flags=w)))
    for j in range(N):
        for i in range(j + 1):
            if 2 in (i, j):
                assert np.all(v[:, :, bidx(i, j)] == 0), "flagged station must vanish"
    w2 = np.ones((N, S))
    w2[:, S1:] = 0.0
    va = o.correlate(o.correct(chan, FS, centres, tau, tau, flags=w2))
    vb = o.correlate(o.correct(np.ascontiguousarray(chan[:, :, :, :S1]), FS, centres, tau, tau))
    assert np.allclose(va, vb, rtol=1e-12, atol=1e-12), "flags = shorter block"
    cnt = o.baseline_counts(w2, N, S)
    assert np.all(cnt == S1)
    assert np.all(o.baseline_counts(None, N, S) == S)
    w3 = np.ones((N, S)); w3[0, :3] = 0.0; w3[1, 5:] = 0.0
    c3 = o.baseline_counts(w3, N, S)
    assert c3[bidx(0, 1)] == 2 and c3[bidx(0, 0)] == S - 3 and c3[bidx(1, 1)] == 5 and c3[bidx(2, 3)] == S


def _plane_wave(seed, SB, N, C, S, centres, delays0, amp=(3.0, 2.0)):
    """corr block of a plane wave whose signal reaches station n delays0[n]
    late: Y_np(s, k) = amp_p exp(i theta_s) exp(-2 pi i f_k delays0[n])."""
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0, 2 * np.pi, S)
    y = np.zeros((SB, C, S, N, 2), dtype=complex)
    for sb in range(SB):
        for k in range(C):
            f = centres[sb] + (k - C / 2) * FS / C
            for p in range(2):
                y[sb, k, :, :, p] = amp[p] * np.exp(1j * theta)[:, None] * np.exp(-2j * np.pi * f * delays0)[None, :]
    return np.stack([y.real, y.imag], axis=-1), theta


def pin_beam_point_source(o):
    """A beam steered at a plane wave adds the stations in phase: voltage
    = amp_p exp(i theta_s) sum_n a_n exactly; a beam at the phase centre sees
    the closed-form array factor |sum_n a_n exp(-2 pi i f_k d_n)|."""
    SB, N, C, S = 2, 5, 8, 6
    rng = np.random.default_rng(21)
    centres = synth.subband_centres(SB)
    d0 = rng.uniform(-3e-6, 3e-6, N)
    a = rng.uniform(0.5, 1.5, N)
    corr, theta = _plane_wave(22, SB, N, C, S, centres, d0)
    v = o.beamform(corr, FS, centres, np.stack([d0, np.zeros(N)]), a, mode=0)
    X = v[..., 0] + 1j * v[..., 1]
    Y = v[..., 2] + 1j * v[..., 3]
    want = np.exp(1j * theta)[None, None, :] * a.sum()
    assert np.allclose(X[:, 0], 3.0 * want, rtol=1e-12, atol=1e-9), "coherent sum, pol X"
    assert np.allclose(Y[:, 0], 2.0 * want, rtol=1e-12, atol=1e-9), "coherent sum, pol Y"
    for sb in range(SB):
        for k in range(C):
            f = centres[sb] + (k - C / 2) * FS / C
            af = abs(np.sum(a * np.exp(-2j * np.pi * f * d0)))
            assert np.allclose(np.abs(X[sb, 1, k]), 3.0 * af, rtol=1e-10), "array factor"
            assert af < a.sum() * 0.999


def pin_beam_station_sum(o):
    """Zero beam delays and unit weights: the beam is the plain station sum;
    a one-hot weight with a beam delay gives that station rotated by
    exp(+2 pi i f_k delay) (channel frequency f_sb + (k - C/2) fs / C)."""
    SB, N, C, S = 2, 3, 4, 5
    corr = synth.noise(23, (SB, C, S, N, 2, 2))
    centres = synth.subband_centres(SB)
    v = o.beamform(corr, FS, centres, np.zeros((1, N)), None, mode=0)
    z = cplx(corr).sum(axis=3)                        # [SB][C][S][P]
    assert np.allclose(v[:, 0, ..., 0] + 1j * v[:, 0, ..., 1], z[..., 0], rtol=1e-12, atol=1e-12)
    assert np.allclose(v[:, 0, ..., 2] + 1j * v[:, 0, ..., 3], z[..., 1], rtol=1e-12, atol=1e-12)
    dl = np.array([[0.0, 2.5e-6, 0.0]])
    w = np.array([0.0, 1.0, 0.0])
    v1 = o.beamform(corr, FS, centres, dl, w, mode=0)
    ym = cplx(corr)[:, :, :, 1, 0]
    for sb in range(SB):
        for k in range(C):
            f = centres[sb] + (k - C / 2) * FS / C
            rot = np.exp(2j * np.pi * f * 2.5e-6)
            got = v1[sb, 0, k, :, 0] + 1j * v1[sb, 0, k, :, 1]
            assert np.allclose(got, rot * ym[sb, k], rtol=1e-10, atol=1e-10)


def pin_stokes(o):
    """Stokes closed forms: Y = X gives Q = V = 0, U = I; X = i Y gives
    Q = U = 0, V = I; Y = 0 gives Q = I, U = V = 0. I^2 = Q^2 + U^2 + V^2 for a
    single spectrum, I^2 >= Q^2 + U^2 + V^2 after integration, and the
    integrated value is the sum of the per-spectrum values."""
    SB, N, C, S = 1, 3, 4, 8
    centres = synth.subband_centres(SB)
    base = cplx(synth.noise(24, (SB, C, S, N, 2)))           # one pol of noise
    dl = np.random.default_rng(25).uniform(-1e-6, 1e-6, (2, N))
    for rel, want in (((1.0, 1.0), "U"), ((1j, 1.0), "V"), ((1.0, 0.0), "Q")):
        y = np.stack([rel[0] * base, rel[1] * base], axis=-1)     # pol X = rel0 * b, pol Y = rel1 * b
        corr = np.stack([y.real, y.imag], axis=-1)
        st = o.beamform(corr, FS, centres, dl, None, mode=2, tint=1)
        I, Q, U, V = (st[..., q] for q in range(4))
        assert np.all(I > 0)
        z = {"U": (Q, V), "V": (Q, U), "Q": (U, V)}[want]
        assert np.allclose(z[0], 0, atol=1e-9 * I.max()) and np.allclose(z[1], 0, atol=1e-9 * I.max())
        assert np.allclose({"U": U, "V": V, "Q": Q}[want], I, rtol=1e-12)
    corr = synth.noise(26, (SB, C, S, N, 2, 2))
    s1 = o.beamform(corr, FS, centres, dl, None, mode=2, tint=1)
    assert np.allclose(s1[..., 0] ** 2, (s1[..., 1:] ** 2).sum(-1), rtol=1e-10)
    s4 = o.beamform(corr, FS, centres, dl, None, mode=2, tint=4)
    assert np.allclose(s4, s1.reshape(SB, 2, C, S // 4, 4, 4).sum(axis=4), rtol=1e-12)
    assert np.all(s4[..., 0] ** 2 >= (s4[..., 1:] ** 2).sum(-1) * (1 - 1e-12))
    i4 = o.beamform(corr, FS, centres, dl, None, mode=1, tint=4)
    assert np.allclose(i4, s4[..., 0], rtol=1e-12)


def pin_incoherent(o):
    """Incoherent beam: a plane wave of amplitude (3, 2) per station gives
    I = (9 + 4) sum_n a_n per spectrum (powers add, phases do not matter),
    against (9 + 4) (sum_n a_n)^2 for the coherent beam steered at it; the
    Stokes closed forms hold per station (Y = X: U = I, Q = V = 0); the sum is
    linear in the station weights; and with one station it equals that
    station's coherent beam at zero delay."""
    SB, N, C, S = 2, 5, 4, 6
    rng = np.random.default_rng(31)
    centres = synth.subband_centres(SB)
    d0 = rng.uniform(-3e-6, 3e-6, N)
    a = rng.uniform(0.5, 1.5, N)
    corr, _ = _plane_wave(32, SB, N, C, S, centres, d0)
    inc = o.beamform_incoherent(corr, a, mode=2, tint=1)
    assert np.allclose(inc[..., 0], 13.0 * a.sum(), rtol=1e-12)
    coh = o.beamform(corr, FS, centres, d0[None, :], a, mode=2, tint=1)
    assert np.allclose(coh[:, 0, ..., 0], 13.0 * a.sum() ** 2, rtol=1e-10)
    y = cplx(synth.noise(33, (SB, C, S, N, 2)))
    same = np.stack([y, y], axis=-1)
    st = o.beamform_incoherent(np.stack([same.real, same.imag], axis=-1), None, mode=2, tint=2)
    assert np.allclose(st[..., 2], st[..., 0], rtol=1e-12)
    assert np.allclose(st[..., 1], 0, atol=1e-9 * st[..., 0].max())
    assert np.allclose(st[..., 3], 0, atol=1e-9 * st[..., 0].max())
    noise = synth.noise(34, (SB, C, S, N, 2, 2))
    whole = o.beamform_incoherent(noise, a, mode=2, tint=3)
    parts = sum(a[n] * o.beamform_incoherent(noise, np.eye(N)[n], mode=2, tint=3) for n in range(N))
    assert np.allclose(whole, parts, rtol=1e-12)
    one = np.ascontiguousarray(noise[:, :, :, 1:2])
    assert np.allclose(o.beamform_incoherent(one, None, mode=2, tint=3)[:, None],
                       o.beamform(one, FS, centres, np.zeros((1, 1)), None, mode=2, tint=3), rtol=1e-12)
    # a one-hot weight picks that station: its zero-delay coherent beam with the same weight
    for m in range(N):
        e = np.eye(N)[m]
        assert np.allclose(o.beamform_incoherent(noise, e, mode=2, tint=3)[:, None],
                           o.beamform(noise, FS, centres, np.zeros((1, N)), e, mode=2, tint=3), rtol=1e-12)


ALL_PINS = [pin_gradient_interp, pin_fir_delta, pin_tone, pin_dft_vs_numpy, pin_point_source, pin_bandpass,
            pin_delay_ramp, pin_correlate_einsum, pin_hermitian, pin_linearity,
            pin_gradient_fd, pin_gradient_truth, pin_fx_chain, pin_ci4_decode, pin_flags,
            pin_beam_point_source, pin_beam_station_sum, pin_stokes, pin_incoherent]
