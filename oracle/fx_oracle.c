/*
 * fx_oracle.c -- plain FP64 CPU oracle for the Cobalt FX correlator hot path
 * (arXiv 1801.04834, Sec. "Signal processing with GPU kernels").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, calls or
 * includes this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it. It shares no code, header, table or constant with the
 * CUDA path.
 *
 * Every function computes its result straight from the definition, in double
 * precision, with no blocking, fusion or reordering:
 *   fxo_channelize  direct T-tap FIR per channel, then a naive O(C^2) DFT
 *   fxo_correct     per-sample delay phase exp(+2 pi i f_k tau(s)) in FP64,
 *                   times bandpass weight and complex gain
 *   fxo_correlate   explicit sum over time of Y_ip * conj(Y_jq), i <= j
 *   fxo_vjp         gradient of a real loss through correct + correlate,
 *                   by the chain rule entry by entry (constant delays)
 *   fxo_vjp_interp  the same with delays interpolated over the block, by the
 *                   chain rule sample by sample (gradients for both ends)
 *   fxo_beamform    coherent beams: per-sample phase-shifted station sum,
 *                   then complex voltages or Stokes I / IQUV
 *   fxo_beamform_incoherent  Stokes per station, then the weighted station sum
 * OpenMP splits independent outer loops (subbands, stations, channels) across
 * host threads, as the paper's host code does over subbands (Sec. "Parallelization
 * libraries"); it does not change any arithmetic.
 *
 * Conventions (readings of the paper, which leaves them unstated):
 *   PPF      u_s[c] = sum_{k<T} h[k*C + c] * x[(s + k)*C + c],  s < S
 *   DFT      X_s[m] = sum_{c<C} u_s[c] * exp(-2 pi i c m / C), unnormalised;
 *            output channel k = (m + C/2) mod C, so channel C/2 is the subband
 *            centre and channel k has sky frequency f_sb + (k - C/2) fs / C
 *   delay    tau_n(s) = tau_begin[n] + (tau_end[n] - tau_begin[n]) * s / S,
 *            correction multiplies by exp(+2 pi i f_k tau_n(s))
 *   visibs   b = j(j+1)/2 + i for stations i <= j, products p q in the order
 *            XX, XY, YX, YY (index 2p + q), V = sum_s Y_ip conj(Y_jq)
 *
 * Layouts (row-major, complex = two doubles re, im unless stated):
 *   raw   [SB][N][L][P] complex int16, int8 or int4, L = (S + T - 1) * C;
 *         int4: one byte per complex sample, real part in the high nibble,
 *         imaginary part in the low nibble, each two's complement in [-8, 7]
 *   chan  [SB][N][P][S][C]      corr [SB][C][S][N][P]      vis [SB][C][B][4]
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FXO_CI16 0
#define FXO_CI8 1
#define FXO_CI4 2

static const double TWO_PI = 6.283185307179586476925286766559;

static double raw_component(const void *raw, int fmt, size_t idx)
{
    if (fmt == FXO_CI16) return (double)((const int16_t *)raw)[idx];
    if (fmt == FXO_CI8) return (double)((const int8_t *)raw)[idx];
    /* int4: component idx of the complex sample in byte idx / 2 */
    const unsigned byte = ((const uint8_t *)raw)[idx / 2];
    const unsigned nib = (idx % 2 == 0) ? (byte >> 4) : (byte & 15u);
    return (nib >= 8) ? (double)nib - 16.0 : (double)nib;
}

/* Polyphase filter bank (Sec. "Hardware requirements and design priorities";
 * Sec. "Signal processing with GPU kernels"): one FIR filter per channel over
 * the decimated sample stream, then the transform that channelises the
 * subband. */
int fxo_channelize(int fmt, const void *raw, int SB, int N, int P, int C, int T, int S,
                   const double *taps, double *chan)
{
    if (fmt != FXO_CI16 && fmt != FXO_CI8 && fmt != FXO_CI4) return -1;
    const size_t L = (size_t)(S + T - 1) * C;
    /* exact twiddle table: angle depends only on (c*m mod C) */
    double *wre = malloc(sizeof(double) * C), *wim = malloc(sizeof(double) * C);
    if (!wre || !wim) { free(wre); free(wim); return -3; }
    for (int r = 0; r < C; ++r) {
        wre[r] = cos(TWO_PI * r / C);
        wim[r] = -sin(TWO_PI * r / C);
    }
    int rc = 0;
#pragma omp parallel for collapse(3) schedule(dynamic)
    for (int sb = 0; sb < SB; ++sb)
        for (int n = 0; n < N; ++n)
            for (int p = 0; p < P; ++p) {
                double *ure = malloc(sizeof(double) * C), *uim = malloc(sizeof(double) * C);
                if (!ure || !uim) { free(ure); free(uim); rc = -3; continue; }
                const size_t base = ((size_t)sb * N + n) * L;   /* time-sample index base */
                for (int s = 0; s < S; ++s) {
                    /* FIR: one T-tap filter per channel over the decimated stream */
                    for (int c = 0; c < C; ++c) {
                        double are = 0.0, aim = 0.0;
                        for (int k = 0; k < T; ++k) {
                            const size_t t = (size_t)(s + k) * C + c;
                            const size_t e = ((base + t) * P + p) * 2;
                            const double h = taps[(size_t)k * C + c];
                            are += h * raw_component(raw, fmt, e);
                            aim += h * raw_component(raw, fmt, e + 1);
                        }
                        ure[c] = are;
                        uim[c] = aim;
                    }
                    /* naive DFT, then reorder to ascending frequency */
                    double *out = chan + ((((size_t)sb * N + n) * P + p) * S + s) * (size_t)C * 2;
                    for (int m = 0; m < C; ++m) {
                        double xre = 0.0, xim = 0.0;
                        for (int c = 0; c < C; ++c) {
                            const int r = (int)(((long long)c * m) % C);
                            xre += ure[c] * wre[r] - uim[c] * wim[r];
                            xim += ure[c] * wim[r] + uim[c] * wre[r];
                        }
                        const int k = (m + C / 2) % C;
                        out[2 * k] = xre;
                        out[2 * k + 1] = xim;
                    }
                }
                free(ure);
                free(uim);
            }
    free(wre);
    free(wim);
    return rc;
}

/* Sky frequency of output channel k of subband sb. */
static double channel_freq(const double *centres, int sb, int k, int C, double fs)
{
    return centres[sb] + (double)(k - C / 2) * fs / C;
}

/* Fine delay compensation + bandpass correction (Sec. "Signal processing with
 * GPU kernels": phase from begin/end delays, linear in time within a block),
 * with the transposing write-back to the per-channel, all-stations layout.
 * bandpass [N][C] real or NULL (= 1); gains [N][P] complex or NULL (= 1);
 * flags [N][S] real weights marking lost data (0 = lost) or NULL (= 1). */
int fxo_correct(const double *chan, int SB, int N, int P, int C, int S, double fs,
                const double *centres, const double *tau_begin, const double *tau_end,
                const double *bandpass, const double *gains, const double *flags, double *corr)
{
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int sb = 0; sb < SB; ++sb)
        for (int k = 0; k < C; ++k) {
            const double f = channel_freq(centres, sb, k, C, fs);
            for (int s = 0; s < S; ++s)
                for (int n = 0; n < N; ++n) {
                    const double tau = tau_begin[n] + (tau_end[n] - tau_begin[n]) * s / S;
                    const double phi = TWO_PI * f * tau;
                    const double b = bandpass ? bandpass[(size_t)n * C + k] : 1.0;
                    const double rre = b * cos(phi), rim = b * sin(phi);
                    for (int p = 0; p < P; ++p) {
                        const double gre = gains ? gains[((size_t)n * P + p) * 2] : 1.0;
                        const double gim = gains ? gains[((size_t)n * P + p) * 2 + 1] : 0.0;
                        const double *x = chan + ((((size_t)sb * N + n) * P + p) * S + s) * (size_t)C * 2 + 2 * k;
                        /* (x * g) * (b e^{i phi}) */
                        const double xgre = x[0] * gre - x[1] * gim;
                        const double xgim = x[0] * gim + x[1] * gre;
                        double *y = corr + (((((size_t)sb * C + k) * S + s) * N + n) * P + p) * 2;
                        /* lost-data weight of (station, spectrum), 1 when no flags */
                        const double w = flags ? flags[(size_t)n * S + s] : 1.0;
                        y[0] = (xgre * rre - xgim * rim) * w;
                        y[1] = (xgre * rim + xgim * rre) * w;
                    }
                }
        }
    return 0;
}

/* X-stage: correlate every station pair (autos included) and every
 * polarisation product, integrated (summed) over the block. */
int fxo_correlate(const double *corr, int SB, int N, int P, int C, int S, double *vis)
{
    if (P != 2) return -1;
    const size_t B = (size_t)N * (N + 1) / 2;
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int sb = 0; sb < SB; ++sb)
        for (int k = 0; k < C; ++k)
            for (int j = 0; j < N; ++j)
                for (int i = 0; i <= j; ++i) {
                    const size_t b = (size_t)j * (j + 1) / 2 + i;
                    for (int p = 0; p < 2; ++p)
                        for (int q = 0; q < 2; ++q) {
                            double vre = 0.0, vim = 0.0;
                            for (int s = 0; s < S; ++s) {
                                const double *y = corr + ((((size_t)sb * C + k) * S + s) * N) * P * 2;
                                const double are = y[(i * P + p) * 2], aim = y[(i * P + p) * 2 + 1];
                                const double bre = y[(j * P + q) * 2], bim = y[(j * P + q) * 2 + 1];
                                /* a * conj(b) */
                                vre += are * bre + aim * bim;
                                vim += aim * bre - are * bim;
                            }
                            double *v = vis + ((((size_t)sb * C + k) * B + b) * 4 + (2 * p + q)) * 2;
                            v[0] = vre;
                            v[1] = vim;
                        }
                }
    return 0;
}

/* Number of spectra that count for each baseline when per-(station, spectrum)
 * weights flag lost data: counts[b(i,j)] = sum_s w_i(s) w_j(s), i <= j. */
int fxo_baseline_counts(const double *flags, int N, int S, double *counts)
{
    for (int j = 0; j < N; ++j)
        for (int i = 0; i <= j; ++i) {
            double c = 0.0;
            for (int s = 0; s < S; ++s)
                c += (flags ? flags[(size_t)i * S + s] : 1.0) * (flags ? flags[(size_t)j * S + s] : 1.0);
            counts[(size_t)j * (j + 1) / 2 + i] = c;
        }
    return 0;
}

/* Whole hot path, raw samples to visibilities. Scratch is allocated here. */
int fxo_fx(int fmt, const void *raw, int SB, int N, int P, int C, int T, int S,
           const double *taps, double fs, const double *centres, const double *tau_begin,
           const double *tau_end, const double *bandpass, const double *gains, double *vis)
{
    const size_t n = (size_t)SB * N * P * S * C * 2;
    double *chan = malloc(sizeof(double) * n), *corr = malloc(sizeof(double) * n);
    int rc = (!chan || !corr) ? -3 : 0;
    if (!rc) rc = fxo_channelize(fmt, raw, SB, N, P, C, T, S, taps, chan);
    if (!rc) rc = fxo_correct(chan, SB, N, P, C, S, fs, centres, tau_begin, tau_end,
                              bandpass, gains, NULL, corr);
    if (!rc) rc = fxo_correlate(corr, SB, N, P, C, S, vis);
    free(chan);
    free(corr);
    return rc;
}

/*
 * Vector-Jacobian product of correct + correlate with respect to the complex
 * per-(station, pol) gains g and the per-station delays tau (held constant
 * over the block). grad_vis [SB][C][B][4][2] holds dL/dRe(V), dL/dIm(V) of a
 * real loss L. Outputs: grad_gains [N][P][2] = dL/dRe(g), dL/dIm(g) and
 * grad_tau [N] = dL/dtau.
 *
 * With constant delays each corrected sample is Y_a = c_a X_a with
 * c_a(k) = g_a b_n(k) exp(2 pi i f_k tau_n), so every visibility factors as
 * V_ab = c_a conj(c_b) R_ab with R the visibilities of the uncorrected data.
 * R is formed here by the explicit time sum; then for every visibility entry
 * dL/dtheta += dL/dRe(V) dRe(V)/dtheta + dL/dIm(V) dIm(V)/dtheta, with the
 * partial derivatives of V_ab written out for each parameter it touches.
 */
int fxo_vjp(const double *chan, int SB, int N, int P, int C, int S, double fs,
            const double *centres, const double *tau, const double *bandpass,
            const double *gains, const double *grad_vis, double *grad_gains, double *grad_tau)
{
    if (P != 2) return -1;
    const size_t B = (size_t)N * (N + 1) / 2;
    for (int a = 0; a < N * P * 2; ++a) grad_gains[a] = 0.0;
    for (int n = 0; n < N; ++n) grad_tau[n] = 0.0;
    const int nthread_slots = SB * C;
    double *gg = calloc((size_t)nthread_slots * N * P * 2, sizeof(double));
    double *gt = calloc((size_t)nthread_slots * N, sizeof(double));
    if (!gg || !gt) { free(gg); free(gt); return -3; }

#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int sb = 0; sb < SB; ++sb)
        for (int k = 0; k < C; ++k) {
            double *my_gg = gg + ((size_t)sb * C + k) * N * P * 2;
            double *my_gt = gt + ((size_t)sb * C + k) * N;
            const double f = channel_freq(centres, sb, k, C, fs);
            for (int j = 0; j < N; ++j)
                for (int i = 0; i <= j; ++i)
                    for (int p = 0; p < 2; ++p)
                        for (int q = 0; q < 2; ++q) {
                            /* R_ab = sum_s X_ip conj(X_jq) */
                            double rre = 0.0, rim = 0.0;
                            for (int s = 0; s < S; ++s) {
                                const double *xa = chan + ((((size_t)sb * N + i) * P + p) * S + s) * (size_t)C * 2 + 2 * k;
                                const double *xb = chan + ((((size_t)sb * N + j) * P + q) * S + s) * (size_t)C * 2 + 2 * k;
                                rre += xa[0] * xb[0] + xa[1] * xb[1];
                                rim += xa[1] * xb[0] - xa[0] * xb[1];
                            }
                            /* e_a = b_i(k) exp(i 2 pi f tau_i), c_a = g_a e_a; same for b */
                            const double ba = bandpass ? bandpass[(size_t)i * C + k] : 1.0;
                            const double bb = bandpass ? bandpass[(size_t)j * C + k] : 1.0;
                            const double pa = TWO_PI * f * tau[i], pb = TWO_PI * f * tau[j];
                            const double eare = ba * cos(pa), eaim = ba * sin(pa);
                            const double ebre = bb * cos(pb), ebim = bb * sin(pb);
                            const double gare = gains ? gains[((size_t)i * P + p) * 2] : 1.0;
                            const double gaim = gains ? gains[((size_t)i * P + p) * 2 + 1] : 0.0;
                            const double gbre = gains ? gains[((size_t)j * P + q) * 2] : 1.0;
                            const double gbim = gains ? gains[((size_t)j * P + q) * 2 + 1] : 0.0;
                            const double care = gare * eare - gaim * eaim, caim = gare * eaim + gaim * eare;
                            const double cbre = gbre * ebre - gbim * ebim, cbim = gbre * ebim + gbim * ebre;
                            /* cb* R */
                            const double cbRre = cbre * rre + cbim * rim;
                            const double cbRim = cbre * rim - cbim * rre;
                            /* V = ca * conj(cb) * R */
                            const double vre = care * cbRre - caim * cbRim;
                            const double vim = care * cbRim + caim * cbRre;

                            const size_t b = (size_t)j * (j + 1) / 2 + i;
                            const double *G = grad_vis + ((((size_t)sb * C + k) * B + b) * 4 + (2 * p + q)) * 2;
                            const double Gre = G[0], Gim = G[1];

                            /* d/dRe(g_a): dV = e_a conj(c_b) R ; d/dIm(g_a): dV = i e_a conj(c_b) R */
                            const double d1re = eare * cbRre - eaim * cbRim;
                            const double d1im = eare * cbRim + eaim * cbRre;
                            my_gg[((size_t)i * P + p) * 2] += Gre * d1re + Gim * d1im;
                            my_gg[((size_t)i * P + p) * 2 + 1] += Gre * (-d1im) + Gim * d1re;

                            /* d/dRe(g_b): dV = c_a conj(e_b) R ; d/dIm(g_b): dV = -i c_a conj(e_b) R */
                            const double ebRre = ebre * rre + ebim * rim;
                            const double ebRim = ebre * rim - ebim * rre;
                            const double d2re = care * ebRre - caim * ebRim;
                            const double d2im = care * ebRim + caim * ebRre;
                            my_gg[((size_t)j * P + q) * 2] += Gre * d2re + Gim * d2im;
                            my_gg[((size_t)j * P + q) * 2 + 1] += Gre * d2im + Gim * (-d2re);

                            /* d/dtau_i: dV = i 2 pi f V ; d/dtau_j: dV = -i 2 pi f V */
                            const double w = TWO_PI * f;
                            const double dtre = -w * vim, dtim = w * vre;
                            my_gt[i] += Gre * dtre + Gim * dtim;
                            my_gt[j] -= Gre * dtre + Gim * dtim;
                        }
        }
    for (int t = 0; t < nthread_slots; ++t) {
        for (int a = 0; a < N * P * 2; ++a) grad_gains[a] += gg[(size_t)t * N * P * 2 + a];
        for (int n = 0; n < N; ++n) grad_tau[n] += gt[(size_t)t * N + n];
    }
    free(gg);
    free(gt);
    return 0;
}

/* Gradient of a real loss L(V) through correct + correlate when each
 * station's delay moves linearly over the block (Sec. "Signal processing
 * with GPU kernels": the phase is formed at the block's start and end and
 * interpolated in between), by the chain rule sample by sample:
 *   Y_a(s) = g_a b_i(k) exp(2 pi i f_k tau_i(s)) X_a(s),
 *   tau_i(s) = tau_begin[i] + (tau_end[i] - tau_begin[i]) s / S,
 *   dY_a(s)/dtau_begin[i] = 2 pi i f_k (1 - s/S) Y_a(s),
 *   dY_a(s)/dtau_end[i]   = 2 pi i f_k (s/S) Y_a(s),
 *   dY_a(s)/dRe(g_a) = U_a(s), dY_a(s)/dIm(g_a) = i U_a(s), U_a = Y_a / g_a,
 * and V_ab = sum_s Y_a(s) conj(Y_b(s)), dL = sum Re(conj(G) dV) with
 * G = dL/dRe(V) + i dL/dIm(V). Outputs grad_gains [N][P][2],
 * grad_tau_begin [N], grad_tau_end [N]. */
int fxo_vjp_interp(const double *chan, int SB, int N, int P, int C, int S, double fs,
                   const double *centres, const double *tau_begin, const double *tau_end,
                   const double *bandpass, const double *gains, const double *grad_vis,
                   double *grad_gains, double *grad_tb, double *grad_te)
{
    if (P != 2) return -1;
    const size_t B = (size_t)N * (N + 1) / 2;
    for (int a = 0; a < N * P * 2; ++a) grad_gains[a] = 0.0;
    for (int n = 0; n < N; ++n) grad_tb[n] = grad_te[n] = 0.0;
    const int slots = SB * C;
    const size_t per = (size_t)N * P * 2 + 2 * (size_t)N;          /* gains, tau_begin, tau_end */
    double *acc = calloc((size_t)slots * per, sizeof(double));
    double *ure = malloc(sizeof(double) * (size_t)slots * N * P * S);
    double *uim = malloc(sizeof(double) * (size_t)slots * N * P * S);
    if (!acc || !ure || !uim) { free(acc); free(ure); free(uim); return -3; }

#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int sb = 0; sb < SB; ++sb)
        for (int k = 0; k < C; ++k) {
            const size_t slot = (size_t)sb * C + k;
            double *my = acc + slot * per;
            double *my_tb = my + (size_t)N * P * 2, *my_te = my_tb + N;
            double *Ur = ure + slot * N * P * S, *Ui = uim + slot * N * P * S;
            const double f = channel_freq(centres, sb, k, C, fs);
            /* U_a(s) = b_i exp(2 pi i f tau_i(s)) X_a(s): the corrected sample before the gain */
            for (int n = 0; n < N; ++n)
                for (int p = 0; p < P; ++p)
                    for (int s = 0; s < S; ++s) {
                        const double *x = chan + ((((size_t)sb * N + n) * P + p) * S + s) * (size_t)C * 2 + 2 * k;
                        const double tau = tau_begin[n] + (tau_end[n] - tau_begin[n]) * (double)s / (double)S;
                        const double ph = TWO_PI * f * tau;
                        const double bw = bandpass ? bandpass[(size_t)n * C + k] : 1.0;
                        const double er = bw * cos(ph), ei = bw * sin(ph);
                        const size_t u = ((size_t)n * P + p) * S + s;
                        Ur[u] = er * x[0] - ei * x[1];
                        Ui[u] = er * x[1] + ei * x[0];
                    }
            for (int j = 0; j < N; ++j)
                for (int i = 0; i <= j; ++i)
                    for (int p = 0; p < 2; ++p)
                        for (int q = 0; q < 2; ++q) {
                            const double gar = gains ? gains[((size_t)i * P + p) * 2] : 1.0;
                            const double gai = gains ? gains[((size_t)i * P + p) * 2 + 1] : 0.0;
                            const double gbr = gains ? gains[((size_t)j * P + q) * 2] : 1.0;
                            const double gbi = gains ? gains[((size_t)j * P + q) * 2 + 1] : 0.0;
                            const size_t b = (size_t)j * (j + 1) / 2 + i;
                            const double *G = grad_vis + (((slot * B) + b) * 4 + (2 * p + q)) * 2;
                            const double Gr = G[0], Gi = G[1];
                            for (int s = 0; s < S; ++s) {
                                const size_t ua = ((size_t)i * P + p) * S + s, ub = ((size_t)j * P + q) * S + s;
                                /* Y = g U */
                                const double yar = gar * Ur[ua] - gai * Ui[ua], yai = gar * Ui[ua] + gai * Ur[ua];
                                const double ybr = gbr * Ur[ub] - gbi * Ui[ub], ybi = gbr * Ui[ub] + gbi * Ur[ub];
                                /* P = Y_a conj(Y_b) */
                                const double pr = yar * ybr + yai * ybi, pi = yai * ybr - yar * ybi;
                                /* dL for dV = c * P, c = i w: Re(conj(G) i w P) = w (-Gr Pi + Gi Pr) */
                                const double w = TWO_PI * f;
                                const double t = w * (-Gr * pi + Gi * pr);
                                const double fe = (double)s / (double)S, fb = 1.0 - fe;
                                my_tb[i] += fb * t;
                                my_te[i] += fe * t;
                                my_tb[j] -= fb * t;
                                my_te[j] -= fe * t;
                                /* gains: dV/dRe(g_a) = U_a conj(Y_b), dV/dIm(g_a) = i U_a conj(Y_b) */
                                const double d1r = Ur[ua] * ybr + Ui[ua] * ybi, d1i = Ui[ua] * ybr - Ur[ua] * ybi;
                                my[((size_t)i * P + p) * 2] += Gr * d1r + Gi * d1i;
                                my[((size_t)i * P + p) * 2 + 1] += Gr * (-d1i) + Gi * d1r;
                                /* dV/dRe(g_b) = Y_a conj(U_b), dV/dIm(g_b) = -i Y_a conj(U_b) */
                                const double d2r = yar * Ur[ub] + yai * Ui[ub], d2i = yai * Ur[ub] - yar * Ui[ub];
                                my[((size_t)j * P + q) * 2] += Gr * d2r + Gi * d2i;
                                my[((size_t)j * P + q) * 2 + 1] += Gr * d2i + Gi * (-d2r);
                            }
                        }
        }
    for (int t = 0; t < slots; ++t) {
        const double *my = acc + (size_t)t * per;
        for (int a = 0; a < N * P * 2; ++a) grad_gains[a] += my[a];
        for (int n = 0; n < N; ++n) {
            grad_tb[n] += my[(size_t)N * P * 2 + n];
            grad_te[n] += my[(size_t)N * P * 2 + N + n];
        }
    }
    free(acc);
    free(ure);
    free(uim);
    return 0;
}

/* Coherent beamformer (Sec. "Signal processing with GPU kernels": after
 * delay and bandpass correction each beam is steered by a phase shift and
 * summed over antenna fields, then optionally converted to Stokes
 * parameters). For beam b, pol p, spectrum s, channel k:
 *   B_bp(s, k) = sum_n a_n exp(+2 pi i f_k delta[b][n]) Y_np(s, k)
 * with delta[b][n] the beam's extra delay for station n (seconds, constant
 * over the block), a_n a real station weight (NULL = 1) and f_k the channel's
 * sky frequency. Output, with X = B_b0 and Y = B_b1:
 *   mode 0  complex voltages  out [SB][NB][C][S][4] = (Re X, Im X, Re Y, Im Y)
 *   mode 1  Stokes I          out [SB][NB][C][S/tint]
 *   mode 2  Stokes IQUV       out [SB][NB][C][S/tint][4]
 *           I = |X|^2 + |Y|^2, Q = |X|^2 - |Y|^2, U = 2 Re(X conj Y),
 *           V = 2 Im(X conj Y), each summed over tint consecutive spectra.
 * corr is the corrected block [SB][C][S][N][P]. */
int fxo_beamform(const double *corr, int SB, int N, int P, int C, int S, double fs, const double *centres,
                 int NB, const double *delays, const double *weights, int mode, int tint, double *out)
{
    if (P != 2 || NB < 1 || mode < 0 || mode > 2 || tint < 1 || S % tint != 0) return -1;
    if (mode == 0 && tint != 1) return -1;
    const int SO = S / tint;
#pragma omp parallel for collapse(3) schedule(dynamic)
    for (int sb = 0; sb < SB; ++sb)
        for (int b = 0; b < NB; ++b)
            for (int k = 0; k < C; ++k) {
                const double f = channel_freq(centres, sb, k, C, fs);
                for (int so = 0; so < SO; ++so) {
                    double acc[4] = {0.0, 0.0, 0.0, 0.0};
                    for (int t = 0; t < tint; ++t) {
                        const int s = so * tint + t;
                        double bx[2][2] = {{0.0, 0.0}, {0.0, 0.0}};   /* [pol][re, im] */
                        for (int n = 0; n < N; ++n) {
                            const double a = weights ? weights[n] : 1.0;
                            const double phi = TWO_PI * f * delays[(size_t)b * N + n];
                            const double wre = a * cos(phi), wim = a * sin(phi);
                            for (int p = 0; p < 2; ++p) {
                                const double *y = corr + (((((size_t)sb * C + k) * S + s) * N + n) * P + p) * 2;
                                bx[p][0] += wre * y[0] - wim * y[1];
                                bx[p][1] += wre * y[1] + wim * y[0];
                            }
                        }
                        if (mode == 0) {
                            double *o = out + ((((size_t)sb * NB + b) * C + k) * S + s) * 4;
                            o[0] = bx[0][0];
                            o[1] = bx[0][1];
                            o[2] = bx[1][0];
                            o[3] = bx[1][1];
                            continue;
                        }
                        const double xx = bx[0][0] * bx[0][0] + bx[0][1] * bx[0][1];
                        const double yy = bx[1][0] * bx[1][0] + bx[1][1] * bx[1][1];
                        /* X conj(Y) */
                        const double cre = bx[0][0] * bx[1][0] + bx[0][1] * bx[1][1];
                        const double cim = bx[0][1] * bx[1][0] - bx[0][0] * bx[1][1];
                        acc[0] += xx + yy;
                        acc[1] += xx - yy;
                        acc[2] += 2.0 * cre;
                        acc[3] += 2.0 * cim;
                    }
                    if (mode == 1) {
                        out[(((size_t)sb * NB + b) * C + k) * SO + so] = acc[0];
                    } else if (mode == 2) {
                        double *o = out + ((((size_t)sb * NB + b) * C + k) * SO + so) * 4;
                        for (int q = 0; q < 4; ++q) o[q] = acc[q];
                    }
                }
            }
    return 0;
}

/* Incoherent beam (Sec. "Signal processing with GPU kernels": incoherent
 * beamforming first computes Stokes parameters and then sums over antenna
 * fields). Per subband, channel and spectrum, each station's Stokes
 * parameters from its own X = Y_n0, Y = Y_n1 (definitions as in
 * fxo_beamform) are multiplied by the station weight a_n (NULL = 1) and
 * summed over stations and over tint consecutive spectra:
 *   mode 1  out [SB][C][S/tint]      Stokes I
 *   mode 2  out [SB][C][S/tint][4]   Stokes I, Q, U, V
 * corr is the corrected block [SB][C][S][N][P]. */
int fxo_beamform_incoherent(const double *corr, int SB, int N, int P, int C, int S, const double *weights, int mode,
                            int tint, double *out)
{
    if (P != 2 || mode < 1 || mode > 2 || tint < 1 || S % tint != 0) return -1;
    const int SO = S / tint;
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int sb = 0; sb < SB; ++sb)
        for (int k = 0; k < C; ++k)
            for (int so = 0; so < SO; ++so) {
                double acc[4] = {0.0, 0.0, 0.0, 0.0};
                for (int t = 0; t < tint; ++t) {
                    const int s = tint * so + t;
                    for (int n = 0; n < N; ++n) {
                        const double wn = weights ? weights[n] : 1.0;
                        const double *y = corr + ((((size_t)sb * C + k) * S + s) * N + n) * P * 2;
                        const double xre = y[0], xim = y[1], yre = y[2], yim = y[3];
                        const double xx = xre * xre + xim * xim;
                        const double yy = yre * yre + yim * yim;
                        acc[0] += wn * (xx + yy);
                        acc[1] += wn * (xx - yy);
                        acc[2] += wn * 2.0 * (xre * yre + xim * yim);    /* 2 Re(X conj Y) */
                        acc[3] += wn * 2.0 * (xim * yre - xre * yim);    /* 2 Im(X conj Y) */
                    }
                }
                if (mode == 1) {
                    out[((size_t)sb * C + k) * SO + so] = acc[0];
                } else {
                    double *o = out + (((size_t)sb * C + k) * SO + so) * 4;
                    for (int q = 0; q < 4; ++q) o[q] = acc[q];
                }
            }
    return 0;
}

int fxo_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
