// adjoint.cu -- differentiation form of correction + correlation: the
// gradient of a real loss L(V) with respect to per-(station, pol) complex
// gains and per-station delays, and the gain/delay application that makes the
// matching forward from raw visibilities.
//
// Paper link: Sec. "Signal processing with GPU kernels" (delay compensation
// is a per-channel phase rotation, bandpass a per-channel weight). With the
// delay held constant over the block, a corrected sample is
//   Y_a(s,k) = c_a(k) X_a(s,k),   c_a(k) = g_a exp(2 pi i f_k tau_n(a)),
// so every visibility factors as V_ab(k) = c_a(k) conj(c_b(k)) R_ab(k), where
// R is the correlation of the bandpass-corrected but otherwise uncorrected
// data (fx_correct with unit gains and zero delays, then fx_correlate).
//
// Backward, given dL/dRe(V) and dL/dIm(V) for every entry:
//   dV/dRe(g_a) = e_a conj(c_b) R          dV/dIm(g_a) = i e_a conj(c_b) R   (a first)
//   dV/dRe(g_b) = c_a conj(e_b) R          dV/dIm(g_b) = -i c_a conj(e_b) R  (b second)
//   dV/dtau_i   = +i 2 pi f_k V            dV/dtau_j   = -i 2 pi f_k V
// with e_a = exp(2 pi i f_k tau_n(a)). One thread per input a visits every
// partner b and adds the terms of the entries in which a takes part (a first
// when station(a) <= station(b), a second when station(b) <= station(a)), so
// each entry is seen from both of its ends and no atomics are needed. Per-input
// sums are kept in FP64 per CTA and reduced across CTAs in a fixed order
// (deterministic). Phases: 2 pi f_k tau in FP64 per (station, channel),
// reduced mod 2 pi, then FP32 sin/cos, as in the forward correction.
#include "internal.h"

namespace fxi {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

__device__ __forceinline__ float2 cm(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cj(float2 a) { return make_float2(a.x, -a.y); }

// e_a = exp(i 2 pi f_k tau_n) and c_a = g_a e_a for every input of channel k
__device__ __forceinline__ void phasors(int a, int k, int C, double f_sb, double fs, const double *tau,
                                        const float2 *gains, float2 &e, float2 &c)
{
    const int n = a >> 1;
    const double f = f_sb + (double)(k - C / 2) * fs / (double)C;
    const double ph = kTwoPi * f * tau[n];
    const float r = (float)(ph - kTwoPi * rint(ph / kTwoPi));
    float s, co;
    sincosf(r, &s, &co);
    e = make_float2(co, s);
    const float2 g = gains ? gains[a] : make_float2(1.f, 0.f);
    c = cm(g, e);
}

// V = c_a conj(c_b) R over all entries; one CTA per (subband, channel)
__global__ void apply_gains_kernel(const float2 *__restrict__ R, const float2 *__restrict__ gains,
                                   const double *__restrict__ tau, const double *__restrict__ centres,
                                   float2 *__restrict__ V, int N, int C, double fs)
{
    extern __shared__ float2 csh[];                 // [I]
    const int I = 2 * N;
    const long long ch = blockIdx.x;
    const int k = (int)(ch % C), sb = (int)(ch / C);
    for (int a = threadIdx.x; a < I; a += blockDim.x) {
        float2 e, c;
        phasors(a, k, C, centres[sb], fs, tau, gains, e, c);
        csh[a] = c;
    }
    __syncthreads();
    const long long B = (long long)N * (N + 1) / 2;
    const float2 *r = R + ch * B * 4;
    float2 *v = V + ch * B * 4;
    for (long long e = threadIdx.x; e < B * 4; e += blockDim.x) {
        const int pq = (int)(e & 3);
        const long long b = e >> 2;
        // invert b = j(j+1)/2 + i
        int j = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
        while ((long long)j * (j + 1) / 2 > b) --j;
        while ((long long)(j + 1) * (j + 2) / 2 <= b) ++j;
        const int i = (int)(b - (long long)j * (j + 1) / 2);
        const float2 ca = csh[2 * i + (pq >> 1)], cb = csh[2 * j + (pq & 1)];
        v[e] = cm(cm(ca, cj(cb)), r[e]);
    }
}

// Per-CTA partial gradients: thread a accumulates (dL/dRe g_a, dL/dIm g_a,
// dL/dtau contribution of input a) over the CTA's channels.
__global__ void adjoint_partial_kernel(const float2 *__restrict__ R, const float2 *__restrict__ G,
                                       const float2 *__restrict__ gains, const double *__restrict__ tau,
                                       const double *__restrict__ centres, double *__restrict__ partial,
                                       int N, int C, long long total_ch, double fs)
{
    extern __shared__ float2 sh[];                  // e[I], c[I]
    const int I = 2 * N;
    float2 *esh = sh, *csh = sh + I;
    const long long B = (long long)N * (N + 1) / 2;
    const int a = threadIdx.x;
    const int ia = a >> 1, pa = a & 1;
    double gre = 0.0, gim = 0.0, gt = 0.0;
    for (long long ch = blockIdx.x; ch < total_ch; ch += gridDim.x) {
        const int k = (int)(ch % C), sb = (int)(ch / C);
        __syncthreads();
        for (int t = threadIdx.x; t < I; t += blockDim.x) {
            float2 e, c;
            phasors(t, k, C, centres[sb], fs, tau, gains, e, c);
            esh[t] = e;
            csh[t] = c;
        }
        __syncthreads();
        if (a >= I) continue;
        const float w = (float)(kTwoPi * (centres[sb] + (double)(k - C / 2) * fs / (double)C));
        const float2 *r = R + ch * B * 4;
        const float2 *g = G + ch * B * 4;
        const float2 ea = esh[a], ca = csh[a];
        float sre = 0.f, sim = 0.f, st = 0.f;
        for (int bi = 0; bi < I; ++bi) {
            const int jb = bi >> 1, pb = bi & 1;
            const float2 cb = csh[bi];
            if (ia <= jb) {                                   // entry (a first, b second)
                const long long idx = ((long long)jb * (jb + 1) / 2 + ia) * 4 + 2 * pa + pb;
                const float2 Rv = r[idx], Gv = g[idx];
                const float2 cbR = cm(cj(cb), Rv);
                const float2 d1 = cm(ea, cbR);
                sre += Gv.x * d1.x + Gv.y * d1.y;
                sim += -Gv.x * d1.y + Gv.y * d1.x;
                const float2 Vv = cm(ca, cbR);
                st += w * (-Gv.x * Vv.y + Gv.y * Vv.x);
            }
            if (jb <= ia) {                                   // entry (b first, a second)
                const long long idx = ((long long)ia * (ia + 1) / 2 + jb) * 4 + 2 * pb + pa;
                const float2 Rv = r[idx], Gv = g[idx];
                const float2 eaR = cm(cj(ea), Rv);
                const float2 d2 = cm(cb, eaR);
                sre += Gv.x * d2.x + Gv.y * d2.y;
                sim += Gv.x * d2.y - Gv.y * d2.x;
                const float2 Vv = cm(cm(cb, cj(ca)), Rv);
                st -= w * (-Gv.x * Vv.y + Gv.y * Vv.x);
            }
        }
        gre += sre;
        gim += sim;
        gt += st;
    }
    if (a < I) {
        double *out = partial + ((long long)blockIdx.x * I + a) * 3;
        out[0] = gre;
        out[1] = gim;
        out[2] = gt;
    }
}

// Fixed-order reduction over CTAs: grad_gains[a] and grad_tau[n] (sum of pols).
__global__ void adjoint_reduce_kernel(const double *__restrict__ partial, int nblk, int N,
                                      float2 *__restrict__ grad_gains, double *__restrict__ grad_tau)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int I = 2 * N;
    double t = 0.0;
    for (int p = 0; p < 2; ++p) {
        const int a = 2 * n + p;
        double re = 0.0, im = 0.0;
        for (int b = 0; b < nblk; ++b) {
            const double *q = partial + ((long long)b * I + a) * 3;
            re += q[0];
            im += q[1];
            t += q[2];
        }
        if (grad_gains) grad_gains[a] = make_float2((float)re, (float)im);
    }
    if (grad_tau) grad_tau[n] = t;
}

// ---- delays moving over the block ------------------------------------------
// With tau_n(s) = tau_begin + (tau_end - tau_begin) s / S the visibility no
// longer factors through R. With unit gains, K = sum_s Y_a conj(Y_b) and
// M1 = sum_s (s/S) Y_a conj(Y_b) of the delay- and bandpass-corrected data Y,
//   V_ab = g_a conj(g_b) K_ab,
//   dV_ab/dtau_end[i]   = +i w g_a conj(g_b) M1_ab          (i = station of a)
//   dV_ab/dtau_begin[i] = +i w g_a conj(g_b) (K_ab - M1_ab)
// (minus for the station of b, w = 2 pi f_k), and the gain terms are those of
// the constant-delay adjoint with R replaced by K and e = 1. M1 is the X-stage
// of the corrected block with spectrum s scaled by sqrt(s/S) on both sides.

// corr *= sqrt(s / S) per spectrum (FP32 spectrum-blocked or FP32 planar layout)
__global__ void weight_spectra_kernel(float *__restrict__ corr, long long n, int planar, int N, int NB, int S,
                                      int S_pad)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        int s;
        if (planar) {
            s = (int)(e % S_pad);                       // [SB][C][2][I_pad][S_pad] floats
        } else {
            const long long f2 = e >> 1;                // [SB][C][NB][N][16][P] float2
            const int r = (int)((f2 >> 1) & 15);
            const long long bk = (f2 / (32LL * N)) % NB;
            s = (int)(bk * 16 + r);
        }
        corr[e] = s < S ? corr[e] * sqrtf((float)s / (float)S) : 0.f;
    }
}

// Per-CTA partial gradients for moving delays: (dL/dRe g_a, dL/dIm g_a,
// dL/dtau_begin and dL/dtau_end contributions of input a).
__global__ void adjoint_interp_partial_kernel(const float2 *__restrict__ K, const float2 *__restrict__ M1,
                                              const float2 *__restrict__ G, const float2 *__restrict__ gains,
                                              const double *__restrict__ centres, double *__restrict__ partial,
                                              int N, int C, long long total_ch, double fs)
{
    extern __shared__ float2 gsh[];                 // g[I]
    const int I = 2 * N;
    const long long B = (long long)N * (N + 1) / 2;
    const int a = threadIdx.x;
    const int ia = a >> 1, pa = a & 1;
    for (int t = threadIdx.x; t < I; t += blockDim.x) gsh[t] = gains ? gains[t] : make_float2(1.f, 0.f);
    __syncthreads();
    double gre = 0.0, gim = 0.0, gtb = 0.0, gte = 0.0;
    if (a < I) {
        const float2 ga = gsh[a];
        for (long long ch = blockIdx.x; ch < total_ch; ch += gridDim.x) {
            const int k = (int)(ch % C), sb = (int)(ch / C);
            const float w = (float)(kTwoPi * (centres[sb] + (double)(k - C / 2) * fs / (double)C));
            const float2 *kv = K + ch * B * 4, *mv = M1 + ch * B * 4, *gv = G + ch * B * 4;
            float sre = 0.f, sim = 0.f, sb_ = 0.f, se = 0.f;
            for (int bi = 0; bi < I; ++bi) {
                const int jb = bi >> 1, pb = bi & 1;
                const float2 gb = gsh[bi];
                if (ia <= jb) {                                   // entry (a first, b second)
                    const long long idx = ((long long)jb * (jb + 1) / 2 + ia) * 4 + 2 * pa + pb;
                    const float2 Kv = kv[idx], Mv = mv[idx], Gv = gv[idx];
                    const float2 d1 = cm(cj(gb), Kv);
                    sre += Gv.x * d1.x + Gv.y * d1.y;
                    sim += -Gv.x * d1.y + Gv.y * d1.x;
                    const float2 cab = cm(ga, cj(gb));
                    const float2 Vm = cm(cab, Mv), Vb = cm(cab, make_float2(Kv.x - Mv.x, Kv.y - Mv.y));
                    se += w * (-Gv.x * Vm.y + Gv.y * Vm.x);
                    sb_ += w * (-Gv.x * Vb.y + Gv.y * Vb.x);
                }
                if (jb <= ia) {                                   // entry (b first, a second)
                    const long long idx = ((long long)ia * (ia + 1) / 2 + jb) * 4 + 2 * pb + pa;
                    const float2 Kv = kv[idx], Mv = mv[idx], Gv = gv[idx];
                    const float2 d2 = cm(gb, Kv);
                    sre += Gv.x * d2.x + Gv.y * d2.y;
                    sim += Gv.x * d2.y - Gv.y * d2.x;
                    const float2 cba = cm(gb, cj(ga));
                    const float2 Vm = cm(cba, Mv), Vb = cm(cba, make_float2(Kv.x - Mv.x, Kv.y - Mv.y));
                    se -= w * (-Gv.x * Vm.y + Gv.y * Vm.x);
                    sb_ -= w * (-Gv.x * Vb.y + Gv.y * Vb.x);
                }
            }
            gre += sre;
            gim += sim;
            gtb += sb_;
            gte += se;
        }
        double *out = partial + ((long long)blockIdx.x * I + a) * 4;
        out[0] = gre;
        out[1] = gim;
        out[2] = gtb;
        out[3] = gte;
    }
}

__global__ void adjoint_interp_reduce_kernel(const double *__restrict__ partial, int nblk, int N,
                                             float2 *__restrict__ grad_gains, double *__restrict__ grad_tb,
                                             double *__restrict__ grad_te)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int I = 2 * N;
    double tb = 0.0, te = 0.0;
    for (int p = 0; p < 2; ++p) {
        const int a = 2 * n + p;
        double re = 0.0, im = 0.0;
        for (int b = 0; b < nblk; ++b) {
            const double *q = partial + ((long long)b * I + a) * 4;
            re += q[0];
            im += q[1];
            tb += q[2];
            te += q[3];
        }
        if (grad_gains) grad_gains[a] = make_float2((float)re, (float)im);
    }
    if (grad_tb) grad_tb[n] = tb;
    if (grad_te) grad_te[n] = te;
}

}  // namespace

int adjoint_blocks(const Handle &h)
{
    const long long total = (long long)h.p.n_subbands * h.p.n_channels;
    const long long want = 2LL * (h.num_sms > 0 ? h.num_sms : 152);
    return (int)(total < want ? total : want);
}

cudaError_t launch_apply_gains(const Handle &h, const float2 *R, const float2 *gains, const double *tau,
                               float2 *V, cudaStream_t st)
{
    const long long total = (long long)h.p.n_subbands * h.p.n_channels;
    if (total > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const size_t smem = sizeof(float2) * h.I;
    apply_gains_kernel<<<(unsigned)total, 256, smem, st>>>(R, gains, tau, h.d_centres, V, h.p.n_stations,
                                                           h.p.n_channels, h.p.sample_rate_hz);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const Handle &h, const float2 *R, const float2 *G, const float2 *gains,
                           const double *tau, float2 *grad_gains, double *grad_tau, cudaStream_t st)
{
    const int I = h.I;
    if (I > 1024) return cudaErrorNotSupported;
    const long long total = (long long)h.p.n_subbands * h.p.n_channels;
    const int nblk = adjoint_blocks(h);
    const int threads = (I + 31) / 32 * 32;
    const size_t smem = 2 * sizeof(float2) * I;
    adjoint_partial_kernel<<<nblk, threads, smem, st>>>(R, G, gains, tau, h.d_centres, h.d_adj_partial,
                                                        h.p.n_stations, h.p.n_channels, total,
                                                        h.p.sample_rate_hz);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adjoint_reduce_kernel<<<(h.p.n_stations + 127) / 128, 128, 0, st>>>(h.d_adj_partial, nblk, h.p.n_stations,
                                                                        grad_gains, grad_tau);
    return cudaGetLastError();
}

}  // namespace fxi

namespace fxi {

cudaError_t launch_weight_spectra(const Handle &h, void *corr, cudaStream_t st)
{
    const int planar = h.p.precision == FX_TF32_SPLIT;
    if (!planar && h.p.precision != FX_F32) return cudaErrorNotSupported;
    const int NB = (h.p.n_spectra + 15) / 16;
    const long long n = planar ? (long long)h.p.n_subbands * h.p.n_channels * 2 * h.I_pad * h.S_pad
                               : (long long)h.p.n_subbands * h.p.n_channels * NB * h.p.n_stations * 16 * kPols * 2;
    const long long want = (n + 255) / 256;
    const unsigned blocks = (unsigned)(want < 8LL * h.num_sms * 8 ? want : 8LL * h.num_sms * 8);
    if (blocks == 0) return cudaSuccess;
    weight_spectra_kernel<<<blocks, 256, 0, st>>>(static_cast<float *>(corr), n, planar, h.p.n_stations, NB,
                                                  h.p.n_spectra, h.S_pad);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_interp(const Handle &h, const float2 *K, const float2 *M1, const float2 *G,
                                  const float2 *gains, float2 *grad_gains, double *grad_tb, double *grad_te,
                                  cudaStream_t st)
{
    const int I = h.I;
    if (I > 1024) return cudaErrorNotSupported;
    const long long total = (long long)h.p.n_subbands * h.p.n_channels;
    const int nblk = adjoint_blocks(h);
    const int threads = (I + 31) / 32 * 32;
    adjoint_interp_partial_kernel<<<nblk, threads, sizeof(float2) * I, st>>>(
        K, M1, G, gains, h.d_centres, h.d_adj_partial, h.p.n_stations, h.p.n_channels, total, h.p.sample_rate_hz);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adjoint_interp_reduce_kernel<<<(h.p.n_stations + 127) / 128, 128, 0, st>>>(h.d_adj_partial, nblk,
                                                                               h.p.n_stations, grad_gains,
                                                                               grad_tb, grad_te);
    return cudaGetLastError();
}

}  // namespace fxi
