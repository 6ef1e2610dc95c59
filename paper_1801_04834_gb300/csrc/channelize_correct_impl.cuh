// channelize_correct_impl.cuh -- kernels and launch templates of the fused
// F-stage; compiled once per sample format (channelize_correct_ci16.cu,
// _ci8.cu, _ci4.cu, in parallel), dispatched by channelize_correct.cu.
#pragma once
//
// The F-stage and the delay/bandpass correction in one
// pass: raw int16/int8 samples in, corrected operands in the X-stage layout
// out, with no channelised intermediate in HBM.
//
// Paper, Sec. "Signal processing with GPU kernels": FIR and FFT channelise
// each subband, then fine delay compensation and bandpass correction end the
// per-station processing and transpose on write-back so the correlator reads
// all stations of a channel together. The paper runs these as separate
// kernels through device memory; fusing them removes the write and re-read of
// the channelised block (8 + 8 bytes per complex sample).
//
// The FIR and FFT are those of ppf.cu (register sliding-window FIR, two-pass
// in-register FFT). After FFT pass 2 each output X(n, p, s, k) is multiplied
// by bandpass(n, k) * gain(n, p) * exp(i phi), phi = phi0(n, k) + s * step(n, k)
// (phi0 reduced mod 2 pi and step formed in FP64 by the phase-table kernel,
// as in fx_correct); exp(i phi) is evaluated in FP32 after a reduction to
// [-pi, pi] with a two-constant Cody-Waite split of 2 pi, then __sincosf
// (absolute error about 4e-7 on that interval), once per (station, channel,
// spectrum) and shared by the two pols.
//
// Kernels (all write zeros for spectra past the block's end):
//   ppf_correct_ws_kernel     C = 16, 64, every output form: FIR and FFT on
//                             separate warps, pass 2 with lane = transform row
//                             so a warp store is one 256-byte run of the FP32
//                             spectrum-blocked layout [SB][C][ceil16(S)/16][N][16][2]
//                             or 2 inputs x 16 spectra of a planar plane;
//   ppf_correct_ws256_kernel  C = 256, planar outputs: one CTA per (station,
//                             pol), pass 2 with lane = spectrum;
//   ppf_correct_kernel        C = 256, FP32 output: FIR and FFT alternating
//                             on the same threads, writing from the pass-2
//                             registers.
// Planar outputs are [SB][C][planes][I_pad][S_pad] (FP16/BF16 x operand_scale,
// hi/lo FP16, or FP32 for the TF32-split X-stage); planar_pad zeroes what the
// F-stage does not write (inputs I..I_pad, spectra past the last round).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fft_reg.cuh"
#include "internal.h"
#include "ppf_common.cuh"

namespace fxi {
namespace {

using namespace ppf;

// OUT: 1 FP32 spectrum-blocked, 2 FP16 planar, 3 BF16 planar, 4 split FP16 planar, 5 FP32 planar.
// ppf_correct_kernel's per-round factor table: [kRound][IC inputs][PHC], rows
// padded so that FFT pass 2 (lanes = 8 or 16 consecutive channels x inputs)
// reads it conflict free
template <int C>
constexpr int fused_phc() { return C + (C == 16 ? 4 : 8); }

template <int C, typename TIn>
constexpr size_t fused_smem_bytes()
{
    using Cfg = PpfCfg<C>;
    return ppf_smem_bytes<C, TIn>() + (size_t)kRound * Cfg::NPC * kPols * fused_phc<C>() * sizeof(float2);
}

__device__ __forceinline__ unsigned short to_bits(float x, int out)
{
    if (out == 3) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return __half_as_ushort(__float2half_rn(x));
}

// lo part of split FP16: x - hi rounded to FP16, hi = the FP16 bits of x
__device__ __forceinline__ unsigned short lo_bits16(float x, unsigned short hi)
{
    return __half_as_ushort(__float2half_rn(x - __half2float(__ushort_as_half(hi))));
}

template <int C, int T, typename TIn, int OUT>
__global__ void __launch_bounds__(PpfCfg<C>::NT, PpfCfg<C>::NT >= 512 ? 1 : 2)
ppf_correct_kernel(const TIn *__restrict__ raw, void *__restrict__ corr, const float *__restrict__ taps,
                   const float2 *__restrict__ twiddle, const float2 *__restrict__ phase,
                   const float *__restrict__ bandpass, const float2 *__restrict__ gains, int N, int S, int I_pad,
                   int S_pad, float scale, int rounds_per_cta, const float *__restrict__ flags, int s_base,
                   int s_end)
{
    using Cfg = PpfCfg<C>;
    constexpr int R = Cfg::R, NPC = Cfg::NPC, NT = Cfg::NT, ROW = Cfg::ROW;
    constexpr int ROW_BYTES = C * kPols * (int)sizeof(TIn);
    constexpr int BUF_BYTES = kRound * NPC * ROW_BYTES;
    constexpr int IC = NPC * kPols;                 // inputs of this CTA
    constexpr int PHC = fused_phc<C>();
    constexpr int PHROW = IC * PHC;                 // factor-table row per spectrum
    static_assert(OUT == 1, "FP32 spectrum-blocked output (planar outputs: the warp-specialised kernels)");
    static_assert(NT >= 512 ? fused_smem_bytes<C, TIn>() <= 227 * 1024
                            : 2 * (fused_smem_bytes<C, TIn>() + 1024) <= 228 * 1024,
                  "two CTAs per SM (one at 512 threads)");
    static_assert(ROW_BYTES % 16 == 0, "rows must be whole 16-byte chunks");

    extern __shared__ __align__(16) unsigned char smem[];
    float2 *tw = reinterpret_cast<float2 *>(smem);
    unsigned char *inbuf = smem + C * sizeof(float2);
    float2 *u = reinterpret_cast<float2 *>(inbuf + 2 * BUF_BYTES);
    float2 *ph = u + Cfg::NTR * ROW;                // [kRound][IC][PHC] per-sample factors

    const int tid = threadIdx.x;
    const int sb = blockIdx.z;
    const int n0 = blockIdx.x * NPC;                // station groups fastest
    // spectra [s_base, s_end) of the block (s_base a multiple of 16); outputs are
    // written at s - s_base with S_pad (planar) or S_pad (FP32: spectra per
    // channel) as the output's spectrum stride
    const int s0 = s_base + blockIdx.y * rounds_per_cta * kRound;
    const int rows_total = S + T - 1;
    const long long L = (long long)rows_total * C;
    const int nrounds = min(rounds_per_cta, (s_end - s0 + kRound - 1) / kRound);
    const int I = N * kPols;

    auto stage = [&](int buf, int r0, int nrows) {
        const int chunks = nrows * ROW_BYTES / 16;
        for (int q = tid; q < NPC * chunks; q += NT) {
            const int st = q / chunks, ch = q - st * chunks;
            const int n = n0 + st;
            const int row_in = (ch * 16) / ROW_BYTES;
            const int byte_in_row = (ch * 16) - row_in * ROW_BYTES;
            unsigned char *dst = inbuf + buf * BUF_BYTES + (row_in * NPC + st) * ROW_BYTES + byte_in_row;
            const bool ok = (n < N) && (r0 + row_in < rows_total);
            const unsigned char *src = reinterpret_cast<const unsigned char *>(raw);
            if (ok) src += ((((long long)sb * N + n) * L + (long long)r0 * C) * kPols) * sizeof(TIn) + ch * 16;
            cp_async16(dst, src, ok ? 16 : 0);
        }
    };

    const int p = tid % kPols;
    const int c = (tid / kPols) % C;
    const int nl = tid / (kPols * C);

    for (int i = tid; i < C; i += NT) tw[i] = twiddle[i];
    // factor ownership: (station, channel) = tid mod NPC*C, spectra j = j0, j0+2, ...
    constexpr int OWN = NPC * C;                    // = NT / 2
    const int own_nc = tid % OWN, own_j0 = tid / OWN;
    const int own_nl = own_nc / C, own_k = own_nc % C;
    const int own_n = min(n0 + own_nl, N - 1);
    const float2 pst = phase[((long long)sb * N + own_n) * C + own_k];   // (phi0, step)
    float2 bgr[kPols];                              // bandpass x gain x scale of both pols
#pragma unroll
    for (int pp = 0; pp < kPols; ++pp) {
        const float b = bandpass ? bandpass[(long long)own_n * C + own_k] : 1.f;
        const float2 g = gains ? gains[own_n * kPols + pp] : make_float2(1.f, 0.f);
        bgr[pp] = make_float2(b * g.x * scale, b * g.y * scale);
    }

    // taps duplicated into (h, h) pairs: one packed FMA filters re and im
    float2 h[T];
#pragma unroll
    for (int k = 0; k < T; ++k) h[k] = make_float2(taps[k * C + c], taps[k * C + c]);

    stage(1, s0, T - 1);
    cp_async_commit();
    stage(0, s0 + T - 1, kRound);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();

    float2 win[T];
    const TIn *in1 = reinterpret_cast<const TIn *>(inbuf + BUF_BYTES);
#pragma unroll
    for (int k = 0; k < T - 1; ++k) win[k] = to_f2(in1[k * NT + tid]);
    win[T - 1] = make_float2(0.f, 0.f);
    __syncthreads();
    if (nrounds > 1) stage(1, s0 + T - 1 + kRound, kRound);
    cp_async_commit();

    for (int b = 0; b < nrounds; ++b) {
        const int sr = s0 + b * kRound;             // first spectrum of this round
        cp_async_wait<1>();
        __syncthreads();
        // ---- FIR over 16 new rows ----
        const TIn *in = reinterpret_cast<const TIn *>(inbuf + (b & 1) * BUF_BYTES);
#pragma unroll
        for (int j = 0; j < kRound; ++j) {
            win[(T - 1 + j) % T] = to_f2(in[j * NT + tid]);
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < T; ++k) {
                acc = __ffma2_rn(h[k], win[(j + k) % T], acc);
            }
            u[(j * IC + nl * kPols + p) * ROW + c] = acc;
        }
        // ---- per-sample factors flag * bandpass * gain * exp(i phi) of this round ----
#pragma unroll
        for (int q = 0; q < kRound / 2; ++q) {
            const int j = own_j0 + 2 * q;
            const float phi = fmaf((float)(sr + j), pst.y, pst.x);
            const float kq = rintf(phi * 0.15915494309189535f);           // phi / (2 pi)
            float r = fmaf(-kq, 6.28125f, phi);                           // 2 pi = 6.28125 + 1.9353...e-3
            r = fmaf(-kq, 1.9353071795864769e-3f, r);
            float sn, cs;
            __sincosf(r, &sn, &cs);
            // lost-data weight of (station, spectrum); 1 without flags
            const float fw = flags ? flags[(long long)own_n * S + min(sr + j, S - 1)] : 1.f;
            cs *= fw;
            sn *= fw;
#pragma unroll
            for (int pp = 0; pp < kPols; ++pp)
                ph[j * PHROW + (own_nl * kPols + pp) * PHC + own_k] =
                    make_float2(bgr[pp].x * cs - bgr[pp].y * sn, bgr[pp].x * sn + bgr[pp].y * cs);
        }
        __syncthreads();
        if (b + 2 < nrounds) stage(b & 1, s0 + T - 1 + (b + 2) * kRound, kRound);
        cp_async_commit();

        // ---- FFT pass 1 (all inputs read before the transposed writes) ----
        float2 y[Cfg::FFT_ITERS][R];
#pragma unroll
        for (int it = 0; it < Cfg::FFT_ITERS; ++it) {
            const int task = it * NT + tid;
            const float2 *row = u + (task / R) * ROW;
#pragma unroll
            for (int n1 = 0; n1 < R; ++n1) y[it][n1] = row[R * n1 + task % R];
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < Cfg::FFT_ITERS; ++it) {
            const int task = it * NT + tid;
            const int tr = task / R, n2 = task % R;
            float2 *row = u + tr * ROW;
            fft_reg<R>(y[it]);
#pragma unroll
            for (int k1 = 1; k1 < R; ++k1) y[it][k1] = cmul(y[it][k1], tw[n2 * k1]);
#pragma unroll
            for (int k1 = 0; k1 < R; ++k1) row[(R + 1) * k1 + n2] = y[it][k1];
        }
        __syncthreads();
        // ---- FFT pass 2 + correction, results held in registers ----
#pragma unroll
        for (int it = 0; it < Cfg::FFT_ITERS; ++it) {
            const int task = it * NT + tid;
            const int tr = task / R, k1 = task % R;  // transform tr = j * IC + il
            const float2 *row = u + tr * ROW;
#pragma unroll
            for (int n2 = 0; n2 < R; ++n2) y[it][n2] = row[(R + 1) * k1 + n2];
            fft_reg<R>(y[it]);
            const int j = tr / IC, il = tr % IC;
#pragma unroll
            for (int k2 = 0; k2 < R; ++k2) {
                const int kout = k1 + R * ((k2 + R / 2) % R);
                y[it][k2] = cmul(y[it][k2], ph[j * PHROW + il * PHC + kout]);
            }
        }
        {
            // ---- write out from registers into the spectrum-blocked FP32 layout
            // [SB][C][S_pad/16][N][16][2] (zeros past s_end) ----
            float2 *out = reinterpret_cast<float2 *>(corr);
            const int NB = S_pad / kRound;
#pragma unroll
            for (int it = 0; it < Cfg::FFT_ITERS; ++it) {
                const int task = it * NT + tid;
                const int tr = task / R, k1 = task % R;
                const int s = sr + tr / IC, i = 2 * n0 + tr % IC;
                if (i < I) {
                    const int so = s - s_base;
#pragma unroll
                    for (int k2 = 0; k2 < R; ++k2) {
                        const int kout = k1 + R * ((k2 + R / 2) % R);
                        out[((((long long)sb * C + kout) * NB + so / kRound) * N + (i >> 1)) * (2 * kRound) +
                            (so % kRound) * 2 + (i & 1)] = s < s_end ? y[it][k2] : make_float2(0.f, 0.f);
                    }
                }
            }
            // the next round's first barrier orders these reads of u before its FIR stores
        }
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Warp-specialised fused kernel, FP32 output (C = 16, 64). As ppf_ws_kernel:
// 128 FIR threads (NPC = 64 / C stations) and 128 FFT threads per CTA, FIR
// round b -> rows u[b & 1] -> FULL[b & 1]; FFT round b -> EMPTY[b & 1] for FIR
// round b + 2. Three further choices keep the shared-memory/L1 pipe (which
// also carries the global stores) below saturation:
//  * rows are input-major (row = input * 16 + spectrum, each input's 16 rows
//    offset by 8 entries so the FIR stores of the two pols use different banks);
//    pass 1 (R lanes per row, as in ppf_ws_kernel) writes its results
//    transposed, P1[k1][n2][row] with row stride NTR + 16/R (conflict free),
//    over u[b & 1] once every FFT thread has read its rows (barrier FFT);
//  * pass 2 runs with lane = row: a warp takes (group of 32 rows, k1) items,
//    so each output store of a warp is one station's 16 spectra x 2 pols of
//    one channel, 256 contiguous bytes of the spectrum-blocked layout;
//  * the FIR threads, which have the lighter share of the work, multiply
//    their FIR output by the input's complex gain x operand scale (the FFT is
//    linear, so this equals multiplying its output) and tabulate
//    bandpass x exp(i phi) x flag per (station, channel, spectrum) of their
//    round into a double-buffered table (one __sincosf per owner and round,
//    then rotations by exp(2 i step)); the FFT threads multiply each output
//    by that one factor.
template <int C>
struct FusedWsCfg {
    static constexpr int R = PpfCfg<C>::R;
    static constexpr int NPC = 64 / C;
    static constexpr int NF = NPC * C * kPols;           // 128 FIR threads, 128 FFT threads
    static constexpr int IC = NPC * kPols;               // inputs of a CTA
    static constexpr int NTR = IC * kRound;              // rows per round
    static constexpr int ROW = PpfCfg<C>::ROW;
    static constexpr int PADG = 8;                       // float2 offset per input (16 rows)
    static constexpr int USZ = NTR * ROW + IC * PADG;    // one row buffer
    static constexpr int RS = NTR + 16 / R;              // P1 row stride
    static constexpr int EJ = kRound + 2;                // phase table: 16 spectra + pad (even: 16-byte pairs)
    static constexpr int ESZ = NPC * C * EJ;             // one phase-table buffer
    static constexpr int ITEMS = (NTR / 32) * (R / 2);   // pass-2 items (row group, pair of k1)
    static_assert(C == 16 || C == 64, "warp-specialised fused kernel: C = 16 or 64");
    static_assert(R * R * RS <= USZ, "P1 fits over the row buffer");
    static_assert(ITEMS % 4 == 0 && NTR % 32 == 0, "four FFT warps share the pass-2 items");
};

template <int C, typename TIn>
constexpr size_t fused_ws_smem_bytes()
{
    using W = FusedWsCfg<C>;
    return (size_t)C * sizeof(float2) + 2ull * kRound * W::NPC * C * kPols * sizeof(TIn) +
           (2ull * W::USZ + 2ull * W::ESZ) * sizeof(float2) + 16;   // + 2 mbarriers
}

// CTAs per SM the shared memory allows: 3 at C = 64, 2 at C = 16 (four stations' rows)
template <int C, typename TIn>
constexpr int fused_ws_ctas()
{
    return 3 * (fused_ws_smem_bytes<C, TIn>() + 1024) <= 228 * 1024 ? 3 : 2;
}


// OUT as ppf_correct_kernel: 1 FP32 spectrum-blocked, 2 FP16 / 3 BF16 / 4 split
// FP16 / 5 FP32 planar ([SB][C][planes][I_pad][s_out], x scale for 2-4).
template <int C, int T, typename TIn, int OUT>
__global__ void __launch_bounds__(2 * FusedWsCfg<C>::NF, fused_ws_ctas<C, TIn>())
ppf_correct_ws_kernel(const TIn *__restrict__ raw, void *__restrict__ corr, const float *__restrict__ taps,
                      const float2 *__restrict__ twiddle, const float2 *__restrict__ phase,
                      const float *__restrict__ bandpass, const float2 *__restrict__ gains, int N, int S, int I_pad,
                      int s_out, float scale, int rounds_per_cta, const float *__restrict__ flags, int s_base,
                      int s_end, int *__restrict__ status, long long budget, int no_loads)
{
    using W = FusedWsCfg<C>;
    constexpr int R = W::R, NPC = W::NPC, NF = W::NF, ROW = W::ROW, PADG = W::PADG, USZ = W::USZ;
    constexpr int RS = W::RS, EJ = W::EJ, ESZ = W::ESZ;
    constexpr int ROW_BYTES = C * kPols * (int)sizeof(TIn);
    constexpr int BUF_BYTES = kRound * NPC * ROW_BYTES;
    constexpr int ALL = 2 * NF;
    static_assert(ROW_BYTES % 16 == 0, "rows must be whole 16-byte chunks");
    static_assert(2 * (fused_ws_smem_bytes<C, TIn>() + 1024) <= 228 * 1024, "at least two CTAs per SM");

    extern __shared__ __align__(16) unsigned char smem[];
    float2 *tw = reinterpret_cast<float2 *>(smem);
    unsigned char *inbuf = smem + C * sizeof(float2);
    float2 *u = reinterpret_cast<float2 *>(inbuf + 2 * BUF_BYTES);   // [2][USZ]
    float2 *et = u + 2 * USZ;                                         // [2][NPC][C][EJ]
    // raw-row mbarriers (one station per CTA: its rows arrive by bulk copy)
    const unsigned rbar = tc::smem_u32(et + 2 * ESZ);

    const int tid = threadIdx.x;
    const int sb = blockIdx.z;
    const int n0 = blockIdx.x * NPC;                // station groups fastest
    const int s0 = s_base + blockIdx.y * rounds_per_cta * kRound;
    const int rows_total = S + T - 1;
    const long long L = (long long)rows_total * C;
    const int nrounds = min(rounds_per_cta, (s_end - s0 + kRound - 1) / kRound);
    auto rowp = [&](float2 *uq, int r) { return uq + r * ROW + (r / kRound) * PADG; };

    for (int i = tid; i < C; i += ALL) tw[i] = twiddle[i];
    if constexpr (NPC == 1) {
        if (tid == 0) {
            tc::mbar_init(rbar, 1);
            tc::mbar_init(rbar + 8, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    __syncthreads();

    if (tid < NF) {
        // ---------------- FIR threads: (station nl, channel c, pol p) ----------------
        // one station (C = 64): thread 0 moves each round's raw rows (one
        // contiguous run) with a bulk copy completing on rbar[buf]; several
        // stations (C = 16): 16-byte cp.async by all FIR threads
        const unsigned char *rows0 = reinterpret_cast<const unsigned char *>(raw) +
                                     (((long long)sb * N + n0) * L) * kPols * sizeof(TIn);
        auto issue = [&](int buf, int r0, int nrows) {
            if (tid == 0 && !no_loads) {            // no_loads: failure-detection test hook
                const int nv = max(0, min(nrows, rows_total - r0));
                bulk_rows_issue(inbuf + buf * BUF_BYTES, rows0 + (long long)r0 * ROW_BYTES,
                                (unsigned)(nv * ROW_BYTES), rbar + 8u * buf);
            }
        };
        auto stage = [&](int buf, int r0, int nrows) {
            const int chunks = nrows * ROW_BYTES / 16;
            for (int q = tid; q < NPC * chunks; q += NF) {
                const int st = q / chunks, ch = q - st * chunks;
                const int n = n0 + st;
                const int row_in = (ch * 16) / ROW_BYTES;
                const int byte_in_row = (ch * 16) - row_in * ROW_BYTES;
                unsigned char *dst = inbuf + buf * BUF_BYTES + (row_in * NPC + st) * ROW_BYTES + byte_in_row;
                const bool ok = (n < N) && (r0 + row_in < rows_total);
                const unsigned char *src = reinterpret_cast<const unsigned char *>(raw);
                if (ok) src += ((((long long)sb * N + n) * L + (long long)r0 * C) * kPols) * sizeof(TIn) + ch * 16;
                cp_async16(dst, src, ok ? 16 : 0);
            }
        };
        const int p = tid % kPols;
        const int c = (tid / kPols) % C;
        const int nl = tid / (kPols * C);
        // phase-table role: (station, channel) = tid mod NPC*C, spectra j0, j0 + 2, ...
        constexpr int OWN = NPC * C;                // = NF / 2
        const int own_nc = tid % OWN, own_j0 = tid / OWN;
        const int own_n = min(n0 + own_nc / C, N - 1);
        const float2 pst = phase[((long long)sb * N + own_n) * C + own_nc % C];   // (phi0, step)
        float sn2, cs2;
        sincosf(2.f * pst.y, &sn2, &cs2);           // exp(2 i step): this owner's spectra are 2 apart
        const float bpo = bandpass ? bandpass[(long long)own_n * C + own_nc % C] : 1.f;
        const int n_fir = min(n0 + nl, N - 1);
        const float2 gg = gains ? gains[n_fir * kPols + p] : make_float2(1.f, 0.f);
        const float2 gsc = make_float2(gg.x * scale, gg.y * scale);
        const float2 rot2 = make_float2(cs2, sn2);
        float2 h[T];
#pragma unroll
        for (int k = 0; k < T; ++k) h[k] = make_float2(taps[k * C + c], taps[k * C + c]);

        if constexpr (NPC == 1) {
            issue(1, s0, T - 1);                        // history rows: buffer 1, phase 0
            issue(0, s0 + T - 1, kRound);               // round 0: buffer 0, phase 0
            raw_wait(rbar + 8, 0, status, budget);
        } else {
            stage(1, s0, T - 1);
            cp_async_commit();
            stage(0, s0 + T - 1, kRound);
            cp_async_commit();
            cp_async_wait<1>();
            named_bar_sync(kBarRaw, NF);
        }
        float2 win[T];
        const TIn *in1 = reinterpret_cast<const TIn *>(inbuf + BUF_BYTES);
#pragma unroll
        for (int k = 0; k < T - 1; ++k) win[k] = to_f2(in1[k * NF + tid]);
        win[T - 1] = make_float2(0.f, 0.f);
        named_bar_sync(kBarRaw, NF);
        if constexpr (NPC == 1) {
            if (tid == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (nrounds > 1) issue(1, s0 + T - 1 + kRound, kRound);    // round 1: buffer 1, phase 1
        } else {
            if (nrounds > 1) stage(1, s0 + T - 1 + kRound, kRound);
            cp_async_commit();
        }

        for (int b = 0; b < nrounds; ++b) {
            const int q = b & 1;
            const int sr = s0 + b * kRound;
            if constexpr (NPC == 1) {
                raw_wait(rbar + 8u * q, (unsigned)(((b + q) / 2) & 1), status, budget);   // round b's rows
            } else {
                cp_async_wait<1>();
                named_bar_sync(kBarRaw, NF);            // raw rows of round b are in
            }
            if (b >= 2) named_bar_sync(kBarEmpty + q, ALL);   // FFT threads are done with u[q], et[q]
            const TIn *in = reinterpret_cast<const TIn *>(inbuf + q * BUF_BYTES);
            float2 *uq = u + q * USZ;
            float2 *fo = rowp(uq, (nl * kPols + p) * kRound) + c;
            // four outputs at a time (four independent FMA chains); tap k of
            // output j takes the sample loaded at output j + k - (T - 1), so the
            // group's new samples stay in t[] until its outputs are formed
#pragma unroll
            for (int j0 = 0; j0 < kRound; j0 += 4) {
                float2 t[4], acc[4];
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    t[qq] = to_f2(in[(j0 + qq) * NF + tid]);
                    acc[qq] = make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int k = 0; k < T; ++k)
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq)
                        acc[qq] = __ffma2_rn(h[k], k >= T - 1 - qq ? t[qq + k - (T - 1)] : win[(j0 + qq + k) % T],
                                             acc[qq]);
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    fo[(j0 + qq) * ROW] = cmul(acc[qq], gsc);   // row (input, spectrum), times gain x scale
                    win[(T - 1 + j0 + qq) % T] = t[qq];
                }
            }
            // exp(i phi) x flag of this round: phi = phi0 + s step reduced to
            // [-pi, pi] (two-constant Cody-Waite split of 2 pi), then __sincosf
            // exp(i phi) at this owner's first spectrum of the round (re-anchored
            // every round), then rotations by exp(2 i step) for the next ones
            float2 *eq = et + q * ESZ + own_nc * EJ;
            float2 e;
            {
                const float phi = fmaf((float)(sr + own_j0), pst.y, pst.x);
                const float kq = rintf(phi * 0.15915494309189535f);
                float r = fmaf(-kq, 6.28125f, phi);
                r = fmaf(-kq, 1.9353071795864769e-3f, r);
                __sincosf(r, &e.y, &e.x);
                e.x *= bpo;
                e.y *= bpo;
            }
#pragma unroll
            for (int qq = 0; qq < kRound / 2; ++qq) {
                const int j = own_j0 + 2 * qq;
                const float fw = flags ? flags[(long long)own_n * S + min(sr + j, S - 1)] : 1.f;
                eq[j] = make_float2(e.x * fw, e.y * fw);
                e = cmul(e, rot2);
            }
            named_bar_arrive(kBarFull + q, ALL);
            named_bar_sync(kBarRaw, NF);                // every FIR thread has read raw buffer q
            if constexpr (NPC == 1) {
                if (tid == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (b + 2 < nrounds) issue(q, s0 + T - 1 + (b + 2) * kRound, kRound);
            } else {
                if (b + 2 < nrounds) stage(q, s0 + T - 1 + (b + 2) * kRound, kRound);
                cp_async_commit();
            }
        }
        if constexpr (NPC != 1) cp_async_wait<0>();
    } else {
        // ---------------- FFT threads ----------------
        const int t = tid - NF;
        const int warp = t / 32, lane = t % 32;
        float2 twr[R];                              // W_C^(n2 k1), n2 = t mod R
#pragma unroll
        for (int k1 = 1; k1 < R; ++k1) twr[k1] = tw[(t % R) * k1];
        const int NB = s_out / kRound;
        const int I = N * kPols;
        constexpr int P1ITERS = W::NTR * R / NF;
        for (int b = 0; b < nrounds; ++b) {
            const int q = b & 1;
            const int sr = s0 + b * kRound;
            float2 *uq = u + q * USZ;
            const float2 *eq = et + q * ESZ;
            named_bar_sync(kBarFull + q, ALL);          // FIR round b is in u[q], et[q]
            // pass 1: R-point FFTs over n1 (stride R), times W_C^(n2 k1)
            float2 v1[P1ITERS][R];
#pragma unroll
            for (int it = 0; it < P1ITERS; ++it) {
                const int task = it * NF + t;
                const float2 *row = rowp(uq, task / R);
#pragma unroll
                for (int n1 = 0; n1 < R; ++n1) v1[it][n1] = row[R * n1 + task % R];
                fft_reg<R>(v1[it]);
#pragma unroll
                for (int k1 = 1; k1 < R; ++k1) v1[it][k1] = cmul(v1[it][k1], twr[k1]);
            }
            named_bar_sync(kBarFft, NF);                // every FFT thread has read its rows of u[q]
#pragma unroll
            for (int it = 0; it < P1ITERS; ++it) {
                const int task = it * NF + t;
#pragma unroll
                for (int k1 = 0; k1 < R; ++k1) uq[(k1 * R + task % R) * RS + task / R] = v1[it][k1];
            }
            named_bar_sync(kBarFft, NF);                // P1 complete
            // pass 2: a half-warp per k1 (two k1 per item), each lane two adjacent
            // rows (input il, spectra j and j + 1), so the rows and the phase
            // factors come in 16-byte loads and the planar stores go out in pairs
#pragma unroll
            for (int it = 0; it < W::ITEMS / 4; ++it) {
                const int item = warp + 4 * it;
                const int g = item / (R / 2), k1 = 2 * (item % (R / 2)) + lane / 16;
                const int r = 32 * g + 2 * (lane % 16);
                const int il = r / kRound, j = r % kRound;
                float2 va[R], vb[R];
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    const float4 w = *reinterpret_cast<const float4 *>(uq + (k1 * R + m) * RS + r);
                    va[m] = make_float2(w.x, w.y);
                    vb[m] = make_float2(w.z, w.w);
                }
                fft_reg<R>(va);
                fft_reg<R>(vb);
                const float2 *e = eq + ((il / kPols) * C) * EJ + j;
#pragma unroll
                for (int k2 = 0; k2 < R; ++k2) {
                    const int kout = k1 + R * ((k2 + R / 2) % R);
                    const float4 f = *reinterpret_cast<const float4 *>(e + kout * EJ);
                    va[k2] = cmul(va[k2], make_float2(f.x, f.y));
                    vb[k2] = cmul(vb[k2], make_float2(f.z, f.w));
                }
                if (it == W::ITEMS / 4 - 1 && b + 2 < nrounds) named_bar_arrive(kBarEmpty + q, ALL);
                const int s = sr + j, i = 2 * n0 + il;
                if (sr + kRound > s_end) {                  // only in the block's last round
#pragma unroll
                    for (int k2 = 0; k2 < R; ++k2) {
                        if (s >= s_end) va[k2] = make_float2(0.f, 0.f);
                        if (s + 1 >= s_end) vb[k2] = make_float2(0.f, 0.f);
                    }
                }
                if (i < I) {
                    if constexpr (OUT == 1) {
                        // one warp store = one station's 16 spectra x 2 pols of two channels
                        float2 *out = reinterpret_cast<float2 *>(corr) +
                                      ((((long long)sb * C) * NB + (sr - s_base) / kRound) * N + (i >> 1)) *
                                          (2 * kRound) + j * 2 + (i & 1);
                        const long long kstride = (long long)NB * N * (2 * kRound);
#pragma unroll
                        for (int k2 = 0; k2 < R; ++k2) {
                            const int kout = k1 + R * ((k2 + R / 2) % R);
                            out[kout * kstride] = va[k2];
                            out[kout * kstride + 2] = vb[k2];
                        }
                    } else {
                        // planar: one warp store = 2 inputs x 16 spectra of two (channel, plane)
                        constexpr int planes = OUT == 4 ? 4 : 2;
                        const long long pstride = (long long)I_pad * s_out;
                        const long long base = (long long)sb * C * planes * pstride + (long long)i * s_out + (s - s_base);
#pragma unroll
                        for (int k2 = 0; k2 < R; ++k2) {
                            const int kout = k1 + R * ((k2 + R / 2) % R);
                            const float2 ya = va[k2], yb = vb[k2];
                            const long long o = base + (long long)kout * planes * pstride;
                            if constexpr (OUT == 5) {
                                float *out = reinterpret_cast<float *>(corr);
                                *reinterpret_cast<float2 *>(out + o) = make_float2(ya.x, yb.x);
                                *reinterpret_cast<float2 *>(out + o + pstride) = make_float2(ya.y, yb.y);
                            } else {
                                unsigned short *out = reinterpret_cast<unsigned short *>(corr);
                                const unsigned short ra = to_bits(ya.x, OUT), ia = to_bits(ya.y, OUT);
                                const unsigned short rb = to_bits(yb.x, OUT), ib = to_bits(yb.y, OUT);
                                *reinterpret_cast<unsigned *>(out + o) = (unsigned)ra | ((unsigned)rb << 16);
                                *reinterpret_cast<unsigned *>(out + o + pstride) = (unsigned)ia | ((unsigned)ib << 16);
                                if constexpr (OUT == 4) {
                                    const unsigned short lra = lo_bits16(ya.x, ra), lia = lo_bits16(ya.y, ia);
                                    const unsigned short lrb = lo_bits16(yb.x, rb), lib = lo_bits16(yb.y, ib);
                                    *reinterpret_cast<unsigned *>(out + o + 2 * pstride) =
                                        (unsigned)lra | ((unsigned)lrb << 16);
                                    *reinterpret_cast<unsigned *>(out + o + 3 * pstride) =
                                        (unsigned)lia | ((unsigned)lib << 16);
                                }
                            }
                        }
                    }
                }
            }
        }
    }
}

// Zero the padding of the planar layout that the fused kernel does not cover:
// inputs [I, I_pad) and spectra [ceil16(S), S_pad) of every (subband, channel, plane).
__global__ void planar_pad_kernel(unsigned short *__restrict__ corr, long long n_rows, int I, int I_pad, int S16,
                                  int S_pad)
{
    const long long row = blockIdx.x;               // (sb, c, plane, i) flattened
    if (row >= n_rows) return;
    const int i = (int)(row % I_pad);
    unsigned short *r = corr + row * S_pad;
    const int from = (i >= I) ? 0 : S16;
    for (int s = from + threadIdx.x; s < S_pad; s += blockDim.x) r[s] = 0;
}

// ---------------------------------------------------------------------------
// Warp-specialised fused kernel for C = 256 with planar outputs (OUT = 2..5):
// one CTA per (station, pol), 256 FIR threads (one channel each) and 256 FFT
// threads in two groups of 128, one CTA per SM. A round's rows (16 spectra
// of one input) fit twice in shared memory at this channel count only per
// input; the CTAs of a station's two pols are neighbours in the grid and read
// the same raw rows (the second read mostly from L2). FIR round b -> u[b & 1]
// and the whole per-sample factor bandpass x gain x flag x exp(i phi) of its
// 16 spectra (one __sincosf per channel and round, multiplied once by
// bandpass x gain, then rotations by exp(i step) computed in FP32 from the
// FP64-derived step; bandpass x gain is constant per channel within a CTA,
// which serves one input) -> FULL[b & 1]. FFT group g takes the rounds
// b = g mod 2 (row buffer g) with its own named barrier, so two rounds are in
// FFT at once and each FFT thread has two transforms in flight per pass
// (36.6 against 39.5 ms at the 8-bit workload with one group of 256): pass 1
// (row = 16 lanes), transposed into P1[k1][n2][row] over u[g] after the
// group's barrier, pass 2 with lane = spectrum (a half-warp per k1), so a
// warp store is 2 x 32 bytes of planar rows.
struct Ws256 {
    static constexpr int C = 256, R = 16, NF = 256;
    static constexpr int ROW = C + 16;                  // FIR row stride (float2)
    static constexpr int USZ = kRound * ROW;            // one row buffer: 16 spectra
    static constexpr int RS = kRound + 1;               // P1 row stride
    static constexpr int EJ = kRound + 1;               // phasor table: [C][EJ]
    static constexpr int ESZ = C * EJ;
    static_assert(R * R * RS <= USZ, "P1 fits over the row buffer");
};

template <typename TIn>
constexpr size_t ws256_smem_bytes()
{
    using W = Ws256;
    return (size_t)W::C * sizeof(float2) + 2ull * kRound * W::C * kPols * sizeof(TIn) +
           (2ull * W::USZ + 2ull * W::ESZ + 2ull * W::C) * sizeof(float2) + 16;   // + 2 mbarriers
}

template <int T, typename TIn, int OUT>
__global__ void __launch_bounds__(2 * Ws256::NF, 1)
ppf_correct_ws256_kernel(const TIn *__restrict__ raw, void *__restrict__ corr, const float *__restrict__ taps,
                         const float2 *__restrict__ twiddle, const float2 *__restrict__ phase,
                         const float *__restrict__ bandpass, const float2 *__restrict__ gains, int N, int S,
                         int I_pad, int s_out, float scale, int rounds_per_cta, const float *__restrict__ flags,
                         int s_base, int s_end, int *__restrict__ status, long long budget, int no_loads)
{
    using W = Ws256;
    constexpr int C = W::C, R = W::R, NF = W::NF, ROW = W::ROW, USZ = W::USZ, RS = W::RS, EJ = W::EJ, ESZ = W::ESZ;
    constexpr int ROW_BYTES = C * kPols * (int)sizeof(TIn);     // one raw time row of the station (both pols)
    constexpr int BUF_BYTES = kRound * ROW_BYTES;
    constexpr int ALL = 2 * NF;
    constexpr int NG = NF / 2;                  // FFT threads per group: group g takes rounds b = g mod 2
    constexpr int HAND = NF + NG;               // FULL / EMPTY: the FIR threads and one FFT group
    static_assert(OUT >= 2 && OUT <= 5, "planar outputs");
    static_assert(ROW_BYTES % 16 == 0, "rows must be whole 16-byte chunks");
    static_assert(ws256_smem_bytes<TIn>() <= 227 * 1024, "one CTA per SM");

    extern __shared__ __align__(16) unsigned char smem[];
    float2 *tw = reinterpret_cast<float2 *>(smem);
    unsigned char *inbuf = smem + C * sizeof(float2);
    float2 *u = reinterpret_cast<float2 *>(inbuf + 2 * BUF_BYTES);   // [2][USZ]
    float2 *et = u + 2 * USZ;                                         // [2][C][EJ]
    float2 *bgt = et + 2 * ESZ;                                       // [C] bandpass x gain x scale
    float2 *tw2 = bgt + C;                                            // [k1][n2] = W_C^(n2 k1): pass-1
                                                                      // lanes (n2) read consecutive entries
    const unsigned rbar = tc::smem_u32(tw2 + C);                      // raw-row mbarriers [2]
    const int tid = threadIdx.x;
    const int sb = blockIdx.z;
    const int n = blockIdx.x / kPols, p = blockIdx.x % kPols;       // (station, pol) fastest
    const int s0 = s_base + blockIdx.y * rounds_per_cta * kRound;
    const int rows_total = S + T - 1;
    const long long L = (long long)rows_total * C;
    const int nrounds = min(rounds_per_cta, (s_end - s0 + kRound - 1) / kRound);

    for (int i = tid; i < C; i += ALL) {
        tw[i] = twiddle[i];
        tw2[i] = twiddle[(i % R) * (i / R)];
        const float b = bandpass ? bandpass[(long long)n * C + i] : 1.f;
        const float2 g = gains ? gains[n * kPols + p] : make_float2(1.f, 0.f);
        bgt[i] = make_float2(b * g.x * scale, b * g.y * scale);
    }
    if (tid == 0) {
        tc::mbar_init(rbar, 1);
        tc::mbar_init(rbar + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (tid < NF) {
        // ---------------- FIR threads: channel c of input (n, p) ----------------
        // the station's raw rows of a round are one contiguous run: thread 0
        // moves it with a bulk copy completing on rbar[buf]
        const unsigned char *rows0 = reinterpret_cast<const unsigned char *>(raw) +
                                     (((long long)sb * N + n) * L) * kPols * sizeof(TIn);
        auto issue = [&](int buf, int r0, int nrows) {
            if (tid == 0 && !no_loads) {            // no_loads: failure-detection test hook
                const int nv = max(0, min(nrows, rows_total - r0));
                bulk_rows_issue(inbuf + buf * BUF_BYTES, rows0 + (long long)r0 * ROW_BYTES,
                                (unsigned)(nv * ROW_BYTES), rbar + 8u * buf);
            }
        };
        const int c = tid;
        const float2 pst = phase[((long long)sb * N + n) * C + c];   // (phi0, step)
        const float2 bgc = bgt[c];                                   // this input's bandpass x gain x scale
        float sn1, cs1;
        sincosf(pst.y, &sn1, &cs1);                                  // exp(i step)
        const float2 rot = make_float2(cs1, sn1);
        float2 h[T];
#pragma unroll
        for (int k = 0; k < T; ++k) h[k] = make_float2(taps[k * C + c], taps[k * C + c]);

        issue(1, s0, T - 1);                            // history rows: buffer 1, phase 0
        issue(0, s0 + T - 1, kRound);                   // round 0: buffer 0, phase 0
        raw_wait(rbar + 8, 0, status, budget);
        float2 win[T];
        const TIn *in1 = reinterpret_cast<const TIn *>(inbuf + BUF_BYTES);
#pragma unroll
        for (int k = 0; k < T - 1; ++k) win[k] = to_f2(in1[k * C * kPols + c * kPols + p]);
        win[T - 1] = make_float2(0.f, 0.f);
        named_bar_sync(kBarRaw, NF);
        if (tid == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (nrounds > 1) issue(1, s0 + T - 1 + kRound, kRound);     // round 1: buffer 1, phase 1

        for (int b = 0; b < nrounds; ++b) {
            const int q = b & 1;
            const int sr = s0 + b * kRound;
            raw_wait(rbar + 8u * q, (unsigned)(((b + q) / 2) & 1), status, budget);   // round b's rows
            if (b >= 2) named_bar_sync(kBarEmpty + q, HAND);
            const TIn *in = reinterpret_cast<const TIn *>(inbuf + q * BUF_BYTES);
            float2 *uq = u + q * USZ;
            // four outputs at a time (see the 16/64-channel kernel)
#pragma unroll
            for (int j0 = 0; j0 < kRound; j0 += 4) {
                float2 t[4], acc[4];
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    t[qq] = to_f2(in[(j0 + qq) * C * kPols + c * kPols + p]);
                    acc[qq] = make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int k = 0; k < T; ++k)
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq)
                        acc[qq] = __ffma2_rn(h[k], k >= T - 1 - qq ? t[qq + k - (T - 1)] : win[(j0 + qq + k) % T],
                                             acc[qq]);
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    uq[(j0 + qq) * ROW + c] = acc[qq];
                    win[(T - 1 + j0 + qq) % T] = t[qq];
                }
            }
            // phasors of this round: phi(sr) reduced to [-pi, pi] (two-constant
            // Cody-Waite split of 2 pi) and __sincosf, then rotations by exp(i step)
            float2 *eq = et + q * ESZ + c * EJ;
            float2 e;
            {
                const float phi = fmaf((float)sr, pst.y, pst.x);
                const float kq = rintf(phi * 0.15915494309189535f);
                float r = fmaf(-kq, 6.28125f, phi);
                r = fmaf(-kq, 1.9353071795864769e-3f, r);
                __sincosf(r, &e.y, &e.x);
            }
            e = cmul(bgc, e);                           // the anchor carries bandpass x gain
            if (flags) {
#pragma unroll
                for (int j = 0; j < kRound; ++j) {
                    const float fw = flags[(long long)n * S + min(sr + j, S - 1)];
                    eq[j] = make_float2(e.x * fw, e.y * fw);     // the whole per-sample factor
                    e = cmul(e, rot);
                }
            } else {
#pragma unroll
                for (int j = 0; j < kRound; ++j) {
                    eq[j] = e;
                    e = cmul(e, rot);
                }
            }
            named_bar_arrive(kBarFull + q, HAND);
            named_bar_sync(kBarRaw, NF);                // every FIR thread has read raw buffer q
            if (tid == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (b + 2 < nrounds) issue(q, s0 + T - 1 + (b + 2) * kRound, kRound);
        }
    } else {
        // ---------------- FFT threads: two groups of NG, group g = buffer g ----------------
        const int t = tid - NF;
        const int g = t / NG, tg = t % NG;
        const int bar_fft = g ? kBarFft2 : kBarFft;
        constexpr int planes = OUT == 4 ? 4 : 2;
        const long long pstride = (long long)I_pad * s_out;
        const int i = n * kPols + p;
        for (int b = g; b < nrounds; b += 2) {
            const int q = b & 1;
            const int sr = s0 + b * kRound;
            float2 *uq = u + q * USZ;
            const float2 *eq = et + q * ESZ;
            named_bar_sync(kBarFull + q, HAND);
            // pass 1: two (row tr = spectrum, column n2) tasks per thread
            float2 v[2][R];
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int task = it * NG + tg;
                const int tr = task / R, n2 = task % R;
#pragma unroll
                for (int n1 = 0; n1 < R; ++n1) v[it][n1] = uq[tr * ROW + R * n1 + n2];
            }
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int n2 = (it * NG + tg) % R;
                fft_reg<R>(v[it]);
#pragma unroll
                for (int k1 = 1; k1 < R; ++k1) v[it][k1] = cmul(v[it][k1], tw2[k1 * R + n2]);
            }
            named_bar_sync(bar_fft, NG);                // every thread of the group has read u[q]
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int task = it * NG + tg;
                const int tr = task / R, n2 = task % R;
#pragma unroll
                for (int k1 = 0; k1 < R; ++k1) uq[(k1 * R + n2) * RS + tr] = v[it][k1];
            }
            named_bar_sync(bar_fft, NG);                // P1 complete
            // pass 2: two (k1, spectrum j) items per thread, a half-warp per k1
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int item = it * NG + tg;
                const int k1 = item / 16, j = item % 16;
#pragma unroll
                for (int m = 0; m < R; ++m) v[it][m] = uq[(k1 * R + m) * RS + j];
            }
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int item = it * NG + tg;
                const int k1 = item / 16, j = item % 16;
                fft_reg<R>(v[it]);
#pragma unroll
                for (int k2 = 0; k2 < R; ++k2) {
                    const int kout = k1 + R * ((k2 + R / 2) % R);
                    v[it][k2] = cmul(v[it][k2], eq[kout * EJ + j]);
                }
            }
            if (b + 2 < nrounds) named_bar_arrive(kBarEmpty + q, HAND);
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int item = it * NG + tg;
                const int k1 = item / 16, j = item % 16;
                const int s = sr + j;
                if (sr + kRound > s_end && s >= s_end) {       // only in the block's last round
#pragma unroll
                    for (int k2 = 0; k2 < R; ++k2) v[it][k2] = make_float2(0.f, 0.f);
                }
                const long long base = (long long)sb * C * planes * pstride + (long long)i * s_out + (s - s_base);
#pragma unroll
                for (int k2 = 0; k2 < R; ++k2) {
                    const int kout = k1 + R * ((k2 + R / 2) % R);
                    const float2 y = v[it][k2];
                    const long long o = base + (long long)kout * planes * pstride;
                    if constexpr (OUT == 5) {
                        float *out = reinterpret_cast<float *>(corr);
                        out[o] = y.x;
                        out[o + pstride] = y.y;
                    } else {
                        unsigned short *out = reinterpret_cast<unsigned short *>(corr);
                        const unsigned short hr = to_bits(y.x, OUT), hi = to_bits(y.y, OUT);
                        out[o] = hr;
                        out[o + pstride] = hi;
                        if constexpr (OUT == 4) {
                            out[o + 2 * pstride] =
                                __half_as_ushort(__float2half_rn(y.x - __half2float(__ushort_as_half(hr))));
                            out[o + 3 * pstride] =
                                __half_as_ushort(__float2half_rn(y.y - __half2float(__ushort_as_half(hi))));
                        }
                    }
                }
            }
        }
    }
}

// Zeros of the planar layout outside what the F-stage wrote: inputs [I, I_pad)
// and spectra [S16, s_out) of every (subband, channel, plane).
cudaError_t planar_pad(const Handle &h, void *corr, int out, int S16, int s_out, cudaStream_t st)
{
    if (h.I_pad <= h.I && s_out <= S16) return cudaSuccess;
    const long long rows = (long long)h.p.n_subbands * h.p.n_channels * (out == 4 ? 4 : 2) * h.I_pad;
    if (rows > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    // zero bits are zero in either element size: FP32 rows are twice as many 16-bit words
    const int w = out == 5 ? 2 : 1;
    planar_pad_kernel<<<(unsigned)rows, 64, 0, st>>>(reinterpret_cast<unsigned short *>(corr), rows, h.I, h.I_pad,
                                                      w * S16, w * s_out);
    return cudaGetLastError();
}

template <int C, int T, typename TIn, int OUT>
cudaError_t launch_t(const Handle &h, const void *raw, void *corr, const float *bandpass, const float2 *gains,
                     const float *flags, const FWindow *win, cudaStream_t st)
{
    using Cfg = PpfCfg<C>;
    const int N = h.p.n_stations, S = h.p.n_spectra, SB = h.p.n_subbands;
    // spectra [s_base, s_end) into an output whose spectrum stride is s_out
    const int s_base = win ? win->s_base : 0;
    const int s_end = win ? win->s_end : S;
    // FP32: the spectrum-blocked layout, s_out a multiple of 16 (ceil16(S) by default)
    const int s_out = win ? win->s_out : (OUT == 1 ? (S + kRound - 1) / kRound * kRound : h.S_pad);
    if (s_base % kRound != 0 || s_end > S || s_base >= s_end || s_end - s_base > s_out ||
        (OUT == 1 && s_out % kRound != 0))
        return cudaErrorInvalidValue;
    const int rounds_total = (s_end - s_base + kRound - 1) / kRound;
    const float scale = (OUT == 1 || OUT == 5) ? 1.f : h.operand_scale;
    if constexpr (C == 16 || C == 64) {
        using W = FusedWsCfg<C>;
        const int sg = (N + W::NPC - 1) / W::NPC;
        // long runs amortise the T-1 history rows each CTA filters first; shorten
        // them only while the grid would be under ~5 waves
        int rpc = 64;
        while (rpc > 1 && (long long)((rounds_total + rpc - 1) / rpc) * sg * SB < 152LL * 16) rpc /= 2;
        dim3 grid(sg, (rounds_total + rpc - 1) / rpc, SB);
        if (grid.x > 0x7fffffffu || grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
        constexpr size_t smem = fused_ws_smem_bytes<C, TIn>();
        auto kern = ppf_correct_ws_kernel<C, T, TIn, OUT>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, 2 * W::NF, smem, st>>>(reinterpret_cast<const TIn *>(raw), corr, h.d_taps, h.d_twiddle,
                                            h.d_phase, bandpass, gains, N, S, h.I_pad, s_out, scale, rpc, flags,
                                            s_base, s_end, h.d_status, h.tc_timeout_cycles, h.tc_test_no_tma);
        e = cudaGetLastError();
        if (e != cudaSuccess || OUT == 1) return e;
        return planar_pad(h, corr, OUT, rounds_total * kRound, s_out, st);
    } else if constexpr (C == 256 && OUT != 1) {
        // one CTA per (station, pol) and SM; long runs of rounds amortise the
        // prologue, shortened only while the grid would be under ~4 waves
        int rpc = 64;
        while (rpc > 1 && (long long)((rounds_total + rpc - 1) / rpc) * N * kPols * SB < 152LL * 4) rpc /= 2;
        dim3 grid(N * kPols, (rounds_total + rpc - 1) / rpc, SB);
        if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
        constexpr size_t smem = ws256_smem_bytes<TIn>();
        auto kern = ppf_correct_ws256_kernel<T, TIn, OUT>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, 2 * Ws256::NF, smem, st>>>(reinterpret_cast<const TIn *>(raw), corr, h.d_taps, h.d_twiddle,
                                                h.d_phase, bandpass, gains, N, S, h.I_pad, s_out, scale, rpc, flags,
                                                s_base, s_end, h.d_status, h.tc_timeout_cycles,
                                                h.tc_test_no_tma);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return planar_pad(h, corr, OUT, rounds_total * kRound, s_out, st);
    } else {
        const int sgroups = (N + Cfg::NPC - 1) / Cfg::NPC;
        // long runs of rounds per CTA amortise the T-1 history rows each CTA reads
        // and filters first; shorten them only while the grid would be under ~8 waves
        int rpc = 32;
        while (rpc > 1 && (long long)((rounds_total + rpc - 1) / rpc) * sgroups * SB < 152LL * 16) rpc /= 2;
        dim3 grid(sgroups, (rounds_total + rpc - 1) / rpc, SB);
        if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
        constexpr size_t smem = fused_smem_bytes<C, TIn>();
        auto kern = ppf_correct_kernel<C, T, TIn, OUT>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, Cfg::NT, smem, st>>>(reinterpret_cast<const TIn *>(raw), corr, h.d_taps, h.d_twiddle, h.d_phase,
                                          bandpass, gains, N, S, h.I_pad, s_out, scale, rpc, flags, s_base, s_end);
        e = cudaGetLastError();
        if (e != cudaSuccess || OUT == 1) return e;
        return planar_pad(h, corr, OUT, rounds_total * kRound, s_out, st);
    }
}

template <int C, int T, typename TIn>
cudaError_t launch_out(const Handle &h, const void *raw, void *corr, const float *bp, const float2 *g, const float *fl,
                       const FWindow *w, cudaStream_t st)
{
    switch (h.p.precision) {
    case FX_F32: return launch_t<C, T, TIn, 1>(h, raw, corr, bp, g, fl, w, st);
    case FX_F16: return launch_t<C, T, TIn, 2>(h, raw, corr, bp, g, fl, w, st);
    case FX_BF16: return launch_t<C, T, TIn, 3>(h, raw, corr, bp, g, fl, w, st);
    case FX_TF32_SPLIT: return launch_t<C, T, TIn, 5>(h, raw, corr, bp, g, fl, w, st);
    default: return launch_t<C, T, TIn, 4>(h, raw, corr, bp, g, fl, w, st);
    }
}

template <int C, typename TIn>
cudaError_t launch_taps(const Handle &h, const void *raw, void *corr, const float *bp, const float2 *g,
                        const float *fl, const FWindow *w, cudaStream_t st)
{
    switch (h.p.n_taps) {
    case 4: return launch_out<C, 4, TIn>(h, raw, corr, bp, g, fl, w, st);
    case 8: return launch_out<C, 8, TIn>(h, raw, corr, bp, g, fl, w, st);
    case 16: return launch_out<C, 16, TIn>(h, raw, corr, bp, g, fl, w, st);
    default: return cudaErrorInvalidValue;
    }
}

template <typename TIn>
cudaError_t launch_fmt(const Handle &h, const void *raw, void *corr, const float *bp, const float2 *g, const float *fl,
                       const FWindow *w, cudaStream_t st)
{
    switch (h.p.n_channels) {
    case 16: return launch_taps<16, TIn>(h, raw, corr, bp, g, fl, w, st);
    case 64: return launch_taps<64, TIn>(h, raw, corr, bp, g, fl, w, st);
    case 256: return launch_taps<256, TIn>(h, raw, corr, bp, g, fl, w, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace fxi
