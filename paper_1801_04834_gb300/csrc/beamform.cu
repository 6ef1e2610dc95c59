// beamform.cu -- coherent beamformer on the tcgen05 tensor cores.
//
// Paper, Sec. "Signal processing with GPU kernels": after delay compensation
// and bandpass correction (done at 256 channels per subband), coherent
// beamforming steers each beam with a phase shift and sums over antenna
// fields, then optionally forms Stokes parameters; without them the complex
// voltages are kept. Per (subband, channel k) and pol this is a complex
// matrix product over stations n:
//   B[s][b] = sum_n Y[s][n] W[b][n],   W[b][n] = a_n exp(+2 pi i f_k delta[b][n])
// done as real GEMMs on planar operands (re plane r, im plane j):
//   Re B = Yr Wr^T - Yj Wj^T          Im B = Yr Wj^T + Yj Wr^T
// The weight table holds three 64-beam planes per quarter, [Wj; Wr; -Wj], so
// that [Wr; -Wj] and [Wj; Wr] are contiguous 128-row B tiles: per pol two
// MMAs of N = 128 give Re B in columns 0-63 and -Im B in columns 64-127,
//   D = Yr [Wr; -Wj]^T - Yj [Wj; Wr]^T     (the minus by the negate-A bit),
// which reads each data tile once per K-step instead of twice.
//
// Operands. A = data: M = 128 spectra x K = 64 stations of one (pol, plane),
// read from the planar FP16/BF16 block the fused F-stage writes for the
// X-stage ([SB][C][re/im][I_pad][S_pad], input i = 2n + p, spectra
// contiguous). A 4-D TMA box {64 spectra, 1 pol, 64 stations} picks one pol
// out of the interleaved inputs; two boxes give the 128 spectra. Spectra are
// contiguous, so A is MN-major (128-byte swizzle: 8 station rows of 64
// spectra per 1024-byte atom, the two 64-spectrum halves 8 KB apart).
// B = weights: N = 128 rows (two 64-beam planes) x K = 64 stations, K-major,
// from a table the weight kernel writes each call ([SB][C][3][NB_pad][64]:
// im, re, -im); its phase per
// (subband, beam, station) is formed in FP64 at the channel-0 frequency and
// per-channel step, reduced mod 2 pi, then stepped over channels in FP32 (as
// the paper does for delay compensation).
//
// Work item = (subband, channel, 128-spectrum tile); each CTA takes whole
// channels. A channel's weights (16 KB per quarter of 64 beams) are loaded
// once and stay resident while its spectrum tiles stream through (two
// channel slots when there are at most 128 beams, so the next channel's
// weights load meanwhile). The CTA loads the four data planes of an item once
// (64 KB, ring of 2) and walks the beams in quarters of 64: 16 MMAs
// (4 K-steps x 2 pols x 2, M = 128, N = 128, K = 16) into (Re X, -Im X),
// (Re Y, -Im Y) (2 x 128 TMEM columns, double buffered: all 512 columns).
// Warp roles (persistent, one CTA per SM): warp 0 TMA producer, warp 1 TMEM
// allocator + MMA issuer, warps 2-9 epilogue (TMEM lane = spectrum; two warps
// per lane quadrant, 32 beams each): complex voltages, or Stokes I / IQUV
// summed over tint consecutive spectra by recursive halving across lanes. Every mbarrier wait is bounded; on expiry the role is recorded in
// the status word, all roles leave, in-flight copies and MMAs are drained
// (bounded) and TMEM is freed, as in the X-stage.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "internal.h"
#include "tc_ptx.cuh"

namespace fxi {
namespace {

using namespace tc;

constexpr int kBfThreads = 320;                      // TMA, MMA, 8 epilogue warps
constexpr int kDS = 2;                               // data stages
constexpr int kWS = 2;                               // weight slots (barrier pairs)
constexpr unsigned kHalfBytes = 64u * 128u;          // 64 stations x 64 spectra x 2 B
constexpr unsigned kPlaneBytes = 2u * kHalfBytes;    // 128 spectra of one (pol, plane)
constexpr unsigned kDataBytes = 4u * kPlaneBytes;    // (pol, plane) = 4 planes: 64 KB
constexpr unsigned kWPlane = 64u * 128u;             // 64 beams x 64 stations x 2 B
constexpr unsigned kWBytes = 3u * kWPlane;           // im, re, -im: 24 KB per beam quarter
constexpr unsigned kWRegion = 4u * kWBytes;          // up to 256 beams of one channel, or 2 x 128
constexpr int kAccCols = 256;                        // Re X, Im X, Re Y, Im Y x 64 beams
constexpr int kTmemCols = 512;
constexpr int kNumBars = 2 * kDS + 2 * kWS + 5;      // dfull, dempty, wfull, wempty, accf 2, acce 2, drain

struct BfParams {
    CUtensorMap mapY;        // 4-D (spectrum, pol, station, sb*C*2 + plane)
    CUtensorMap mapW;        // 3-D (station, beam, sb*C*3 + plane)
    float *out;
    int *status;
    long long n_ch;          // SB * C
    int ntile;               // 128-spectrum tiles per channel
    int C, S, NB, NBQ;       // channels, spectra, beams, beam quarters
    unsigned bf16;
    float inv_scale, inv_scale2;
    long long timeout_cycles;
    int no_tma;              // failure-detection test hook: issue no loads
};

// Bounded wait: false on timeout (sets abort + status) or when another role aborted.
__device__ __forceinline__ bool bwait(unsigned bar, unsigned parity, volatile int *abort_flag, const BfParams &P,
                                      int code)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > P.timeout_cycles) {
            *abort_flag = 1;
            atomicCAS(P.status, 0, code);
            atomicExch(P.status + 1, (int)blockIdx.x);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ unsigned short weight_bits(float x, unsigned bf16)
{
    return bf16 ? __bfloat16_as_ushort(__float2bfloat16_rn(x)) : __half_as_ushort(__float2half_rn(x));
}

// Weight table W[sb][k][3][NB_pad][64], planes (im, re, -im): one thread per
// (subband, beam, station slot), looping over channels. Padding is zero.
__global__ void bf_weight_kernel(const double *__restrict__ delays, const float *__restrict__ weights,
                                 const double *__restrict__ centres, unsigned short *__restrict__ W, int SB, int C,
                                 int N, int NB, int NB_pad, double fs, unsigned bf16)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)SB * NB_pad * 64) return;
    const int n = (int)(idx % 64);
    const int b = (int)((idx / 64) % NB_pad);
    const int sb = (int)(idx / (64LL * NB_pad));
    const long long plane = (long long)NB_pad * 64;
    unsigned short *w = W + (long long)sb * C * 3 * plane + (long long)b * 64 + n;
    if (b >= NB || n >= N) {
        for (int k = 0; k < C; ++k) {
            w[(3LL * k) * plane] = 0;
            w[(3LL * k + 1) * plane] = 0;
            w[(3LL * k + 2) * plane] = 0;
        }
        return;
    }
    const double two_pi = 6.283185307179586476925286766559;
    const double d = delays[(long long)b * N + n];
    // phase at channel 0 (frequency centre - fs/2) and step per channel (fs / C), mod 2 pi
    double p0 = two_pi * (centres[sb] - 0.5 * fs) * d;
    p0 -= two_pi * rint(p0 / two_pi);
    double dp = two_pi * (fs / C) * d;
    dp -= two_pi * rint(dp / two_pi);
    const float a = weights ? weights[n] : 1.f;
    const float p0f = (float)p0, dpf = (float)dp;
    for (int k = 0; k < C; ++k) {
        const float phi = fmaf((float)k, dpf, p0f);
        const float kq = rintf(phi * 0.15915494309189535f);           // phi / (2 pi)
        float r = fmaf(-kq, 6.28125f, phi);                           // 2 pi = 6.28125 + 1.9353...e-3
        r = fmaf(-kq, 1.9353071795864769e-3f, r);
        float sn, cs;
        __sincosf(r, &sn, &cs);
        w[(3LL * k) * plane] = weight_bits(a * sn, bf16);
        w[(3LL * k + 1) * plane] = weight_bits(a * cs, bf16);
        w[(3LL * k + 2) * plane] = weight_bits(-(a * sn), bf16);
    }
}

// Sum v[0..M) over aligned groups of T lanes by recursive halving: at each
// step a lane keeps half of its values (the upper half when the step's lane
// bit is set) and adds its partner's copy of that half, so after the steps
// over lane bits 1, 2, 4, ... (up to 8) lane l holds 16 / min(T, 16) sums, of
// beams i + 8 b0 + 4 b1 + 2 b2 + b3 (b_k = bit k of l); a group of 32 adds a
// final plain exchange across the half-warps.
template <int M, int O, int T>
__device__ __forceinline__ void halve(float (&v)[16], int lane)
{
    if constexpr (O < T && M > 1) {
        const bool upper = (lane & O) != 0;
#pragma unroll
        for (int i = 0; i < M / 2; ++i) {
            const float send = upper ? v[i] : v[i + M / 2];
            const float keep = upper ? v[i + M / 2] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
        }
        halve<M / 2, O * 2, T>(v, lane);
    } else if constexpr (O < T) {
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], O);
        halve<1, O * 2, T>(v, lane);
    }
}

// MODE 0 voltages, 1 Stokes I, 2 Stokes IQUV; TINT spectra summed per output
template <int MODE, int TINT>
__global__ void __launch_bounds__(kBfThreads, 1) beamform_kernel(const __grid_constant__ BfParams P)
{
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment for the 128-byte-swizzled tiles
    const unsigned base_u32 = smem_u32(smem_raw);
    const unsigned pad = (1024 - (base_u32 & 1023)) & 1023;
    const unsigned data_u32 = base_u32 + pad;
    const unsigned w_u32 = data_u32 + kDS * kDataBytes;
    unsigned char *ctrl = smem_raw + pad + kDS * kDataBytes + kWRegion;
    const unsigned bar0 = smem_u32(ctrl);
    auto dfull = [&](int s) { return bar0 + 8u * s; };
    auto dempty = [&](int s) { return bar0 + 8u * (kDS + s); };
    auto wfull = [&](int s) { return bar0 + 8u * (2 * kDS + s); };
    auto wempty = [&](int s) { return bar0 + 8u * (2 * kDS + kWS + s); };
    auto accf = [&](int b) { return bar0 + 8u * (2 * kDS + 2 * kWS + b); };
    auto acce = [&](int b) { return bar0 + 8u * (2 * kDS + 2 * kWS + 2 + b); };
    const unsigned drain_bar = bar0 + 8u * (kNumBars - 1);
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(ctrl + 8 * kNumBars);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kDS; ++s) {
            mbar_init(dfull(s), 1);
            mbar_init(dempty(s), 1);
        }
        for (int s = 0; s < kWS; ++s) {
            mbar_init(wfull(s), 1);
            mbar_init(wempty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf(b), 1);
            mbar_init(acce(b), 8);
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const unsigned tmem_base = *tmem_slot;

    // weight slots: one channel's NBQ quarters each; two slots (next channel's
    // weights load while this channel computes) when NBQ <= 2
    const int nslots = P.NBQ <= 2 ? 2 : 1;
    const unsigned slot_bytes = P.NBQ <= 2 ? 2u * kWBytes : 4u * kWBytes;

    if (warp == 0) {
        // ================= TMA producer =================
        if (lane == 0) {
            long long d_issued = 0, w_issued = 0;
            bool ok = true;
            for (long long gch = blockIdx.x; gch < P.n_ch && ok; gch += gridDim.x) {
                const int sl = (int)(w_issued % nslots);
                if (!bwait(wempty(sl), (unsigned)((w_issued / nslots) & 1) ^ 1u, abort_flag, P, 1)) {
                    ok = false;
                    break;
                }
                if (P.no_tma) {
                    ++w_issued;
                    continue;
                }
                mbar_arrive_expect_tx(wfull(sl), (unsigned)P.NBQ * kWBytes);
                for (int q = 0; q < P.NBQ; ++q)
                    for (int pl = 0; pl < 3; ++pl)
                        tma_load_3d(w_u32 + (unsigned)sl * slot_bytes + (unsigned)q * kWBytes + (unsigned)pl * kWPlane,
                                    &P.mapW, wfull(sl), 0, q * 64, (int)(gch * 3 + pl));
                ++w_issued;
                for (int st = 0; st < P.ntile; ++st) {
                    const int ds = (int)(d_issued % kDS);
                    if (!bwait(dempty(ds), (unsigned)((d_issued / kDS) & 1) ^ 1u, abort_flag, P, 1)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(dfull(ds), kDataBytes);
                    const unsigned dst = data_u32 + (unsigned)ds * kDataBytes;
                    for (int p = 0; p < 2; ++p)
                        for (int pl = 0; pl < 2; ++pl)
                            for (int hh = 0; hh < 2; ++hh)
                                tma_load_4d(dst + (unsigned)(p * 2 + pl) * kPlaneBytes + (unsigned)hh * kHalfBytes,
                                            &P.mapY, dfull(ds), st * 128 + hh * 64, p, 0, (int)(gch * 2 + pl));
                    ++d_issued;
                }
            }
            if (!ok && !P.no_tma) {
                // the last loads issued into each ring may still be in flight
                for (long long u = d_issued > kDS ? d_issued - kDS : 0; u < d_issued; ++u)
                    drain_wait(dfull((int)(u % kDS)), (unsigned)((u / kDS) & 1), P.timeout_cycles);
                for (long long u = w_issued > nslots ? w_issued - nslots : 0; u < w_issued; ++u)
                    drain_wait(wfull((int)(u % nslots)), (unsigned)((u / nslots) & 1), P.timeout_cycles);
            }
        }
    } else if (warp == 1) {
        // ================= MMA issuer =================
        if (lane == 0) {
            long long dit = 0, wit = 0, ait = 0;
            bool ok = true, issued = false;
            const unsigned idesc = make_idesc_major(P.bf16, 128, false, true, false);
            const unsigned idesc_neg = make_idesc_major(P.bf16, 128, true, true, false);
            for (long long gch = blockIdx.x; gch < P.n_ch && ok; gch += gridDim.x, ++wit) {
                const int sl = (int)(wit % nslots);
                if (!bwait(wfull(sl), (unsigned)((wit / nslots) & 1), abort_flag, P, 2)) {
                    ok = false;
                    break;
                }
                for (int st = 0; st < P.ntile && ok; ++st, ++dit) {
                    const int ds = (int)(dit % kDS);
                    if (!bwait(dfull(ds), (unsigned)((dit / kDS) & 1), abort_flag, P, 2)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned dtile = data_u32 + (unsigned)ds * kDataBytes;
                    for (int q = 0; q < P.NBQ; ++q, ++ait) {
                        const int ab = (int)(ait & 1);
                        if (!bwait(acce(ab), (unsigned)((ait >> 1) & 1) ^ 1u, abort_flag, P, 2)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const unsigned wt = w_u32 + (unsigned)sl * slot_bytes + (unsigned)q * kWBytes;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {      // 16 stations per K-step
                            const unsigned acc = kk ? 1u : 0u;
                            const unsigned long long b_jr = smem_desc(wt + kk * 32);             // [Wj; Wr]
                            const unsigned long long b_rn = smem_desc(wt + kWPlane + kk * 32);   // [Wr; -Wj]
#pragma unroll
                            for (int p = 0; p < 2; ++p) {
                                const unsigned at = dtile + (unsigned)(p * 2) * kPlaneBytes + (unsigned)kk * 2048u;
                                const unsigned long long ayr = smem_desc_mn(at, kHalfBytes, 1024);
                                const unsigned long long ayj = smem_desc_mn(at + kPlaneBytes, kHalfBytes, 1024);
                                const unsigned d = tmem_base + (unsigned)(ab * kAccCols + p * 128);   // (Re, -Im)
                                mma_f16(d, ayr, b_rn, idesc, acc);
                                mma_f16(d, ayj, b_jr, idesc_neg, 1u);
                            }
                        }
                        issued = true;
                        mma_commit(accf(ab));                 // accumulators ready for the epilogue
                    }
                    if (!ok) break;
                    mma_commit(dempty(ds));                   // data stage free after the last quarter
                }
                if (!ok) break;
                mma_commit(wempty(sl));                       // weight slot free after the channel
            }
            if (!ok && issued) {
                mma_commit(drain_bar);
                drain_wait(drain_bar, 0, P.timeout_cycles);
            }
        }
        __syncwarp();
    } else {
        // ================= epilogue (warps 2..9) =================
        const int qd = warp & 3;                              // TMEM lane quadrant of this warp
        const int hf = (warp - 2) >> 2;                       // which 32 of the quarter's 64 beams
        const unsigned lane_off = (unsigned)(32 * qd) << 16;
        long long ait = 0;
        bool live = true;
        for (long long gch = blockIdx.x; gch < P.n_ch && live; gch += gridDim.x)
          for (int st = 0; st < P.ntile && live; ++st) {
            const long long sb = gch / P.C;
            const int c = (int)(gch % P.C);
            const int s = st * 128 + 32 * qd + lane;          // this lane's spectrum
            for (int q = 0; q < P.NBQ; ++q, ++ait) {
                const int ab = (int)(ait & 1);
                const bool got = bwait(accf(ab), (unsigned)((ait >> 1) & 1), abort_flag, P, 3);
                if (!__all_sync(0xffffffffu, got)) {
                    live = false;
                    break;
                }
                tc_fence_after();
                const unsigned t0 = tmem_base + lane_off + (unsigned)(ab * kAccCols);
#pragma unroll 1
                for (int cc = 2 * hf; cc < 2 * hf + 2; ++cc) {
                    const int b0 = q * 64 + cc * 16;
                    if (b0 >= P.NB) break;
                    float xr[16], xj[16], yr[16], yj[16];
                    tmem_ld16(t0 + 16 * cc, xr);
                    tmem_ld16(t0 + 64 + 16 * cc, xj);
                    tmem_ld16(t0 + 128 + 16 * cc, yr);
                    tmem_ld16(t0 + 192 + 16 * cc, yj);
                    tmem_ld_wait();
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {            // columns 64-127 of a pol hold -Im
                        xj[jj] = -xj[jj];
                        yj[jj] = -yj[jj];
                    }
                    if constexpr (MODE == 0) {
                        if (s < P.S) {
                            const float is = P.inv_scale;
#pragma unroll
                            for (int jj = 0; jj < 16; ++jj) {
                                const int b = b0 + jj;
                                if (b < P.NB)
                                    *reinterpret_cast<float4 *>(P.out + (((sb * P.NB + b) * P.C + c) * P.S + s) * 4) =
                                        make_float4(xr[jj] * is, xj[jj] * is, yr[jj] * is, yj[jj] * is);
                            }
                        }
                    } else {
                        // Stokes of this lane's spectrum for 16 beams (padded spectra are zero)
                        float sI[16], sQ[16], sU[16], sV[16];
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj) {
                            const float xx = fmaf(xr[jj], xr[jj], xj[jj] * xj[jj]);
                            const float yy = fmaf(yr[jj], yr[jj], yj[jj] * yj[jj]);
                            sI[jj] = xx + yy;
                            if constexpr (MODE == 2) {
                                sQ[jj] = xx - yy;
                                sU[jj] = 2.f * fmaf(xr[jj], yr[jj], xj[jj] * yj[jj]);    // 2 Re(X conj Y)
                                sV[jj] = 2.f * fmaf(xj[jj], yr[jj], -xr[jj] * yj[jj]);   // 2 Im(X conj Y)
                            }
                        }
                        // sum over the TINT spectra of each lane group; lane then holds kM beams
                        halve<16, 1, TINT>(sI, lane);
                        if constexpr (MODE == 2) {
                            halve<16, 1, TINT>(sQ, lane);
                            halve<16, 1, TINT>(sU, lane);
                            halve<16, 1, TINT>(sV, lane);
                        }
                        constexpr int kG = TINT < 16 ? TINT : 16;       // lanes sharing one set of beams
                        constexpr int kM = 16 / kG;                     // beams held per lane
                        int boff = 0;                                   // first beam of this lane's share
#pragma unroll
                        for (int k = 0; (1 << k) < kG; ++k) boff += ((lane >> k) & 1) * (8 >> k);
                        const int sg = s - lane % TINT;                 // first spectrum of the lane group
                        const bool writer = sg < P.S && (TINT < 32 || lane < 16);
                        const long long so = sg / TINT;
                        const float is2 = P.inv_scale2;
#pragma unroll
                        for (int i = 0; i < kM; ++i) {
                            const int b = b0 + boff + i;
                            if (!writer || b >= P.NB) continue;
                            const long long o = ((sb * P.NB + b) * P.C + c) * (P.S / TINT) + so;
                            if constexpr (MODE == 1)
                                P.out[o] = sI[i] * is2;
                            else
                                *reinterpret_cast<float4 *>(P.out + o * 4) =
                                    make_float4(sI[i] * is2, sQ[i] * is2, sU[i] * is2, sV[i] * is2);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce(ab));
            }
        }
    }

    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                     : "memory");
    }
}

// ---- incoherent beam ---------------------------------------------------------
// Sec. "Signal processing with GPU kernels": incoherent beamforming first forms
// Stokes parameters per antenna field and then sums over fields. Per
// (subband, channel) and spectrum s: sum_n a_n Stokes(X_n(s), Y_n(s)), summed
// over tint consecutive spectra. No contraction, so CUDA cores: one thread per
// spectrum (lanes = consecutive spectra, so each station's planes are read in
// coalesced runs), stations accumulated in registers, tint lanes summed with
// shuffles. SRC: 0 FP32 spectrum-blocked [SB][C][ceil16(S)/16][N][16][2]
// (16 lanes read one station's 256-byte run), 1 FP16 planar, 2 BF16 planar,
// 3 FP32 planar ([SB][C][2][I_pad][S_pad]).
template <int MODE, int SRC>
__global__ void __launch_bounds__(128) incoherent_kernel(const void *__restrict__ corr, const float *__restrict__ weights,
                                                         float *__restrict__ out, int N, int S, int I_pad, int S_pad,
                                                         int tint, float inv_scale2, int sblocks)
{
    const long long gch = blockIdx.x / sblocks;
    const int s = (int)(blockIdx.x % sblocks) * 128 + threadIdx.x;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const bool in = SRC == 0 ? s < S : s < S_pad;
    if (in) {
        for (int n = 0; n < N; ++n) {
            const float a = weights ? __ldg(weights + n) : 1.f;
            float xr, xj, yr, yj;
            if constexpr (SRC == 0) {
                const long long NB = (S + 15) / 16;
                const float4 v = *reinterpret_cast<const float4 *>(
                    reinterpret_cast<const float2 *>(corr) + (((gch * NB + s / 16) * N + n) * 16 + s % 16) * 2);
                xr = v.x; xj = v.y; yr = v.z; yj = v.w;
            } else if constexpr (SRC == 3) {
                const float *re = reinterpret_cast<const float *>(corr) + gch * 2 * (long long)I_pad * S_pad;
                const float *im = re + (long long)I_pad * S_pad;
                xr = re[(long long)(2 * n) * S_pad + s];
                xj = im[(long long)(2 * n) * S_pad + s];
                yr = re[(long long)(2 * n + 1) * S_pad + s];
                yj = im[(long long)(2 * n + 1) * S_pad + s];
            } else {
                const unsigned short *re =
                    reinterpret_cast<const unsigned short *>(corr) + gch * 2 * (long long)I_pad * S_pad;
                const unsigned short *im = re + (long long)I_pad * S_pad;
                auto f = [](unsigned short b) {
                    return SRC == 2 ? __bfloat162float(__ushort_as_bfloat16(b)) : __half2float(__ushort_as_half(b));
                };
                xr = f(re[(long long)(2 * n) * S_pad + s]);
                xj = f(im[(long long)(2 * n) * S_pad + s]);
                yr = f(re[(long long)(2 * n + 1) * S_pad + s]);
                yj = f(im[(long long)(2 * n + 1) * S_pad + s]);
            }
            const float xx = fmaf(xr, xr, xj * xj), yy = fmaf(yr, yr, yj * yj);
            acc[0] = fmaf(a, xx + yy, acc[0]);
            if constexpr (MODE == 2) {
                acc[1] = fmaf(a, xx - yy, acc[1]);
                acc[2] = fmaf(a, 2.f * fmaf(xr, yr, xj * yj), acc[2]);     // 2 Re(X conj Y)
                acc[3] = fmaf(a, 2.f * fmaf(xj, yr, -xr * yj), acc[3]);    // 2 Im(X conj Y)
            }
        }
    }
    constexpr int NQ = MODE == 1 ? 1 : 4;
    for (int off = 1; off < tint; off <<= 1)
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
    if (s < S && (threadIdx.x % tint) == 0) {
        const long long o = gch * (S / tint) + s / tint;
        if constexpr (MODE == 1)
            out[o] = acc[0] * inv_scale2;
        else
            *reinterpret_cast<float4 *>(out + o * 4) =
                make_float4(acc[0] * inv_scale2, acc[1] * inv_scale2, acc[2] * inv_scale2, acc[3] * inv_scale2);
    }
}

// ---- host side ----------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn bf_encode_fn()
{
    static EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<EncodeTiledFn>(p);
        return static_cast<EncodeTiledFn>(nullptr);
    }();
    return fn;
}

constexpr size_t bf_smem_bytes() { return 1024 + (size_t)kDS * kDataBytes + (size_t)kWRegion + 8 * kNumBars + 16; }
static_assert(bf_smem_bytes() <= 227 * 1024, "beamformer stages exceed the shared memory of one CTA");

template <int MODE, int TINT>
cudaError_t bf_launch(const BfParams &P, unsigned grid, cudaStream_t st)
{
    constexpr size_t smem = bf_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(beamform_kernel<MODE, TINT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    beamform_kernel<MODE, TINT><<<grid, kBfThreads, smem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_beamform_incoherent(const Handle &h, const void *corr, const float *weights, int mode, int tint,
                                       float *out, cudaStream_t st)
{
    const int SB = h.p.n_subbands, C = h.p.n_channels, N = h.p.n_stations, S = h.p.n_spectra;
    const long long n_ch = (long long)SB * C;
    const int sblocks = ((h.p.precision == FX_F32 ? S : h.S_pad) + 127) / 128;
    const long long blocks = n_ch * sblocks;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const float is2 = 1.0f / (h.operand_scale * h.operand_scale);
    auto go = [&](auto kern) {
        kern<<<(unsigned)blocks, 128, 0, st>>>(corr, weights, out, N, S, h.I_pad, h.S_pad, tint, is2, sblocks);
        return cudaGetLastError();
    };
    switch (h.p.precision * 4 + mode) {
    case FX_F32 * 4 + 1: return go(incoherent_kernel<1, 0>);
    case FX_F32 * 4 + 2: return go(incoherent_kernel<2, 0>);
    case FX_F16 * 4 + 1: return go(incoherent_kernel<1, 1>);
    case FX_F16 * 4 + 2: return go(incoherent_kernel<2, 1>);
    case FX_BF16 * 4 + 1: return go(incoherent_kernel<1, 2>);
    case FX_BF16 * 4 + 2: return go(incoherent_kernel<2, 2>);
    case FX_TF32_SPLIT * 4 + 1: return go(incoherent_kernel<1, 3>);
    case FX_TF32_SPLIT * 4 + 2: return go(incoherent_kernel<2, 3>);
    default: return cudaErrorNotSupported;
    }
}

size_t bf_weight_bytes(const Handle &h, int n_beams)
{
    const size_t nb_pad = (size_t)(n_beams + 63) / 64 * 64;
    return (size_t)h.p.n_subbands * h.p.n_channels * 3 * nb_pad * 64 * sizeof(unsigned short);
}

cudaError_t launch_beamform(const Handle &h, const void *corr, int NB, const double *delays, const float *weights,
                            int mode, int tint, float *out, cudaStream_t st)
{
    EncodeTiledFn enc = bf_encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int SB = h.p.n_subbands, C = h.p.n_channels, N = h.p.n_stations, S = h.p.n_spectra;
    const int NB_pad = (NB + 63) / 64 * 64;
    const unsigned bf16 = h.p.precision == FX_BF16 ? 1u : 0u;
    const long long planes = (long long)SB * C * 2;
    if (planes / 2 * 3 > 0x7fffffffLL) return cudaErrorInvalidValue;

    // weight table for this call
    const long long wthreads = (long long)SB * NB_pad * 64;
    bf_weight_kernel<<<(unsigned)((wthreads + 255) / 256), 256, 0, st>>>(
        delays, weights, h.d_centres, h.d_bfw, SB, C, N, NB, NB_pad, h.p.sample_rate_hz, bf16);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    BfParams P;
    memset(&P, 0, sizeof(P));
    // data: (spectrum, pol, station, plane row) over [SB][C][2][I_pad][S_pad], input i = 2n + p
    {
        const cuuint64_t gdim[4] = {(cuuint64_t)h.S_pad, 2, (cuuint64_t)(h.I_pad / 2), (cuuint64_t)planes};
        const cuuint64_t gstride[3] = {(cuuint64_t)h.S_pad * 2, (cuuint64_t)h.S_pad * 4,
                                       (cuuint64_t)h.S_pad * 2 * h.I_pad};
        const cuuint32_t box[4] = {64, 1, 64, 1};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        if (enc(&P.mapY, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<void *>(corr), gdim, gstride, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    // weights: (station, beam, plane row) over [SB][C][3][NB_pad][64]
    {
        const cuuint64_t gdim[3] = {64, (cuuint64_t)NB_pad, (cuuint64_t)(planes / 2 * 3)};
        const cuuint64_t gstride[2] = {64 * 2, (cuuint64_t)NB_pad * 64 * 2};
        const cuuint32_t box[3] = {64, 64, 1};
        const cuuint32_t estr[3] = {1, 1, 1};
        if (enc(&P.mapW, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, h.d_bfw, gdim, gstride, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    P.out = out;
    P.status = h.d_status;
    P.ntile = (S + 127) / 128;
    P.n_ch = planes / 2;
    P.C = C;
    P.S = S;
    P.NB = NB;
    P.NBQ = NB_pad / 64;
    P.bf16 = bf16;
    P.inv_scale = 1.0f / h.operand_scale;
    P.inv_scale2 = 1.0f / (h.operand_scale * h.operand_scale);
    P.timeout_cycles = h.tc_timeout_cycles;
    P.no_tma = h.tc_test_no_tma;
    const long long grid = std::min<long long>(P.n_ch, h.num_sms);
    if (grid <= 0) return cudaSuccess;
    switch (mode * 64 + tint) {
    case 0 * 64 + 1: return bf_launch<0, 1>(P, (unsigned)grid, st);
    case 1 * 64 + 1: return bf_launch<1, 1>(P, (unsigned)grid, st);
    case 1 * 64 + 2: return bf_launch<1, 2>(P, (unsigned)grid, st);
    case 1 * 64 + 4: return bf_launch<1, 4>(P, (unsigned)grid, st);
    case 1 * 64 + 8: return bf_launch<1, 8>(P, (unsigned)grid, st);
    case 1 * 64 + 16: return bf_launch<1, 16>(P, (unsigned)grid, st);
    case 1 * 64 + 32: return bf_launch<1, 32>(P, (unsigned)grid, st);
    case 2 * 64 + 1: return bf_launch<2, 1>(P, (unsigned)grid, st);
    case 2 * 64 + 2: return bf_launch<2, 2>(P, (unsigned)grid, st);
    case 2 * 64 + 4: return bf_launch<2, 4>(P, (unsigned)grid, st);
    case 2 * 64 + 8: return bf_launch<2, 8>(P, (unsigned)grid, st);
    case 2 * 64 + 16: return bf_launch<2, 16>(P, (unsigned)grid, st);
    case 2 * 64 + 32: return bf_launch<2, 32>(P, (unsigned)grid, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fxi
