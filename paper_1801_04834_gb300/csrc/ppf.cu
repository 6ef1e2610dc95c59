// ppf.cu -- polyphase filter bank: int16/int8 -> FP32 conversion, T-tap FIR
// per channel and C-point FFT, per (subband, station, polarisation).
//
// Paper: Sec. "Signal processing with GPU kernels" (FIR and FFT kernels
// channelise each subband, FIR history is carried across blocks) and
// Sec. "Processing steps" (fixed-point input converted to floating point).
// The paper's FFT was a cuFFT call; here the FFT is fused behind the FIR.
//
// Work decomposition of ppf_kernel (C = 256; C = 16 and 64 use the
// warp-specialised ppf_ws_kernel below, same FIR and FFT, overlapped): one CTA
// = NPC stations x 2 pols x all C channels x a run of spectra:
//   * Raw samples stream through shared memory 16 time rows (one row = C
//     samples) at a time with cp.async, double buffered.
//   * FIR: thread (station, channel c, pol p) keeps the last T samples of its
//     channel in registers as a circular buffer and its T taps in registers;
//     each new row costs one 4-byte (int16) or 2-byte (int8) shared load and
//     2T FMAs. Rounds are 16 spectra long, a multiple of T, so the circular
//     indices are compile-time constants.
//   * FFT: C = R*R. Pass 1: R threads per transform, each an R-point FFT over
//     stride-R samples in registers, times the inter-pass twiddle (host-FP64
//     table); pass 2: R threads per transform, R-point FFTs along the other
//     index. Shared memory holds the 16-spectrum batch between passes, one
//     row per transform in spectrum-major order (row j * IC + input), which
//     keeps the FIR stores and both passes free of bank conflicts.
//   * Output channel k = (m + C/2) mod C (ascending sky frequency).
#include "internal.h"
#include "fft_reg.cuh"
#include "ppf_common.cuh"

namespace fxi {
namespace {

using namespace ppf;

// A separate FFT pass-1 output buffer saves one barrier per round where it
// still leaves room for the same number of CTAs per SM (two below 512 threads).
template <int C, typename TIn>
constexpr bool ppf_split_u()
{
    using Cfg = PpfCfg<C>;
    constexpr size_t b = ppf_smem_bytes<C, TIn>() + (size_t)Cfg::NTR * Cfg::ROW * sizeof(float2);
    return Cfg::NT >= 512 ? b <= 227 * 1024 : 2 * (b + 1024) <= 228 * 1024;
}

template <int C, int T, typename TIn>
__global__ void __launch_bounds__(PpfCfg<C>::NT)
ppf_kernel(const TIn *__restrict__ raw, float2 *__restrict__ chan, const float *__restrict__ taps,
           const float2 *__restrict__ twiddle, int N, int S, int rounds_per_cta)
{
    using Cfg = PpfCfg<C>;
    constexpr int R = Cfg::R, NPC = Cfg::NPC, NT = Cfg::NT, ROW = Cfg::ROW;
    constexpr int ROW_BYTES = C * kPols * (int)sizeof(TIn);     // one time row of one station
    constexpr int BUF_BYTES = kRound * NPC * ROW_BYTES;
    constexpr int IC = NPC * kPols;                                // inputs of this CTA
    static_assert(ROW_BYTES % 16 == 0, "rows must be whole 16-byte chunks");
    constexpr bool kSplitU = ppf_split_u<C, TIn>();

    extern __shared__ __align__(16) unsigned char smem[];
    float2 *tw = reinterpret_cast<float2 *>(smem);
    unsigned char *inbuf = smem + C * sizeof(float2);
    float2 *u = reinterpret_cast<float2 *>(inbuf + 2 * BUF_BYTES);
    float2 *u2 = kSplitU ? u + Cfg::NTR * ROW : u;                    // FFT pass-1 output

    const int tid = threadIdx.x;
    const int sb = blockIdx.z;
    const int n0 = blockIdx.y * NPC;
    const int s0 = blockIdx.x * rounds_per_cta * kRound;
    const int rows_total = S + T - 1;
    const long long L = (long long)rows_total * C;
    const int nrounds = min(rounds_per_cta, (S - s0 + kRound - 1) / kRound);

    // stage rows [r0, r0 + nrows) of the CTA's stations into buffer `buf`
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

    // FIR role of this thread
    const int p = tid % kPols;
    const int c = (tid / kPols) % C;
    const int nl = tid / (kPols * C);

    for (int i = tid; i < C; i += NT) tw[i] = twiddle[i];
    // taps duplicated into (h, h) pairs: one packed FMA filters re and im
    float2 h[T];
#pragma unroll
    for (int k = 0; k < T; ++k) h[k] = make_float2(taps[k * C + c], taps[k * C + c]);

    // warm-up rows (FIR history) into buffer 1, first round into buffer 0
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
            u[(j * IC + nl * kPols + p) * ROW + c] = acc;     // transform row j * IC + input
        }
        __syncthreads();
        if (b + 2 < nrounds) stage(b & 1, s0 + T - 1 + (b + 2) * kRound, kRound);
        cp_async_commit();

        // ---- FFT pass 1: R-point FFTs over n1 (stride R), times W_C^(n2 k1) ----
        // With a second buffer (u2) the outputs go there; in place, every
        // task's inputs are read before any output is written, because the
        // outputs go to other positions (row k1 of length R + 1)
        float2 v1[Cfg::FFT_ITERS][R];
#pragma unroll
        for (int it = 0; it < Cfg::FFT_ITERS; ++it) {
            const int task = it * NT + tid;
            const float2 *row = u + (task / R) * ROW;
#pragma unroll
            for (int n1 = 0; n1 < R; ++n1) v1[it][n1] = row[R * n1 + task % R];
        }
        if constexpr (!kSplitU) __syncthreads();
#pragma unroll
        for (int it = 0; it < Cfg::FFT_ITERS; ++it) {
            const int task = it * NT + tid;
            const int tr = task / R, n2 = task % R;
            float2 *row = u2 + tr * ROW;
            fft_reg<R>(v1[it]);
#pragma unroll
            for (int k1 = 1; k1 < R; ++k1) v1[it][k1] = cmul(v1[it][k1], tw[n2 * k1]);
#pragma unroll
            for (int k1 = 0; k1 < R; ++k1) row[(R + 1) * k1 + n2] = v1[it][k1];
        }
        __syncthreads();
        // ---- FFT pass 2: R-point FFTs over n2, X[k1 + R k2] ----
#pragma unroll
        for (int it = 0; it < Cfg::FFT_ITERS; ++it) {
            const int task = it * NT + tid;
            const int tr = task / R, k1 = task % R;
            const float2 *row = u2 + tr * ROW;
            float2 v[R];
#pragma unroll
            for (int n2 = 0; n2 < R; ++n2) v[n2] = row[(R + 1) * k1 + n2];
            fft_reg<R>(v);
            const int j = tr / IC, il = tr % IC;
            const int pp = il % kPols;
            const int n = n0 + il / kPols;
            const int s = s0 + b * kRound + j;
            if (s < S && n < N) {
                float2 *out = chan + ((((long long)blockIdx.z * N + n) * kPols + pp) * S + s) * C;
#pragma unroll
                for (int k2 = 0; k2 < R; ++k2) out[k1 + R * ((k2 + R / 2) % R)] = v[k2];
            }
        }
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Warp-specialised form (C = 16, 64): the FIR (CUDA-core FMA bound) and the
// FFT (shared-memory bound) of consecutive rounds overlap instead of
// alternating between CTA-wide barriers. A CTA holds NF FIR threads (NPC
// stations x 2 pols x C channels, the sliding-window FIR above) and NF FFT
// threads:
//   FIR round b -> transform rows u[b & 1]; bar.arrive FULL[b & 1]
//   FFT round b: bar.sync FULL[b & 1], both FFT passes in place in u[b & 1],
//                output; bar.arrive EMPTY[b & 1], which FIR round b + 2 waits for
// Each transform row is handled by R consecutive lanes of one FFT warp, so the
// in-place pass 1 (every lane reads its column of the row before any lane
// writes the row back transposed) and pass 2 need only __syncwarp. Raw rows
// are staged by the FIR threads alone (barrier RAW). Named barriers are
// hardware barriers with fixed arrival counts; every FIR thread and every FFT
// thread runs the same number of rounds, so each barrier instance completes.
// 128 FIR + 128 FFT threads at <= 85 registers and <= 56 KB of shared memory
// leave room for three CTAs per SM.
template <int C>
struct PpfWsCfg {
    static constexpr int R = PpfCfg<C>::R;
    static constexpr int NPC = 64 / C;                       // C = 64: 1 station, C = 16: 4
    static constexpr int NF = NPC * C * kPols;               // 128 FIR threads (and 128 FFT threads)
    static constexpr int NTR = NPC * kPols * kRound;         // transforms per round
    static constexpr int ROW = PpfCfg<C>::ROW;
    static constexpr int ITERS = NTR * R / NF;               // FFT tasks per FFT thread per round
    static_assert(C == 16 || C == 64, "warp-specialised PPF: C = 16 or 64");
    static_assert(NTR * R % NF == 0 && 32 % R == 0, "a transform row stays inside one warp");
};

template <int C, typename TIn>
constexpr size_t ppf_ws_smem_bytes()
{
    using W = PpfWsCfg<C>;
    return (size_t)C * sizeof(float2) + 2ull * kRound * W::NPC * C * kPols * sizeof(TIn) +
           2ull * W::NTR * W::ROW * sizeof(float2) + 16;   // + 2 raw-row mbarriers
}

template <int C, int T, typename TIn>
__global__ void __launch_bounds__(2 * PpfWsCfg<C>::NF, 3)
ppf_ws_kernel(const TIn *__restrict__ raw, float2 *__restrict__ chan, const float *__restrict__ taps,
              const float2 *__restrict__ twiddle, int N, int S, int rounds_per_cta, int *__restrict__ status,
              long long budget, int no_loads)
{
    using W = PpfWsCfg<C>;
    constexpr int R = W::R, NPC = W::NPC, NF = W::NF, ROW = W::ROW, NTR = W::NTR;
    constexpr int ROW_BYTES = C * kPols * (int)sizeof(TIn);
    constexpr int BUF_BYTES = kRound * NPC * ROW_BYTES;
    constexpr int IC = NPC * kPols;
    constexpr int ALL = 2 * NF;
    static_assert(ROW_BYTES % 16 == 0, "rows must be whole 16-byte chunks");
    static_assert(3 * (ppf_ws_smem_bytes<C, TIn>() + 1024) <= 228 * 1024, "three CTAs per SM");

    extern __shared__ __align__(16) unsigned char smem[];
    float2 *tw = reinterpret_cast<float2 *>(smem);
    unsigned char *inbuf = smem + C * sizeof(float2);
    float2 *u = reinterpret_cast<float2 *>(inbuf + 2 * BUF_BYTES);   // [2][NTR][ROW]
    const unsigned rbar = tc::smem_u32(u + 2 * NTR * ROW);            // raw-row mbarriers [2]

    const int tid = threadIdx.x;
    const int sb = blockIdx.z;
    const int n0 = blockIdx.y * NPC;
    const int s0 = blockIdx.x * rounds_per_cta * kRound;
    const int rows_total = S + T - 1;
    const long long L = (long long)rows_total * C;
    const int nrounds = min(rounds_per_cta, (S - s0 + kRound - 1) / kRound);

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
        // ---- FIR threads: thread = (station nl, channel c, pol p) ----
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
        float2 h[T];
#pragma unroll
        for (int k = 0; k < T; ++k) h[k] = make_float2(taps[k * C + c], taps[k * C + c]);

        if constexpr (NPC == 1) {
            issue(1, s0, T - 1);                        // FIR history: buffer 1, phase 0
            issue(0, s0 + T - 1, kRound);               // round 0: buffer 0, phase 0
            raw_wait(rbar + 8, 0, status, budget);
        } else {
            stage(1, s0, T - 1);                        // FIR history
            cp_async_commit();
            stage(0, s0 + T - 1, kRound);               // round 0
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
            if constexpr (NPC == 1) {
                raw_wait(rbar + 8u * q, (unsigned)(((b + q) / 2) & 1), status, budget);   // round b's rows
            } else {
                cp_async_wait<1>();
                named_bar_sync(kBarRaw, NF);              // raw rows of round b are in
            }
            if (b >= 2) named_bar_sync(kBarEmpty + q, ALL);   // the FFT threads are done with u[q]
            const TIn *in = reinterpret_cast<const TIn *>(inbuf + q * BUF_BYTES);
            float2 *uq = u + q * NTR * ROW;
#pragma unroll
            for (int j = 0; j < kRound; ++j) {
                win[(T - 1 + j) % T] = to_f2(in[j * NF + tid]);
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < T; ++k) acc = __ffma2_rn(h[k], win[(j + k) % T], acc);
                uq[(j * IC + nl * kPols + p) * ROW + c] = acc;     // transform row j * IC + input
            }
            named_bar_arrive(kBarFull + q, ALL);
            named_bar_sync(kBarRaw, NF);                  // every FIR thread has read raw buffer q
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
        // ---- FFT threads: task = (transform row, column); R lanes of one warp per row ----
        const int t = tid - NF;
        float2 twr[R];                              // W_C^(n2 k1) of this thread's column n2 = t mod R
#pragma unroll
        for (int k1 = 1; k1 < R; ++k1) twr[k1] = tw[(t % R) * k1];
        float2 *obase = chan + ((long long)sb * N + n0) * kPols * S * C;
        for (int b = 0; b < nrounds; ++b) {
            const int q = b & 1;
            float2 *uq = u + q * NTR * ROW;
            named_bar_sync(kBarFull + q, ALL);            // FIR round b is in u[q]
#pragma unroll
            for (int it = 0; it < W::ITERS; ++it) {
                const int task = it * NF + t;
                const int tr = task / R, n2 = task % R;
                float2 *row = uq + tr * ROW;
                float2 v[R];
                // pass 1: R-point FFT over n1 (stride R), times W_C^(n2 k1)
#pragma unroll
                for (int n1 = 0; n1 < R; ++n1) v[n1] = row[R * n1 + n2];
                fft_reg<R>(v);
#pragma unroll
                for (int k1 = 1; k1 < R; ++k1) v[k1] = cmul(v[k1], twr[k1]);
                __syncwarp();                       // the row's R lanes have read it
#pragma unroll
                for (int k1 = 0; k1 < R; ++k1) row[(R + 1) * k1 + n2] = v[k1];
                __syncwarp();
                // pass 2: R-point FFT over n2 of row k1 = this lane's column, X[k1 + R k2]
                const int k1 = n2;
#pragma unroll
                for (int m = 0; m < R; ++m) v[m] = row[(R + 1) * k1 + m];
                if (it == W::ITERS - 1 && b + 2 < nrounds) named_bar_arrive(kBarEmpty + q, ALL);
                fft_reg<R>(v);
                const int j = tr / IC, il = tr % IC;
                const int s = s0 + b * kRound + j;
                if (s < S && n0 + il / kPols < N) {
                    float2 *out = obase + ((long long)il * S + s) * C;
#pragma unroll
                    for (int k2 = 0; k2 < R; ++k2) out[k1 + R * ((k2 + R / 2) % R)] = v[k2];
                }
            }
        }
    }
}

template <int C, int T, typename TIn>
cudaError_t launch_ws(const Handle &h, const void *raw, float2 *chan, cudaStream_t st)
{
    using W = PpfWsCfg<C>;
    const int N = h.p.n_stations, S = h.p.n_spectra, SB = h.p.n_subbands;
    const int rounds_total = (S + kRound - 1) / kRound;
    const int sgroups = (N + W::NPC - 1) / W::NPC;
    // long runs amortise the T-1 history rows each CTA filters first; shorten
    // them only while the grid would be under ~5 waves of three CTAs per SM
    int rpc = 64;
    while (rpc > 1 && (long long)((rounds_total + rpc - 1) / rpc) * sgroups * SB < 152LL * 16) rpc /= 2;
    dim3 grid((rounds_total + rpc - 1) / rpc, sgroups, SB);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
    constexpr size_t smem = ppf_ws_smem_bytes<C, TIn>();
    auto kern = ppf_ws_kernel<C, T, TIn>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 2 * W::NF, smem, st>>>(reinterpret_cast<const TIn *>(raw), chan, h.d_taps, h.d_twiddle, N, S, rpc,
                                        h.d_status, h.tc_timeout_cycles, h.tc_test_no_tma);
    return cudaGetLastError();
}

template <int C, int T, typename TIn>
cudaError_t launch_t(const Handle &h, const void *raw, float2 *chan, cudaStream_t st)
{
    if constexpr (C == 16 || C == 64) {
        return launch_ws<C, T, TIn>(h, raw, chan, st);
    } else {
        // C = 256: one CTA of 512 FIR lanes alternating FIR and FFT
        using Cfg = PpfCfg<C>;
        const int N = h.p.n_stations, S = h.p.n_spectra, SB = h.p.n_subbands;
        const int rounds_total = (S + kRound - 1) / kRound;
        const int sgroups = (N + Cfg::NPC - 1) / Cfg::NPC;
        // long runs of rounds per CTA amortise the T-1 history rows each CTA reads
        // and filters first; shorten them only while the grid would be under ~8 waves
        int rpc = 32;
        while (rpc > 1 && (long long)((rounds_total + rpc - 1) / rpc) * sgroups * SB < 152LL * 16) rpc /= 2;
        dim3 grid((rounds_total + rpc - 1) / rpc, sgroups, SB);
        if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
        constexpr size_t smem =
            ppf_smem_bytes<C, TIn>() + (ppf_split_u<C, TIn>() ? (size_t)Cfg::NTR * Cfg::ROW * sizeof(float2) : 0);
        auto kern = ppf_kernel<C, T, TIn>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, Cfg::NT, smem, st>>>(reinterpret_cast<const TIn *>(raw), chan, h.d_taps, h.d_twiddle,
                                          N, S, rpc);
        return cudaGetLastError();
    }
}

template <int C, typename TIn>
cudaError_t launch_taps(const Handle &h, const void *raw, float2 *chan, cudaStream_t st)
{
    switch (h.p.n_taps) {
    case 4: return launch_t<C, 4, TIn>(h, raw, chan, st);
    case 8: return launch_t<C, 8, TIn>(h, raw, chan, st);
    case 16: return launch_t<C, 16, TIn>(h, raw, chan, st);
    default: return cudaErrorInvalidValue;
    }
}

template <typename TIn>
cudaError_t launch_fmt(const Handle &h, const void *raw, float2 *chan, cudaStream_t st)
{
    switch (h.p.n_channels) {
    case 16: return launch_taps<16, TIn>(h, raw, chan, st);
    case 64: return launch_taps<64, TIn>(h, raw, chan, st);
    case 256: return launch_taps<256, TIn>(h, raw, chan, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool ppf_supported(int C, int T)
{
    return (C == 16 || C == 64 || C == 256) && (T == 4 || T == 8 || T == 16);
}

cudaError_t launch_ppf(const Handle &h, const void *raw, float2 *chan, cudaStream_t st)
{
    if (h.p.format == FX_CI16) return launch_fmt<short2>(h, raw, chan, st);
    if (h.p.format == FX_CI8) return launch_fmt<char2>(h, raw, chan, st);
    return launch_fmt<ci4_t>(h, raw, chan, st);
}

}  // namespace fxi
