// ppf_common.cuh -- CTA geometry and copy helpers shared by the polyphase
// filter-bank kernels (ppf.cu: channelise only; channelize_correct_impl.cuh:
// channelise + delay/bandpass correction in one pass).
#pragma once
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace fxi {
namespace ppf {

constexpr int kRound = 16;  // spectra per round; a multiple of every supported T

// One CTA = NPC stations x 2 pols x C channels. C = R * R for the two-pass FFT.
template <int C>
struct PpfCfg {
    static constexpr int R = (C == 16) ? 4 : (C == 64) ? 8 : 16;  // C = R * R
    static constexpr int NPC = (C * kPols >= 256) ? 1 : 256 / (C * kPols);  // stations per CTA
    static constexpr int NT = NPC * C * kPols;                    // threads per CTA
    // smem row of one transform: C + R float2, which holds the pass-1 output
    // as R rows of R + 1 (the odd row length keeps pass-2 reads conflict free),
    // padded for R >= 8 to 8 mod 16 entries so that the FIR stores of the two
    // pols of a channel (rows one apart) fall on different banks
    static constexpr int ROW = R * (R + 1) + (R >= 8 ? ((8 - (R * (R + 1)) % 16) + 16) % 16 : 0);
    static constexpr int NTR = NPC * kPols * kRound;              // transforms per round
    static constexpr int FFT_ITERS = NTR * R / NT;
    static_assert(R * R == C, "C must be a square of R");
    static_assert(NTR * R % NT == 0, "FFT tasks must tile the CTA");
};

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, int src_bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Raw rows by the bulk-copy (TMA) engine: one contiguous run of a station's
// time rows (global and shared addresses 16-byte aligned, a multiple of 16
// bytes) lands in shared memory and completes on an mbarrier with its byte
// count, so the FIR threads issue no per-chunk copies.
__device__ __forceinline__ void bulk_rows(void *smem_dst, const void *gsrc, unsigned bytes, unsigned bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(smem_dst)),
                 "l"(gsrc), "r"(bytes), "r"(bar)
                 : "memory");
}
// Expect `bytes` on `bar` (one arrival) and start the copy; a zero-byte run
// (rows past the block's end) only completes the phase.
__device__ __forceinline__ void bulk_rows_issue(void *smem_dst, const void *gsrc, unsigned bytes, unsigned bar)
{
    tc::mbar_arrive_expect_tx(bar, bytes);
    if (bytes) bulk_rows(smem_dst, gsrc, bytes, bar);
}
// Bounded wait for a raw-row phase: after `budget` clock cycles the wait gives
// up, records code 6 (F-stage loader) in the status word and returns, so the
// kernel finishes (on stale rows) instead of hanging; fx_poll_status reports it.
constexpr int kStatusLoader = 6;
__device__ __forceinline__ void raw_wait(unsigned bar, unsigned parity, int *status, long long budget)
{
    if (tc::mbar_try_wait(bar, parity)) return;
    const long long t0 = clock64();
    while (!tc::mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) {
            if (status) atomicCAS(status, 0, kStatusLoader);
            return;
        }
    }
}

// Named CTA barriers (hardware barriers with fixed arrival counts, like
// __syncthreads, which uses id 0) for the warp-specialised kernels: FIR warps
// and FFT warps hand rounds over with bar.arrive (producer) / bar.sync
// (consumer); every participant of a barrier runs the same number of rounds.
enum {
    kBarRaw = 1,     // FIR threads: raw rows staged / consumed
    kBarFft = 2,     // FFT threads among themselves
    kBarFull = 3,    // FULL[0], FULL[1]: FIR round in the row buffer (ids 3, 4)
    kBarEmpty = 5,   // EMPTY[0], EMPTY[1]: FFT threads done with it (ids 5, 6)
    kBarFft2 = 7,    // the second FFT group of the 256-channel kernel among itself
};
__device__ __forceinline__ void named_bar_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_bar_arrive(int id, int n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ float2 to_f2(short2 v) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ float2 to_f2(char2 v) { return make_float2((float)v.x, (float)v.y); }
// 4-bit complex sample: real part in the high nibble, imaginary part in the low
// nibble, two's complement (sign-extended by arithmetic shifts of a signed byte)
struct ci4_t {
    unsigned char v;
};
__device__ __forceinline__ float2 to_f2(ci4_t s)
{
    const int b = (int)(signed char)s.v;
    return make_float2((float)(b >> 4), (float)((int)(signed char)(s.v << 4) >> 4));
}

// twiddles + double-buffered raw rows + one round of FFT rows
template <int C, typename TIn>
constexpr size_t ppf_smem_bytes()
{
    using Cfg = PpfCfg<C>;
    return (size_t)C * sizeof(float2) + 2ull * kRound * Cfg::NPC * C * kPols * sizeof(TIn) +
           (size_t)Cfg::NTR * Cfg::ROW * sizeof(float2);
}

}  // namespace ppf
}  // namespace fxi
