// xcorr_tf32.cu -- FP32-accurate X-stage on the tcgen05 tensor cores, any
// station count: FP32 corrected samples split in the kernel into hi + lo,
// V ~ hi hi' + hi lo' + lo hi' (lo lo' dropped), the main term hi hi' as TF32
// MMAs and the two cross terms as BF16 MMAs, FP32 accumulation in TMEM, chunk
// sums added in IEEE FP32.
//
// Paper, Sec. "Signal processing with GPU kernels": the correlator forms
// V[a][b] = sum_s Y[s][a] conj(Y[s][b]) for all input pairs and integrates over
// the block, in single precision. TF32 keeps FP32's exponent range with an
// 11-bit significand; hi = x with its 13 low mantissa bits cleared is exactly
// a TF32 value and lo = x - hi is exact in FP32 with |lo| < 2^-10 |x|. The
// cross terms hi lo' and lo hi' are each below 2^-10 of the product, so they
// tolerate BF16 operands: rounding hi and lo to BF16 (8-bit significand, FP32
// exponent range, round to nearest) changes a cross term by at most 2^-8 of
// itself, i.e. 2^-18 of the product in the worst case and about 2^-21 RMS,
// with zero mean; the dropped lo lo' term is below 2^-20 of the product. BF16
// MMAs run at twice the TF32 rate, so one K-step of 16 spectra costs the time
// of 8 TF32 MMAs (4 TF32 + 4 BF16 of twice the depth) instead of 12 with all
// three products in TF32, and reads two thirds of the shared-memory bytes.
//
// Complex product as one real MMA of twice the width. With planar operands
// (re plane R, im plane J) and, for the column inputs, three consecutive
// shared-memory planes [R; J; -R] of n rows each,
//   D[a][0:n)  += R_a . R_b + J_a . J_b   = Re V[a][b]
//   D[a][n:2n) += R_a . J_b - J_a . R_b   = -Im V[a][b]
// come from two MMAs of N = 2n: A = R rows against B = [R; J] (planes 0-1),
// and A = J rows against B = [J; -R] (planes 1-2). Per stage of 16 spectra:
//   TF32 (K = 8, two K-steps):  hiR.[hiR; hiJ], hiJ.[hiJ; -hiR]
//   BF16 (K = 16, one K-step):  hiR.[loR; loJ], hiJ.[loJ; -loR],
//                               loR.[hiR; hiJ], loJ.[hiJ; -hiR]
// At n = 128 each MMA reads 4 KB of A and 8 KB of B from shared memory.
//
// Work items. Rows come in blocks of 128 inputs (M = 128); an item is
// (subband x channel, row block, column block) over the upper block
// triangle: the diagonal item of a row block covers columns
// [row0, row0 + min(128, I_pad - row0)), off-diagonal items cover the columns
// right of it in tiles of at most NT (64 or 128) inputs. 64 stations (128
// inputs) is one diagonal item per channel; 76 stations (160 inputs) is a
// 128-column diagonal item, a 32-column off-diagonal item and a 32-row
// diagonal item.
//
// Shared memory, one stage = 16 spectra:
//   B region: TF32 planes hi R, hi J, -hi R of n rows each (64-byte rows,
//             64-byte swizzle, plane pitch n x 64 bytes), then BF16 planes
//             hi R, hi J, -hi R, lo R, lo J, -lo R (32-byte rows, 32-byte
//             swizzle, pitch n x 32 bytes) from byte 3 n x 64. On a diagonal
//             item the A operands are TF32 planes 0, 1 and BF16 planes 0, 1,
//             3, 4 of the same region read as 128-row tiles (rows past n are
//             other planes' data and only reach accumulator rows the
//             epilogue ignores; the region is at least 48 KB, so these reads
//             stay inside the stage).
//   A region (off-diagonal items): TF32 hi R, hi J (8 KB each), then BF16
//             hi R, hi J, lo R, lo J (4 KB each), before the B region.
// TMA writes the raw FP32 R and J rows into the TF32 hi planes, where they
// stay as they are: a kind::tf32 MMA reads the upper 19 bits of each 32-bit
// operand and ignores the 13 low mantissa bits, so the raw value acts as hi
// (the kernel tests on operands with non-zero low bits check this against an
// FP64 reference). Converter warps write -hi R and the BF16 planes, fence the
// async proxy and release the stage to the MMA thread.
//
// Accumulation. The tensor core's FP32 accumulator does not round each
// addition to nearest, so a long chain of MMAs into one accumulator drifts
// (about 2^-24 of the running value per MMA). The accumulator is restarted
// every `chunk` stages (64 spectra by default); the epilogue writes the first
// chunk's sums and adds every later chunk's into the visibilities with
// vector FP32 reductions in L2 (red.global.add.v4.f32, round to nearest; no
// read back into the SM, so the epilogue never waits on memory). Each
// visibility entry is owned by one lane of one CTA, which issues its chunks in
// order, so the sum order is fixed and results are reproducible.
//
// Warp roles (persistent, one CTA per SM, 448 threads):
//   warp 0      TMA producer
//   warp 1      TMEM allocator + MMA issuer (tcgen05.mma kind::tf32 and
//               kind::f16 with BF16 operands, into the same accumulator)
//   warps 2-9   epilogue: two warps per TMEM lane quadrant (warp % 4), each
//               taking every other 32-column group of the upper triangle
//   warps 10-13 converter
// Two accumulators of 256 columns (double buffered) fill the 512 TMEM columns.
// Every mbarrier wait is bounded; on expiry the role is recorded in the status
// word, all roles leave, in-flight copies and MMAs are drained (bounded) and
// TMEM is freed.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"

namespace fxi {
namespace {

using namespace tc;

constexpr int kT3Threads = 448;
constexpr int kT3EpiWarps = 8;
constexpr int kT3ConvWarp0 = 2 + kT3EpiWarps;
constexpr int kT3K = 16;                              // spectra per stage (64-byte FP32 rows)
constexpr unsigned kT3RowBytes = 64;
constexpr unsigned kT3APlane = 128u * kT3RowBytes;    // one 128-row TF32 plane: 8 KB
constexpr unsigned kT3BfRowBytes = 32;                // one BF16 row: 16 spectra
constexpr unsigned kT3ABfPlane = 128u * kT3BfRowBytes; // one 128-row BF16 plane: 4 KB
constexpr unsigned kT3ABf = 2u * kT3APlane;           // BF16 planes of the A region
constexpr unsigned kT3BRegionMin = 6u * kT3APlane;    // diagonal item at n = 128: 48 KB
constexpr int kT3MaxStages = 6;
constexpr int kT3MaxItems = 64;                       // items per channel
constexpr int kT3TmemCols = 512;
constexpr int kT3AccCols = 256;
constexpr int kT3Bars = 3 * kT3MaxStages + 5;         // full, conv, empty per stage; accf 2, acce 2, drain
constexpr unsigned kT3SmemBudget = 200u * 1024u;

struct T3Params {
    CUtensorMap map128;       // 3-D (spectrum, input, sb*C*2 + plane), box {16, 128, 1}
    CUtensorMap map16;        // same tensor, box {16, 16, 1}
    int4 items[kT3MaxItems];  // per channel: (row0, col0, n, diagonal)
    float2 *vis;
    int *status;
    long long n_items;        // SB * C * ipc
    long long B;              // baselines
    long long timeout_cycles;
    int ipc;                  // items per channel
    int N, nk, chunk;         // stations, stages per item, stages per accumulator chain
    int stages;
    unsigned stage_bytes;
    unsigned a_off;           // byte offset of the B region when an A region precedes it
    int no_tma;               // failure-detection test hook: issue no loads
    int accumulate;           // add every chunk to vis (also the first)
};

__device__ __forceinline__ bool t3wait(unsigned bar, unsigned parity, volatile int *abort_flag, const T3Params &P,
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

// Shared-memory matrix descriptor: K-major, 64-byte swizzle (8-row atoms of
// 512 bytes, SBO = 512), LBO unused for this layout, descriptor version 1.
__device__ __forceinline__ unsigned long long sdesc64(unsigned addr)
{
    return (unsigned long long)((addr & 0x3FFFF) >> 4) | (1ull << 16) | ((unsigned long long)(512 >> 4) << 32) |
           (1ull << 46) | (4ull << 61);
}

// The same for the BF16 planes: K-major, 32-byte swizzle (8-row atoms of 256
// bytes, SBO = 256); one 32-byte row is the whole K = 16 of a stage.
__device__ __forceinline__ unsigned long long sdesc32(unsigned addr)
{
    return (unsigned long long)((addr & 0x3FFFF) >> 4) | (1ull << 16) | ((unsigned long long)(256 >> 4) << 32) |
           (1ull << 46) | (6ull << 61);
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major, M = 128.
__device__ __forceinline__ unsigned idesc_tf32(int n, bool neg_a)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((neg_a ? 1u : 0u) << 13) | ((unsigned)(n >> 3) << 17) |
           ((unsigned)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(unsigned d_tmem, unsigned long long adesc, unsigned long long bdesc,
                                         unsigned idesc, unsigned accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
                 : "memory");
}

// Vector FP32 reduction into global memory (performed in L2, round to nearest).
__device__ __forceinline__ void red_add4(float2 *addr, float4 v)
{
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w)
                 : "memory");
}

__device__ __forceinline__ unsigned hi_bits(unsigned x) { return x & 0xFFFFE000u; }
__device__ __forceinline__ unsigned lo_bits(unsigned x, unsigned h)
{
    return __float_as_uint(__uint_as_float(x) - __uint_as_float(h));
}

// Byte offset, in a 32-byte-swizzled BF16 plane, of the 4 elements that the
// 16-byte chunk q of a 64-byte-swizzled FP32 plane holds. Both swizzles XOR
// the 16-byte chunk index with address bits 7 and up (64-byte rows: chunk ^=
// (row / 2) mod 4; 32-byte rows: chunk ^= (row / 4) mod 2) and both plane
// bases are aligned to their atoms, so the logical position follows from q.
__device__ __forceinline__ unsigned bf_chunk_off(int q)
{
    const int r = q >> 2;
    const int lc = (q & 3) ^ ((r >> 1) & 3);          // logical chunk: spectra 4 lc .. 4 lc + 3
    return (unsigned)(r * 32 + 16 * ((lc >> 1) ^ ((r >> 2) & 1)) + 8 * (lc & 1));
}

// 4 FP32 -> 4 BF16 (round to nearest even) in element order
__device__ __forceinline__ uint2 bf16x4(uint4 v)
{
    const __nv_bfloat162 a = __floats2bfloat162_rn(__uint_as_float(v.x), __uint_as_float(v.y));
    const __nv_bfloat162 b = __floats2bfloat162_rn(__uint_as_float(v.z), __uint_as_float(v.w));
    return make_uint2(*reinterpret_cast<const unsigned *>(&a), *reinterpret_cast<const unsigned *>(&b));
}

__device__ __forceinline__ uint2 neg_bf16x4(uint2 v) { return make_uint2(v.x ^ 0x80008000u, v.y ^ 0x80008000u); }

// Split one R plane and one J plane of `rows` rows (raw FP32 in the TF32
// planes at tf, pitch tf_pitch, left unchanged: the TF32 MMA reads them as
// hi) into hi and lo and write the BF16 planes at bf (pitch bf_pitch): for
// the column operand (col) -hi R after the two TF32 planes and BF16 hi R,
// hi J, -hi R, lo R, lo J, -lo R; for the row operand of an off-diagonal item
// BF16 hi R, hi J, lo R, lo J.
__device__ __forceinline__ void convert_split(unsigned char *tf, unsigned tf_pitch, unsigned char *bf,
                                              unsigned bf_pitch, int rows, bool col, int t)
{
    const int nq = rows * (int)(kT3RowBytes / 16);
    for (int q = t; q < nq; q += 128) {
        const uint4 x = reinterpret_cast<const uint4 *>(tf)[q];
        const uint4 y = reinterpret_cast<const uint4 *>(tf + tf_pitch)[q];
        uint4 xh, xl, yh, yl;
        xh.x = hi_bits(x.x); xh.y = hi_bits(x.y); xh.z = hi_bits(x.z); xh.w = hi_bits(x.w);
        yh.x = hi_bits(y.x); yh.y = hi_bits(y.y); yh.z = hi_bits(y.z); yh.w = hi_bits(y.w);
        xl.x = lo_bits(x.x, xh.x); xl.y = lo_bits(x.y, xh.y); xl.z = lo_bits(x.z, xh.z); xl.w = lo_bits(x.w, xh.w);
        yl.x = lo_bits(y.x, yh.x); yl.y = lo_bits(y.y, yh.y); yl.z = lo_bits(y.z, yh.z); yl.w = lo_bits(y.w, yh.w);
        const uint2 xhb = bf16x4(xh), yhb = bf16x4(yh), xlb = bf16x4(xl), ylb = bf16x4(yl);
        unsigned char *o = bf + bf_chunk_off(q);
        if (col) {
            const unsigned sg = 0x80000000u;
            reinterpret_cast<uint4 *>(tf + 2 * tf_pitch)[q] = make_uint4(xh.x ^ sg, xh.y ^ sg, xh.z ^ sg, xh.w ^ sg);
            *reinterpret_cast<uint2 *>(o) = xhb;
            *reinterpret_cast<uint2 *>(o + bf_pitch) = yhb;
            *reinterpret_cast<uint2 *>(o + 2 * bf_pitch) = neg_bf16x4(xhb);
            *reinterpret_cast<uint2 *>(o + 3 * bf_pitch) = xlb;
            *reinterpret_cast<uint2 *>(o + 4 * bf_pitch) = ylb;
            *reinterpret_cast<uint2 *>(o + 5 * bf_pitch) = neg_bf16x4(xlb);
        } else {
            *reinterpret_cast<uint2 *>(o) = xhb;
            *reinterpret_cast<uint2 *>(o + bf_pitch) = yhb;
            *reinterpret_cast<uint2 *>(o + 2 * bf_pitch) = xlb;
            *reinterpret_cast<uint2 *>(o + 3 * bf_pitch) = ylb;
        }
    }
}

__global__ void __launch_bounds__(kT3Threads, 1) xcorr_tf32_kernel(const __grid_constant__ T3Params P)
{
    extern __shared__ unsigned char smem_raw[];
    const unsigned base_u32 = smem_u32(smem_raw);
    const unsigned pad = (1024 - (base_u32 & 1023)) & 1023;
    unsigned char *tiles = smem_raw + pad;
    const unsigned tiles_u32 = base_u32 + pad;
    unsigned char *ctrl = tiles + (size_t)P.stages * P.stage_bytes;
    const unsigned bar0 = smem_u32(ctrl);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto conv_bar = [&](int s) { return bar0 + 8u * (kT3MaxStages + s); };
    auto empty_bar = [&](int s) { return bar0 + 8u * (2 * kT3MaxStages + s); };
    auto accf_bar = [&](int b) { return bar0 + 8u * (3 * kT3MaxStages + b); };
    auto acce_bar = [&](int b) { return bar0 + 8u * (3 * kT3MaxStages + 2 + b); };
    const unsigned drain_bar = bar0 + 8u * (3 * kT3MaxStages + 4);
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(ctrl + 8 * kT3Bars);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < P.stages; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(conv_bar(s), 4);              // one arrival per converter warp
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), kT3EpiWarps);    // one arrival per epilogue warp
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kT3TmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const unsigned tmem_base = *tmem_slot;
    const int n_chunks = P.nk / P.chunk;

    if (warp == 0) {
        // ================= TMA producer =================
        if (lane == 0) {
            long long it = 0;
            bool ok = true;
            for (long long w = blockIdx.x; w < P.n_items && ok; w += gridDim.x) {
                const int4 itm = P.items[(int)(w % P.ipc)];
                const long long gch = w / P.ipc;
                const int row0 = itm.x, col0 = itm.y, n = itm.z;
                const bool diag = itm.w != 0;
                const bool full_diag = diag && n == 128;
                const unsigned boff = diag ? 0u : P.a_off;
                const unsigned tx = (diag ? 0u : 2u * kT3APlane) + 2u * (unsigned)n * kT3RowBytes;
                for (int kc = 0; kc < P.nk; ++kc, ++it) {
                    const int s = (int)(it % P.stages);
                    if (!t3wait(empty_bar(s), (unsigned)((it / P.stages) & 1) ^ 1u, abort_flag, P, 1)) {
                        ok = false;
                        break;
                    }
                    if (P.no_tma) continue;
                    mbar_arrive_expect_tx(full_bar(s), tx);
                    const unsigned dst = tiles_u32 + (unsigned)s * P.stage_bytes;
                    for (int pl = 0; pl < 2; ++pl) {
                        const int z = (int)(gch * 2 + pl);
                        if (!diag)         // row inputs: A region planes 0 (R) and 1 (J)
                            tma_load_3d(dst + (unsigned)pl * kT3APlane, &P.map128, full_bar(s), kc * kT3K, row0, z);
                        const unsigned bdst = dst + boff + (unsigned)pl * (unsigned)n * kT3RowBytes;
                        if (full_diag) {
                            tma_load_3d(bdst, &P.map128, full_bar(s), kc * kT3K, col0, z);
                        } else {
                            for (int r = 0; r < n; r += 16)
                                tma_load_3d(bdst + (unsigned)r * kT3RowBytes, &P.map16, full_bar(s), kc * kT3K,
                                            col0 + r, z);
                        }
                    }
                }
            }
            if (!ok && !P.no_tma) {
                const long long first = it > P.stages ? it - P.stages : 0;
                for (long long u = first; u < it; ++u)
                    drain_wait(full_bar((int)(u % P.stages)), (unsigned)((u / P.stages) & 1), P.timeout_cycles);
            }
        }
    } else if (warp == 1) {
        // ================= MMA issuer =================
        if (lane == 0) {
            long long it = 0, acc_it = 0;
            bool ok = true, issued = false;
            for (long long w = blockIdx.x; w < P.n_items && ok; w += gridDim.x) {
                const int4 itm = P.items[(int)(w % P.ipc)];
                const int n = itm.z;
                const bool diag = itm.w != 0;
                const unsigned pitch = (unsigned)n * kT3RowBytes;
                const unsigned bpitch = (unsigned)n * kT3BfRowBytes;
                const unsigned idesc = idesc_tf32(2 * n, false);
                const unsigned idesc_bf = make_idesc(1u, 2 * n, false);
                for (int ch = 0; ch < n_chunks && ok; ++ch, ++acc_it) {
                    const int ab = (int)(acc_it & 1);
                    if (!t3wait(acce_bar(ab), (unsigned)((acc_it >> 1) & 1) ^ 1u, abort_flag, P, 2)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned d = tmem_base + (unsigned)(ab * kT3AccCols);
                    for (int kc = 0; kc < P.chunk; ++kc, ++it) {
                        const int s = (int)(it % P.stages);
                        if (!t3wait(conv_bar(s), (unsigned)((it / P.stages) & 1), abort_flag, P, 2)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const unsigned st = tiles_u32 + (unsigned)s * P.stage_bytes;
                        const unsigned bb = diag ? st : st + P.a_off;      // TF32 hi R, hi J, -hi R
                        const unsigned bf = bb + 3 * pitch;                 // BF16 hi R, hi J, -hi R, lo R, lo J, -lo R
                        // A planes: TF32 hi R, hi J; BF16 hi R, hi J, lo R, lo J
                        const unsigned a_hr = diag ? bb : st;
                        const unsigned a_hj = diag ? bb + pitch : st + kT3APlane;
                        const unsigned a_bhr = diag ? bf : st + kT3ABf;
                        const unsigned a_bhj = diag ? bf + bpitch : st + kT3ABf + kT3ABfPlane;
                        const unsigned a_blr = diag ? bf + 3 * bpitch : st + kT3ABf + 2 * kT3ABfPlane;
                        const unsigned a_blj = diag ? bf + 4 * bpitch : st + kT3ABf + 3 * kT3ABfPlane;
#pragma unroll
                        for (int kk = 0; kk < kT3K / 8; ++kk) {    // 8 FP32 = 32 bytes per TF32 K-step
                            const unsigned acc = (kc | kk) ? 1u : 0u;
                            const unsigned o = (unsigned)kk * 32u;
                            mma_tf32(d, sdesc64(a_hr + o), sdesc64(bb + o), idesc, acc);           // [hi R; hi J]
                            mma_tf32(d, sdesc64(a_hj + o), sdesc64(bb + pitch + o), idesc, 1u);    // [hi J; -hi R]
                        }
                        // cross terms, K = 16 spectra in one BF16 MMA each
                        mma_f16(d, sdesc32(a_bhr), sdesc32(bf + 3 * bpitch), idesc_bf, 1u);    // [lo R; lo J]
                        mma_f16(d, sdesc32(a_bhj), sdesc32(bf + 4 * bpitch), idesc_bf, 1u);    // [lo J; -lo R]
                        mma_f16(d, sdesc32(a_blr), sdesc32(bf), idesc_bf, 1u);                 // [hi R; hi J]
                        mma_f16(d, sdesc32(a_blj), sdesc32(bf + bpitch), idesc_bf, 1u);        // [hi J; -hi R]
                        issued = true;
                        mma_commit(empty_bar(s));
                    }
                    if (!ok) break;
                    mma_commit(accf_bar(ab));
                }
            }
            if (!ok && issued) {
                mma_commit(drain_bar);
                drain_wait(drain_bar, 0, P.timeout_cycles);
            }
        }
        __syncwarp();
    } else if (warp >= kT3ConvWarp0) {
        // ================= converter (warps 10..13) =================
        const int ct = threadIdx.x - kT3ConvWarp0 * 32; // 0..127
        long long it = 0;
        bool ok = true;
        for (long long w = blockIdx.x; w < P.n_items && ok; w += gridDim.x) {
            const int4 itm = P.items[(int)(w % P.ipc)];
            const int n = itm.z;
            const bool diag = itm.w != 0;
            const unsigned pitch = (unsigned)n * kT3RowBytes;
            for (int kc = 0; kc < P.nk; ++kc, ++it) {
                const int s = (int)(it % P.stages);
                const bool got = t3wait(full_bar(s), (unsigned)((it / P.stages) & 1), abort_flag, P, 4);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                unsigned char *st = tiles + (size_t)s * P.stage_bytes;
                unsigned char *bb = diag ? st : st + P.a_off;
                if (!diag)   // row inputs: BF16 planes after the two TF32 planes of the A region
                    convert_split(st, kT3APlane, st + kT3ABf, kT3ABfPlane, 128, false, ct);
                convert_split(bb, pitch, bb + 3 * pitch, (unsigned)n * kT3BfRowBytes, n, true, ct);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(conv_bar(s));
            }
        }
    } else {
        // ================= epilogue (warps 2..9) =================
        const int qd = warp & 3;                        // TMEM lane quadrant
        const int half = (warp - 2) >> 2;               // which 32-column groups
        long long acc_it = 0;
        bool live = true;
        for (long long w = blockIdx.x; w < P.n_items && live; w += gridDim.x) {
            const int4 itm = P.items[(int)(w % P.ipc)];
            const long long gch = w / P.ipc;
            const int row0 = itm.x, col0 = itm.y, n = itm.z;
            const int ia = row0 + 32 * qd + lane;        // this lane's row input
            const int i = ia >> 1, p = ia & 1;
            const int i_warp_min = (row0 + 32 * qd) >> 1;
            const int ncc = n / 16;
            float2 *vrow = P.vis + gch * P.B * 4;
            for (int ch = 0; ch < n_chunks; ++ch, ++acc_it) {
                const int ab = (int)(acc_it & 1);
                const bool got = t3wait(accf_bar(ab), (unsigned)((acc_it >> 1) & 1), abort_flag, P, 3);
                if (!__all_sync(0xffffffffu, got)) {
                    live = false;
                    break;
                }
                tc_fence_after();
                const bool store = (ch == 0) && !P.accumulate;
                const unsigned t = tmem_base + ((unsigned)(32 * qd) << 16) + (unsigned)(ab * kT3AccCols);
                if (i_warp_min < P.N) {
                    for (int cc = 2 * half; cc < ncc; cc += 4) {
                        const int j0 = (col0 >> 1) + 8 * cc;     // first station of this pair of chunks
                        if (j0 >= P.N) break;
                        if (j0 + 15 < i_warp_min) continue;     // both chunks below the diagonal
                        float re[2][16], ni[2][16];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            if (cc + u < ncc) {
                                tmem_ld16(t + 16 * (cc + u), re[u]);
                                tmem_ld16(t + (unsigned)n + 16 * (cc + u), ni[u]);
                            }
                        }
                        tmem_ld_wait();
#pragma unroll
                        for (int u = 0; u < 2; ++u)
#pragma unroll
                            for (int jj = 0; jj < 8; ++jj) {
                                const int j = j0 + 8 * u + jj;
                                if (cc + u < ncc && i <= j && j < P.N) {
                                    const float4 v = make_float4(re[u][2 * jj], -ni[u][2 * jj], re[u][2 * jj + 1],
                                                                 -ni[u][2 * jj + 1]);
                                    float2 *dst = vrow + ((long long)j * (j + 1) / 2 + i) * 4 + 2 * p;
                                    if (store)
                                        *reinterpret_cast<float4 *>(dst) = v;
                                    else
                                        red_add4(dst, v);
                                }
                            }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce_bar(ab));
            }
        }
    }

    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kT3TmemCols)
                     : "memory");
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn t3_encode_fn()
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

// Item list of one channel and the stage geometry it needs.
struct T3Plan {
    std::vector<int4> items;
    unsigned stage_bytes = 0, a_off = 0;
    int stages = 0;
};

bool t3_plan(int I_pad, int NT, T3Plan &pl)
{
    pl.items.clear();
    bool off = false;
    int nmax_off = 0;
    for (int row0 = 0; row0 < I_pad; row0 += 128) {
        const int nd = std::min(128, I_pad - row0);
        pl.items.push_back(make_int4(row0, row0, nd, 1));
        for (int c0 = row0 + 128; c0 < I_pad; c0 += NT) {
            const int n = std::min(NT, I_pad - c0);
            pl.items.push_back(make_int4(row0, c0, n, 0));
            off = true;
            nmax_off = std::max(nmax_off, n);
        }
    }
    if ((int)pl.items.size() > kT3MaxItems) return false;
    pl.a_off = off ? 4u * kT3APlane : 0u;
    pl.stage_bytes = std::max(kT3BRegionMin, pl.a_off + 6u * (unsigned)nmax_off * kT3RowBytes);
    pl.stage_bytes = (pl.stage_bytes + 1023u) / 1024u * 1024u;
    pl.stages = std::min(kT3MaxStages, (int)(kT3SmemBudget / pl.stage_bytes));
    return pl.stages >= 2;
}

}  // namespace

bool xtf32_supported(int I_pad, int S_pad)
{
    T3Plan pl;
    return S_pad % (kT3K * 4) == 0 && t3_plan(I_pad, 64, pl);
}

cudaError_t launch_xcorr_tf32(const Handle &h, const float *corr, float2 *vis, cudaStream_t st, bool accumulate)
{
    EncodeTiledFn enc = t3_encode_fn();
    if (!enc) return cudaErrorNotSupported;
    T3Plan pl;
    if (!t3_plan(h.I_pad, 64, pl)) return cudaErrorNotSupported;
    const int chunk = 4;                                // stages per accumulator chain: 64 spectra
    if (h.S_pad % (kT3K * chunk) != 0) return cudaErrorNotSupported;
    const long long planes = (long long)h.p.n_subbands * h.p.n_channels * 2;
    if (planes > 0x7fffffffLL) return cudaErrorInvalidValue;
    T3Params P;
    memset(&P, 0, sizeof(P));
    const cuuint64_t gdim[3] = {(cuuint64_t)h.S_pad, (cuuint64_t)h.I_pad, (cuuint64_t)planes};
    const cuuint64_t gstride[2] = {(cuuint64_t)h.S_pad * 4, (cuuint64_t)h.S_pad * 4 * h.I_pad};
    const cuuint32_t estr[3] = {1, 1, 1};
    const cuuint32_t box128[3] = {(cuuint32_t)kT3K, 128, 1};
    const cuuint32_t box16[3] = {(cuuint32_t)kT3K, 16, 1};
    if (enc(&P.map128, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<float *>(corr), gdim, gstride, box128, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    if (enc(&P.map16, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<float *>(corr), gdim, gstride, box16, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    for (size_t k = 0; k < pl.items.size(); ++k) P.items[k] = pl.items[k];
    P.ipc = (int)pl.items.size();
    P.vis = vis;
    P.status = h.d_status;
    P.n_items = planes / 2 * P.ipc;
    P.N = h.p.n_stations;
    P.nk = h.S_pad / kT3K;
    P.chunk = chunk;
    P.B = h.B;
    P.stages = pl.stages;
    P.stage_bytes = pl.stage_bytes;
    P.a_off = pl.a_off;
    P.timeout_cycles = h.tc_timeout_cycles;
    P.no_tma = h.tc_test_no_tma;
    P.accumulate = accumulate ? 1 : 0;
    const size_t smem = 1024 + (size_t)pl.stages * pl.stage_bytes + 8 * kT3Bars + 16;
    cudaError_t e = cudaFuncSetAttribute(xcorr_tf32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long grid = std::min<long long>(P.n_items, h.num_sms);
    if (grid <= 0) return cudaSuccess;
    xcorr_tf32_kernel<<<(unsigned)grid, kT3Threads, smem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace fxi
