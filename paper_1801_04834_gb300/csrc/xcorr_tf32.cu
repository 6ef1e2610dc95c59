// xcorr_tf32.cu -- FP32-accurate X-stage on the tcgen05 tensor cores:
// FP32 corrected samples split in the kernel into hi + lo TF32 parts,
// V ~ hi hi' + hi lo' + lo hi' (lo lo' dropped) with FP32 accumulation in TMEM.
//
// Paper, Sec. "Signal processing with GPU kernels": the correlator forms
// V[a][b] = sum_s Y[s][a] conj(Y[s][b]) for all input pairs and integrates over
// the block, in single precision. TF32 keeps FP32's exponent range with an
// 11-bit significand; hi = x with its 13 low mantissa bits cleared is exactly
// a TF32 value and lo = x - hi is exact in FP32, so x = hi + lo and the
// dropped lo lo' term is below 2^-20 of each product, which keeps the FP32
// path's error bound while running on the tensor cores.
// On planar operands (re plane R, im plane J) as in the FP16 X-stage:
//   Re V = R R^T + J J^T          Im V = J R^T - R J^T
// each product expanded into its three hi/lo terms (12 MMAs per K-step).
//
// Layout: corr [SB][C][2][I_pad][S_pad] FP32 (spectra contiguous), I_pad <= 128
// (up to 64 stations): one work item per (subband, channel), all inputs in one
// 128-row tile, so A and B are the same tile (M = 128, N = I_pad, K = 8).
// Stage = 32 spectra (128-byte rows, 128-byte swizzle) of both planes: 32 KB
// of hi (converted in place) + 32 KB of lo, ring of 3.
//
// Warp roles (persistent, one CTA per SM, 320 threads):
//   warp 0     TMA producer
//   warp 1     TMEM allocator + MMA issuer (tcgen05.mma kind::tf32)
//   warps 2-5  epilogue: tcgen05.ld of their TMEM lane quadrant, upper triangle
//   warps 6-9  converter: hi = x & ~0x1FFF written in place, lo = x - hi into
//              the stage's lo half, then a proxy fence so the tensor cores see
//              the generic-proxy writes
// Every mbarrier wait is bounded; on expiry the role is recorded in the status
// word, all roles leave, in-flight copies and MMAs are drained (bounded) and
// TMEM is freed.
//
// Accumulation. The tensor core's FP32 accumulator does not round each
// addition to nearest, so a long chain of MMAs into one accumulator drifts
// (measured: 2.5e-5 normwise after 768 spectra, growing with the chain). The
// accumulator is therefore restarted every kChunk stages (64 spectra) and the
// epilogue adds the chunk sums into the visibilities in IEEE FP32 (the rows
// of one channel stay in L2 while its chunks are summed).
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "internal.h"
#include "tc_ptx.cuh"

namespace fxi {
namespace {

using namespace tc;

constexpr int kT3Threads = 320;
constexpr int kT3Stages = 3;
constexpr int kT3K = 32;                              // spectra per stage (128-byte FP32 rows)
constexpr unsigned kT3Plane = 128u * 128u;            // 128 rows x 128 B
constexpr unsigned kT3Hi = 2u * kT3Plane;             // re + im, hi (converted in place)
constexpr unsigned kT3Stage = 2u * kT3Hi;             // hi + lo
constexpr int kT3TmemCols = 512;
constexpr int kT3Bars = 4 * kT3Stages + 5;            // full, conv, empty per stage; accf 2, acce 2, drain
constexpr int kChunk = 2;                             // stages per accumulator chain (64 spectra)

struct T3Params {
    CUtensorMap map;          // 3-D (spectrum, input, sb*C*2 + plane), box {32, 128, 1}
    float2 *vis;
    int *status;
    long long n_items;        // SB * C
    int N, I_pad, nk;         // stations, padded inputs, stages per item (a multiple of kChunk)
    long long B;              // baselines
    long long timeout_cycles;
    int no_tma;               // failure-detection test hook: issue no loads
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

__global__ void __launch_bounds__(kT3Threads, 1) xcorr_tf32_kernel(const __grid_constant__ T3Params P)
{
    extern __shared__ unsigned char smem_raw[];
    const unsigned base_u32 = smem_u32(smem_raw);
    const unsigned pad = (1024 - (base_u32 & 1023)) & 1023;
    unsigned char *tiles = smem_raw + pad;
    const unsigned tiles_u32 = base_u32 + pad;
    unsigned char *ctrl = tiles + kT3Stages * kT3Stage;
    const unsigned bar0 = smem_u32(ctrl);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto conv_bar = [&](int s) { return bar0 + 8u * (kT3Stages + s); };
    auto empty_bar = [&](int s) { return bar0 + 8u * (2 * kT3Stages + s); };
    auto accf_bar = [&](int b) { return bar0 + 8u * (3 * kT3Stages + b); };
    auto acce_bar = [&](int b) { return bar0 + 8u * (3 * kT3Stages + 2 + b); };
    const unsigned drain_bar = bar0 + 8u * (3 * kT3Stages + 4);
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(ctrl + 8 * kT3Bars);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kT3Stages; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(conv_bar(s), 4);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), 4);
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
    const int ncols = P.I_pad;                        // N of every MMA and accumulator width

    if (warp == 0) {
        // ================= TMA producer =================
        if (lane == 0) {
            long long it = 0;
            bool ok = true;
            for (long long w = blockIdx.x; w < P.n_items && ok; w += gridDim.x) {
                for (int kc = 0; kc < P.nk; ++kc, ++it) {
                    const int s = (int)(it % kT3Stages);
                    if (!t3wait(empty_bar(s), (unsigned)((it / kT3Stages) & 1) ^ 1u, abort_flag, P, 1)) {
                        ok = false;
                        break;
                    }
                    if (P.no_tma) continue;
                    mbar_arrive_expect_tx(full_bar(s), kT3Hi);
                    const unsigned dst = tiles_u32 + (unsigned)s * kT3Stage;
                    for (int pl = 0; pl < 2; ++pl)
                        tma_load_3d(dst + (unsigned)pl * kT3Plane, &P.map, full_bar(s), kc * kT3K, 0,
                                    (int)(w * 2 + pl));
                }
            }
            if (!ok && !P.no_tma) {
                const long long first = it > kT3Stages ? it - kT3Stages : 0;
                for (long long u = first; u < it; ++u)
                    drain_wait(full_bar((int)(u % kT3Stages)), (unsigned)((u / kT3Stages) & 1), P.timeout_cycles);
            }
        }
    } else if (warp == 1) {
        // ================= MMA issuer =================
        if (lane == 0) {
            long long it = 0, acc_it = 0;
            bool ok = true, issued = false;
            const unsigned idesc = idesc_tf32(ncols, false);
            const unsigned idesc_neg = idesc_tf32(ncols, true);
            for (long long w = blockIdx.x; w < P.n_items && ok; w += gridDim.x) {
              for (int ch = 0; ch < P.nk / kChunk && ok; ++ch, ++acc_it) {
                const int ab = (int)(acc_it & 1);
                if (!t3wait(acce_bar(ab), (unsigned)((acc_it >> 1) & 1) ^ 1u, abort_flag, P, 2)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const unsigned d_re = tmem_base + (unsigned)(ab * 256);
                const unsigned d_im = d_re + 128;
                for (int kc = 0; kc < kChunk; ++kc, ++it) {
                    const int s = (int)(it % kT3Stages);
                    if (!t3wait(conv_bar(s), (unsigned)((it / kT3Stages) & 1), abort_flag, P, 2)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned hi = tiles_u32 + (unsigned)s * kT3Stage;
                    const unsigned lo = hi + kT3Hi;
#pragma unroll
                    for (int kk = 0; kk < kT3K / 8; ++kk) {     // 8 FP32 = 32 bytes per K-step
                        const unsigned acc = (kc | kk) ? 1u : 0u;
                        const unsigned long long rh = smem_desc(hi + kk * 32);
                        const unsigned long long jh = smem_desc(hi + kT3Plane + kk * 32);
                        const unsigned long long rl = smem_desc(lo + kk * 32);
                        const unsigned long long jl = smem_desc(lo + kT3Plane + kk * 32);
                        // Re V = R R^T + J J^T
                        mma_tf32(d_re, rh, rh, idesc, acc);
                        mma_tf32(d_re, jh, jh, idesc, 1u);
                        mma_tf32(d_re, rh, rl, idesc, 1u);
                        mma_tf32(d_re, jh, jl, idesc, 1u);
                        mma_tf32(d_re, rl, rh, idesc, 1u);
                        mma_tf32(d_re, jl, jh, idesc, 1u);
                        // Im V = J R^T - R J^T
                        mma_tf32(d_im, jh, rh, idesc, acc);
                        mma_tf32(d_im, rh, jh, idesc_neg, 1u);
                        mma_tf32(d_im, jh, rl, idesc, 1u);
                        mma_tf32(d_im, rh, jl, idesc_neg, 1u);
                        mma_tf32(d_im, jl, rh, idesc, 1u);
                        mma_tf32(d_im, rl, jh, idesc_neg, 1u);
                    }
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
    } else if (warp >= 6) {
        // ================= converter (warps 6..9) =================
        const int ct = threadIdx.x - 6 * 32;            // 0..127
        long long it = 0;
        bool ok = true;
        for (long long w = blockIdx.x; w < P.n_items && ok; w += gridDim.x) {
            for (int kc = 0; kc < P.nk; ++kc, ++it) {
                const int s = (int)(it % kT3Stages);
                const bool got = t3wait(full_bar(s), (unsigned)((it / kT3Stages) & 1), abort_flag, P, 4);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                uint4 *h4 = reinterpret_cast<uint4 *>(tiles + (size_t)s * kT3Stage);
                uint4 *l4 = reinterpret_cast<uint4 *>(tiles + (size_t)s * kT3Stage + kT3Hi);
#pragma unroll 4
                for (int q = ct; q < (int)(kT3Hi / 16); q += 128) {
                    const uint4 x = h4[q];
                    uint4 hv, lv;
                    hv.x = x.x & 0xFFFFE000u;
                    hv.y = x.y & 0xFFFFE000u;
                    hv.z = x.z & 0xFFFFE000u;
                    hv.w = x.w & 0xFFFFE000u;
                    lv.x = __float_as_uint(__uint_as_float(x.x) - __uint_as_float(hv.x));
                    lv.y = __float_as_uint(__uint_as_float(x.y) - __uint_as_float(hv.y));
                    lv.z = __float_as_uint(__uint_as_float(x.z) - __uint_as_float(hv.z));
                    lv.w = __float_as_uint(__uint_as_float(x.w) - __uint_as_float(hv.w));
                    h4[q] = hv;
                    l4[q] = lv;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(conv_bar(s));
            }
        }
    } else {
        // ================= epilogue (warps 2..5) =================
        const int qd = warp & 3;
        long long acc_it = 0;
        bool live = true;
        for (long long w = blockIdx.x; w < P.n_items && live; w += gridDim.x) {
          for (int ch = 0; ch < P.nk / kChunk; ++ch, ++acc_it) {
            const int ab = (int)(acc_it & 1);
            const bool got = t3wait(accf_bar(ab), (unsigned)((acc_it >> 1) & 1), abort_flag, P, 3);
            if (!__all_sync(0xffffffffu, got)) {
                live = false;
                break;
            }
            tc_fence_after();
            const int ia = 32 * qd + lane;               // this lane's row input
            const int i = ia >> 1, p = ia & 1;
            const int i_warp_min = (32 * qd) >> 1;
            const unsigned t_re = tmem_base + ((unsigned)(32 * qd) << 16) + (unsigned)(ab * 256);
            const unsigned t_im = t_re + 128;
            float2 *vrow = P.vis + w * P.B * 4;
            // two 16-column chunks at a time: TMEM loads and the loads of the
            // running sums are all issued before any add or store
            const int ncc = ncols / 16;
            for (int cc0 = 0; cc0 < ncc; cc0 += 2) {
                if (8 * cc0 >= P.N) break;
                if (8 * cc0 + 15 < i_warp_min) continue;    // both chunks below the diagonal for this warp
                float re[2][16], im[2][16];
                float4 old[2][8];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (cc0 + u < ncc) {
                        tmem_ld16(t_re + 16 * (cc0 + u), re[u]);
                        tmem_ld16(t_im + 16 * (cc0 + u), im[u]);
                    }
                }
                if (ch > 0) {
#pragma unroll
                    for (int u = 0; u < 2; ++u)
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            const int j = 8 * (cc0 + u) + jj;
                            if (cc0 + u < ncc && i <= j && j < P.N)
                                old[u][jj] = *reinterpret_cast<const float4 *>(
                                    vrow + ((long long)j * (j + 1) / 2 + i) * 4 + 2 * p);
                        }
                }
                tmem_ld_wait();
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        const int j = 8 * (cc0 + u) + jj;
                        if (cc0 + u < ncc && i <= j && j < P.N) {
                            float4 v = make_float4(re[u][2 * jj], im[u][2 * jj], re[u][2 * jj + 1], im[u][2 * jj + 1]);
                            if (ch > 0) {                // add this chunk to the sum so far (FP32, RN)
                                v.x += old[u][jj].x;
                                v.y += old[u][jj].y;
                                v.z += old[u][jj].z;
                                v.w += old[u][jj].w;
                            }
                            *reinterpret_cast<float4 *>(vrow + ((long long)j * (j + 1) / 2 + i) * 4 + 2 * p) = v;
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

}  // namespace

cudaError_t launch_xcorr_tf32(const Handle &h, const float *corr, float2 *vis, cudaStream_t st)
{
    EncodeTiledFn enc = t3_encode_fn();
    if (!enc) return cudaErrorNotSupported;
    if (h.I_pad > 128 || h.S_pad % (kT3K * kChunk) != 0) return cudaErrorNotSupported;
    const long long planes = (long long)h.p.n_subbands * h.p.n_channels * 2;
    if (planes > 0x7fffffffLL) return cudaErrorInvalidValue;
    T3Params P;
    memset(&P, 0, sizeof(P));
    const cuuint64_t gdim[3] = {(cuuint64_t)h.S_pad, (cuuint64_t)h.I_pad, (cuuint64_t)planes};
    const cuuint64_t gstride[2] = {(cuuint64_t)h.S_pad * 4, (cuuint64_t)h.S_pad * 4 * h.I_pad};
    const cuuint32_t box[3] = {(cuuint32_t)kT3K, 128, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&P.map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<float *>(corr), gdim, gstride, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    P.vis = vis;
    P.status = h.d_status;
    P.n_items = planes / 2;
    P.N = h.p.n_stations;
    P.I_pad = h.I_pad;
    P.nk = h.S_pad / kT3K;
    P.B = h.B;
    P.timeout_cycles = h.tc_timeout_cycles;
    P.no_tma = h.tc_test_no_tma;
    const size_t smem = 1024 + (size_t)kT3Stages * kT3Stage + 8 * kT3Bars + 16;
    cudaError_t e = cudaFuncSetAttribute(xcorr_tf32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long grid = std::min<long long>(P.n_items, h.num_sms);
    if (grid <= 0) return cudaSuccess;
    xcorr_tf32_kernel<<<(unsigned)grid, kT3Threads, smem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace fxi
