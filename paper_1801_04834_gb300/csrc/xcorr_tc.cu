// xcorr_tc.cu -- X-stage correlator on the 5th-generation (tcgen05) tensor
// cores: FP16 or BF16 operands, FP32 accumulation in tensor memory (TMEM).
//
// Paper, Sec. "Signal processing with GPU kernels": the last kernel correlates
// all antenna-field pairs and integrates over the block. The paper ran this in
// FP32 on CUDA cores; here the same contraction
//   V[a][b] = sum_s Y[s][a] * conj(Y[s][b])        (a, b inputs = station x pol)
// is split into real GEMMs on planar operands (re plane R, im plane J):
//   Re V = R R^T + J J^T          Im V = J R^T - R J^T
// with the subtraction done by the MMA's negate-A bit, so both accumulators
// come out ready to store (no transpose in the epilogue). The split-FP16 form
// (value = hi + lo) adds the hi*lo' and lo*hi' cross terms the same way
// (lo*lo' is dropped).
//
// One work item = (subband, channel, row block rb): rows are inputs
// [128 rb, 128 rb + 128) (M = 128), columns are inputs [128 rb, I_pad)
// (N = I_pad - 128 rb <= 256), so only blocks on or above the diagonal are
// computed. The operand tile for a K-chunk of 64 spectra is one TMA box of
// rows [128 rb, 128 rb + R) x 64 spectra per plane, 128-byte swizzled; A and
// B are the same shared-memory tile (A = its first 128 rows).
//
// Warp roles (192 threads, persistent, one CTA per SM):
//   warp 0     TMA producer: one elected thread fills a ring of STAGES tiles
//   warp 1     TMEM allocator + MMA issuer: one elected thread issues
//              tcgen05.mma and tcgen05.commit (stage release, accumulator full)
//   warps 2-5  epilogue: tcgen05.ld of their 32-lane TMEM quadrant, scale by
//              1/operand_scale^2, store the upper-triangle baselines only
// Accumulators are double buffered in TMEM when 4 * N <= 512 columns, so the
// epilogue of one item overlaps the main loop of the next.
//
// Every mbarrier wait is bounded (clock64 budget). On expiry the thread
// records a code in the handle's status word and raises a shared abort flag;
// all roles leave their loops, the producer waits (bounded) for the loads it
// still has in flight, the MMA thread waits (bounded) for its issued MMAs, and
// the TMEM is freed before the CTA exits.
#include <cuda.h>

#include "internal.h"

namespace fxi {
namespace {

constexpr int kBK = 64;               // spectra per stage (128-byte rows of 16-bit values)
constexpr int kThreads = 192;
constexpr int kTmemCols = 512;
constexpr int kMaxStages = 8;

struct TcArgs {
    float2 *vis;
    int *status;
    long long total_ch;               // SB * C
    long long n_items;                // total_ch * nrb
    long long B;                      // baselines
    int N, I_pad, planes, nk, nrb, rload, ncm, acc_stride, nacc, stages;
    unsigned stage_bytes;
    unsigned bf16;                    // operand type: 0 F16, 1 BF16
    float inv_scale2;
    long long timeout_cycles;
    int no_tma;                       // failure-detection test: issue no loads
};

// ---- PTX wrappers ----------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait: false on timeout (sets abort + status) or when another role aborted.
__device__ __forceinline__ bool wait_bounded(unsigned bar, unsigned parity, volatile int *abort_flag,
                                             const TcArgs &a, int code)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > a.timeout_cycles) {
            *abort_flag = 1;
            atomicCAS(a.status, 0, code);
            atomicExch(a.status + 1, (int)blockIdx.x);
            return false;
        }
    }
    return true;
}
// Bounded wait used while draining after an abort (ignores the abort flag).
__device__ __forceinline__ void drain_wait(unsigned bar, unsigned parity, long long budget)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > budget) return;
}

__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *map, unsigned bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO); LBO unused for this layout; descriptor version 1.
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr)
{
    return (unsigned long long)((addr & 0x3FFFF) >> 4) | ((unsigned long long)(16 >> 4) << 16) |
           ((unsigned long long)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor, kind::f16: D = F32, A/B = F16 or BF16, both K-major.
__device__ __forceinline__ unsigned make_idesc(unsigned bf16, int n, bool neg_a)
{
    return (1u << 4) | (bf16 << 7) | (bf16 << 10) | ((neg_a ? 1u : 0u) << 13) |
           ((unsigned)(n >> 3) << 17) | ((unsigned)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(unsigned d_tmem, unsigned long long adesc, unsigned long long bdesc,
                                        unsigned idesc, unsigned accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
                 : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16])
{
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---- the kernel --------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1)
xcorr_tc_kernel(const __grid_constant__ CUtensorMap tmap, const TcArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte alignment for the 128-byte-swizzled operand tiles
    const unsigned base_u32 = smem_u32(smem_raw);
    const unsigned pad = (1024 - (base_u32 & 1023)) & 1023;
    unsigned char *smem = smem_raw + pad;
    const unsigned tiles_u32 = base_u32 + pad;
    unsigned char *ctrl = smem + (size_t)a.stages * a.stage_bytes;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(ctrl);
    // barriers: full[S], empty[S], acc_full[2], acc_empty[2], drain
    const unsigned bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (kMaxStages + s); };
    auto accf_bar = [&](int b) { return bar0 + 8u * (2 * kMaxStages + b); };
    auto acce_bar = [&](int b) { return bar0 + 8u * (2 * kMaxStages + 2 + b); };
    const unsigned drain_bar = bar0 + 8u * (2 * kMaxStages + 4);
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(ctrl + 8 * (2 * kMaxStages + 5));
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(full_bar(s), 1);
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
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const unsigned tmem_base = *tmem_slot;

    if (warp == 0) {
        // ================= TMA producer =================
        if (lane == 0) {
            long long it = 0;
            bool ok = true;
            for (long long w = blockIdx.x; w < a.n_items && ok; w += gridDim.x) {
                const long long gch = w / a.nrb;
                const int rb = (int)(w % a.nrb);
                for (int kc = 0; kc < a.nk; ++kc, ++it) {
                    const int s = (int)(it % a.stages);
                    const unsigned ph = (unsigned)((it / a.stages) & 1);
                    if (!wait_bounded(empty_bar(s), ph ^ 1u, abort_flag, a, 1)) { ok = false; break; }
                    if (a.no_tma) continue;
                    mbar_arrive_expect_tx(full_bar(s), a.stage_bytes);
                    const unsigned dst = tiles_u32 + (unsigned)s * a.stage_bytes;
                    for (int pl = 0; pl < a.planes; ++pl)
                        tma_load_3d(dst + (unsigned)pl * a.rload * 128u, &tmap, full_bar(s), kc * kBK, 128 * rb,
                                    (int)(gch * a.planes + pl));
                }
            }
            if (!ok && !a.no_tma) {
                // drain: the last `stages` loads issued may still be in flight
                const long long first = it > a.stages ? it - a.stages : 0;
                for (long long u = first; u < it; ++u)
                    drain_wait(full_bar((int)(u % a.stages)), (unsigned)((u / a.stages) & 1), a.timeout_cycles);
            }
        }
    } else if (warp == 1) {
        // ================= MMA issuer =================
        if (lane == 0) {
            long long it = 0, acc_it = 0;
            bool ok = true, issued = false;
            for (long long w = blockIdx.x; w < a.n_items && ok; w += gridDim.x, ++acc_it) {
                const int rb = (int)(w % a.nrb);
                const int ncols = a.I_pad - 128 * rb;
                const unsigned idesc = make_idesc(a.bf16, ncols, false);
                const unsigned idesc_neg = make_idesc(a.bf16, ncols, true);
                const int ab = (int)(acc_it % a.nacc);
                const unsigned aph = (unsigned)((acc_it / a.nacc) & 1);
                if (!wait_bounded(acce_bar(ab), aph ^ 1u, abort_flag, a, 2)) { ok = false; break; }
                tc_fence_after();
                const unsigned d_re = tmem_base + (unsigned)(ab * a.acc_stride);
                const unsigned d_im = d_re + (unsigned)a.ncm;
                for (int kc = 0; kc < a.nk; ++kc, ++it) {
                    const int s = (int)(it % a.stages);
                    const unsigned ph = (unsigned)((it / a.stages) & 1);
                    if (!wait_bounded(full_bar(s), ph, abort_flag, a, 2)) { ok = false; break; }
                    tc_fence_after();
                    const unsigned tile = tiles_u32 + (unsigned)s * a.stage_bytes;
                    const unsigned plane_bytes = (unsigned)a.rload * 128u;
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const unsigned acc = (kc | kk) ? 1u : 0u;
                        // descriptors of each plane at this K step (A and B share the tile)
                        const unsigned long long r0 = smem_desc(tile + 0 * plane_bytes + kk * 32);
                        const unsigned long long j0 = smem_desc(tile + 1 * plane_bytes + kk * 32);
                        if (a.planes == 2) {
                            mma_f16(d_re, r0, r0, idesc, acc);
                            mma_f16(d_re, j0, j0, idesc, 1u);
                            mma_f16(d_im, j0, r0, idesc, acc);
                            mma_f16(d_im, r0, j0, idesc_neg, 1u);
                        } else {
                            const unsigned long long r1 = smem_desc(tile + 2 * plane_bytes + kk * 32);
                            const unsigned long long j1 = smem_desc(tile + 3 * plane_bytes + kk * 32);
                            // (hi, hi)
                            mma_f16(d_re, r0, r0, idesc, acc);
                            mma_f16(d_re, j0, j0, idesc, 1u);
                            mma_f16(d_im, j0, r0, idesc, acc);
                            mma_f16(d_im, r0, j0, idesc_neg, 1u);
                            // (hi, lo)
                            mma_f16(d_re, r0, r1, idesc, 1u);
                            mma_f16(d_re, j0, j1, idesc, 1u);
                            mma_f16(d_im, j0, r1, idesc, 1u);
                            mma_f16(d_im, r0, j1, idesc_neg, 1u);
                            // (lo, hi)
                            mma_f16(d_re, r1, r0, idesc, 1u);
                            mma_f16(d_re, j1, j0, idesc, 1u);
                            mma_f16(d_im, j1, r0, idesc, 1u);
                            mma_f16(d_im, r1, j0, idesc_neg, 1u);
                        }
                    }
                    issued = true;
                    mma_commit(empty_bar(s));          // stage free once these MMAs have read it
                }
                if (!ok) break;
                mma_commit(accf_bar(ab));              // accumulator ready for the epilogue
            }
            if (!ok && issued) {
                mma_commit(drain_bar);
                drain_wait(drain_bar, 0, a.timeout_cycles);
            }
        }
        __syncwarp();
    } else {
        // ================= epilogue (warps 2..5) =================
        const int qd = warp & 3;                      // TMEM lane quadrant of this warp
        long long acc_it = 0;
        for (long long w = blockIdx.x; w < a.n_items; w += gridDim.x, ++acc_it) {
            const long long gch = w / a.nrb;
            const int rb = (int)(w % a.nrb);
            const int ncols = a.I_pad - 128 * rb;
            const int ab = (int)(acc_it % a.nacc);
            const unsigned aph = (unsigned)((acc_it / a.nacc) & 1);
            const bool got = wait_bounded(accf_bar(ab), aph, abort_flag, a, 3);
            if (!__all_sync(0xffffffffu, got)) break;   // warp-uniform exit
            tc_fence_after();
            const int ia = 128 * rb + 32 * qd + lane;  // this lane's row input
            const int i = ia >> 1, p = ia & 1;
            const int i_warp_min = (128 * rb + 32 * qd) >> 1;
            const unsigned lane_off = (unsigned)(32 * qd) << 16;
            const unsigned t_re = tmem_base + lane_off + (unsigned)(ab * a.acc_stride);
            const unsigned t_im = t_re + (unsigned)a.ncm;
            float2 *vrow = a.vis + gch * a.B * 4;
            for (int cc = 0; cc < ncols / 16; ++cc) {
                const int j0 = 64 * rb + 8 * cc;      // first station of this 16-column chunk
                if (j0 >= a.N) break;
                if (j0 + 7 < i_warp_min) continue;    // whole chunk below the diagonal for this warp
                float re[16], im[16];
                tmem_ld16(t_re + 16 * cc, re);
                tmem_ld16(t_im + 16 * cc, im);
                tmem_ld_wait();
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const int j = j0 + jj;
                    if (i <= j && j < a.N) {
                        const long long b = (long long)j * (j + 1) / 2 + i;
                        const float s = a.inv_scale2;
                        *reinterpret_cast<float4 *>(vrow + b * 4 + 2 * p) =
                            make_float4(re[2 * jj] * s, im[2 * jj] * s, re[2 * jj + 1] * s, im[2 * jj + 1] * s);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce_bar(ab));
        }
    }

    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                     : "memory");
    }
}

// ---- host side ----------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

}  // namespace

bool xtc_plan(const Handle &h, int *rload, int *stages, unsigned *stage_bytes)
{
    const int planes = h.p.precision == FX_F16_SPLIT ? 4 : 2;
    if (h.I_pad > 256) return false;
    const int rl = h.I_pad > 128 ? h.I_pad : 128;
    const unsigned sb = (unsigned)(planes * rl * 128);
    const int st = (int)((200u * 1024u) / sb);
    if (st < 2) return false;
    *rload = rl;
    *stages = st > kMaxStages ? kMaxStages : st;
    *stage_bytes = sb;
    return true;
}

cudaError_t launch_xcorr_tc(const Handle &h, const void *corr, float2 *vis, cudaStream_t st)
{
    int rload, stages;
    unsigned stage_bytes;
    if (!xtc_plan(h, &rload, &stages, &stage_bytes)) return cudaErrorNotSupported;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int planes = h.p.precision == FX_F16_SPLIT ? 4 : 2;
    const long long total_ch = (long long)h.p.n_subbands * h.p.n_channels;
    if (total_ch * planes > 0x7fffffffLL) return cudaErrorInvalidValue;

    CUtensorMap map;
    const cuuint64_t gdim[3] = {(cuuint64_t)h.S_pad, (cuuint64_t)h.I_pad, (cuuint64_t)(total_ch * planes)};
    const cuuint64_t gstride[2] = {(cuuint64_t)h.S_pad * 2, (cuuint64_t)h.S_pad * 2 * h.I_pad};
    const cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)rload, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void *>(corr), gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;

    TcArgs a;
    a.vis = vis;
    a.status = h.d_status;
    a.total_ch = total_ch;
    a.nrb = (h.I_pad + 127) / 128;
    a.n_items = total_ch * a.nrb;
    a.B = h.B;
    a.N = h.p.n_stations;
    a.I_pad = h.I_pad;
    a.planes = planes;
    a.nk = h.S_pad / kBK;
    a.rload = rload;
    a.ncm = (h.I_pad + 31) / 32 * 32;
    a.acc_stride = 2 * a.ncm;
    a.nacc = (2 * a.acc_stride <= kTmemCols) ? 2 : 1;
    a.stages = stages;
    a.stage_bytes = stage_bytes;
    a.bf16 = h.p.precision == FX_BF16 ? 1u : 0u;
    a.inv_scale2 = 1.0f / (h.operand_scale * h.operand_scale);
    a.timeout_cycles = h.tc_timeout_cycles;
    a.no_tma = h.tc_test_no_tma;

    const size_t ctrl = 8 * (2 * kMaxStages + 5) + 16;
    const size_t smem = 1024 + (size_t)stages * stage_bytes + ctrl;
    cudaError_t e = cudaFuncSetAttribute(xcorr_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long grid = a.n_items < h.num_sms ? a.n_items : h.num_sms;
    xcorr_tc_kernel<<<(unsigned)grid, kThreads, smem, st>>>(map, a);
    return cudaGetLastError();
}

}  // namespace fxi
