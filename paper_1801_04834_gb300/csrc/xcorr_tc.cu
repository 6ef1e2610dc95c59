// xcorr_tc.cu -- X-stage correlator on the 5th-generation (tcgen05) tensor
// cores: FP16 or BF16 operands, FP32 accumulation in tensor memory (TMEM),
// for one job (fx_correlate) or a batch of uneven jobs in one persistent
// launch (fx_correlate_batched).
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
// Work items. Rows of the I_pad x I_pad product come in blocks of 128 inputs
// (M = 128); only column ranges at or right of the row block are computed.
//   wide  : one item per (channel, row block rb): columns [128 rb, I_pad),
//           N = I_pad - 128 rb <= 256. One TMA box per plane holds rows
//           [128 rb, 128 rb + R) x 64 spectra; A and B are the same tile.
//   split : items (channel, rb, cb): columns [128 rb + NT cb, +NT) with
//           NT = 64 or 128. A is a 128-row box; B is either inside A (the
//           diagonal tile) or a second NT-row box. Any station count; the
//           accumulators (2 x NT columns) are always double buffered.
// A batch carries up to kMaxJobs jobs (each its own tensor maps, shape and
// output) and a device list of items sorted by cost (longest first), walked
// round-robin by the persistent CTAs.
//
// Warp roles (192 threads, persistent, one CTA per SM):
//   warp 0     TMA producer: one elected thread fills a ring of STAGES tiles
//   warp 1     TMEM allocator + MMA issuer: one elected thread issues
//              tcgen05.mma and tcgen05.commit (stage release, accumulator full)
//   warps 2-5  epilogue: tcgen05.ld of their 32-lane TMEM quadrant, scale by
//              1/operand_scale^2, store the upper-triangle baselines only
//
// Accumulator chains. FP16/BF16 accumulate an item's whole block in one TMEM
// accumulator. Split FP16 restarts it every 4 stages (256 spectra): the tensor
// core's FP32 accumulation truncates each addition, so a long chain drifts by
// about 2^-24 of the running value per MMA, more than the lo planes win back.
// The epilogue stores an item's first chain and adds the later ones with
// vector FP32 reductions in L2 (red.global.add.v4.f32, round to nearest);
// each entry has one owner lane, which issues its chains in order.
//
// Every mbarrier wait is bounded (clock64 budget). On expiry the thread
// records a code in the status word and raises a shared abort flag; all roles
// leave their loops, the producer waits (bounded) for the loads it still has
// in flight, the MMA thread waits (bounded) for its issued MMAs, and the TMEM
// is freed before the CTA exits.
#include <cuda.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"

namespace fxi {
namespace {

using namespace tc;

constexpr int kBK = 64;               // spectra per stage (128-byte rows of 16-bit values)
constexpr int kThreads = 192;
constexpr int kTmemCols = 512;
constexpr int kMaxStages = 8;
constexpr int kMaxJobs = 64;
constexpr unsigned kSmemBudget = 200u * 1024u;

struct TcJob {
    CUtensorMap mapA;                 // box rows ra_job (wide: max(128, I_pad); split: 128)
    CUtensorMap mapB;                 // split: box rows NT
    float2 *vis;
    long long B;                      // baselines
    long long n_ch;                   // SB * C
    int N, I_pad, nk, items_per_ch;
    int ra;                           // rows of this job's A box
};

struct TcCommon {
    int *status;
    const int4 *items;                // (job, rb, cb, gch) sorted by cost, or null for one job
    long long n_items;
    int mode;                         // 0 wide, 1 split
    int NT;                           // split column tile
    int planes, stages;
    unsigned stage_bytes;
    int ra_max;                       // rows reserved per plane for the A region
    int rbr;                          // rows reserved per plane for the B region (split)
    int ncm, acc_stride, nacc;
    unsigned bf16;                    // operand type: 0 F16, 1 BF16
    float inv_scale2;
    long long timeout_cycles;
    int no_tma;                       // failure-detection test: issue no loads
    int accumulate;                   // add to the visibilities instead of writing them
    int chunk;                        // stages per accumulator chain (0: the whole item)
};

template <int MAXJ>
struct TcParams {
    TcJob jobs[MAXJ];
    TcCommon c;
};

struct Item {
    int job, rb, cb;
    long long gch;
};

// Bounded wait: false on timeout (sets abort + status) or when another role aborted.
__device__ __forceinline__ bool wait_bounded(unsigned bar, unsigned parity, volatile int *abort_flag,
                                             const TcCommon &a, int code)
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
// Vector FP32 reduction into global memory (performed in L2, round to nearest).
__device__ __forceinline__ void red_add4(float2 *addr, float4 v)
{
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w)
                 : "memory");
}

// ---- work-item decoding --------------------------------------------------------
template <int MAXJ>
__device__ __forceinline__ Item decode(const TcParams<MAXJ> &P, long long w)
{
    Item it;
    if (P.c.items) {
        const int4 v = P.c.items[w];
        it.job = v.x;
        it.rb = v.y;
        it.cb = v.z;
        it.gch = v.w;
        return it;
    }
    const TcJob &J = P.jobs[0];
    it.job = 0;
    it.gch = w / J.items_per_ch;
    int r = (int)(w % J.items_per_ch);
    if (P.c.mode == 0) {
        it.rb = r;
        it.cb = 0;
    } else {
        int rb = 0;
        for (;;) {
            const int n = (J.I_pad - 128 * rb + P.c.NT - 1) / P.c.NT;
            if (r < n) break;
            r -= n;
            ++rb;
        }
        it.rb = rb;
        it.cb = r;
    }
    return it;
}

// column range of an item
template <int MAXJ>
__device__ __forceinline__ void item_cols(const TcParams<MAXJ> &P, const TcJob &J, const Item &it, int &row0,
                                          int &col0, int &ncols)
{
    row0 = 128 * it.rb;
    if (P.c.mode == 0) {
        col0 = row0;
        ncols = J.I_pad - row0;
    } else {
        col0 = row0 + P.c.NT * it.cb;
        ncols = min(P.c.NT, J.I_pad - col0);
    }
}

// ---- the kernel --------------------------------------------------------------
template <int MAXJ>
__global__ void __launch_bounds__(kThreads, 1) xcorr_tc_kernel(const __grid_constant__ TcParams<MAXJ> P)
{
    const TcCommon &a = P.c;
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
    const unsigned a_region = (unsigned)a.planes * a.ra_max * 128u;   // bytes of the A part of a stage
    const unsigned a_plane = (unsigned)a.ra_max * 128u;
    const unsigned b_plane = (unsigned)a.rbr * 128u;

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
                const Item itm = decode(P, w);
                const TcJob &J = P.jobs[itm.job];
                int row0, col0, ncols;
                item_cols(P, J, itm, row0, col0, ncols);
                const bool diag = (col0 == row0);
                const unsigned tx = (unsigned)a.planes * 128u * (J.ra + (diag ? 0 : a.NT));
                for (int kc = 0; kc < J.nk; ++kc, ++it) {
                    const int s = (int)(it % a.stages);
                    const unsigned ph = (unsigned)((it / a.stages) & 1);
                    if (!wait_bounded(empty_bar(s), ph ^ 1u, abort_flag, a, 1)) { ok = false; break; }
                    if (a.no_tma) continue;
                    mbar_arrive_expect_tx(full_bar(s), tx);
                    const unsigned dst = tiles_u32 + (unsigned)s * a.stage_bytes;
                    for (int pl = 0; pl < a.planes; ++pl) {
                        const int z = (int)(itm.gch * a.planes + pl);
                        tma_load_3d(dst + (unsigned)pl * a_plane, &J.mapA, full_bar(s), kc * kBK, row0, z);
                        if (!diag)
                            tma_load_3d(dst + a_region + (unsigned)pl * b_plane, &J.mapB, full_bar(s), kc * kBK,
                                        col0, z);
                    }
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
            for (long long w = blockIdx.x; w < a.n_items && ok; w += gridDim.x) {
                const Item itm = decode(P, w);
                const TcJob &J = P.jobs[itm.job];
                int row0, col0, ncols;
                item_cols(P, J, itm, row0, col0, ncols);
                const bool diag = (col0 == row0);
                const unsigned idesc = make_idesc(a.bf16, ncols, false);
                const unsigned idesc_neg = make_idesc(a.bf16, ncols, true);
                const int clen = a.chunk > 0 ? a.chunk : J.nk;   // stages per accumulator chain
                for (int k0 = 0; k0 < J.nk && ok; k0 += clen, ++acc_it) {
                    const int ab = (int)(acc_it % a.nacc);
                    const unsigned aph = (unsigned)((acc_it / a.nacc) & 1);
                    if (!wait_bounded(acce_bar(ab), aph ^ 1u, abort_flag, a, 2)) { ok = false; break; }
                    tc_fence_after();
                    const unsigned d_re = tmem_base + (unsigned)(ab * a.acc_stride);
                    const unsigned d_im = d_re + (unsigned)a.ncm;
                    const int k1 = min(J.nk, k0 + clen);
                    for (int kc = k0; kc < k1; ++kc, ++it) {
                        const int s = (int)(it % a.stages);
                        const unsigned ph = (unsigned)((it / a.stages) & 1);
                        if (!wait_bounded(full_bar(s), ph, abort_flag, a, 2)) { ok = false; break; }
                        tc_fence_after();
                        const unsigned tile = tiles_u32 + (unsigned)s * a.stage_bytes;
                        const unsigned btile = diag ? tile : tile + a_region;
                        const unsigned bpl = diag ? a_plane : b_plane;
#pragma unroll
                        for (int kk = 0; kk < kBK / 16; ++kk) {
                            const unsigned acc = (kc != k0 || kk) ? 1u : 0u;
                            // A operand rows = the row block, B operand rows = the column block
                            const unsigned long long ar0 = smem_desc(tile + 0 * a_plane + kk * 32);
                            const unsigned long long aj0 = smem_desc(tile + 1 * a_plane + kk * 32);
                            const unsigned long long br0 = smem_desc(btile + 0 * bpl + kk * 32);
                            const unsigned long long bj0 = smem_desc(btile + 1 * bpl + kk * 32);
                            if (a.planes == 2) {
                                mma_f16(d_re, ar0, br0, idesc, acc);
                                mma_f16(d_re, aj0, bj0, idesc, 1u);
                                mma_f16(d_im, aj0, br0, idesc, acc);
                                mma_f16(d_im, ar0, bj0, idesc_neg, 1u);
                            } else {
                                const unsigned long long ar1 = smem_desc(tile + 2 * a_plane + kk * 32);
                                const unsigned long long aj1 = smem_desc(tile + 3 * a_plane + kk * 32);
                                const unsigned long long br1 = smem_desc(btile + 2 * bpl + kk * 32);
                                const unsigned long long bj1 = smem_desc(btile + 3 * bpl + kk * 32);
                                // (hi, hi)
                                mma_f16(d_re, ar0, br0, idesc, acc);
                                mma_f16(d_re, aj0, bj0, idesc, 1u);
                                mma_f16(d_im, aj0, br0, idesc, acc);
                                mma_f16(d_im, ar0, bj0, idesc_neg, 1u);
                                // (hi, lo)
                                mma_f16(d_re, ar0, br1, idesc, 1u);
                                mma_f16(d_re, aj0, bj1, idesc, 1u);
                                mma_f16(d_im, aj0, br1, idesc, 1u);
                                mma_f16(d_im, ar0, bj1, idesc_neg, 1u);
                                // (lo, hi)
                                mma_f16(d_re, ar1, br0, idesc, 1u);
                                mma_f16(d_re, aj1, bj0, idesc, 1u);
                                mma_f16(d_im, aj1, br0, idesc, 1u);
                                mma_f16(d_im, ar1, bj0, idesc_neg, 1u);
                            }
                        }
                        issued = true;
                        mma_commit(empty_bar(s));          // stage free once these MMAs have read it
                    }
                    if (!ok) break;
                    mma_commit(accf_bar(ab));              // accumulator ready for the epilogue
                }
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
        bool live = true;
        for (long long w = blockIdx.x; w < a.n_items && live; w += gridDim.x) {
            const Item itm = decode(P, w);
            const TcJob &J = P.jobs[itm.job];
            int row0, col0, ncols;
            item_cols(P, J, itm, row0, col0, ncols);
            const int clen = a.chunk > 0 ? a.chunk : J.nk;
            const int ia = row0 + 32 * qd + lane;       // this lane's row input
            const int i = ia >> 1, p = ia & 1;
            const int i_warp_min = (row0 + 32 * qd) >> 1;
            const unsigned lane_off = (unsigned)(32 * qd) << 16;
            float2 *vrow = J.vis + itm.gch * J.B * 4;
            for (int k0 = 0; k0 < J.nk; k0 += clen, ++acc_it) {
                const int ab = (int)(acc_it % a.nacc);
                const unsigned aph = (unsigned)((acc_it / a.nacc) & 1);
                const bool got = wait_bounded(accf_bar(ab), aph, abort_flag, a, 3);
                if (!__all_sync(0xffffffffu, got)) {   // warp-uniform exit
                    live = false;
                    break;
                }
                tc_fence_after();
                // the first chain of an item is written (or, accumulating, added by
                // load + add + store); later chains are added by FP32 reductions in L2
                const bool first = (k0 == 0);
                const unsigned t_re = tmem_base + lane_off + (unsigned)(ab * a.acc_stride);
                const unsigned t_im = t_re + (unsigned)a.ncm;
                for (int cc = 0; cc < ncols / 16; ++cc) {
                    const int j0 = (col0 >> 1) + 8 * cc;   // first station of this 16-column chunk
                    if (j0 >= J.N) break;
                    if (j0 + 7 < i_warp_min) continue;    // whole chunk below the diagonal for this warp
                    float re[16], im[16];
                    tmem_ld16(t_re + 16 * cc, re);
                    tmem_ld16(t_im + 16 * cc, im);
                    // accumulating: the sums of earlier time pieces, loaded while TMEM is read
                    float4 old[8];
                    if (a.accumulate && first) {
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            const int j = j0 + jj;
                            old[jj] = (i <= j && j < J.N) ? *reinterpret_cast<const float4 *>(
                                                                vrow + ((long long)j * (j + 1) / 2 + i) * 4 + 2 * p)
                                                          : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    }
                    tmem_ld_wait();
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        const int j = j0 + jj;
                        if (i <= j && j < J.N) {
                            const long long b = (long long)j * (j + 1) / 2 + i;
                            const float s = a.inv_scale2;
                            float4 v = make_float4(re[2 * jj] * s, im[2 * jj] * s, re[2 * jj + 1] * s,
                                                   im[2 * jj + 1] * s);
                            float2 *dst = vrow + b * 4 + 2 * p;
                            if (!first) {
                                red_add4(dst, v);
                                continue;
                            }
                            if (a.accumulate) {
                                v.x += old[jj].x;
                                v.y += old[jj].y;
                                v.z += old[jj].z;
                                v.w += old[jj].w;
                            }
                            *reinterpret_cast<float4 *>(dst) = v;
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
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Shape of one job as the kernel sees it.
struct JobShape {
    int N, I_pad, S_pad;
    long long n_ch;
    const void *corr;
    float2 *vis;
};

// Launch configuration (the "tile plan"): item shape, pipeline depth, order.
struct TcConfig {
    int mode = 0;      // 0 wide, 1 split
    int NT = 128;      // split column tile
    int stages = 0;    // 0: as many as fit
    int sorted = 1;    // batch: items longest first
};

int planes_of(int precision) { return precision == FX_F16_SPLIT ? 4 : 2; }

int job_ra(const TcConfig &cfg, int I_pad) { return cfg.mode == 0 ? std::max(128, I_pad) : 128; }

// Can this configuration run these jobs? Fills stage geometry.
bool geometry(const TcConfig &cfg, int precision, const std::vector<JobShape> &jobs, TcCommon &c)
{
    const int planes = planes_of(precision);
    int ra_max = 128, ncm = 0;
    for (const auto &j : jobs) {
        if (cfg.mode == 0 && j.I_pad > 256) return false;
        ra_max = std::max(ra_max, job_ra(cfg, j.I_pad));
        ncm = std::max(ncm, cfg.mode == 0 ? j.I_pad : std::min(cfg.NT, j.I_pad));
    }
    if (cfg.mode == 1 && cfg.NT != 64 && cfg.NT != 128) return false;
    c.mode = cfg.mode;
    c.NT = cfg.NT;
    c.planes = planes;
    c.ra_max = ra_max;
    c.rbr = cfg.mode == 1 ? cfg.NT : 0;
    c.stage_bytes = (unsigned)(planes * (ra_max + c.rbr) * 128);
    int fit = (int)(kSmemBudget / c.stage_bytes);
    if (fit < 2) return false;
    c.stages = std::min(kMaxStages, cfg.stages > 0 ? std::min(cfg.stages, fit) : fit);
    c.ncm = (ncm + 31) / 32 * 32;
    c.acc_stride = 2 * c.ncm;
    c.nacc = (2 * c.acc_stride <= kTmemCols) ? 2 : 1;
    // Split FP16: the tensor core's FP32 accumulation truncates each addition
    // (about 2^-24 of the running value per MMA, 24 MMAs per accumulator and
    // 64-spectrum stage), which would undo what the lo planes win back over a
    // long integration (3.8e-5 over 3072 spectra in one chain); chains of 4
    // stages (256 spectra) are added in IEEE FP32 instead (3.1e-6, 6% more
    // time for the L2 reductions; 128-spectrum chains 1.5e-6 at 13% more).
    // Plain FP16/BF16 keep one chain per item: they are the fast forms, well
    // inside their bounds.
    c.chunk = (planes == 4 && c.nacc == 2) ? 4 : 0;
    c.bf16 = precision == FX_BF16 ? 1u : 0u;
    return true;
}

int items_per_ch(const TcConfig &cfg, int I_pad)
{
    const int nrb = (I_pad + 127) / 128;
    if (cfg.mode == 0) return nrb;
    int n = 0;
    for (int rb = 0; rb < nrb; ++rb) n += (I_pad - 128 * rb + cfg.NT - 1) / cfg.NT;
    return n;
}

bool encode_job(const TcConfig &cfg, int precision, const JobShape &js, int nk, TcJob &J)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const int planes = planes_of(precision);
    const cuuint64_t gdim[3] = {(cuuint64_t)js.S_pad, (cuuint64_t)js.I_pad, (cuuint64_t)(js.n_ch * planes)};
    const cuuint64_t gstride[2] = {(cuuint64_t)js.S_pad * 2, (cuuint64_t)js.S_pad * 2 * js.I_pad};
    const cuuint32_t estr[3] = {1, 1, 1};
    J.ra = job_ra(cfg, js.I_pad);
    const cuuint32_t boxA[3] = {(cuuint32_t)kBK, (cuuint32_t)J.ra, 1};
    CUresult r = enc(&J.mapA, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void *>(js.corr), gdim, gstride, boxA,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    if (cfg.mode == 1) {
        const cuuint32_t boxB[3] = {(cuuint32_t)kBK, (cuuint32_t)cfg.NT, 1};
        r = enc(&J.mapB, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void *>(js.corr), gdim, gstride, boxB, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    } else {
        J.mapB = J.mapA;
    }
    J.vis = js.vis;
    J.B = (long long)js.N * (js.N + 1) / 2;
    J.n_ch = js.n_ch;
    J.N = js.N;
    J.I_pad = js.I_pad;
    J.nk = nk;
    J.items_per_ch = items_per_ch(cfg, js.I_pad);
    return true;
}

template <int MAXJ>
cudaError_t launch_params(const TcParams<MAXJ> &P, int num_sms, cudaStream_t st)
{
    const size_t ctrl = 8 * (2 * kMaxStages + 5) + 16;
    const size_t smem = 1024 + (size_t)P.c.stages * P.c.stage_bytes + ctrl;
    cudaError_t e = cudaFuncSetAttribute(xcorr_tc_kernel<MAXJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long grid = std::min<long long>(P.c.n_items, num_sms);
    if (grid <= 0) return cudaSuccess;
    xcorr_tc_kernel<MAXJ><<<(unsigned)grid, kThreads, smem, st>>>(P);
    return cudaGetLastError();
}

TcConfig default_config(int precision, int I_pad)
{
    TcConfig cfg;
    const int planes = planes_of(precision);
    if (planes == 2) {
        cfg.mode = I_pad <= 256 ? 0 : 1;
        cfg.NT = 128;
    } else {
        cfg.mode = I_pad <= 128 ? 0 : 1;
        cfg.NT = 64;
    }
    return cfg;
}

void fill_common(TcCommon &c, int *status, float scale, long long timeout, int no_tma)
{
    c.status = status;
    c.inv_scale2 = 1.0f / (scale * scale);
    c.timeout_cycles = timeout;
    c.no_tma = no_tma;
    c.accumulate = 0;
}

}  // namespace

bool xtc_plan(const Handle &h, int *rload, int *stages, unsigned *stage_bytes)
{
    TcConfig cfg = default_config(h.p.precision, h.I_pad);
    std::vector<JobShape> js(1);
    js[0].I_pad = h.I_pad;
    js[0].N = h.p.n_stations;
    TcCommon c{};
    if (!geometry(cfg, h.p.precision, js, c)) return false;
    *rload = c.ra_max;
    *stages = c.stages;
    *stage_bytes = c.stage_bytes;
    return true;
}

cudaError_t launch_xcorr_tc(const Handle &h, const void *corr, float2 *vis, cudaStream_t st, bool accumulate)
{
    TcConfig cfg = default_config(h.p.precision, h.I_pad);
    std::vector<JobShape> js(1);
    js[0] = JobShape{h.p.n_stations, h.I_pad, h.S_pad, (long long)h.p.n_subbands * h.p.n_channels, corr, vis};
    if (js[0].n_ch * planes_of(h.p.precision) > 0x7fffffffLL) return cudaErrorInvalidValue;
    TcParams<1> P;
    memset(&P, 0, sizeof(P));
    if (!geometry(cfg, h.p.precision, js, P.c)) return cudaErrorNotSupported;
    if (!encode_job(cfg, h.p.precision, js[0], h.S_pad / kBK, P.jobs[0])) return cudaErrorInvalidValue;
    fill_common(P.c, h.d_status, h.operand_scale, h.tc_timeout_cycles, h.tc_test_no_tma);
    P.c.accumulate = accumulate ? 1 : 0;
    P.c.items = nullptr;
    P.c.n_items = js[0].n_ch * P.jobs[0].items_per_ch;
    return launch_params(P, h.num_sms, st);
}

}  // namespace fxi

// ============================ batched form =====================================
// A plan owns the device item list, the per-job tensor maps (baked into the
// launch parameters) and the status word; fx_correlate_batched is one kernel
// launch with no host work beyond it, so it can be captured in a CUDA graph.

struct fx_batch {
    int precision = FX_F16;
    float scale = 1.f;
    int device = 0;
    int num_sms = 152;
    std::vector<fxi::JobShape> jobs;
    std::vector<int> nk;
    fxi::TcConfig cfg;
    fxi::TcParams<fxi::kMaxJobs> P;
    int4 *d_items = nullptr;
    long long max_items = 0;
    int *d_status = nullptr;
    std::string signature;
    char desc[256] = "";
};

namespace fxi {
namespace {

std::map<std::string, TcConfig> &tune_cache()
{
    static std::map<std::string, TcConfig> m;
    return m;
}
std::mutex &tune_mu()
{
    static std::mutex m;
    return m;
}

long long batch_items(const fx_batch &b, const TcConfig &cfg)
{
    long long n = 0;
    for (const auto &j : b.jobs) n += j.n_ch * items_per_ch(cfg, j.I_pad);
    return n;
}

// Build the launch parameters and the item list for one configuration.
cudaError_t batch_prepare(fx_batch &b, const TcConfig &cfg, cudaStream_t st)
{
    fx_batch &B = b;
    memset(&B.P, 0, sizeof(B.P));
    if (!geometry(cfg, B.precision, B.jobs, B.P.c)) return cudaErrorNotSupported;
    std::vector<std::pair<long long, int4>> items;
    for (size_t j = 0; j < B.jobs.size(); ++j) {
        if (!encode_job(cfg, B.precision, B.jobs[j], B.nk[j], B.P.jobs[j])) return cudaErrorInvalidValue;
        const JobShape &js = B.jobs[j];
        const int nrb = (js.I_pad + 127) / 128;
        for (long long g = 0; g < js.n_ch; ++g)
            for (int rb = 0; rb < nrb; ++rb) {
                const int ncb = cfg.mode == 0 ? 1 : (js.I_pad - 128 * rb + cfg.NT - 1) / cfg.NT;
                for (int cb = 0; cb < ncb; ++cb) {
                    const int ncols = cfg.mode == 0 ? js.I_pad - 128 * rb
                                                    : std::min(cfg.NT, js.I_pad - 128 * rb - cfg.NT * cb);
                    const long long cost = (long long)B.nk[j] * (ncols + 32);
                    items.push_back({cost, make_int4((int)j, rb, cb, (int)g)});
                }
            }
    }
    if (cfg.sorted)
        std::stable_sort(items.begin(), items.end(),
                         [](const std::pair<long long, int4> &x, const std::pair<long long, int4> &y) {
                             return x.first > y.first;
                         });
    if ((long long)items.size() > B.max_items) return cudaErrorInvalidValue;
    std::vector<int4> flat(items.size());
    for (size_t k = 0; k < items.size(); ++k) flat[k] = items[k].second;
    cudaError_t e = cudaMemcpyAsync(B.d_items, flat.data(), sizeof(int4) * flat.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    fill_common(B.P.c, B.d_status, B.scale, 4000000000LL, 0);
    B.P.c.items = B.d_items;
    B.P.c.n_items = (long long)flat.size();
    B.cfg = cfg;
    snprintf(B.desc, sizeof(B.desc), "mode=%s NT=%d stages=%d acc_buffers=%d order=%s items=%lld",
             cfg.mode == 0 ? "wide" : "split", cfg.mode == 0 ? 0 : cfg.NT, B.P.c.stages, B.P.c.nacc,
             cfg.sorted ? "longest-first" : "job-major", B.P.c.n_items);
    return cudaSuccess;
}

}  // namespace
}  // namespace fxi

cudaError_t fxi_batch_create(const fx_job *jobs, int n_jobs, int precision, float scale, int num_sms,
                             fx_batch **out, const char **why)
{
    using namespace fxi;
    *out = nullptr;
    if (n_jobs < 1 || n_jobs > kMaxJobs) { *why = "n_jobs must be in 1..64"; return cudaErrorInvalidValue; }
    fx_batch *b = new fx_batch();
    b->precision = precision;
    b->scale = scale;
    b->num_sms = num_sms;
    cudaGetDevice(&b->device);
    std::string sig = std::to_string(precision) + ":";
    for (int j = 0; j < n_jobs; ++j) {
        const fx_job &J = jobs[j];
        JobShape s;
        s.N = J.n_stations;
        s.I_pad = (2 * J.n_stations + 15) / 16 * 16;
        s.S_pad = (J.n_spectra + 63) / 64 * 64;
        s.n_ch = (long long)J.n_subbands * J.n_channels;
        s.corr = J.d_corr;
        s.vis = reinterpret_cast<float2 *>(J.d_vis);
        if (s.n_ch * planes_of(precision) > 0x7fffffffLL || s.n_ch > 0x7fffffffLL) {
            delete b;
            *why = "job too large";
            return cudaErrorInvalidValue;
        }
        b->jobs.push_back(s);
        b->nk.push_back(s.S_pad / kBK);
        sig += std::to_string(s.N) + "," + std::to_string(s.n_ch) + "," + std::to_string(s.S_pad) + ";";
    }
    b->signature = sig;
    // room for the largest item list of any configuration (split NT=64 has the most)
    TcConfig most;
    most.mode = 1;
    most.NT = 64;
    b->max_items = batch_items(*b, most);
    cudaError_t e = cudaMalloc(&b->d_items, sizeof(int4) * b->max_items);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int) * 4);
    if (e != cudaSuccess) {
        cudaFree(b->d_items);
        cudaFree(b->d_status);
        delete b;
        *why = "device allocation failed";
        return e;
    }
    // a configuration tuned earlier for the same shapes, else the default
    TcConfig cfg;
    {
        std::lock_guard<std::mutex> lk(tune_mu());
        auto it = tune_cache().find(sig);
        if (it != tune_cache().end()) {
            cfg = it->second;
        } else {
            int I_max = 0;
            for (const auto &s : b->jobs) I_max = std::max(I_max, s.I_pad);
            cfg = default_config(precision, I_max);
        }
    }
    e = batch_prepare(*b, cfg, 0);
    if (e != cudaSuccess) {
        cudaFree(b->d_items);
        cudaFree(b->d_status);
        delete b;
        *why = "no kernel configuration fits these jobs";
        return e;
    }
    *out = b;
    return cudaSuccess;
}

cudaError_t fxi_batch_launch(fx_batch *b, cudaStream_t st) { return fxi::launch_params(b->P, b->num_sms, st); }

// Time every candidate configuration on the batch itself (CUDA events, `reps`
// launches each after one warm-up), keep the fastest, remember it for this
// batch signature.
cudaError_t fxi_batch_autotune(fx_batch *b, int reps, cudaStream_t st)
{
    using namespace fxi;
    std::vector<TcConfig> cands;
    for (int sorted = 1; sorted >= 0; --sorted) {
        TcConfig w;
        w.mode = 0;
        w.sorted = sorted;
        cands.push_back(w);
        for (int nt : {128, 64}) {
            TcConfig s;
            s.mode = 1;
            s.NT = nt;
            s.sorted = sorted;
            cands.push_back(s);
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    TcConfig best_cfg = b->cfg;
    for (const TcConfig &cfg : cands) {
        if (batch_prepare(*b, cfg, st) != cudaSuccess) continue;
        cudaError_t e = fxi_batch_launch(b, st);
        if (e != cudaSuccess) return e;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r) fxi_batch_launch(b, st);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) return e;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_cfg = cfg;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaError_t e = batch_prepare(*b, best_cfg, st);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(tune_mu());
    tune_cache()[b->signature] = best_cfg;
    return cudaSuccess;
}

void fxi_batch_destroy(fx_batch *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    cudaFree(b->d_items);
    cudaFree(b->d_status);
    delete b;
}

const char *fxi_batch_describe(const fx_batch *b) { return b->desc; }
int *fxi_batch_status(fx_batch *b) { return b->d_status; }
int fxi_batch_device(const fx_batch *b) { return b->device; }
