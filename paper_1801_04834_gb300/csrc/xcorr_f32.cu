// xcorr_f32.cu -- X-stage correlator in FP32 on the CUDA cores (FFMA).
//
// Paper, Sec. "Signal processing with GPU kernels": the last kernel correlates
// all pairs of antenna fields and integrates to ~1 s. Sec. "Hardware
// requirements and design priorities": the correlator is compute bound and
// can run close to peak.
//
//   V[sb][k][b(i,j)][2p+q] = sum_s Y[s][i,p] * conj(Y[s][j,q]),  i <= j
//
// Input is the FP32 corrected layout, spectrum-blocked:
// [SB][C][ceil16(S)/16][N][16][2] complex (one channel's block is contiguous;
// within it, 16 spectra x 2 pols of one station are one 256-byte run).
//
// Register tiling over the station triangle: a thread owns RS stations (rows,
// 2 RS inputs) x 4 stations (columns, 8 inputs). RS = 2: 32 complex
// accumulators, 64 packed FP32 FMAs (FFMA2) per time sample against 6
// shared-memory vector loads; RS = 4: 64 accumulators, 128 FFMA2 against 8
// loads (fewer loads and operand copies per FMA, fewer threads per SM). Tiles
// (row block r, column quad q) are kept only where some pair i <= j exists
// (RS r <= 4q+3): for 64 stations 272 (RS = 2) or 136 (RS = 4) tiles, 4.6%
// more MACs than the triangle.
//
// Threads are numbered over the flattened (channel, tile) index, up to 512 per
// CTA (16 warps, 4 per scheduler), so a CTA covers the tiles of one to a few
// channels whatever the station count; it streams the time samples of every
// channel it touches through shared memory in chunks of KC samples with
// double-buffered cp.async (consecutive threads copy consecutive spectra of
// one station, so each warp reads whole 256-byte runs; time rows are padded
// by one 16-byte entry so those copies land on distinct banks). Within a time
// row the 16-byte station entries are
// grouped by station index: RS = 2 stores
// [even stations][odd stations], RS = 4 stores [stations = 0 mod 4][1 mod 4]
// [2 mod 4][3 mod 4], so the row loads of consecutive row tiles fall on
// consecutive 16-byte words (no bank conflicts); column loads are mostly
// broadcasts.
#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace fxi {
namespace {

constexpr int kMaxThreads = 512;   // 16 warps
constexpr size_t kSmemBudget = 200 * 1024;

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, int src_bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Thread g = blockIdx.x * blockDim.x + threadIdx.x works on tile g % ntiles of
// channel g / ntiles; the CTA stages the rows of channels [ch_first, ch_first + max_ch).
// kKC time samples per shared-memory chunk (32, or less for very many stations).
template <int kKC, int RS, bool G3>
__global__ void __launch_bounds__(G3 ? 384 : (RS == 4 ? 256 : kMaxThreads), 1)
xcorr_f32_kernel(const float2 *__restrict__ corr, float2 *__restrict__ vis,
                 const int2 *__restrict__ tiles, int ntiles, int N, int S, int IP, int max_ch,
                 long long total_ch, int accumulate)
{
    extern __shared__ float4 sm[];   // [2][max_ch][KC][IP/2 + 1] float4
    const int row4 = IP / 2;                       // float4 (= station entries) per time row
    const int rowp = row4 + 1;                     // padded row stride
    const int half = IP / 4;                       // RS = 2: offset of the odd-station half
    const int quarter = IP / 8;                    // RS = 4: offset between the residue groups
    const int stage_f4 = max_ch * kKC * rowp;
    const int NB = (S + 15) / 16;                  // 16-spectrum blocks of the input layout
    const int tid = threadIdx.x;
    const long long g0 = (long long)blockIdx.x * blockDim.x;
    const long long ch_first = g0 / ntiles;
    const long long ch_last = (g0 + blockDim.x - 1) / ntiles + 1;
    const long long ch_end = ch_last < total_ch ? ch_last : total_ch;
    const int nch = (int)(ch_end - ch_first);
    const int nthr = blockDim.x;

    // element v = (cl * row4 + x) * KC + s: the thread's sample s = tid mod KC is
    // the same in every chunk (nthr is a multiple of KC); its first (x, cl) is
    // found once and advanced by nthr / KC with a carry (no division per element)
    const int s_l = tid % kKC;
    const int e_first = tid / kKC, de = nthr / kKC;
    const int x_first = e_first % row4, c_first = e_first / row4;
    const int dx = de % row4, dc = de / row4;
    auto load_chunk = [&](int stage, int s0) {
        float4 *dst0 = sm + stage * stage_f4;
        const int total = nch * row4;
        const int sa = s0 + s_l;
        const bool s_ok = sa < S;
        const long long run = (long long)(sa >> 4) * N;  // block of this sample
        int x = x_first, cl = c_first;
        for (int e = e_first; e < total; e += de) {
            const long long gch = ch_first + cl;
            const bool ok = s_ok && (x < N);
            const float2 *src = corr;
            if (ok) src = corr + ((gch * NB * N + run + x) * 16 + (sa & 15)) * 2;
            const int xs = RS == 4 ? (x & 3) * quarter + (x >> 2)    // [0 mod 4][1][2][3]
                                   : (x & 1) * half + (x >> 1);      // [even stations][odd stations]
            cp_async16(dst0 + (cl * kKC + s_l) * rowp + xs, src, ok ? 16 : 0);
            x += dx;
            cl += dc;
            if (x >= row4) {
                x -= row4;
                ++cl;
            }
        }
    };

    const long long g = g0 + tid;
    const long long gch = g / ntiles;
    const int tl = (int)(g - gch * ntiles);
    const int cl = (int)(gch - ch_first);
    const bool active = gch < total_ch;
    int2 rq = make_int2(0, 0);
    if (active) rq = tiles[tl];
    const int r = rq.x, q = rq.y;

    // acc[a][b] = (re, im) of x_a conj(y_b), updated with packed FP32 FMAs:
    //   acc += (xr, xi) * (yr, yr);  acc += (xi, -xr) * (yi, yi)
    // (per component the same two FMAs in the same order as the scalar form)
    constexpr int RA = 2 * RS;                     // row inputs of a tile
    // G3 (three-multiplication form): t12[a][b] = (sum xr yr, sum xi yi) by one
    // packed FMA on the natural (xr, xi), (yr, yi) pairs, t3[a][b] = sum
    // (xr + xi)(yr - yi) by one scalar FMA; then re = t1 + t2 and
    // im = t3 - t1 + t2 (3 FMAs per complex MAC instead of 4, no operand copies)
    constexpr int RG = G3 ? RA : 1;
    float2 acc[RA][8];
    float t3[RG][8];
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < RG; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) t3[a][b] = 0.f;

    const int nchunks = (S + kKC - 1) / kKC;
    load_chunk(0, 0);
    cp_async_commit();
    for (int kc = 0; kc < nchunks; ++kc) {
        if (kc + 1 < nchunks) load_chunk((kc + 1) & 1, (kc + 1) * kKC);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        if (active) {
            const float4 *base = sm + (kc & 1) * stage_f4 + cl * kKC * rowp;
#pragma unroll 2
            for (int s = 0; s < kKC; ++s) {
                const float4 *row = base + s * rowp;
                float2 xv[RA];
                if constexpr (RS == 2) {
                    // row stations 2r (even half) and 2r+1 (odd half)
                    const float4 x0 = row[r], x1 = row[half + r];
                    xv[0] = make_float2(x0.x, x0.y);
                    xv[1] = make_float2(x0.z, x0.w);
                    xv[2] = make_float2(x1.x, x1.y);
                    xv[3] = make_float2(x1.z, x1.w);
                } else {
                    // row stations 4r .. 4r+3
                    const float4 x0 = row[r], x1 = row[quarter + r], x2 = row[2 * quarter + r],
                                 x3 = row[3 * quarter + r];
                    xv[0] = make_float2(x0.x, x0.y);
                    xv[1] = make_float2(x0.z, x0.w);
                    xv[2] = make_float2(x1.x, x1.y);
                    xv[3] = make_float2(x1.z, x1.w);
                    xv[4] = make_float2(x2.x, x2.y);
                    xv[5] = make_float2(x2.z, x2.w);
                    xv[6] = make_float2(x3.x, x3.y);
                    xv[7] = make_float2(x3.z, x3.w);
                }
                // column stations 4q, 4q+1, 4q+2, 4q+3
                float4 y0, y1, y2, y3;
                if constexpr (RS == 2) {
                    y0 = row[2 * q];
                    y1 = row[half + 2 * q];
                    y2 = row[2 * q + 1];
                    y3 = row[half + 2 * q + 1];
                } else {
                    y0 = row[q];
                    y1 = row[quarter + q];
                    y2 = row[2 * quarter + q];
                    y3 = row[3 * quarter + q];
                }
                if constexpr (G3) {
                    const float2 yv[8] = {make_float2(y0.x, y0.y), make_float2(y0.z, y0.w),
                                          make_float2(y1.x, y1.y), make_float2(y1.z, y1.w),
                                          make_float2(y2.x, y2.y), make_float2(y2.z, y2.w),
                                          make_float2(y3.x, y3.y), make_float2(y3.z, y3.w)};
                    float dy[8];
#pragma unroll
                    for (int b = 0; b < 8; ++b) dy[b] = yv[b].x - yv[b].y;
#pragma unroll
                    for (int a = 0; a < RA; ++a) {
                        const float sx = xv[a].x + xv[a].y;
#pragma unroll
                        for (int b = 0; b < 8; ++b) {
                            acc[a][b] = __ffma2_rn(xv[a], yv[b], acc[a][b]);   // (xr yr, xi yi)
                            t3[a % RG][b] = fmaf(sx, dy[b], t3[a % RG][b]);   // (xr + xi)(yr - yi)
                        }
                    }
                    continue;
                }
                const float yr[8] = {y0.x, y0.z, y1.x, y1.z, y2.x, y2.z, y3.x, y3.z};
                const float yi[8] = {y0.y, y0.w, y1.y, y1.w, y2.y, y2.w, y3.y, y3.w};
#pragma unroll
                for (int a = 0; a < RA; ++a) {
                    const float2 xs = make_float2(xv[a].y, -xv[a].x);
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        // x * conj(y)
                        acc[a][b] = __ffma2_rn(xv[a], make_float2(yr[b], yr[b]), acc[a][b]);
                        acc[a][b] = __ffma2_rn(xs, make_float2(yi[b], yi[b]), acc[a][b]);
                    }
                }
            }
        }
        __syncthreads();
    }
    if (!active) return;
    const long long B = (long long)N * (N + 1) / 2;
#pragma unroll
    for (int a = 0; a < RA; ++a) {
        const int i = RS * r + a / 2, p = a % 2;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int j = 4 * q + jj;
            if (i <= j && j < N) {
                const long long b = (long long)j * (j + 1) / 2 + i;
                float4 v;
                if constexpr (G3) {
                    const float2 u0 = acc[a][2 * jj], u1 = acc[a][2 * jj + 1];
                    v = make_float4(u0.x + u0.y, (t3[a % RG][2 * jj] - u0.x) + u0.y, u1.x + u1.y,
                                    (t3[a % RG][2 * jj + 1] - u1.x) + u1.y);
                } else {
                    v = make_float4(acc[a][2 * jj].x, acc[a][2 * jj].y, acc[a][2 * jj + 1].x, acc[a][2 * jj + 1].y);
                }
                float4 *dst = reinterpret_cast<float4 *>(vis + (gch * B + b) * 4 + 2 * p);
                if (accumulate) {                      // add to the sums of earlier time chunks
                    const float4 o = *dst;
                    v.x += o.x;
                    v.y += o.y;
                    v.z += o.z;
                    v.w += o.w;
                }
                *dst = v;
            }
        }
    }
}

}  // namespace

// Tiles (r, q): row stations RS r .. RS r + RS - 1; column stations 4q..4q+3;
// kept where RS r <= 4q + 3. Ordered by q, then r, so a warp mostly shares
// its column loads.
int xf32_build_tiles(int N, int RS, int2 *out)
{
    const int NR = (N + RS - 1) / RS, NQ = (N + 3) / 4;
    int n = 0;
    for (int q = 0; q < NQ; ++q)
        for (int r = 0; r < NR; ++r)
            if (RS * r <= 4 * q + 3) {
                if (out) out[n] = make_int2(r, q);
                ++n;
            }
    return n;
}

// CTA size (largest of 512, 384, 256, 128, 96, 64, 32 threads) whose touched
// channels fit in shared memory, shrunk while the grid would not fill the GPU.
bool xf32_geometry(int N, long long total_ch, int ntiles, int kc, int mode, int *threads, int *max_ch)
{
    const int IP = 8 * ((N + 3) / 4);
    const size_t row_bytes = (size_t)kc * (IP + 2) * sizeof(float2);   // rows padded by one entry
    static const int cand[] = {512, 384, 256, 128, 96, 64, 32};
    // 4x4 tiles (64 accumulators): at most 256 threads; three-multiplication form: 384
    int t = 0, mc = 0, k = mode == 1 ? 2 : mode == 2 ? 1 : 0;
    for (; k < 7; ++k) {
        mc = (cand[k] + ntiles - 1) / ntiles + 1;
        if (2 * mc * row_bytes <= kSmemBudget) {
            t = cand[k];
            break;
        }
    }
    if (!t) return false;
    while (k + 1 < 7 && (total_ch * ntiles + t - 1) / t < 2 * 152) {
        ++k;
        t = cand[k];
        mc = (t + ntiles - 1) / ntiles + 1;
    }
    *threads = t;
    *max_ch = mc;
    return true;
}

cudaError_t launch_xcorr_f32(const Handle &h, const float2 *corr, float2 *vis, cudaStream_t st, bool accumulate)
{
    const int N = h.p.n_stations, S = h.p.n_spectra;
    const int IP = 8 * ((N + 3) / 4);
    const int mode = h.xf32_mode;                   // 0: 2x4, 1: 4x4, 2: 2x4 three-multiplication
    const int nt = h.xf32_ntiles;
    const long long total = (long long)h.p.n_subbands * h.p.n_channels;
    int threads = 0, max_ch = 0, kc = 32;
    for (; kc >= 4; kc /= 2)
        if (xf32_geometry(N, total, nt, kc, mode, &threads, &max_ch)) break;
    if (kc < 4) return cudaErrorNotSupported;   // > ~800 stations
    const size_t smem = 2ull * max_ch * kc * (IP + 2) * sizeof(float2);
    const long long blocks = (total * nt + threads - 1) / threads;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    auto pick = [&](auto rs, auto g3) {
        constexpr int R = decltype(rs)::value;
        constexpr bool G = decltype(g3)::value;
        return kc == 32 ? xcorr_f32_kernel<32, R, G> : kc == 16 ? xcorr_f32_kernel<16, R, G>
                                                  : kc == 8     ? xcorr_f32_kernel<8, R, G>
                                                                : xcorr_f32_kernel<4, R, G>;
    };
    auto kern = mode == 1   ? pick(std::integral_constant<int, 4>{}, std::false_type{})
                : mode == 2 ? pick(std::integral_constant<int, 2>{}, std::true_type{})
                            : pick(std::integral_constant<int, 2>{}, std::false_type{});
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)blocks, threads, smem, st>>>(corr, vis, h.d_xf32_tiles, nt, N, S, IP, max_ch, total,
                                                   accumulate ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace fxi
