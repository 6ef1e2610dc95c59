// fft_reg.cuh -- small complex helpers and an in-register radix-2 FFT of
// size R in {2, 4, 8, 16}, used for both passes of the C = R*R point
// channelising FFT. Twiddles are the exact 16th roots of unity written as
// decimal constants (cos and sin of multiples of pi/8), so multiplications by
// 1 and -i fold away at compile time.
#pragma once
#include <cuda_runtime.h>

namespace fxi {

// complex add / subtract as one packed FP32 add (FADD2) each; same rounding as
// the two scalar adds
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// b * exp(-2 pi i m / 16) for a compile-time m in [0, 8)
template <int M>
__device__ __forceinline__ float2 rot16(float2 b)
{
    constexpr float c1 = 0.92387953251128675613f;  // cos(pi/8)
    constexpr float s1 = 0.38268343236508977173f;  // sin(pi/8)
    constexpr float r2 = 0.70710678118654752440f;  // sqrt(2)/2
    if constexpr (M == 0) return b;
    else if constexpr (M == 4) return make_float2(b.y, -b.x);
    else if constexpr (M == 2) return make_float2(r2 * (b.x + b.y), r2 * (b.y - b.x));
    else if constexpr (M == 6) return make_float2(r2 * (b.y - b.x), -r2 * (b.x + b.y));
    else {
        constexpr float wr = (M == 1) ? c1 : (M == 3) ? s1 : (M == 5) ? -s1 : -c1;
        constexpr float wi = (M == 1) ? -s1 : (M == 3) ? -c1 : (M == 5) ? -c1 : -s1;
        return make_float2(fmaf(b.x, wr, -b.y * wi), fmaf(b.x, wi, b.y * wr));
    }
}

constexpr int bitrev(int i, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

template <int R, int HALF, int BASE, int J>
__device__ __forceinline__ void fft_bfly(float2 (&t)[R])
{
    if constexpr (J < HALF) {
        constexpr int M = J * (8 / HALF);
        const float2 bw = rot16<M>(t[BASE + J + HALF]);
        const float2 a = t[BASE + J];
        t[BASE + J] = cadd(a, bw);
        t[BASE + J + HALF] = csub(a, bw);
        fft_bfly<R, HALF, BASE, J + 1>(t);
    }
}

template <int R, int HALF, int BASE>
__device__ __forceinline__ void fft_stage(float2 (&t)[R])
{
    if constexpr (BASE < R) {
        fft_bfly<R, HALF, BASE, 0>(t);
        fft_stage<R, HALF, BASE + 2 * HALF>(t);
    }
}

template <int R, int HALF>
__device__ __forceinline__ void fft_stages(float2 (&t)[R])
{
    if constexpr (HALF < R) {
        fft_stage<R, HALF, 0>(t);
        fft_stages<R, HALF * 2>(t);
    }
}

// v[k] <- sum_n v[n] exp(-2 pi i n k / R), in place, natural order in and out.
template <int R>
__device__ __forceinline__ void fft_reg(float2 (&v)[R])
{
    static_assert(R == 2 || R == 4 || R == 8 || R == 16, "R must be 2, 4, 8 or 16");
    float2 t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) t[bitrev(i, ilog2(R))] = v[i];
    fft_stages<R, 1>(t);
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = t[i];
}

}  // namespace fxi
