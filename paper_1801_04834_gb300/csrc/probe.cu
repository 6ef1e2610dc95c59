// probe.cu -- FP32 FMA throughput probe: a kernel that does nothing but
// packed FP32 FMAs (FFMA2) on register operands, so that the FP32 peak
// derived from the unit counts (SMs x 128 lanes x 2 flop x clock) can be
// checked by measurement on the device at hand.
#include "internal.h"

namespace fxi {
namespace {

constexpr int kProbeChains = 8;      // independent accumulator chains per thread

__global__ void __launch_bounds__(256) ffma_probe_kernel(int iterations, float2 m, float *sink)
{
    float2 acc[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) acc[k] = make_float2((float)threadIdx.x + k, (float)blockIdx.x - k);
    const float2 c = make_float2(1e-7f, -1e-7f);
    for (int it = 0; it < iterations; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int k = 0; k < kProbeChains; ++k) acc[k] = __ffma2_rn(acc[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += acc[k].x + acc[k].y;
    if (s == 12345.678f) sink[0] = s;    // keeps the chains live; practically never taken
}

}  // namespace

cudaError_t launch_ffma_probe(int iterations, int blocks, float *sink, cudaStream_t st)
{
    ffma_probe_kernel<<<blocks, 256, 0, st>>>(iterations, make_float2(0.999999f, 1.000001f), sink);
    return cudaGetLastError();
}

}  // namespace fxi
