// channelize_correct_ci16.cu -- the fused F-stage for ci16 input samples
// (kernels in channelize_correct_impl.cuh; one translation unit per format).
#include "channelize_correct_impl.cuh"

namespace fxi {

cudaError_t launch_channelize_correct_ci16(const Handle &h, const void *raw, const float *bandpass,
                                            const float2 *gains, void *corr, cudaStream_t st, const float *flags,
                                            const FWindow *window)
{
    return launch_fmt<short2>(h, raw, corr, bandpass, gains, flags, window, st);
}

}  // namespace fxi
