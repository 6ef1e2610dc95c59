// channelize_correct.cu -- entry of the fused F-stage (channelise + delay /
// bandpass correction in one pass): dispatch on the sample format. The
// kernels are in channelize_correct_impl.cuh, compiled once per format.
#include "internal.h"

namespace fxi {

cudaError_t launch_channelize_correct_ci16(const Handle &, const void *, const float *, const float2 *, void *,
                                           cudaStream_t, const float *, const FWindow *);
cudaError_t launch_channelize_correct_ci8(const Handle &, const void *, const float *, const float2 *, void *,
                                          cudaStream_t, const float *, const FWindow *);
cudaError_t launch_channelize_correct_ci4(const Handle &, const void *, const float *, const float2 *, void *,
                                          cudaStream_t, const float *, const FWindow *);

cudaError_t launch_channelize_correct(const Handle &h, const void *raw, const float *bandpass, const float2 *gains,
                                      void *corr, cudaStream_t st, const float *flags, const FWindow *window)
{
    if (h.p.format == FX_CI16) return launch_channelize_correct_ci16(h, raw, bandpass, gains, corr, st, flags, window);
    if (h.p.format == FX_CI8) return launch_channelize_correct_ci8(h, raw, bandpass, gains, corr, st, flags, window);
    return launch_channelize_correct_ci4(h, raw, bandpass, gains, corr, st, flags, window);
}

}  // namespace fxi
