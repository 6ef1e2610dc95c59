// xcorr_tc.cu -- X-stage correlator on the tcgen05 tensor cores (placeholder
// until the tensor-core kernel lands; reports "not supported").
#include "internal.h"

namespace fxi {
cudaError_t launch_xcorr_tc(const Handle &, const void *, float2 *, cudaStream_t)
{
    return cudaErrorNotSupported;
}
}  // namespace fxi
