// Fused objective pass (placeholder until the fused kernel lands): reports
// "not supported" so that callers must select the multi-pass evaluation.
#include "internal.h"

cudaError_t launch_ngf_fused(reg_ctx *, int, const float *, const float *, const double *, float *, double *,
                             int *, cudaStream_t)
{
    return cudaErrorNotSupported;
}
