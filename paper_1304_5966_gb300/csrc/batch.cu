// batch.cu -- sw_align_batch: many pairs in one persistent launch.
#include "ctx.h"

extern "C" int sw_align_batch(sw_ctx *ctx, const sw_pair *, int32_t, const sw_scheme *, int32_t,
                              sw_result *outs)
{
    if (!ctx || !outs) return SW_EINVAL;
    return SW_ENOTIMPL;
}
