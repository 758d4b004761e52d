// align.cu -- sw_align: start point and linear-space reconstruction.
#include "ctx.h"

extern "C" int sw_align(sw_ctx *ctx, const uint8_t *, int64_t, const uint8_t *, int64_t,
                        const sw_scheme *, int32_t, sw_result *out)
{
    if (!ctx || !out) return SW_EINVAL;
    return SW_ENOTIMPL;
}
