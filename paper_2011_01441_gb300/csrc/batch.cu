// Batch of independent pairs (placeholder until the batch engine lands).
#include "../../include/paco_lcs.h"
#include "ctx.hpp"

namespace paco {
struct BatchState {};
void batch_release(paco_ctx *ctx) {
    delete ctx->batch;
    ctx->batch = nullptr;
}
}  // namespace paco

extern "C" int paco_lcs_batch(paco_ctx *ctx, const uint8_t *, const int64_t *, const uint8_t *,
                              const int64_t *, const int64_t *, const int64_t *, int32_t, int32_t *,
                              int32_t *, const int64_t *, int32_t *, const int64_t *, void *) {
    if (!ctx) return PACO_EINVAL;
    return PACO_EINVAL;
}
