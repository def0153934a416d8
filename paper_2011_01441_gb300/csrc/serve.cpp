// Serving engine (placeholder until the serving loop lands).
#include "../../include/paco_lcs.h"
#include "ctx.hpp"

namespace paco {
struct ServeEngine {};
void serve_shutdown(paco_ctx *ctx) {
    delete ctx->serve;
    ctx->serve = nullptr;
}
}  // namespace paco

extern "C" {
int paco_lcs_submit(paco_ctx *ctx, const uint8_t *, int64_t, const uint8_t *, int64_t, int, uint64_t *) {
    return ctx ? PACO_EINVAL : PACO_EINVAL;
}
int paco_lcs_poll(paco_ctx *ctx, uint64_t, int32_t *, int32_t *, int32_t *) {
    return ctx ? PACO_ENOTFOUND : PACO_EINVAL;
}
int paco_serve_get_stats(paco_ctx *ctx, paco_serve_stats *out) {
    return (ctx && out) ? PACO_EINVAL : PACO_EINVAL;
}
}
