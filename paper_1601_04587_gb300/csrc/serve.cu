// Serving: continuous batching of propagator solves (filled in below).
#include "ddp_host.h"

extern "C" {

int ddp_serve_reset(ddp_ctx *ctx) {
    (void)ctx;
    return DDP_OK;
}

int ddp_serve_config(ddp_ctx *ctx, uint64_t mem_budget_bytes, int max_active, int precision) {
    (void)ctx; (void)mem_budget_bytes; (void)max_active; (void)precision;
    return DDP_ERR_UNSUPPORTED;
}
int ddp_submit(ddp_ctx *ctx, const ddp_solve_req *req, uint64_t *ticket) {
    (void)ctx; (void)req; (void)ticket;
    return DDP_ERR_UNSUPPORTED;
}
int ddp_serve_step(ddp_ctx *ctx, int *in_flight) {
    (void)ctx; (void)in_flight;
    return DDP_ERR_UNSUPPORTED;
}
int ddp_poll(ddp_ctx *ctx, uint64_t ticket, int *done, ddp_solve_info *info) {
    (void)ctx; (void)ticket; (void)done; (void)info;
    return DDP_ERR_UNSUPPORTED;
}
}
