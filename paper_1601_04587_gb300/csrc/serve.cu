// C ABI of the continuous-batching server (serve_engine.cuh holds the engine).
#include <cstring>

#include "ddp_host.h"

using namespace ddp;

namespace {

bool on_device(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

ServerBase *server(ddp_ctx *ctx) { return reinterpret_cast<ServerBase *>(ctx->serve); }

struct Dev {
    int prev = -1;
    explicit Dev(int d) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d);
    }
    ~Dev() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

uint64_t g_ticket = 0;

}  // namespace

extern "C" {

int ddp_serve_reset(ddp_ctx *ctx) {
    if (!ctx) return DDP_ERR_INVALID_ARG;
    if (ctx->serve) {
        Dev d(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        delete server(ctx);
        ctx->serve = nullptr;
    }
    return DDP_OK;
}

int ddp_serve_config(ddp_ctx *ctx, uint64_t mem_budget_bytes, int max_active, int precision) {
    if (!ctx || max_active < 1 || precision < 0 || precision > 3) return DDP_ERR_INVALID_ARG;
    ddp_serve_reset(ctx);
    Dev d(ctx->device);
    if (mem_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return DDP_ERR_CUDA;
        mem_budget_bytes = (uint64_t)(0.8 * (double)fr);
    }
    int st = DDP_OK;
    ServerBase *s = nullptr;
    switch (precision) {
        case DDP_PREC_FP64: s = make_server<PF64>(ctx, precision, mem_budget_bytes, max_active, &st); break;
        case DDP_PREC_MIXED_FP32: s = make_server<PF32>(ctx, precision, mem_budget_bytes, max_active, &st); break;
        case DDP_PREC_MIXED_FP16: s = make_server<PF16>(ctx, precision, mem_budget_bytes, max_active, &st); break;
        default: s = make_server<PBF16>(ctx, precision, mem_budget_bytes, max_active, &st); break;
    }
    if (!s) return st ? st : DDP_ERR_OOM;
    ctx->serve = s;
    return DDP_OK;
}

int ddp_submit(ddp_ctx *ctx, const ddp_solve_req *r, uint64_t *ticket) {
    if (!ctx || !r || !ticket) return DDP_ERR_INVALID_ARG;
    if (!ctx->serve) return DDP_ERR_INVALID_ARG;
    if (r->csw != 0.0) return DDP_ERR_UNSUPPORTED;
    if (!(r->kappa > 0) || !(r->tol > 0) || !on_device(r->out)) return DDP_ERR_INVALID_ARG;
    if (r->eta && !on_device(r->eta)) return DDP_ERR_INVALID_ARG;
    auto di = ctx->domains.find(r->domain_id);
    if (di == ctx->domains.end()) return DDP_ERR_NOT_FOUND;
    auto gi = ctx->gauges.find(di->second.gauge_id);
    if (gi == ctx->gauges.end()) return DDP_ERR_NOT_FOUND;
    const DomainDev &d = di->second;
    const GaugeDev &g = *gi->second;
    Job j;
    memset(&j, 0, sizeof(j));
    j.g = &g;
    memcpy(j.o, d.o, sizeof(j.o));
    memcpy(j.e, d.e, sizeof(j.e));
    j.kappa = r->kappa;
    j.tol = r->tol;
    j.out = r->out;
    if (r->eta) {
        if (r->ncol < 1) return DDP_ERR_INVALID_ARG;
        j.ncol = r->ncol;
        j.eta = r->eta;
    } else {
        j.ncol = 12;
        int k[4];
        for (int m = 0; m < 4; m++) {
            if (r->src[m] < 0 || r->src[m] >= g.L[m]) return DDP_ERR_INVALID_ARG;
            k[m] = ((r->src[m] - d.o[m]) % g.L[m] + g.L[m]) % g.L[m];
            if (k[m] >= d.e[m]) return DDP_ERR_INVALID_ARG;
        }
        j.src_l = ((k[0] * d.e[1] + k[1]) * d.e[2] + k[2]) * d.e[3] + k[3];
    }
    uint64_t t = ++g_ticket;
    int rc = server(ctx)->submit(j, t);
    if (rc == DDP_OK) *ticket = t;
    return rc;
}

int ddp_serve_step(ddp_ctx *ctx, int *in_flight) {
    if (!ctx || !in_flight) return DDP_ERR_INVALID_ARG;
    if (!ctx->serve) {
        *in_flight = 0;
        return DDP_OK;
    }
    Dev d(ctx->device);
    StreamJoin sj(ctx);
    return server(ctx)->step(in_flight);
}

int ddp_poll(ddp_ctx *ctx, uint64_t ticket, int *done, ddp_solve_info *info) {
    if (!ctx || !done) return DDP_ERR_INVALID_ARG;
    if (!ctx->serve) return DDP_ERR_NOT_FOUND;
    return server(ctx)->poll(ticket, done, info);
}
}
