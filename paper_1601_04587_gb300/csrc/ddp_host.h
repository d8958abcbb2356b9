// Host-side state of a libddp context: gauge fields, domains, workspaces and
// the solver engine interface shared by the translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "ddp.h"
#include "ddp_kernels.cuh"
#include "clover.cuh"

namespace ddp {

// Clover fields T = 1 + 2 kappa C and T^-1 of one (gauge, kappa, c_sw) (clover.cuh).
struct CloverDev {
    double kappa = 0, csw = 0;
    double2 *t64 = nullptr, *ti64 = nullptr;  // [36][V]
    float4 *t32 = nullptr, *ti32 = nullptr;   // [18][V]
    ~CloverDev();
};

// Resident gauge field: FP64 full links and 2-row low-precision copies, all
// in the global even-odd order [mu][chunk][V].
struct GaugeDev {
    int L[4];
    int64_t V;
    int bc;
    double2 *u64 = nullptr;  // [4][9][V]
    float4 *u32 = nullptr;   // [4][3][V]
    uint2 *u16 = nullptr;    // [4][3][V]
    uint2 *ub16 = nullptr;   // [4][3][V]
    std::vector<std::unique_ptr<CloverDev>> clov;  // clover fields built for this field
    const void *links(int prec) const {
        switch (prec) {
            case DDP_PREC_FP64: return u64;
            case DDP_PREC_MIXED_FP32: return u32;
            case DDP_PREC_MIXED_FP16: return u16;
            default: return ub16;
        }
    }
};

struct DomainDev {
    int gauge_id;
    int o[4], e[4];
    int64_t n;
};

// One solve request inside the engine (all buffers on the device).
struct Job {
    const GaugeDev *g;
    int o[4], e[4];
    double kappa;
    double tol;
    int ncol;
    const double *eta;  // device, user layout; nullptr: 12 point sources at src_l
    int src_l;
    double *out;        // device, user layout
    const CloverDev *clov;  // clover term of (g, kappa, c_sw), or nullptr (c_sw = 0)
};

struct JobInfo {
    int status = DDP_OK;
    int outer = 0;
    int inner = 0;
    int64_t column_iters = 0;  // inner iterations summed over columns
    std::vector<double> relres;
};

struct EngineParams {
    int max_outer = 40;
    int max_inner = 30000;
    double floor_delta[4] = {1e-12, 5e-6, 5e-4, 1e-2};
    int TS = 0, CG = 0;         // 0: heuristic
    int CG_prec[4] = {0, 0, 0, 0};  // columns per block chosen by ddp_autotune, per storage format
    int use_conditional = 1;    // device-driven while loop in a CUDA graph
    int host_chunk = 16;        // iterations per host check without conditional nodes
    // preferred shared-memory carveout of the inner-loop stencils, percent (-1: the driver's
    // choice): 28 rounds up to the smallest carveout that holds three 19.6 KB blocks and
    // leaves the rest of the unified memory (about 192 KB) as L1 for the neighbour gathers
    int carveout = 28;
    // the carveout ddp_autotune chose for a storage format (-2: none, use carveout)
    int carveout_prec[4] = {-2, -2, -2, -2};
    int contract_dd = 1;        // nucleon contraction in double-FP32 arithmetic (0: FP64)
    int proj_tc = 1;            // projector-cut Gram blocks and colourless sums on the tensor cores (0: FP64 kernels)
    // ddp_propagator_series with host outputs: solve the smaller nested domains first and
    // download their results while the largest solves (0: one batched solve, then downloads)
    int overlap_downloads = 1;
};

// The stencil carveout of a storage format: the autotuner's choice, else the context's.
inline int carveout_for(const EngineParams &p, int prec) {
    return (prec >= 0 && prec < 4 && p.carveout_prec[prec] != -2) ? p.carveout_prec[prec] : p.carveout;
}

// A growable device arena owned by the context.
struct Arena {
    char *base = nullptr;
    size_t bytes = 0;
    size_t used = 0;
    cudaError_t reserve(size_t need);
    void reset() { used = 0; }
    void *take(size_t n) {
        size_t a = (used + 255) & ~size_t(255);
        used = a + ((n + 255) & ~size_t(255));
        return base + a;
    }
    ~Arena();
};

struct Timing {
    // CUDA events around the hot kernels of the last solve, for measurement.
    float hop_ms = 0;
    long hop_launches = 0;
};

}  // namespace ddp

struct ddp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;       // the library's own non-blocking work stream
    cudaStream_t user_stream = nullptr;  // the caller's stream (may be the legacy default stream)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::map<int, std::unique_ptr<ddp::GaugeDev>> gauges;
    std::map<int, ddp::DomainDev> domains;
    int next_gauge = 1;
    int next_domain = 1;
    char last_error[512] = {0};
    ddp::EngineParams prm;
    ddp::Arena ws;        // solver workspace
    ddp::Arena scratch;   // staging of host buffers, contraction partials
    ddp::Arena results;   // device-resident propagators and series terms of ddp_propagator_series
    ddp::Arena aux;       // partial sums of the projector-cut kernels
    cudaStream_t copy_stream = nullptr;  // device-to-host copies overlapped with compute (created on first use)
    void *serve = nullptr;
    // instrumentation: per-kernel-class launch counts of the last solve
    long launches = 0;
};

namespace ddp {

// Orders the work stream after the caller's stream on entry to an API call
// and the caller's stream after the work stream on exit.
struct StreamJoin {
    ddp_ctx *c;
    explicit StreamJoin(ddp_ctx *ctx) : c(ctx) {
        cudaEventRecord(c->ev_in, c->user_stream);
        cudaStreamWaitEvent(c->stream, c->ev_in, 0);
    }
    ~StreamJoin() {
        cudaEventRecord(c->ev_out, c->stream);
        cudaStreamWaitEvent(c->user_stream, c->ev_out, 0);
    }
};

int set_cuda_error(ddp_ctx *ctx, cudaError_t e, const char *where);

// The clover fields of (g, kappa, c_sw), built on first use and cached with g
// (least recently used first out, CLOVER_CACHE pairs).
constexpr int CLOVER_CACHE = 4;
int clover_for(ddp_ctx *ctx, GaugeDev &g, double kappa, double csw, const CloverDev **out);
// Largest number of columns (modes) of the tensor-core Gram blocks and colourless sums
// of the projector cut: one 128-row MMA tile holds the rows of a Gram block.
constexpr int TC_MMAX = 128;
// Colourless-spinor time-slice sums on the tensor cores (m <= TC_MMAX; device fields;
// X zeroed by the caller).
int colourless_tc(ddp_ctx *ctx, const double2 *A, int64_t n, int m, int form, int64_t slice_n, int nslice, int o0,
                  int L0, double2 *X);
// Gram blocks of nseg row segments on the tensor cores (m <= TC_MMAX; device buffers).
int gram_tc(ddp_ctx *ctx, const double2 *A, int64_t cs, int m, int64_t seg, int nseg, double2 *out);

#define DDP_CUDA(ctx, call)                                          \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return set_cuda_error(ctx, e_, #call); \
    } while (0)

// Solve a list of jobs with storage format P (templated engine, one
// instantiation per translation unit).
template <class P>
int solve_jobs(ddp_ctx *ctx, int prec, std::vector<Job> &jobs, std::vector<JobInfo> &infos);

int solve_jobs_dispatch(ddp_ctx *ctx, int prec, std::vector<Job> &jobs, std::vector<JobInfo> &infos);

// Continuous-batching server (one per context); see serve_engine.cuh.
struct ServerBase {
    int prec = 0;
    virtual ~ServerBase() {}
    virtual int submit(const Job &job, uint64_t ticket) = 0;
    virtual int step(int *in_flight) = 0;
    virtual int poll(uint64_t ticket, int *done, ddp_solve_info *info) = 0;
};

template <class P>
ServerBase *make_server(ddp_ctx *ctx, int prec, uint64_t budget, int max_active, int *status);

// Build the work table of a list of boxes (shared by the engine and apply).
struct Plan {
    std::vector<Item> items;
    int TS = 32, CG = 12;
    int64_t nfield = 0;    // site-columns per parity field
    int64_t npart = 0;     // partial slots
    int nblocks = 0;
    int nsolve = 0;
};

void make_plan(const std::vector<Job> &jobs, int prec, const EngineParams &prm, Plan &plan);

template <class P>
inline size_t field_bytes(int64_t nfield) {
    size_t b = (size_t)nfield * sizeof(typename P::chunk) * P::NCH;
    if (P::SCALED) b += ((size_t)nfield * sizeof(float) + 255) & ~size_t(255);
    return b + 256;
}

template <class P>
inline FieldView carve_field(Arena &a, int64_t nfield) {
    FieldView f;
    f.stride = nfield;
    f.p = a.take((size_t)nfield * sizeof(typename P::chunk) * P::NCH);
    f.scale = P::SCALED ? (float *)a.take((size_t)nfield * sizeof(float)) : nullptr;
    return f;
}

}  // namespace ddp
