// Continuous batching of domain-propagator solves.
//
// The server owns one fixed-capacity set of solver fields sized by its memory
// budget.  A request is admitted when an active slot and a contiguous range of
// site-columns are free (otherwise DDP_ERR_BUSY); from then on its sources and
// FP64 solution stay resident in that range.  Every step runs one
// defect-correction cycle (FP64 residual, inner BiCGStab loop, FP64
// accumulation) for all active requests in one launch sequence: requests
// admitted since the previous step join the running ones, converged requests
// are unpacked into their output buffers and retire, freeing their range.
//
// A request goes through the same sequence of cycles whatever else is active
// (its reductions are per request and in a fixed order, its inner iterations
// stop on its own criterion), so its result does not depend on the mix.
#pragma once

#include <chrono>
#include <map>

#include "engine.cuh"

namespace ddp {

template <class P>
struct Server : ServerBase {
    struct Req {
        Job job;
        int64_t off = 0, len = 0;
        bool fresh = true;
        std::vector<SolveState> st;
        int outer = 0;
        std::chrono::steady_clock::time_point t0;
        bool done = false;
        ddp_solve_info info;
    };

    ddp_ctx *ctx = nullptr;
    Engine<P> eng;
    Arena arena;
    int64_t cap = 0, npart_cap = 0;
    int max_active = 0, nsolve_cap = 0;
    std::map<uint64_t, Req> reqs;
    std::vector<uint64_t> active;
    std::map<int64_t, int64_t> free_;  // offset -> length of free site-column ranges

    static constexpr int MAX_NCOL = 16;

    int init(ddp_ctx *c, int precision, uint64_t budget, int maxact) {
        ctx = c;
        prec = precision;
        eng.ctx = c;
        eng.prec = precision;
        max_active = maxact;
        nsolve_cap = MAX_NCOL * maxact;
        // bytes per site-column of capacity (fields) plus the per-tile partials
        double per = (double)Engine<P>::bytes_needed(1 << 20, 0, 0, 0) / (1 << 20) + 2.0 * 24.0 / 32.0;
        cap = (int64_t)((double)budget / per);
        cap = (cap / 32) * 32;
        if (cap < 1024) return DDP_ERR_OOM;
        npart_cap = cap / 32 + (int64_t)nsolve_cap + 64;
        size_t need = Engine<P>::bytes_needed(cap, npart_cap, maxact, nsolve_cap);
        cudaError_t e = arena.reserve(need);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "serving arena");
        eng.carve(arena, cap, npart_cap, maxact, nsolve_cap);
        free_[0] = cap;
        return DDP_OK;
    }

    bool alloc(int64_t len, int64_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                *off = it->first;
                int64_t rest = it->second - len;
                int64_t noff = it->first + len;
                free_.erase(it);
                if (rest > 0) free_[noff] = rest;
                return true;
            }
        }
        return false;
    }

    void release(int64_t off, int64_t len) {
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

    int submit(const Job &job, uint64_t ticket) override {
        if (job.ncol > MAX_NCOL) return DDP_ERR_UNSUPPORTED;
        int64_t nh = (int64_t)job.e[0] * job.e[1] * job.e[2] * job.e[3] / 2;
        int64_t len = nh * job.ncol;
        if (len > cap) return DDP_ERR_OOM;  // can never fit this server
        if ((int)active.size() >= max_active) return DDP_ERR_BUSY;
        int64_t off;
        if (!alloc(len, &off)) return DDP_ERR_BUSY;
        Req r;
        r.job = job;
        r.off = off;
        r.len = len;
        r.t0 = std::chrono::steady_clock::now();
        memset(&r.info, 0, sizeof(r.info));
        reqs[ticket] = r;
        active.push_back(ticket);
        return DDP_OK;
    }

    int step(int *in_flight) override {
        if (active.empty()) {
            *in_flight = 0;
            return DDP_OK;
        }
        std::vector<Job> jobs;
        for (uint64_t t : active) jobs.push_back(reqs[t].job);
        make_plan(jobs, prec, ctx->prm, eng.plan);
        eng.clov = false;  // serving refuses the clover term (ddp_submit)
        std::vector<SolveState> states(eng.plan.nsolve);
        for (size_t i = 0; i < active.size(); i++) {
            Req &r = reqs[active[i]];
            Item &it = eng.plan.items[i];
            it.fbase = r.off;
            for (int c = 0; c < it.ncol; c++) {
                SolveState S = r.fresh ? eng.fresh_state((int)i, c, r.job.tol) : r.st[c];
                S.item = (int)i;
                S.col = c;
                states[it.solve0 + c] = S;
            }
        }
        int rc = eng.upload(states);
        if (rc) return rc;
        for (size_t i = 0; i < active.size(); i++) {
            Req &r = reqs[active[i]];
            if (r.fresh && (rc = eng.pack_source((int)i, r.job))) return rc;
        }
        eng.source_norms();
        eng.residual(false);  // x = 0 for fresh requests: exactly eta, as in a one-shot solve
        if ((rc = eng.download_states())) return rc;
        std::vector<char> retire(active.size(), 0);
        bool any_work = false;
        for (size_t i = 0; i < active.size(); i++) {
            Req &r = reqs[active[i]];
            const Item &it = eng.plan.items[i];
            bool done = true;
            for (int c = 0; c < it.ncol; c++) done = done && eng.h_st[it.solve0 + c].outer_done;
            if (done || r.outer >= ctx->prm.max_outer) {
                retire[i] = 1;
                // requests that stop here must not be corrected again
                for (int c = 0; c < it.ncol; c++) {
                    eng.h_st[it.solve0 + c].sigma = 0;
                    eng.h_st[it.solve0 + c].scale = 0;
                }
            } else {
                any_work = true;
            }
        }
        if (any_work) {
            DDP_CUDA(ctx, cudaMemcpyAsync(eng.d_st, eng.h_st.data(), eng.plan.nsolve * sizeof(SolveState),
                                          cudaMemcpyHostToDevice, ctx->stream));
            eng.drop_graph();
            if ((rc = eng.build_loop_graph())) return rc;
            if ((rc = eng.correction(false))) return rc;
            if ((rc = eng.download_states())) return rc;
        }
        std::vector<uint64_t> keep;
        for (size_t i = 0; i < active.size(); i++) {
            Req &r = reqs[active[i]];
            const Item &it = eng.plan.items[i];
            r.st.assign(eng.h_st.begin() + it.solve0, eng.h_st.begin() + it.solve0 + it.ncol);
            r.fresh = false;
            if (!retire[i]) {
                r.outer++;
                keep.push_back(active[i]);
                continue;
            }
            if ((rc = eng.unpack_result((int)i, r.job.out))) return rc;
            r.done = true;
            ddp_solve_info &inf = r.info;
            inf.ncol = it.ncol;
            inf.outer_cycles = r.outer;
            double mx = 0;
            int inner = 0;
            int64_t colit = 0;
            bool ok = true;
            for (int c = 0; c < it.ncol; c++) {
                const SolveState &S = r.st[c];
                double rr = (S.bnorm2 > 0) ? sqrt(S.rr64 / S.bnorm2) : 0.0;
                if (c < DDP_INFO_COLS) inf.rel_residual[c] = rr;
                if (!(rr <= mx)) mx = rr;
                ok = ok && (rr <= r.job.tol);
                inner = std::max(inner, S.total_iters);
                colit += S.total_iters;
            }
            inf.max_rel_residual = mx;
            inf.inner_iters = inner;
            inf.column_iters = colit;
            inf.status = ok ? DDP_OK : DDP_ERR_NOT_CONVERGED;
            release(r.off, r.len);
        }
        DDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        auto now = std::chrono::steady_clock::now();
        for (size_t i = 0; i < active.size(); i++)
            if (retire[i]) {
                Req &r = reqs[active[i]];
                r.info.seconds = std::chrono::duration<double>(now - r.t0).count();
            }
        active.swap(keep);
        ctx->launches += eng.launches;
        eng.launches = 0;
        *in_flight = (int)active.size();
        return DDP_OK;
    }

    int poll(uint64_t ticket, int *done, ddp_solve_info *info) override {
        auto it = reqs.find(ticket);
        if (it == reqs.end()) return DDP_ERR_NOT_FOUND;
        *done = it->second.done ? 1 : 0;
        if (it->second.done) {
            if (info) *info = it->second.info;
            reqs.erase(it);
        }
        return DDP_OK;
    }
};

template <class P>
ServerBase *make_server(ddp_ctx *ctx, int prec, uint64_t budget, int max_active, int *status) {
    Server<P> *s = new Server<P>();
    *status = s->init(ctx, prec, budget, max_active);
    if (*status) {
        delete s;
        return nullptr;
    }
    return s;
}

}  // namespace ddp
