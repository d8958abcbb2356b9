// Solver engine: domain propagators S = D_Gamma^{-1} eta (Sec. 2, Eq. diric)
// for a batch of independent requests.
//
// Outer loop (FP64 defect correction): r = eta - D_Gamma x with FP64 links and
// vectors; stop a column when |r| <= tol |eta|.  Otherwise solve
// (2 kappa D_Gamma) e' = 2 kappa r / |r| with the even-odd Schur complement
//   (1 - kappa^2 H_eo H_oe) e'_e = r'_e + kappa H_eo r'_o,  e'_o = r'_o + kappa H_oe e'_e
// by BiCGStab in the storage format P to a relative tolerance delta, and
// accumulate x += |r| e' in FP64.
//
// Inner loop: every column of every request iterates together; per-column
// scalars live on the device and the loop runs inside a CUDA graph whose
// conditional WHILE node is driven by the device (no host round trip per
// iteration).  Converged columns freeze (alpha = omega = 0).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "ddp_host.h"

namespace ddp {

// One launch of the hopping term (CL: with the clover term of the items that have one).
template <class Q, int EPI, int DOT, bool CL = false>
inline void launch_hop(ddp_ctx *ctx, int nblocks, int threads, const HopArgs &a) {
    k_hop<Q, EPI, DOT, CL><<<nblocks, threads, 0, ctx->stream>>>(a);
}

// Preferred shared-memory carveout of the inner-loop stencils (percent of the unified
// L1/shared memory; the rest is L1 for the neighbour gathers), set outside graph capture.
template <class Q, bool CL>
inline cudaError_t set_hop_carveout(int percent) {
    if (percent < 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_hop<Q, EPI_PLAIN, DOT_NONE, CL>,
                                         cudaFuncAttributePreferredSharedMemoryCarveout, percent);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_hop<Q, EPI_MHAT, DOT_RHAT, CL>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 percent);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_hop<Q, EPI_MHAT, DOT_TS, CL>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 percent);
    return e;
}

template <class P>
struct Engine {
    ddp_ctx *ctx;
    int prec;
    Plan plan;
    FieldView be, bo, xe, xo, re64, ro64;      // FP64
    FieldView r, rh, p, v, s, t, xi, tmp, ro;  // storage format P (rh: ShadowOf<P>)
    Partials A, B;
    Item *d_items = nullptr;
    SolveState *d_st = nullptr;
    LoopCtl *d_ctl = nullptr;
    int loop_mode = 0;  // how the iteration body being captured ends (see FinArgs)
    cudaGraphConditionalHandle loop_handle = 0;
    std::vector<SolveState> h_st;
    Launch L;
    int threads = 0;
    cudaGraphExec_t loop_exec = nullptr;
    cudaGraph_t loop_graph = nullptr;
    long launches = 0;
    bool clov = false;  // some item of the plan has a clover term

    ~Engine() {
        if (loop_exec) cudaGraphExecDestroy(loop_exec);
        if (loop_graph) cudaGraphDestroy(loop_graph);
    }

    HopArgs hop_args(int par, FieldView in, FieldView out, FieldView v1, FieldView v2, FieldView rhv,
                     Partials part, int skip = 0) {
        HopArgs a;
        a.st = d_st;
        a.skip = skip;
        a.L = L;
        a.p = par;
        a.in = in;
        a.out = out;
        a.v1 = v1;
        a.v2 = v2;
        a.rh = rhv;
        a.part = part;
        return a;
    }

    template <class Q, int EPI, int DOT, bool CL = false>
    void hop(const HopArgs &a) {
        launch_hop<Q, EPI, DOT, CL>(ctx, plan.nblocks, threads, a);
        launches++;
    }

    template <class Q, int OP>
    void blas(Partials part, int skip = 1) {
        BlasArgs a;
        a.skip = skip;
        a.L = L;
        a.x = xi;
        a.r = r;
        a.rh = rh;
        a.p = p;
        a.v = v;
        a.s = s;
        a.t = t;
        a.st = d_st;
        a.part = part;
        k_blas<Q, OP><<<plan.nblocks, threads, 0, ctx->stream>>>(a);
        launches++;
    }

    template <int FIN>
    void fin() {
        FinArgs a;
        a.items = d_items;
        a.st = d_st;
        a.nsolve = plan.nsolve;
        a.A = A;
        a.B = B;
        a.ctl = d_ctl;
        a.loop_mode = FIN == FIN_RHO ? loop_mode : 0;
        a.loop = loop_handle;
        k_fin<FIN><<<plan.nsolve, 256, 0, ctx->stream>>>(a);
        launches++;
    }

    void norm64(FieldView f, Partials part) {
        BlasArgs a;
        memset(&a, 0, sizeof(a));
        a.skip = 0;
        a.L = L;
        a.x = f;
        a.st = d_st;
        a.part = part;
        k_blas<PF64, OP_NORM><<<plan.nblocks, threads, 0, ctx->stream>>>(a);
        launches++;
    }

    // to_low: lo = scale hi (times T^-1 of the site when clov_inv); else hi += sigma lo
    void conv(bool to_low, FieldView lo, FieldView hi, int par = 0, bool clov_inv = false) {
        ConvArgs a;
        a.L = L;
        a.lo = lo;
        a.hi = hi;
        a.st = d_st;
        a.p = par;
        a.clov = clov_inv ? 1 : 0;
        if (to_low)
            k_to_low<P><<<plan.nblocks, threads, 0, ctx->stream>>>(a);
        else
            k_accum<P><<<plan.nblocks, threads, 0, ctx->stream>>>(a);
        launches++;
    }

    // One BiCGStab iteration on the Schur complement (van der Vorst 1992); with the
    // clover term the operator is 1 - kappa^2 T_ee^-1 H_eo T_oo^-1 H_oe.
    template <bool CL>
    void iteration_body_t() {
        FieldView none = {nullptr, nullptr, 0};
        hop<P, EPI_PLAIN, DOT_NONE, CL>(hop_args(1, p, tmp, none, none, none, A, 1));   // tmp = T^-1 H_oe p
        hop<P, EPI_MHAT, DOT_RHAT, CL>(hop_args(0, tmp, v, p, none, rh, A, 1));        // v = p - k^2 T^-1 H_eo tmp
        fin<FIN_ALPHA>();                                                               // alpha = rho / (rh, v)
        blas<P, OP_S_UPDATE>(A);                                                        // s = r - alpha v
        hop<P, EPI_PLAIN, DOT_NONE, CL>(hop_args(1, s, tmp, none, none, none, A, 1));   // tmp = T^-1 H_oe s
        hop<P, EPI_MHAT, DOT_TS, CL>(hop_args(0, tmp, t, s, none, none, A, 1));        // t = s - k^2 T^-1 H_eo tmp
        fin<FIN_OMEGA>();                                                               // omega = (t,s)/(t,t)
        blas<P, OP_XR_UPDATE>(A);                                                       // x, r; (rh,r), (r,r)
        fin<FIN_RHO>();                                                                 // beta, convergence
        blas<P, OP_P_UPDATE>(A);                                                        // p = r + beta (p - omega v)
    }
    void iteration_body() {
        if (clov)
            iteration_body_t<true>();
        else
            iteration_body_t<false>();
    }

    int build_loop_graph() {
        cudaStream_t st = ctx->stream;
        DDP_CUDA(ctx, (set_hop_carveout<P, false>(carveout_for(ctx->prm, prec))));
        DDP_CUDA(ctx, (set_hop_carveout<P, true>(carveout_for(ctx->prm, prec))));
        if (ctx->prm.use_conditional) {
            DDP_CUDA(ctx, cudaGraphCreate(&loop_graph, 0));
            cudaGraphConditionalHandle h;
            DDP_CUDA(ctx, cudaGraphConditionalHandleCreate(&h, loop_graph, 1, cudaGraphCondAssignDefault));
            // the parameter union has no default constructor: build it in zeroed storage
            alignas(cudaGraphNodeParams) unsigned char cp_buf[sizeof(cudaGraphNodeParams)];
            memset(cp_buf, 0, sizeof(cp_buf));
            cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_buf);
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t node;
            DDP_CUDA(ctx, cudaGraphAddNode(&node, loop_graph, nullptr, nullptr, 0, &cp));
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            DDP_CUDA(ctx, cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0,
                                                        cudaStreamCaptureModeThreadLocal));
            loop_mode = 1;
            loop_handle = h;
            iteration_body();  // its last kernel sets the loop condition
            loop_mode = 0;
            cudaGraph_t captured;
            cudaError_t e = cudaStreamEndCapture(st, &captured);
            if (e != cudaSuccess) return set_cuda_error(ctx, e, "capture of the inner loop");
            DDP_CUDA(ctx, cudaGraphInstantiate(&loop_exec, loop_graph, 0));
        } else {
            DDP_CUDA(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            loop_mode = 2;
            for (int i = 0; i < ctx->prm.host_chunk; i++) iteration_body();
            loop_mode = 0;
            cudaError_t e = cudaStreamEndCapture(st, &loop_graph);
            if (e != cudaSuccess) return set_cuda_error(ctx, e, "capture of the inner loop");
            DDP_CUDA(ctx, cudaGraphInstantiate(&loop_exec, loop_graph, 0));
        }
        return DDP_OK;
    }

    int run_inner() {
        // launches per iteration: 4 stencils, 3 vector updates, 3 scalar-recurrence
        // kernels (the last of which also runs the loop control)
        const long per_iter = 10;
        if (ctx->prm.use_conditional) {
            DDP_CUDA(ctx, cudaGraphLaunch(loop_exec, ctx->stream));
        } else {
            LoopCtl hc;
            for (int guard = 0; guard < 1 + ctx->prm.max_inner / std::max(1, ctx->prm.host_chunk); guard++) {
                DDP_CUDA(ctx, cudaGraphLaunch(loop_exec, ctx->stream));
                DDP_CUDA(ctx, cudaMemcpyAsync(&hc, d_ctl, sizeof(hc), cudaMemcpyDeviceToHost, ctx->stream));
                DDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
                if (!hc.pad) break;
            }
        }
        LoopCtl hc;
        DDP_CUDA(ctx, cudaMemcpyAsync(&hc, d_ctl, sizeof(hc), cudaMemcpyDeviceToHost, ctx->stream));
        DDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        launches += per_iter * (long)hc.iter;
        return DDP_OK;
    }

    // ----------------------------------------------------------- building blocks

    static size_t bytes_needed(int64_t cap, int64_t npart, int nitems, int nsolve) {
        return 6 * field_bytes<PF64>(cap) + 9 * field_bytes<P>(cap) +
               2 * ((size_t)npart * (sizeof(double2) + sizeof(double)) + 1024) + (size_t)nitems * sizeof(Item) +
               (size_t)nsolve * sizeof(SolveState) + sizeof(LoopCtl) + 8192;
    }

    // Every field gets room for cap site-columns per parity (stride cap).
    void carve(Arena &a, int64_t cap, int64_t npart, int nitems, int nsolve) {
        a.reset();
        be = carve_field<PF64>(a, cap);
        bo = carve_field<PF64>(a, cap);
        xe = carve_field<PF64>(a, cap);
        xo = carve_field<PF64>(a, cap);
        re64 = carve_field<PF64>(a, cap);
        ro64 = carve_field<PF64>(a, cap);
        r = carve_field<P>(a, cap);
        rh = carve_field<typename ShadowOf<P>::type>(a, cap);
        p = carve_field<P>(a, cap);
        v = carve_field<P>(a, cap);
        s = carve_field<P>(a, cap);
        t = carve_field<P>(a, cap);
        xi = carve_field<P>(a, cap);
        tmp = carve_field<P>(a, cap);
        ro = carve_field<P>(a, cap);
        A.c = (double2 *)a.take(npart * sizeof(double2));
        A.n = (double *)a.take(npart * sizeof(double));
        B.c = (double2 *)a.take(npart * sizeof(double2));
        B.n = (double *)a.take(npart * sizeof(double));
        d_items = (Item *)a.take(nitems * sizeof(Item));
        d_st = (SolveState *)a.take(nsolve * sizeof(SolveState));
        d_ctl = (LoopCtl *)a.take(sizeof(LoopCtl));
    }

    // Upload the work table of the current plan and the per-column states.
    int upload(const std::vector<SolveState> &states) {
        cudaStream_t st = ctx->stream;
        L.items = d_items;
        L.nitems = (int)plan.items.size();
        L.TS = plan.TS;
        L.CG = plan.CG;
        threads = plan.TS * plan.CG;
        h_st = states;
        DDP_CUDA(ctx, cudaMemcpyAsync(d_items, plan.items.data(), plan.items.size() * sizeof(Item),
                                      cudaMemcpyHostToDevice, st));
        DDP_CUDA(ctx, cudaMemcpyAsync(d_st, h_st.data(), plan.nsolve * sizeof(SolveState), cudaMemcpyHostToDevice,
                                      st));
        LoopCtl c0 = {0, 0, ctx->prm.max_inner, 0, 0};
        DDP_CUDA(ctx, cudaMemcpyAsync(d_ctl, &c0, sizeof(c0), cudaMemcpyHostToDevice, st));
        return DDP_OK;
    }

    SolveState fresh_state(int item, int col, double tol) const {
        SolveState S;
        memset(&S, 0, sizeof(S));
        S.item = item;
        S.col = col;
        S.tol = tol;
        S.floor_delta = ctx->prm.floor_delta[prec];
        S.maxit = ctx->prm.max_inner;
        S.status = 4;
        return S;
    }

    // eta (or the point sources) of item i into the FP64 source fields; x = 0 there.
    int pack_source(int i, const Job &job) {
        cudaStream_t st = ctx->stream;
        PackArgs pa;
        memset(&pa, 0, sizeof(pa));
        pa.it = plan.items[i];
        pa.user = (const double2 *)job.eta;
        pa.fe = be;
        pa.fo = bo;
        pa.src_l = job.src_l;
        pa.xe = xe;
        pa.xo = xo;
        int64_t nt = 2 * (int64_t)pa.it.nh * pa.it.ncol;
        k_pack<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(pa);
        launches++;
        return DDP_OK;
    }

    int unpack_result(int i, double *out) {
        PackArgs pa;
        memset(&pa, 0, sizeof(pa));
        pa.it = plan.items[i];
        pa.uout = (double2 *)out;
        pa.fe = xe;
        pa.fo = xo;
        int64_t nt = 2 * (int64_t)pa.it.nh * pa.it.ncol;
        k_unpack<<<(unsigned)((nt + 255) / 256), 256, 0, ctx->stream>>>(pa);
        launches++;
        DDP_CUDA(ctx, cudaGetLastError());
        return DDP_OK;
    }

    void source_norms() {
        norm64(be, A);
        norm64(bo, B);
        fin<FIN_BNORM>();
    }

    // r64 = eta - D_Gamma x (FP64 links and vectors); skip_hop: x is known to be 0,
    // so r64 = eta and the partials of |eta|^2 left by source_norms() are reused.
    void residual(bool skip_hop) {
        FieldView none = {nullptr, nullptr, 0};
        if (!skip_hop) {
            if (clov) {
                hop<PF64, EPI_RESID, DOT_NORM, true>(hop_args(0, xo, re64, xe, be, none, A, 2));
                hop<PF64, EPI_RESID, DOT_NORM, true>(hop_args(1, xe, ro64, xo, bo, none, B, 2));
            } else {
                hop<PF64, EPI_RESID, DOT_NORM>(hop_args(0, xo, re64, xe, be, none, A, 2));
                hop<PF64, EPI_RESID, DOT_NORM>(hop_args(1, xe, ro64, xo, bo, none, B, 2));
            }
        }
        fin<FIN_RESID>();
    }

    int download_states() {
        DDP_CUDA(ctx, cudaMemcpyAsync(h_st.data(), d_st, plan.nsolve * sizeof(SolveState), cudaMemcpyDeviceToHost,
                                      ctx->stream));
        DDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        return DDP_OK;
    }

    // One correction: inner solve of the normalised defect and FP64 accumulation.
    // With 2 kappa D = [[T_ee, -k H_eo], [-k H_oe, T_oo]] and r' the normalised defect:
    //   (1 - k^2 T_ee^-1 H_eo T_oo^-1 H_oe) e_e = T_ee^-1 (r'_e + k H_eo T_oo^-1 r'_o),
    //   e_o = T_oo^-1 r'_o + k T_oo^-1 H_oe e_e   (T = 1 without the clover term).
    template <bool CL>
    int correction_t(bool r_is_eta) {
        FieldView none = {nullptr, nullptr, 0};
        conv(true, s, r_is_eta ? be : re64, 0);
        conv(true, ro, r_is_eta ? bo : ro64, 1, CL);                                  // ro = T_oo^-1 r'_o
        hop<P, EPI_RHS, DOT_NORM, CL>(hop_args(0, ro, r, s, none, none, A));         // r = T_ee^-1 (r'_e + k H_eo ro)
        blas<P, OP_INIT>(A, 0);
        DDP_CUDA(ctx, cudaMemsetAsync(d_ctl, 0, 2 * sizeof(int), ctx->stream));
        fin<FIN_INIT>();
        DDP_CUDA(ctx, cudaGetLastError());
        int rc = run_inner();
        if (rc) return rc;
        hop<P, EPI_AXPY_K, DOT_NONE, CL>(hop_args(1, xi, tmp, ro, none, none, A));  // e_o = ro + k T^-1 H_oe e_e
        conv(false, xi, xe);
        conv(false, tmp, xo);
        return DDP_OK;
    }
    int correction(bool r_is_eta) { return clov ? correction_t<true>(r_is_eta) : correction_t<false>(r_is_eta); }

    void drop_graph() {
        if (loop_exec) cudaGraphExecDestroy(loop_exec);
        if (loop_graph) cudaGraphDestroy(loop_graph);
        loop_exec = nullptr;
        loop_graph = nullptr;
    }

    // ----------------------------------------------------------- one-shot solve

    int run(std::vector<Job> &jobs, std::vector<JobInfo> &infos) {
        const EngineParams &prm = ctx->prm;
        make_plan(jobs, prec, prm, plan);
        clov = false;
        for (auto &j : jobs) clov = clov || j.clov;
        DDP_CUDA(ctx, ctx->ws.reserve(bytes_needed(plan.nfield, plan.npart, (int)plan.items.size(), plan.nsolve)));
        carve(ctx->ws, plan.nfield, plan.npart, (int)plan.items.size(), plan.nsolve);
        std::vector<SolveState> states(plan.nsolve);
        for (size_t i = 0; i < plan.items.size(); i++)
            for (int c = 0; c < plan.items[i].ncol; c++)
                states[plan.items[i].solve0 + c] = fresh_state((int)i, c, jobs[i].tol);
        int rc = upload(states);
        if (rc) return rc;
        for (size_t i = 0; i < jobs.size(); i++)
            if ((rc = pack_source((int)i, jobs[i]))) return rc;
        source_norms();
        DDP_CUDA(ctx, cudaGetLastError());
        if ((rc = build_loop_graph())) return rc;
        int cycles = 0;
        for (int cyc = 0; cyc <= prm.max_outer; cyc++) {
            residual(cyc == 0);
            if ((rc = download_states())) return rc;
            bool all_done = true;
            for (auto &S : h_st) all_done = all_done && S.outer_done;
            if (all_done || cyc == prm.max_outer) break;
            cycles++;
            if ((rc = correction(cyc == 0))) return rc;
        }
        for (size_t i = 0; i < jobs.size(); i++)
            if ((rc = unpack_result((int)i, jobs[i].out))) return rc;
        DDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        infos.assign(jobs.size(), JobInfo());
        for (size_t i = 0; i < jobs.size(); i++) {
            const Item &it = plan.items[i];
            JobInfo &inf = infos[i];
            inf.outer = cycles;
            inf.relres.resize(it.ncol);
            bool ok = true;
            int inner = 0;
            for (int c = 0; c < it.ncol; c++) {
                const SolveState &S = h_st[it.solve0 + c];
                double rr = (S.bnorm2 > 0) ? sqrt(S.rr64 / S.bnorm2) : 0.0;
                inf.relres[c] = rr;
                ok = ok && (rr <= jobs[i].tol);
                inner = std::max(inner, S.total_iters);
                inf.column_iters += S.total_iters;
            }
            inf.inner = inner;
            inf.status = ok ? DDP_OK : DDP_ERR_NOT_CONVERGED;
        }
        ctx->launches += launches;
        launches = 0;
        return DDP_OK;
    }
};

template <class P>
int solve_jobs(ddp_ctx *ctx, int prec, std::vector<Job> &jobs, std::vector<JobInfo> &infos) {
    Engine<P> eng;
    eng.ctx = ctx;
    eng.prec = prec;
    return eng.run(jobs, infos);
}

// out = D_Gamma psi with the stencil of storage format P (App. A, Sec. 2).
template <class P>
int apply_dirac_impl(ddp_ctx *ctx, const Job &job, const double *psi, double *out, int prec) {
    std::vector<Job> jobs(1, job);
    Plan plan;
    make_plan(jobs, prec, ctx->prm, plan);
    const int64_t NF = plan.nfield;
    size_t need = 4 * field_bytes<P>(NF) + sizeof(Item) + 1024;
    DDP_CUDA(ctx, ctx->scratch.reserve(need));
    Arena &a = ctx->scratch;
    a.reset();
    FieldView ie = carve_field<P>(a, NF), io = carve_field<P>(a, NF);
    FieldView oe = carve_field<P>(a, NF), oo = carve_field<P>(a, NF);
    Item *d_items = (Item *)a.take(sizeof(Item));
    cudaStream_t st = ctx->stream;
    DDP_CUDA(ctx, cudaMemcpyAsync(d_items, plan.items.data(), sizeof(Item), cudaMemcpyHostToDevice, st));
    PackArgs pa;
    memset(&pa, 0, sizeof(pa));
    pa.it = plan.items[0];
    pa.user = (const double2 *)psi;
    pa.uout = (double2 *)out;
    int64_t nt = 2 * (int64_t)pa.it.nh * pa.it.ncol;
    unsigned nb = (unsigned)((nt + 255) / 256);
    k_pack_low<P><<<nb, 256, 0, st>>>(pa, ie, io);
    Launch L;
    L.items = d_items;
    L.nitems = 1;
    L.TS = plan.TS;
    L.CG = plan.CG;
    FieldView none = {nullptr, nullptr, 0};
    HopArgs h;
    h.st = nullptr;
    h.skip = 0;
    h.L = L;
    h.v2 = none;
    h.rh = none;
    h.part.c = nullptr;
    h.part.n = nullptr;
    h.p = 0;
    h.in = io;
    h.out = oe;
    h.v1 = ie;
    auto dirac = [&]() {
        if (job.clov)
            launch_hop<P, EPI_DIRAC, DOT_NONE, true>(ctx, plan.nblocks, plan.TS * plan.CG, h);
        else
            launch_hop<P, EPI_DIRAC, DOT_NONE>(ctx, plan.nblocks, plan.TS * plan.CG, h);
    };
    dirac();
    h.p = 1;
    h.in = ie;
    h.out = oo;
    h.v1 = io;
    dirac();
    k_unpack_low<P><<<nb, 256, 0, st>>>(pa, oe, oo);
    ctx->launches += 4;
    DDP_CUDA(ctx, cudaGetLastError());
    return DDP_OK;
}

// out *= s over n complex numbers.
static __global__ void k_scale_complex(double2 *out, int64_t n, double s) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_double2(s * out[i].x, s * out[i].y);
}

// out = (kappa D_hop)^p psi on a domain in FP64 (Eq. HPEtr with the
// Dirichlet-restricted hopping term of Sec. 2): p pairs of plain hop launches
// (odd -> even, even -> odd) between two even-odd field pairs, then kappa^p
// applied once to the unpacked result.  psi and out: device pointers.
template <class P>
int hop_power_impl(ddp_ctx *ctx, const Job &job, int p, const double *psi, double *out) {
    static_assert(P::IS64, "the hopping power is an FP64 operation");
    std::vector<Job> jobs(1, job);
    Plan plan;
    make_plan(jobs, DDP_PREC_FP64, ctx->prm, plan);
    const int64_t NF = plan.nfield;
    size_t need = 4 * field_bytes<P>(NF) + sizeof(Item) + 1024;
    DDP_CUDA(ctx, ctx->scratch.reserve(need));
    Arena &a = ctx->scratch;
    a.reset();
    FieldView f[2][2] = {{carve_field<P>(a, NF), carve_field<P>(a, NF)}, {carve_field<P>(a, NF), carve_field<P>(a, NF)}};
    Item *d_items = (Item *)a.take(sizeof(Item));
    cudaStream_t st = ctx->stream;
    DDP_CUDA(ctx, cudaMemcpyAsync(d_items, plan.items.data(), sizeof(Item), cudaMemcpyHostToDevice, st));
    PackArgs pa;
    memset(&pa, 0, sizeof(pa));
    pa.it = plan.items[0];
    pa.user = (const double2 *)psi;
    pa.uout = (double2 *)out;
    const int64_t nt = 2 * (int64_t)pa.it.nh * pa.it.ncol;
    const unsigned nb = (unsigned)((nt + 255) / 256);
    k_pack_low<P><<<nb, 256, 0, st>>>(pa, f[0][0], f[0][1]);
    Launch L;
    L.items = d_items;
    L.nitems = 1;
    L.TS = plan.TS;
    L.CG = plan.CG;
    FieldView none = {nullptr, nullptr, 0};
    HopArgs h;
    h.st = nullptr;
    h.skip = 0;
    h.L = L;
    h.v1 = none;
    h.v2 = none;
    h.rh = none;
    h.part.c = nullptr;
    h.part.n = nullptr;
    int cur = 0;
    for (int k = 0; k < p; k++) {
        const int nxt = cur ^ 1;
        h.p = 0;
        h.in = f[cur][1];
        h.out = f[nxt][0];
        launch_hop<P, EPI_PLAIN, DOT_NONE>(ctx, plan.nblocks, plan.TS * plan.CG, h);
        h.p = 1;
        h.in = f[cur][0];
        h.out = f[nxt][1];
        launch_hop<P, EPI_PLAIN, DOT_NONE>(ctx, plan.nblocks, plan.TS * plan.CG, h);
        cur = nxt;
    }
    k_unpack_low<P><<<nb, 256, 0, st>>>(pa, f[cur][0], f[cur][1]);
    const int64_t nc = (int64_t)pa.it.ncol * 2 * pa.it.nh * 12;
    k_scale_complex<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>((double2 *)out, nc, std::pow(job.kappa, p));
    ctx->launches += 3 + 2 * (long)p;
    DDP_CUDA(ctx, cudaGetLastError());
    return DDP_OK;
}

// Timing of one inner-loop stencil variant on fields of the given domain
// (contents: zeros, which does not change the kernel's work), CUDA events on
// the context's stream around `iters` back-to-back launches after 3 warm-up
// launches.  kernel: DDP_HOP_PLAIN  tmp = H_oe p;  DDP_HOP_SCHUR_RHAT  v = p -
// kappa^2 H_eo tmp with the (rh, v) partials;  DDP_HOP_SCHUR_TS  t = s -
// kappa^2 H_eo tmp with the (t, s), (t, t) partials.  Algorithmic bytes per
// launch: the spinors the variant reads or writes once per output
// site-column (2, 4 and 3 of them; the shadow residual of the (rh, v) variant
// in its own storage, BF16 for FP32 storage) plus the 8 links touching each
// output site once for all columns.
template <class P>
int time_hop_impl(ddp_ctx *ctx, const Job &job, int prec, int kernel, int iters, float *ms, double *bytes) {
    std::vector<Job> jobs(1, job);
    Plan plan;
    make_plan(jobs, prec, ctx->prm, plan);
    const int64_t NF = plan.nfield;
    size_t need = 4 * field_bytes<P>(NF) + 2 * ((size_t)plan.npart * 24 + 1024) + sizeof(Item) + 1024;
    DDP_CUDA(ctx, ctx->scratch.reserve(need));
    Arena &a = ctx->scratch;
    a.reset();
    FieldView in = carve_field<P>(a, NF), v1 = carve_field<P>(a, NF), rhv = carve_field<P>(a, NF),
              out = carve_field<P>(a, NF);
    Partials A;
    A.c = (double2 *)a.take(plan.npart * sizeof(double2));
    A.n = (double *)a.take(plan.npart * sizeof(double));
    Item *d_items = (Item *)a.take(sizeof(Item));
    cudaStream_t st = ctx->stream;
    DDP_CUDA(ctx, cudaMemcpyAsync(d_items, plan.items.data(), sizeof(Item), cudaMemcpyHostToDevice, st));
    size_t fb = (size_t)NF * sizeof(typename P::chunk) * P::NCH;
    DDP_CUDA(ctx, cudaMemsetAsync(in.p, 0, fb, st));
    DDP_CUDA(ctx, cudaMemsetAsync(v1.p, 0, fb, st));
    DDP_CUDA(ctx, cudaMemsetAsync(rhv.p, 0, fb, st));
    if (P::SCALED) {
        DDP_CUDA(ctx, cudaMemsetAsync(in.scale, 0, NF * sizeof(float), st));
        DDP_CUDA(ctx, cudaMemsetAsync(v1.scale, 0, NF * sizeof(float), st));
        DDP_CUDA(ctx, cudaMemsetAsync(rhv.scale, 0, NF * sizeof(float), st));
    }
    Launch L;
    L.items = d_items;
    L.nitems = 1;
    L.TS = plan.TS;
    L.CG = plan.CG;
    HopArgs h;
    FieldView none = {nullptr, nullptr, 0};
    h.st = nullptr;
    h.skip = 0;
    h.L = L;
    h.p = (kernel == DDP_HOP_PLAIN) ? 1 : 0;
    h.in = in;
    h.out = out;
    h.v1 = (kernel == DDP_HOP_PLAIN) ? none : v1;
    h.v2 = none;
    h.rh = (kernel == DDP_HOP_SCHUR_RHAT) ? rhv : none;
    h.part = A;
    DDP_CUDA(ctx, (set_hop_carveout<P, false>(carveout_for(ctx->prm, prec))));
    auto launch = [&]() {
        if (kernel == DDP_HOP_PLAIN)
            launch_hop<P, EPI_PLAIN, DOT_NONE>(ctx, plan.nblocks, plan.TS * plan.CG, h);
        else if (kernel == DDP_HOP_SCHUR_RHAT)
            launch_hop<P, EPI_MHAT, DOT_RHAT>(ctx, plan.nblocks, plan.TS * plan.CG, h);
        else
            launch_hop<P, EPI_MHAT, DOT_TS>(ctx, plan.nblocks, plan.TS * plan.CG, h);
    };
    cudaEvent_t e0, e1;
    DDP_CUDA(ctx, cudaEventCreate(&e0));
    DDP_CUDA(ctx, cudaEventCreate(&e1));
    for (int i = 0; i < 3; i++) launch();
    DDP_CUDA(ctx, cudaEventRecord(e0, st));
    for (int i = 0; i < iters; i++) launch();
    DDP_CUDA(ctx, cudaEventRecord(e1, st));
    DDP_CUDA(ctx, cudaEventSynchronize(e1));
    float t = 0;
    DDP_CUDA(ctx, cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    DDP_CUDA(ctx, cudaGetLastError());
    ctx->launches += 3 + iters;
    *ms = t / iters;
    const double site_cols = (double)plan.items[0].nh * job.ncol;
    const double spinor = (double)sizeof(typename P::chunk) * P::NCH + (P::SCALED ? 4.0 : 0.0);
    const double link = P::IS64 ? 144.0 : (std::is_same<P, PF32>::value ? 48.0 : 24.0);
    using SH = typename ShadowOf<P>::type;
    const double shadow = (double)sizeof(typename SH::chunk) * SH::NCH + (SH::SCALED ? 4.0 : 0.0);
    // spinors of the storage format read or written once per output site-column, plus
    // the shadow residual (in its own format) of the (rh, v) variant
    const double per_col = (kernel == DDP_HOP_PLAIN) ? 2 * spinor
                           : (kernel == DDP_HOP_SCHUR_RHAT) ? 3 * spinor + shadow : 3 * spinor;
    // every link touching an output site: 8 per output site (4 forward + 4 backward)
    *bytes = site_cols * per_col + (double)plan.items[0].nh * 8.0 * link;
    return DDP_OK;
}

}  // namespace ddp
