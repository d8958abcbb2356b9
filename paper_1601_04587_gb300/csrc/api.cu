// C ABI of libddp: contexts, resident gauge fields, domains, solves, series
// terms.  Contractions live in contract.cu, serving in serve.cu and the
// templated solver engine in engine.cuh (one instantiation per storage format).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>

#include "ddp_host.h"

using namespace ddp;

namespace ddp {

int set_cuda_error(ddp_ctx *ctx, cudaError_t e, const char *where) {
    if (ctx) snprintf(ctx->last_error, sizeof(ctx->last_error), "%s: %s", where, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return DDP_ERR_OOM;
    return DDP_ERR_CUDA;
}

cudaError_t Arena::reserve(size_t need) {
    if (need <= bytes) return cudaSuccess;
    if (base) {
        cudaError_t e = cudaFree(base);
        if (e != cudaSuccess) return e;
        base = nullptr;
        bytes = 0;
    }
    size_t want = need + need / 8;
    cudaError_t e = cudaMalloc(&base, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&base, need);
        if (e != cudaSuccess) {
            base = nullptr;
            return e;
        }
        want = need;
    }
    bytes = want;
    return cudaSuccess;
}

Arena::~Arena() {
    if (base) cudaFree(base);
}

void make_plan(const std::vector<Job> &jobs, int prec, const EngineParams &prm, Plan &plan) {
    int maxcol = 1;
    for (auto &j : jobs) maxcol = std::max(maxcol, j.ncol);
    int tuned = (prec >= 0 && prec < 4) ? prm.CG_prec[prec] : 0;
    int CG = std::min(prm.CG ? prm.CG : (tuned ? tuned : maxcol), HOP_MAX_CG);
    int TS = HOP_TS;
    plan.TS = TS;
    plan.CG = CG;
    plan.items.clear();
    int64_t fbase = 0, pbase = 0;
    int blk = 0, solve = 0;
    for (auto &j : jobs) {
        Item it;
        memset(&it, 0, sizeof(it));
        int par = 0;
        for (int m = 0; m < 4; m++) {
            it.L[m] = j.g->L[m];
            it.o[m] = ((j.o[m] % it.L[m]) + it.L[m]) % it.L[m];
            it.e[m] = j.e[m];
            if (j.e[m] < it.L[m]) it.rmask |= 1 << m;
            par += it.o[m];
        }
        it.par_o = par & 1;
        it.bc = j.g->bc;
        int64_t n = (int64_t)it.e[0] * it.e[1] * it.e[2] * it.e[3];
        it.nh = (int)(n / 2);
        it.ntiles = (it.nh + TS - 1) / TS;
        it.ncol = j.ncol;
        it.ncg = (j.ncol + CG - 1) / CG;
        it.blk0 = blk;
        it.solve0 = solve;
        it.fbase = fbase;
        it.pbase = pbase;
        it.kappa = j.kappa;
        it.links = j.g->links(prec);
        it.links64 = j.g->u64;
        it.gV = j.g->V;
        if (j.clov) {
            it.clov = (prec == DDP_PREC_FP64) ? (const void *)j.clov->t64 : (const void *)j.clov->t32;
            it.clovinv = (prec == DDP_PREC_FP64) ? (const void *)j.clov->ti64 : (const void *)j.clov->ti32;
            it.clov64 = j.clov->t64;
        }
        blk += it.ntiles * it.ncg;
        solve += j.ncol;
        fbase += (int64_t)j.ncol * it.nh;
        pbase += (int64_t)j.ncol * it.ntiles;
        plan.items.push_back(it);
    }
    plan.nblocks = blk;
    plan.nsolve = solve;
    plan.nfield = std::max<int64_t>(fbase, 1);
    plan.npart = std::max<int64_t>(pbase, 1);
}

int solve_jobs_dispatch(ddp_ctx *ctx, int prec, std::vector<Job> &jobs, std::vector<JobInfo> &infos) {
    switch (prec) {
        case DDP_PREC_FP64: return solve_jobs<PF64>(ctx, prec, jobs, infos);
        case DDP_PREC_MIXED_FP32: return solve_jobs<PF32>(ctx, prec, jobs, infos);
        case DDP_PREC_MIXED_FP16: return solve_jobs<PF16>(ctx, prec, jobs, infos);
        case DDP_PREC_MIXED_BF16: return solve_jobs<PBF16>(ctx, prec, jobs, infos);
    }
    return DDP_ERR_INVALID_ARG;
}

template <class P>
int apply_dirac_impl(ddp_ctx *ctx, const Job &job, const double *psi, double *out, int prec);
template <class P>
int hop_power_impl(ddp_ctx *ctx, const Job &job, int p, const double *psi, double *out);
template <class P>
int time_hop_impl(ddp_ctx *ctx, const Job &job, int prec, int kernel, int iters, float *ms, double *bytes);

}  // namespace ddp

// ---------------------------------------------------------------- helpers

namespace {

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A user buffer staged on the device when it lives in host memory.
struct Staged {
    ddp_ctx *ctx;
    const void *user;
    void *dev = nullptr;
    size_t bytes;
    bool owned = false;
    int init(ddp_ctx *c, const void *u, size_t b, bool copy_in) {
        ctx = c;
        user = u;
        bytes = b;
        if (!u) return DDP_ERR_INVALID_ARG;
        if (is_device_ptr(u)) {
            dev = const_cast<void *>(u);
            return DDP_OK;
        }
        cudaError_t e = cudaMallocAsync(&dev, b, c->stream);
        if (e != cudaSuccess) return set_cuda_error(c, e, "staging allocation");
        owned = true;
        if (copy_in) {
            e = cudaMemcpyAsync(dev, u, b, cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) return set_cuda_error(c, e, "host to device copy");
        }
        return DDP_OK;
    }
    int copy_out() {
        if (!owned) return DDP_OK;
        cudaError_t e = cudaMemcpyAsync(const_cast<void *>(user), dev, bytes, cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "device to host copy");
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "synchronize");
        return DDP_OK;
    }
    ~Staged() {
        if (owned && dev) cudaFreeAsync(dev, ctx->stream);
    }
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// ---------------------------------------------------------- gauge packing
//
// Copies the links of (part of) a lattice into the resident formats: FP64
// full matrices and 2-row FP32/FP16/BF16, all in the even-odd site order.
// Also measures max |U^+ U - 1| and |det U - 1| (non-finite values count as
// infinite) so that fields the 2-row formats cannot represent are rejected.

struct GaugePackArgs {
    const double2 *U;     // [4][nsrc][9]
    int64_t nsrc;         // sites provided (V, or the box size)
    int o[4], e[4];       // box (e = L for a whole lattice)
    int L[4];
    int64_t V;
    double2 *u64;
    float4 *u32;
    uint2 *u16, *ub16;
    float *maxdev;        // device scalar (>= 0), atomically maximised via int bits
};

__device__ __forceinline__ void atomic_max_nonneg(float *a, float v) {
    atomicMax(reinterpret_cast<int *>(a), __float_as_int(v));
}

__global__ void k_pack_gauge(GaugePackArgs a) {
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= 4 * a.nsrc) return;
    int mu = (int)(g / a.nsrc);
    int64_t l = g - mu * a.nsrc;
    int k[4];
    int64_t r = l;
    for (int m = 3; m >= 0; m--) {
        k[m] = (int)(r % a.e[m]);
        r /= a.e[m];
    }
    int x[4];
    for (int m = 0; m < 4; m++) x[m] = (a.o[m] + k[m]) % a.L[m];
    int64_t lex = (((int64_t)x[0] * a.L[1] + x[1]) * a.L[2] + x[2]) * a.L[3] + x[3];
    int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    int64_t row = (par ? a.V / 2 : 0) + (lex >> 1);
    double2 u[9];
    const double2 *src = a.U + ((int64_t)mu * a.nsrc + l) * 9;
    bool finite = true;
    for (int j = 0; j < 9; j++) {
        u[j] = src[j];
        finite = finite && isfinite(u[j].x) && isfinite(u[j].y);
    }
    // deviation from SU(3)
    double dev = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double re = 0, im = 0;
            for (int c = 0; c < 3; c++) {  // (U^+ U)_{ij} = sum_c conj(U_ci) U_cj
                double2 a1 = u[c * 3 + i], b1 = u[c * 3 + j];
                re += a1.x * b1.x + a1.y * b1.y;
                im += a1.x * b1.y - a1.y * b1.x;
            }
            if (i == j) re -= 1.0;
            dev = fmax(dev, sqrt(re * re + im * im));
        }
    // determinant
    double2 m0 = u[0], m1 = u[1], m2 = u[2], m3 = u[3], m4 = u[4], m5 = u[5], m6 = u[6], m7 = u[7], m8 = u[8];
    auto cm = [](double2 p, double2 q) { return make_double2(p.x * q.x - p.y * q.y, p.x * q.y + p.y * q.x); };
    auto cs = [](double2 p, double2 q) { return make_double2(p.x - q.x, p.y - q.y); };
    double2 c0 = cs(cm(m4, m8), cm(m5, m7));
    double2 c1 = cs(cm(m5, m6), cm(m3, m8));
    double2 c2 = cs(cm(m3, m7), cm(m4, m6));
    double2 d0 = cm(m0, c0), d1 = cm(m1, c1), d2 = cm(m2, c2);
    double dre = d0.x + d1.x + d2.x - 1.0, dim = d0.y + d1.y + d2.y;
    dev = fmax(dev, sqrt(dre * dre + dim * dim));
    if (!finite || !(dev == dev)) dev = 1e30;
    atomic_max_nonneg(a.maxdev, (float)fmin(dev, 1e30));
    for (int j = 0; j < 9; j++) a.u64[((int64_t)mu * 9 + j) * a.V + row] = u[j];
    float4 f0 = make_float4((float)u[0].x, (float)u[0].y, (float)u[1].x, (float)u[1].y);
    float4 f1 = make_float4((float)u[2].x, (float)u[2].y, (float)u[3].x, (float)u[3].y);
    float4 f2 = make_float4((float)u[4].x, (float)u[4].y, (float)u[5].x, (float)u[5].y);
    a.u32[((int64_t)mu * 3 + 0) * a.V + row] = f0;
    a.u32[((int64_t)mu * 3 + 1) * a.V + row] = f1;
    a.u32[((int64_t)mu * 3 + 2) * a.V + row] = f2;
    a.u16[((int64_t)mu * 3 + 0) * a.V + row] = make_uint2(f2h(f0.x, f0.y), f2h(f0.z, f0.w));
    a.u16[((int64_t)mu * 3 + 1) * a.V + row] = make_uint2(f2h(f1.x, f1.y), f2h(f1.z, f1.w));
    a.u16[((int64_t)mu * 3 + 2) * a.V + row] = make_uint2(f2h(f2.x, f2.y), f2h(f2.z, f2.w));
    a.ub16[((int64_t)mu * 3 + 0) * a.V + row] = make_uint2(f2b(f0.x, f0.y), f2b(f0.z, f0.w));
    a.ub16[((int64_t)mu * 3 + 1) * a.V + row] = make_uint2(f2b(f1.x, f1.y), f2b(f1.z, f1.w));
    a.ub16[((int64_t)mu * 3 + 2) * a.V + row] = make_uint2(f2b(f2.x, f2.y), f2b(f2.z, f2.w));
}

// Domain index maps: global site index and even-odd index per local site.
__global__ void k_domain_maps(Item it, int64_t *gidx, int64_t *eoidx) {
    int64_t n = 2 * (int64_t)it.nh;
    int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (l >= n) return;
    int k[4];
    local_coords(it, (int)l, k);
    int x[4];
    for (int m = 0; m < 4; m++) x[m] = (it.o[m] + k[m]) % it.L[m];
    if (gidx) gidx[l] = global_lex(it, x);
    if (eoidx) eoidx[l] = l >> 1;
}

// Series term T = S_big - E S_small (Eq. Dseries): thread per (column, big-box site).
struct SeriesArgs {
    Item big, small;
    const double2 *Sb, *Ss;
    double2 *T;
    int ncol;
};

__global__ void k_series(SeriesArgs a) {
    int64_t nb = 2 * (int64_t)a.big.nh, ns = 2 * (int64_t)a.small.nh;
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nb * a.ncol) return;
    int col = (int)(g / nb);
    int l = (int)(g - col * nb);
    int k[4];
    local_coords(a.big, l, k);
    int ks[4];
    bool inside = true;
    for (int m = 0; m < 4; m++) {
        int x = (a.big.o[m] + k[m]) % a.big.L[m];
        int d = x - a.small.o[m];
        if (d < 0) d += a.big.L[m];
        ks[m] = d;
        inside = inside && (d < a.small.e[m]);
    }
    const double2 *sb = a.Sb + ((int64_t)col * nb + l) * 12;
    double2 *t = a.T + ((int64_t)col * nb + l) * 12;
    if (inside) {
        int ls = local_lex(a.small, ks);
        const double2 *ss = a.Ss + ((int64_t)col * ns + ls) * 12;
        for (int j = 0; j < 12; j++) t[j] = make_double2(sb[j].x - ss[j].x, sb[j].y - ss[j].y);
    } else {
        for (int j = 0; j < 12; j++) t[j] = sb[j];
    }
}

// sigma = -D[to, from minus to] psi (Eq. blkdec): for every site y of `to`, the hops
// of D_hop that the Dirichlet boundary of `to` drops and that start at a site of
// `from`; D = 1/(2 kappa) - D_hop / 2, so sigma = + D_hop[to, from minus to] psi / 2.
struct BoundaryArgs {
    Item to, from;
    const double2 *psi;  // [ncol][n_from][12]
    double2 *sigma;      // [ncol][n_to][12]
    int ncol;
};

template <int D>
__device__ __forceinline__ void boundary_hop(const BoundaryArgs &a, const int x[4], int px, int col,
                                             cx<double> acc[4][3]) {
    constexpr int MU = D >> 1;
    constexpr bool FWD = !(D & 1);
    const Item &t = a.to;
    int w[4] = {x[0], x[1], x[2], x[3]};
    double f = 1.0;
    if (FWD) {
        w[MU] = x[MU] + 1;
        if (w[MU] == t.L[MU]) {
            w[MU] = 0;
            if (MU == 0 && t.bc == 2) return;
            if (MU == 0 && t.bc == 1) f = -1.0;
        }
    } else {
        w[MU] = x[MU] - 1;
        if (w[MU] < 0) {
            w[MU] = t.L[MU] - 1;
            if (MU == 0 && t.bc == 2) return;
            if (MU == 0 && t.bc == 1) f = -1.0;
        }
    }
    int kt[4], kf[4];
    bool in_to = true, in_from = true;
    for (int m = 0; m < 4; m++) {
        int dt = w[m] - t.o[m], df = w[m] - a.from.o[m];
        if (dt < 0) dt += t.L[m];
        if (df < 0) df += t.L[m];
        kt[m] = dt;
        kf[m] = df;
        in_to = in_to && (dt < t.e[m]);
        in_from = in_from && (df < a.from.e[m]);
    }
    if (in_to || !in_from) return;
    const int64_t nf = 2 * (int64_t)a.from.nh;
    const double2 *ps = a.psi + ((int64_t)col * nf + local_lex(a.from, kf)) * 12;
    double v[24];
    for (int j = 0; j < 12; j++) {
        const double2 c = ps[j];
        v[2 * j] = c.x;
        v[2 * j + 1] = c.y;
    }
    cx<double> u[3][3];
    if (FWD) {
        load_link<PF64>(t.links64, t.gV, MU, link_row(t, x, px), u);
    } else {
        cx<double> b[3][3];
        load_link<PF64>(t.links64, t.gV, MU, link_row(t, w, px ^ 1), b);
        for (int i = 0; i < 3; i++)
            for (int k = 0; k < 3; k++) u[i][k] = conj(b[k][i]);
    }
    for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++) u[i][k] = f * u[i][k];
    hop_step<D, true>(v, u, acc, 1.0);
}

__global__ void k_boundary_source(BoundaryArgs a) {
    const int64_t nt = 2 * (int64_t)a.to.nh;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nt * a.ncol) return;
    const int col = (int)(g / nt);
    const int l = (int)(g - col * nt);
    int k[4], x[4];
    local_coords(a.to, l, k);
    int px = 0;
    for (int m = 0; m < 4; m++) {
        x[m] = (a.to.o[m] + k[m]) % a.to.L[m];
        px += x[m];
    }
    px &= 1;
    cx<double> acc[4][3];
    for (int s2 = 0; s2 < 4; s2++)
        for (int c = 0; c < 3; c++) acc[s2][c] = mk(0.0, 0.0);
    boundary_hop<0>(a, x, px, col, acc);
    boundary_hop<1>(a, x, px, col, acc);
    boundary_hop<2>(a, x, px, col, acc);
    boundary_hop<3>(a, x, px, col, acc);
    boundary_hop<4>(a, x, px, col, acc);
    boundary_hop<5>(a, x, px, col, acc);
    boundary_hop<6>(a, x, px, col, acc);
    boundary_hop<7>(a, x, px, col, acc);
    double2 *out = a.sigma + ((int64_t)col * nt + l) * 12;
    for (int s2 = 0; s2 < 4; s2++)
        for (int c = 0; c < 3; c++) out[3 * s2 + c] = make_double2(0.5 * acc[s2][c].re, 0.5 * acc[s2][c].im);
}

int check_box(const GaugeDev &g, const int o[4], const int e[4]) {
    for (int m = 0; m < 4; m++)
        if (e[m] < 1 || e[m] > g.L[m]) return DDP_ERR_INVALID_ARG;
    if (e[3] % 2) return DDP_ERR_UNSUPPORTED;
    (void)o;
    return DDP_OK;
}

Item item_of(const GaugeDev &g, const DomainDev &d, int ncol, int prec) {
    Job j;
    memset(&j, 0, sizeof(j));
    j.g = &g;
    memcpy(j.o, d.o, sizeof(j.o));
    memcpy(j.e, d.e, sizeof(j.e));
    j.ncol = ncol;
    j.kappa = 0.1;
    std::vector<Job> js(1, j);
    Plan pl;
    EngineParams prm;
    make_plan(js, prec, prm, pl);
    return pl.items[0];
}

int local_index_of(const GaugeDev &g, const DomainDev &d, const int src[4], int *l) {
    int k[4];
    for (int m = 0; m < 4; m++) {
        if (src[m] < 0 || src[m] >= g.L[m]) return DDP_ERR_INVALID_ARG;
        k[m] = ((src[m] - d.o[m]) % g.L[m] + g.L[m]) % g.L[m];
        if (k[m] >= d.e[m]) return DDP_ERR_INVALID_ARG;
    }
    *l = ((k[0] * d.e[1] + k[1]) * d.e[2] + k[2]) * d.e[3] + k[3];
    return DDP_OK;
}

const char *const kErr[] = {"ok",
                            "invalid argument",
                            "unsupported",
                            "out of device memory",
                            "solver did not converge",
                            "CUDA error",
                            "busy",
                            "not found"};

}  // namespace

// =================================================================== C ABI

extern "C" {

const char *ddp_error_string(int status) {
    if (status < 0 || status > 7) return "unknown status";
    return kErr[status];
}

const char *ddp_last_error(const ddp_ctx *ctx) { return ctx ? ctx->last_error : ""; }

int ddp_version(void) { return 10000; }

int ddp_create(ddp_ctx **out, int device, void *stream) {
    if (!out) return DDP_ERR_INVALID_ARG;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return DDP_ERR_INVALID_ARG;
    }
    ddp_ctx *c = new ddp_ctx();
    c->device = device;
    c->user_stream = (cudaStream_t)stream;
    DeviceGuard dg(device);
    // staging buffers of host-memory arguments come from the device's stream-ordered
    // pool; keep freed blocks in the pool instead of returning them at every sync
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    if (cudaFree(0) != cudaSuccess || cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return DDP_ERR_CUDA;
    }
    *out = c;
    return DDP_OK;
}

int ddp_serve_reset(ddp_ctx *ctx);

int ddp_destroy(ddp_ctx *ctx) {
    if (!ctx) return DDP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ddp_serve_reset(ctx);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    cudaGetLastError();
    for (auto &kv : ctx->gauges) {
        cudaFree(kv.second->u64);
        cudaFree(kv.second->u32);
        cudaFree(kv.second->u16);
        cudaFree(kv.second->ub16);
    }
    cudaEventDestroy(ctx->ev_in);
    cudaEventDestroy(ctx->ev_out);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    cudaStreamDestroy(ctx->stream);
    delete ctx;
    return DDP_OK;
}

int ddp_set_stream(ddp_ctx *ctx, void *stream) {
    if (!ctx) return DDP_ERR_INVALID_ARG;
    ctx->user_stream = (cudaStream_t)stream;
    return DDP_OK;
}

static int load_links(ddp_ctx *ctx, GaugeDev &g, const double *U, const int o[4], const int e[4]) {
    int64_t nsrc = (int64_t)e[0] * e[1] * e[2] * e[3];
    Staged su;
    int rc = su.init(ctx, U, (size_t)4 * nsrc * 9 * sizeof(double2), true);
    if (rc) return rc;
    float *d_dev = nullptr;
    DDP_CUDA(ctx, cudaMallocAsync((void **)&d_dev, sizeof(float), ctx->stream));
    DDP_CUDA(ctx, cudaMemsetAsync(d_dev, 0, sizeof(float), ctx->stream));
    GaugePackArgs a;
    a.U = (const double2 *)su.dev;
    a.nsrc = nsrc;
    for (int m = 0; m < 4; m++) {
        a.o[m] = o[m];
        a.e[m] = e[m];
        a.L[m] = g.L[m];
    }
    a.V = g.V;
    a.u64 = g.u64;
    a.u32 = g.u32;
    a.u16 = g.u16;
    a.ub16 = g.ub16;
    a.maxdev = d_dev;
    int64_t nt = 4 * nsrc;
    k_pack_gauge<<<(unsigned)((nt + 255) / 256), 256, 0, ctx->stream>>>(a);
    ctx->launches++;
    float h_dev = 0;
    DDP_CUDA(ctx, cudaGetLastError());
    DDP_CUDA(ctx, cudaMemcpyAsync(&h_dev, d_dev, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    DDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFreeAsync(d_dev, ctx->stream);
    if (!(h_dev <= 1e-8f)) {
        snprintf(ctx->last_error, sizeof(ctx->last_error), "links are not SU(3): max deviation %g", h_dev);
        return DDP_ERR_INVALID_ARG;
    }
    return DDP_OK;
}

static int alloc_gauge(ddp_ctx *ctx, GaugeDev &g) {
    cudaError_t e;
    e = cudaMalloc((void **)&g.u64, (size_t)4 * 9 * g.V * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&g.u32, (size_t)4 * 3 * g.V * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc((void **)&g.u16, (size_t)4 * 3 * g.V * sizeof(uint2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&g.ub16, (size_t)4 * 3 * g.V * sizeof(uint2));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(g.u64);
        cudaFree(g.u32);
        cudaFree(g.u16);
        cudaFree(g.ub16);
        g.u64 = nullptr;
        g.u32 = nullptr;
        g.u16 = g.ub16 = nullptr;
        return set_cuda_error(ctx, e, "gauge allocation");
    }
    return DDP_OK;
}

static void free_gauge(GaugeDev &g) {
    cudaFree(g.u64);
    cudaFree(g.u32);
    cudaFree(g.u16);
    cudaFree(g.ub16);
}

int ddp_load_gauge(ddp_ctx *ctx, const double *U, const int L[4], int time_bc, int *gauge_id) {
    if (!ctx || !U || !L || !gauge_id) return DDP_ERR_INVALID_ARG;
    if (time_bc < 0 || time_bc > 2) return DDP_ERR_INVALID_ARG;
    for (int m = 0; m < 4; m++) {
        if (L[m] < 2) return DDP_ERR_INVALID_ARG;
        if (L[m] % 2) return DDP_ERR_UNSUPPORTED;
    }
    DeviceGuard dg(ctx->device);
    StreamJoin sj(ctx);
    auto g = std::make_unique<GaugeDev>();
    g->V = 1;
    for (int m = 0; m < 4; m++) {
        g->L[m] = L[m];
        g->V *= L[m];
    }
    if (g->V > (int64_t)1 << 31) return DDP_ERR_UNSUPPORTED;
    g->bc = time_bc;
    int rc = alloc_gauge(ctx, *g);
    if (rc) return rc;
    int o[4] = {0, 0, 0, 0};
    rc = load_links(ctx, *g, U, o, g->L);
    if (rc) {
        cudaStreamSynchronize(ctx->stream);
        free_gauge(*g);
        return rc;
    }
    int id = ctx->next_gauge++;
    ctx->gauges[id] = std::move(g);
    *gauge_id = id;
    return DDP_OK;
}

int ddp_load_gauge_region(ddp_ctx *ctx, int base_gauge_id, const int origin[4], const int extent[4],
                          const double *U_box, int *gauge_id) {
    if (!ctx || !origin || !extent || !U_box || !gauge_id) return DDP_ERR_INVALID_ARG;
    auto it = ctx->gauges.find(base_gauge_id);
    if (it == ctx->gauges.end()) return DDP_ERR_NOT_FOUND;
    const GaugeDev &b = *it->second;
    int o[4];
    for (int m = 0; m < 4; m++) {
        if (extent[m] < 1 || extent[m] > b.L[m]) return DDP_ERR_INVALID_ARG;
        o[m] = ((origin[m] % b.L[m]) + b.L[m]) % b.L[m];
    }
    DeviceGuard dg(ctx->device);
    StreamJoin sj(ctx);
    auto g = std::make_unique<GaugeDev>();
    memcpy(g->L, b.L, sizeof(g->L));
    g->V = b.V;
    g->bc = b.bc;
    int rc = alloc_gauge(ctx, *g);
    if (rc) return rc;
    DDP_CUDA(ctx, cudaMemcpyAsync(g->u64, b.u64, (size_t)4 * 9 * b.V * sizeof(double2), cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    DDP_CUDA(ctx, cudaMemcpyAsync(g->u32, b.u32, (size_t)4 * 3 * b.V * sizeof(float4), cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    DDP_CUDA(ctx, cudaMemcpyAsync(g->u16, b.u16, (size_t)4 * 3 * b.V * sizeof(uint2), cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    DDP_CUDA(ctx, cudaMemcpyAsync(g->ub16, b.ub16, (size_t)4 * 3 * b.V * sizeof(uint2), cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    rc = load_links(ctx, *g, U_box, o, extent);
    if (rc) {
        cudaStreamSynchronize(ctx->stream);
        free_gauge(*g);
        return rc;
    }
    int id = ctx->next_gauge++;
    ctx->gauges[id] = std::move(g);
    *gauge_id = id;
    return DDP_OK;
}

int ddp_free_gauge(ddp_ctx *ctx, int gauge_id) {
    if (!ctx) return DDP_ERR_INVALID_ARG;
    auto it = ctx->gauges.find(gauge_id);
    if (it == ctx->gauges.end()) return DDP_ERR_NOT_FOUND;
    for (auto &d : ctx->domains)
        if (d.second.gauge_id == gauge_id) return DDP_ERR_BUSY;
    DeviceGuard dg(ctx->device);
    StreamJoin sj(ctx);
    cudaStreamSynchronize(ctx->stream);
    free_gauge(*it->second);
    ctx->gauges.erase(it);
    return DDP_OK;
}

int ddp_set_domain(ddp_ctx *ctx, int gauge_id, const int origin[4], const int extent[4], int *domain_id) {
    if (!ctx || !origin || !extent || !domain_id) return DDP_ERR_INVALID_ARG;
    auto it = ctx->gauges.find(gauge_id);
    if (it == ctx->gauges.end()) return DDP_ERR_NOT_FOUND;
    int rc = check_box(*it->second, origin, extent);
    if (rc) return rc;
    DomainDev d;
    d.gauge_id = gauge_id;
    d.n = 1;
    for (int m = 0; m < 4; m++) {
        d.o[m] = ((origin[m] % it->second->L[m]) + it->second->L[m]) % it->second->L[m];
        d.e[m] = extent[m];
        d.n *= extent[m];
    }
    int id = ctx->next_domain++;
    ctx->domains[id] = d;
    *domain_id = id;
    return DDP_OK;
}

int ddp_free_domain(ddp_ctx *ctx, int domain_id) {
    if (!ctx) return DDP_ERR_INVALID_ARG;
    return ctx->domains.erase(domain_id) ? DDP_OK : DDP_ERR_NOT_FOUND;
}

static int find_domain(ddp_ctx *ctx, int domain_id, const DomainDev **d, const GaugeDev **g) {
    auto it = ctx->domains.find(domain_id);
    if (it == ctx->domains.end()) return DDP_ERR_NOT_FOUND;
    auto gi = ctx->gauges.find(it->second.gauge_id);
    if (gi == ctx->gauges.end()) return DDP_ERR_NOT_FOUND;
    *d = &it->second;
    *g = gi->second.get();
    return DDP_OK;
}

int ddp_domain_sites(ddp_ctx *ctx, int domain_id, int64_t *n_sites, int64_t *gidx, int64_t *eoidx) {
    if (!ctx) return DDP_ERR_INVALID_ARG;
    const DomainDev *d;
    const GaugeDev *g;
    int rc = find_domain(ctx, domain_id, &d, &g);
    if (rc) return rc;
    if (n_sites) *n_sites = d->n;
    if (!gidx && !eoidx) return DDP_OK;
    DeviceGuard dg(ctx->device);
    StreamJoin sj(ctx);
    Item it = item_of(*g, *d, 1, DDP_PREC_FP64);
    Staged sg, se;
    if (gidx && (rc = sg.init(ctx, gidx, d->n * sizeof(int64_t), false))) return rc;
    if (eoidx && (rc = se.init(ctx, eoidx, d->n * sizeof(int64_t), false))) return rc;
    k_domain_maps<<<(unsigned)((d->n + 255) / 256), 256, 0, ctx->stream>>>(it, gidx ? (int64_t *)sg.dev : nullptr,
                                                                       eoidx ? (int64_t *)se.dev : nullptr);
    ctx->launches++;
    DDP_CUDA(ctx, cudaGetLastError());
    if (gidx && (rc = sg.copy_out())) return rc;
    if (eoidx && (rc = se.copy_out())) return rc;
    DDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return DDP_OK;
}

int ddp_apply_dirac(ddp_ctx *ctx, int domain_id, double kappa, double csw, const double *psi, double *out, int ncol,
                    int precision) {
    if (!ctx || !psi || !out || ncol < 1 || !(kappa > 0) || !std::isfinite(csw)) return DDP_ERR_INVALID_ARG;
    if (precision < 0 || precision > 3) return DDP_ERR_INVALID_ARG;
    const DomainDev *d;
    const GaugeDev *g;
    int rc = find_domain(ctx, domain_id, &d, &g);
    if (rc) return rc;
    DeviceGuard dg(ctx->device);
    StreamJoin sj(ctx);
    size_t bytes = (size_t)ncol * d->n * 12 * sizeof(double2);
    Staged si, so;
    if ((rc = si.init(ctx, psi, bytes, true))) return rc;
    if ((rc = so.init(ctx, out, bytes, false))) return rc;
    Job j;
    memset(&j, 0, sizeof(j));
    j.g = g;
    memcpy(j.o, d->o, sizeof(j.o));
    memcpy(j.e, d->e, sizeof(j.e));
    j.kappa = kappa;
    j.ncol = ncol;
    if (csw != 0.0 && (rc = clover_for(ctx, *const_cast<GaugeDev *>(g), kappa, csw, &j.clov))) return rc;
    switch (precision) {
        case DDP_PREC_FP64: rc = apply_dirac_impl<PF64>(ctx, j, (const double *)si.dev, (double *)so.dev, precision); break;
        case DDP_PREC_MIXED_FP32: rc = apply_dirac_impl<PF32>(ctx, j, (const double *)si.dev, (double *)so.dev, precision); break;
        case DDP_PREC_MIXED_FP16: rc = apply_dirac_impl<PF16>(ctx, j, (const double *)si.dev, (double *)so.dev, precision); break;
        default: rc = apply_dirac_impl<PBF16>(ctx, j, (const double *)si.dev, (double *)so.dev, precision); break;
    }
    if (rc) return rc;
    if ((rc = so.copy_out())) return rc;
    DDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return DDP_OK;
}

// (kappa D_hop)^p psi on a domain, FP64 (Eq. HPEtr, Sec. 2 restriction).
int ddp_hop_power(ddp_ctx *ctx, int domain_id, double kappa, int p, const double *psi, double *out, int ncol) {
    if (!ctx || !psi || !out || ncol < 1 || !(kappa > 0) || p < 0 || p > 64) return DDP_ERR_INVALID_ARG;
    const DomainDev *d;
    const GaugeDev *g;
    int rc = find_domain(ctx, domain_id, &d, &g);
    if (rc) return rc;
    DeviceGuard dg(ctx->device);
    StreamJoin sj(ctx);
    size_t bytes = (size_t)ncol * d->n * 12 * sizeof(double2);
    Staged si, so;
    if ((rc = si.init(ctx, psi, bytes, true))) return rc;
    if ((rc = so.init(ctx, out, bytes, false))) return rc;
    Job j;
    memset(&j, 0, sizeof(j));
    j.g = g;
    memcpy(j.o, d->o, sizeof(j.o));
    memcpy(j.e, d->e, sizeof(j.e));
    j.kappa = kappa;
    j.ncol = ncol;
    if ((rc = hop_power_impl<PF64>(ctx, j, p, (const double *)si.dev, (double *)so.dev))) return rc;
    if ((rc = so.copy_out())) return rc;
    DDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return DDP_OK;
}

// Average duration of one inner-loop stencil variant on a domain, timed with
// CUDA events on the context's stream over `iters` back-to-back launches.
int ddp_time_hop(ddp_ctx *ctx, int domain_id, double kappa, int ncol, int precision, int kernel, int iters,
                 float *ms_per_launch, double *bytes_per_launch) {
    if (!ctx || ncol < 1 || iters < 1 || !ms_per_launch) return DDP_ERR_INVALID_ARG;
    if (kernel < DDP_HOP_PLAIN || kernel > DDP_HOP_SCHUR_TS) return DDP_ERR_INVALID_ARG;
    const DomainDev *d;
    const GaugeDev *g;
    int rc = find_domain(ctx, domain_id, &d, &g);
    if (rc) return rc;
    DeviceGuard dg(ctx->device);
    StreamJoin sj(ctx);
    Job j;
    memset(&j, 0, sizeof(j));
    j.g = g;
    memcpy(j.o, d->o, sizeof(j.o));
    memcpy(j.e, d->e, sizeof(j.e));
    j.kappa = kappa;
    j.ncol = ncol;
    double bytes = 0;
    switch (precision) {
        case DDP_PREC_FP64: rc = time_hop_impl<PF64>(ctx, j, precision, kernel, iters, ms_per_launch, &bytes); break;
        case DDP_PREC_MIXED_FP32: rc = time_hop_impl<PF32>(ctx, j, precision, kernel, iters, ms_per_launch, &bytes); break;
        case DDP_PREC_MIXED_FP16: rc = time_hop_impl<PF16>(ctx, j, precision, kernel, iters, ms_per_launch, &bytes); break;
        case DDP_PREC_MIXED_BF16: rc = time_hop_impl<PBF16>(ctx, j, precision, kernel, iters, ms_per_launch, &bytes); break;
        default: return DDP_ERR_INVALID_ARG;
    }
    if (bytes_per_launch) *bytes_per_launch = bytes;
    return rc;
}

static int run_solves(ddp_ctx *ctx, const ddp_solve_req *reqs, int n, int precision, ddp_solve_info *infos) {
    if (precision < 0 || precision > 3) return DDP_ERR_INVALID_ARG;
    auto t0 = std::chrono::steady_clock::now();
    std::vector<Job> jobs(n);
    std::vector<std::unique_ptr<Staged>> st_in(n), st_out(n);
    int clover_pairs = 0;
    for (int i = 0; i < n; i++) {
        const ddp_solve_req &r = reqs[i];
        if (!(r.kappa > 0) || !(r.tol > 0) || !r.out || !std::isfinite(r.csw)) return DDP_ERR_INVALID_ARG;
        const DomainDev *d;
        const GaugeDev *g;
        int rc = find_domain(ctx, r.domain_id, &d, &g);
        if (rc) return rc;
        Job &j = jobs[i];
        memset(&j, 0, sizeof(j));
        j.g = g;
        if (r.csw != 0.0) {
            // clover term of (gauge, kappa, c_sw): at most CLOVER_CACHE distinct pairs per call
            bool seen = false;
            for (int k = 0; k < i; k++)
                seen = seen || (reqs[k].csw != 0.0 && jobs[k].g == g && reqs[k].kappa == r.kappa &&
                                reqs[k].csw == r.csw);
            if (!seen && ++clover_pairs > CLOVER_CACHE) return DDP_ERR_UNSUPPORTED;
            if ((rc = clover_for(ctx, *const_cast<GaugeDev *>(g), r.kappa, r.csw, &j.clov))) return rc;
        }
        memcpy(j.o, d->o, sizeof(j.o));
        memcpy(j.e, d->e, sizeof(j.e));
        j.kappa = r.kappa;
        j.tol = r.tol;
        if (r.eta) {
            if (r.ncol < 1) return DDP_ERR_INVALID_ARG;
            j.ncol = r.ncol;
            st_in[i].reset(new Staged());
            if ((rc = st_in[i]->init(ctx, r.eta, (size_t)r.ncol * d->n * 12 * sizeof(double2), true))) return rc;
            j.eta = (const double *)st_in[i]->dev;
        } else {
            j.ncol = 12;
            if ((rc = local_index_of(*g, *d, r.src, &j.src_l))) return rc;
        }
        st_out[i].reset(new Staged());
        if ((rc = st_out[i]->init(ctx, r.out, (size_t)j.ncol * d->n * 12 * sizeof(double2), false))) return rc;
        j.out = (double *)st_out[i]->dev;
    }
    std::vector<JobInfo> ji;
    int rc = solve_jobs_dispatch(ctx, precision, jobs, ji);
    if (rc) return rc;
    for (int i = 0; i < n; i++)
        if ((rc = st_out[i]->copy_out())) return rc;
    double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int worst = DDP_OK;
    for (int i = 0; i < n; i++) {
        if (ji[i].status != DDP_OK) worst = ji[i].status;
        if (infos) {
            ddp_solve_info &inf = infos[i];
            memset(&inf, 0, sizeof(inf));
            inf.status = ji[i].status;
            inf.ncol = jobs[i].ncol;
            inf.outer_cycles = ji[i].outer;
            inf.inner_iters = ji[i].inner;
            inf.column_iters = ji[i].column_iters;
            inf.seconds = secs;
            double mx = 0;
            for (int c = 0; c < jobs[i].ncol; c++) {
                double r = ji[i].relres[c];
                if (!(r <= mx)) mx = r;
                if (c < DDP_INFO_COLS) inf.rel_residual[c] = r;
            }
            inf.max_rel_residual = mx;
        }
    }
    return worst;
}

int ddp_solve_propagator(ddp_ctx *ctx, int domain_id, double kappa, double csw, const int src[4], double tol,
                         int precision, double *S_out, ddp_solve_info *info) {
    if (!ctx || !src || !S_out) return DDP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    StreamJoin sj(ctx);
    ddp_solve_req r;
    memset(&r, 0, sizeof(r));
    r.domain_id = domain_id;
    r.kappa = kappa;
    r.csw = csw;
    memcpy(r.src, src, sizeof(r.src));
    r.ncol = 12;
    r.tol = tol;
    r.out = S_out;
    return run_solves(ctx, &r, 1, precision, info);
}

int ddp_solve_sources(ddp_ctx *ctx, int domain_id, double kappa, double csw, const double *eta, int ncol, double tol,
                      int precision, double *psi_out, ddp_solve_info *info) {
    if (!ctx || !eta || !psi_out || ncol < 1) return DDP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    StreamJoin sj(ctx);
    ddp_solve_req r;
    memset(&r, 0, sizeof(r));
    r.domain_id = domain_id;
    r.kappa = kappa;
    r.csw = csw;
    r.eta = eta;
    r.ncol = ncol;
    r.tol = tol;
    r.out = psi_out;
    return run_solves(ctx, &r, 1, precision, info);
}

int ddp_solve_batch(ddp_ctx *ctx, const ddp_solve_req *reqs, int n, int precision, ddp_solve_info *infos) {
    if (!ctx || !reqs || n < 1) return DDP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    StreamJoin sj(ctx);
    return run_solves(ctx, reqs, n, precision, infos);
}

int ddp_series_terms(ddp_ctx *ctx, int domain_small, const double *S_small, int domain_big, const double *S_big,
                     double *T_out, int ncol) {
    if (!ctx || !S_small || !S_big || !T_out || ncol < 1) return DDP_ERR_INVALID_ARG;
    const DomainDev *ds, *db;
    const GaugeDev *gs, *gb;
    int rc = find_domain(ctx, domain_small, &ds, &gs);
    if (rc) return rc;
    if ((rc = find_domain(ctx, domain_big, &db, &gb))) return rc;
    for (int m = 0; m < 4; m++)
        if (gs->L[m] != gb->L[m]) return DDP_ERR_INVALID_ARG;
    // containment: every site of the small box lies in the big box
    for (int m = 0; m < 4; m++) {
        if (db->e[m] == gb->L[m]) continue;
        int d0 = ((ds->o[m] - db->o[m]) % gb->L[m] + gb->L[m]) % gb->L[m];
        if (ds->e[m] > db->e[m] || d0 + ds->e[m] > db->e[m]) return DDP_ERR_INVALID_ARG;
    }
    DeviceGuard dg(ctx->device);
    StreamJoin sj(ctx);
    Staged a, b, t;
    if ((rc = a.init(ctx, S_small, (size_t)ncol * ds->n * 12 * sizeof(double2), true))) return rc;
    if ((rc = b.init(ctx, S_big, (size_t)ncol * db->n * 12 * sizeof(double2), true))) return rc;
    if ((rc = t.init(ctx, T_out, (size_t)ncol * db->n * 12 * sizeof(double2), false))) return rc;
    SeriesArgs sa;
    sa.big = item_of(*gb, *db, ncol, DDP_PREC_FP64);
    sa.small = item_of(*gs, *ds, ncol, DDP_PREC_FP64);
    sa.Sb = (const double2 *)b.dev;
    sa.Ss = (const double2 *)a.dev;
    sa.T = (double2 *)t.dev;
    sa.ncol = ncol;
    int64_t nt = (int64_t)ncol * db->n;
    k_series<<<(unsigned)((nt + 255) / 256), 256, 0, ctx->stream>>>(sa);
    ctx->launches++;
    DDP_CUDA(ctx, cudaGetLastError());
    if ((rc = t.copy_out())) return rc;
    DDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return DDP_OK;
}

// Point-source propagators of nested domains Gamma_0 in ... in Gamma_{n-1} solved
// together, the series terms S^(i) - E S^(i-1) (Eq. Dseries) and the contractions
// of every S^(i), with all intermediate results kept on the device: outputs in
// host memory are only ever downloaded, on a second stream while later kernels
// run, never uploaded again.
int ddp_propagator_series(ddp_ctx *ctx, int n, const int *domain_ids, double kappa, double csw, const int src[4],
                          double tol, int precision, double *const *S_out, double *const *T_out, int contract_mask,
                          double *C_out, ddp_solve_info *infos) {
    if (!ctx || n < 1 || !domain_ids || !src) return DDP_ERR_INVALID_ARG;
    const int allowed = (1 << DDP_CONTRACT_PSEUDO_LOCAL) | (1 << DDP_CONTRACT_NUCLEON) | (1 << DDP_CONTRACT_PION);
    if (contract_mask & ~allowed) return DDP_ERR_INVALID_ARG;
    if (contract_mask && !C_out) return DDP_ERR_INVALID_ARG;
    std::vector<const DomainDev *> dom(n);
    std::vector<const GaugeDev *> gau(n);
    for (int i = 0; i < n; i++) {
        int rc = find_domain(ctx, domain_ids[i], &dom[i], &gau[i]);
        if (rc) return rc;
        if (gau[i] != gau[0]) return DDP_ERR_INVALID_ARG;
    }
    const GaugeDev &g = *gau[0];
    // nesting: every site of domain i-1 lies in domain i
    for (int i = 1; i < n; i++)
        for (int m = 0; m < 4; m++) {
            if (dom[i]->e[m] == g.L[m]) continue;
            int d0 = ((dom[i - 1]->o[m] - dom[i]->o[m]) % g.L[m] + g.L[m]) % g.L[m];
            if (dom[i - 1]->e[m] > dom[i]->e[m] || d0 + dom[i - 1]->e[m] > dom[i]->e[m]) return DDP_ERR_INVALID_ARG;
        }
    DeviceGuard dg(ctx->device);
    StreamJoin sj(ctx);
    const int L0 = g.L[0];
    // device buffers: the caller's where they are device memory, else the results arena
    std::vector<size_t> sb(n);
    size_t need = 0;
    for (int i = 0; i < n; i++) {
        sb[i] = (size_t)12 * dom[i]->n * 12 * sizeof(double2);
        if (!(S_out && S_out[i] && is_device_ptr(S_out[i]))) need += sb[i] + 256;
        if (i > 0 && T_out && T_out[i - 1] && !is_device_ptr(T_out[i - 1])) need += sb[i] + 256;
    }
    const size_t cbytes = (size_t)n * 4 * 2 * L0 * sizeof(double);
    const bool c_dev = contract_mask && is_device_ptr(C_out);
    if (contract_mask && !c_dev) need += cbytes + 256;
    DDP_CUDA(ctx, ctx->results.reserve(need + 1024));
    Arena &ar = ctx->results;
    ar.reset();
    std::vector<double *> dS(n), dT(n, nullptr);
    std::vector<char> s_host(n, 0), t_host(n, 0);
    for (int i = 0; i < n; i++) {
        if (S_out && S_out[i] && is_device_ptr(S_out[i])) {
            dS[i] = S_out[i];
        } else {
            dS[i] = (double *)ar.take(sb[i]);
            s_host[i] = S_out && S_out[i];
        }
        if (i > 0 && T_out && T_out[i - 1]) {
            if (is_device_ptr(T_out[i - 1])) {
                dT[i] = T_out[i - 1];
            } else {
                dT[i] = (double *)ar.take(sb[i]);
                t_host[i] = 1;
            }
        }
    }
    double *dC = nullptr;
    if (contract_mask) dC = c_dev ? C_out : (double *)ar.take(cbytes);
    std::vector<ddp_solve_req> reqs(n);
    for (int i = 0; i < n; i++) {
        ddp_solve_req &r = reqs[i];
        memset(&r, 0, sizeof(r));
        r.domain_id = domain_ids[i];
        r.kappa = kappa;
        r.csw = csw;
        memcpy(r.src, src, sizeof(r.src));
        r.ncol = 12;
        r.tol = tol;
        r.out = dS[i];
    }
    // With host outputs the smaller nested domains are solved first and their
    // propagators and series terms are copied to the host while the largest domain
    // solves; with device outputs all domains share one batched solve.  A domain's
    // result does not depend on the batch it is solved in.
    bool host_out = false;
    for (int i = 0; i < n; i++) host_out = host_out || s_host[i] || t_host[i];
    const int first = (host_out && n > 1 && ctx->prm.overlap_downloads) ? n - 1 : n;
    auto combine = [](int a, int b) {
        if (a != DDP_OK && a != DDP_ERR_NOT_CONVERGED) return a;
        if (b != DDP_OK && b != DDP_ERR_NOT_CONVERGED) return b;
        return (a == DDP_ERR_NOT_CONVERGED || b == DDP_ERR_NOT_CONVERGED) ? (int)DDP_ERR_NOT_CONVERGED : (int)DDP_OK;
    };
    int worst = run_solves(ctx, reqs.data(), first, precision, infos);
    if (worst != DDP_OK && worst != DDP_ERR_NOT_CONVERGED) return worst;
    if (!ctx->copy_stream) DDP_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    cudaStream_t cs = ctx->copy_stream;
    cudaEvent_t ev;
    DDP_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    auto download = [&](void *dst, const void *srcp, size_t bytes) -> int {
        DDP_CUDA(ctx, cudaEventRecord(ev, ctx->stream));
        DDP_CUDA(ctx, cudaStreamWaitEvent(cs, ev, 0));
        DDP_CUDA(ctx, cudaMemcpyAsync(dst, srcp, bytes, cudaMemcpyDeviceToHost, cs));
        return DDP_OK;
    };
    // series term T_i = S_i - E S_{i-1} on the device, then its copy to the host
    auto series = [&](int i) -> int {
        if (!dT[i]) return DDP_OK;
        SeriesArgs sa;
        sa.big = item_of(g, *dom[i], 12, DDP_PREC_FP64);
        sa.small = item_of(g, *dom[i - 1], 12, DDP_PREC_FP64);
        sa.Sb = (const double2 *)dS[i];
        sa.Ss = (const double2 *)dS[i - 1];
        sa.T = (double2 *)dT[i];
        sa.ncol = 12;
        const int64_t nt = (int64_t)12 * dom[i]->n;
        k_series<<<(unsigned)((nt + 255) / 256), 256, 0, ctx->stream>>>(sa);
        ctx->launches++;
        if (cudaPeekAtLastError() != cudaSuccess) return set_cuda_error(ctx, cudaGetLastError(), "series term");
        return t_host[i] ? download(T_out[i - 1], dT[i], sb[i]) : DDP_OK;
    };
    int rc = DDP_OK;
    for (int i = 0; i < first && !rc; i++)
        if (s_host[i]) rc = download(S_out[i], dS[i], sb[i]);
    for (int i = 1; i < first && !rc; i++) rc = series(i);
    if (!rc && first < n) {
        const int w = run_solves(ctx, reqs.data() + first, n - first, precision, infos ? infos + first : nullptr);
        if (w != DDP_OK && w != DDP_ERR_NOT_CONVERGED) rc = w;
        worst = combine(worst, w);
        for (int i = first; i < n && !rc; i++)
            if (s_host[i]) rc = download(S_out[i], dS[i], sb[i]);
        for (int i = first; i < n && !rc; i++) rc = series(i);
    }
    for (int i = 0; i < n && !rc && contract_mask; i++)
        for (int k = 0; k < 4 && !rc; k++) {
            if (!((contract_mask >> k) & 1)) continue;
            rc = ddp_contract(ctx, k, domain_ids[i], dS[i], nullptr, 12, src, dC + ((size_t)i * 4 + k) * 2 * L0);
        }
    if (!rc && contract_mask && !c_dev) rc = download(C_out, dC, cbytes);
    cudaError_t e1 = cudaStreamSynchronize(cs), e2 = cudaStreamSynchronize(ctx->stream);
    cudaEventDestroy(ev);
    if (rc) return rc;
    if (e1 != cudaSuccess) return set_cuda_error(ctx, e1, "device to host copies");
    if (e2 != cudaSuccess) return set_cuda_error(ctx, e2, "synchronize");
    return worst;
}

// Boundary coupling of two domains of one gauge field (Eq. blkdec), the source of
// the second solve of the factorized propagator (Eq. approxlong).
int ddp_boundary_source(ddp_ctx *ctx, int domain_from, const double *psi, int domain_to, double *sigma, int ncol) {
    if (!ctx || !psi || !sigma || ncol < 1) return DDP_ERR_INVALID_ARG;
    const DomainDev *df, *dt;
    const GaugeDev *gf, *gt;
    int rc = find_domain(ctx, domain_from, &df, &gf);
    if (rc) return rc;
    if ((rc = find_domain(ctx, domain_to, &dt, &gt))) return rc;
    if (gf != gt) return DDP_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    StreamJoin sj(ctx);
    Staged a, b;
    if ((rc = a.init(ctx, psi, (size_t)ncol * df->n * 12 * sizeof(double2), true))) return rc;
    if ((rc = b.init(ctx, sigma, (size_t)ncol * dt->n * 12 * sizeof(double2), false))) return rc;
    BoundaryArgs ba;
    ba.to = item_of(*gt, *dt, ncol, DDP_PREC_FP64);
    ba.from = item_of(*gf, *df, ncol, DDP_PREC_FP64);
    ba.psi = (const double2 *)a.dev;
    ba.sigma = (double2 *)b.dev;
    ba.ncol = ncol;
    const int64_t nt = (int64_t)ncol * dt->n;
    k_boundary_source<<<(unsigned)((nt + 255) / 256), 256, 0, ctx->stream>>>(ba);
    ctx->launches++;
    DDP_CUDA(ctx, cudaGetLastError());
    if ((rc = b.copy_out())) return rc;
    DDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return DDP_OK;
}

// Storage-format index of a "<name>_fp64" ... "<name>_bf16" parameter, or -1.
static int prec_suffix(const std::string &n, const char *stem) {
    static const char *suf[4] = {"_fp64", "_fp32", "_fp16", "_bf16"};
    for (int k = 0; k < 4; k++)
        if (n == std::string(stem) + suf[k]) return k;
    return -1;
}

// Tuning knobs of the solver (names: max_outer, max_inner, delta_fp32,
// delta_fp16, delta_bf16, delta_fp64, tile_sites, tile_cols, conditional, stencil_carveout, projector_tensor_cores, contraction_double_fp32,
// overlap_downloads, tuned_cols_*, tuned_carveout_*).
int ddp_set_param(ddp_ctx *ctx, const char *name, double value) {
    if (!ctx || !name) return DDP_ERR_INVALID_ARG;
    EngineParams &p = ctx->prm;
    std::string n(name);
    if (n == "max_outer") p.max_outer = (int)value;
    else if (n == "max_inner") p.max_inner = (int)value;
    else if (n == "delta_fp64") p.floor_delta[0] = value;
    else if (n == "delta_fp32") p.floor_delta[1] = value;
    else if (n == "delta_fp16") p.floor_delta[2] = value;
    else if (n == "delta_bf16") p.floor_delta[3] = value;
    else if (n == "tile_sites") {
        if (value != 0 && value != HOP_TS) return DDP_ERR_INVALID_ARG;
    } else if (n == "tile_cols") {
        if (value < 0 || value > HOP_MAX_CG) return DDP_ERR_INVALID_ARG;
        p.CG = (int)value;
    } else if (n == "conditional") p.use_conditional = value != 0;
    else if (n == "projector_tensor_cores") p.proj_tc = value != 0;
    else if (n == "contraction_double_fp32") p.contract_dd = value != 0;
    else if (n == "overlap_downloads") p.overlap_downloads = value != 0;
    else if (n == "stencil_carveout") {
        if (value < -1 || value > 100) return DDP_ERR_INVALID_ARG;
        p.carveout = (int)value;
    }
    else if (n == "tuned_cols_fp64" || n == "tuned_cols_fp32" || n == "tuned_cols_fp16" || n == "tuned_cols_bf16") {
        if (value < 0 || value > HOP_MAX_CG) return DDP_ERR_INVALID_ARG;
        int k = n == "tuned_cols_fp64" ? 0 : n == "tuned_cols_fp32" ? 1 : n == "tuned_cols_fp16" ? 2 : 3;
        p.CG_prec[k] = (int)value;
    }
    else if (prec_suffix(n, "tuned_carveout") >= 0) {
        if (value < -2 || value > 100) return DDP_ERR_INVALID_ARG;
        p.carveout_prec[prec_suffix(n, "tuned_carveout")] = (int)value;
    }
    else return DDP_ERR_INVALID_ARG;
    return DDP_OK;
}

int ddp_get_param(const ddp_ctx *ctx, const char *name, double *value) {
    if (!ctx || !name || !value) return DDP_ERR_INVALID_ARG;
    const EngineParams &p = ctx->prm;
    const std::string n(name);
    if (n == "max_outer") *value = p.max_outer;
    else if (n == "max_inner") *value = p.max_inner;
    else if (prec_suffix(n, "delta") >= 0) *value = p.floor_delta[prec_suffix(n, "delta")];
    else if (n == "tile_sites") *value = HOP_TS;
    else if (n == "tile_cols") *value = p.CG;
    else if (n == "conditional") *value = p.use_conditional;
    else if (n == "projector_tensor_cores") *value = p.proj_tc;
    else if (n == "contraction_double_fp32") *value = p.contract_dd;
    else if (n == "overlap_downloads") *value = p.overlap_downloads;
    else if (n == "stencil_carveout") *value = p.carveout;
    else if (prec_suffix(n, "tuned_cols") >= 0) *value = p.CG_prec[prec_suffix(n, "tuned_cols")];
    else if (prec_suffix(n, "tuned_carveout") >= 0) *value = p.carveout_prec[prec_suffix(n, "tuned_carveout")];
    else return DDP_ERR_INVALID_ARG;
    return DDP_OK;
}

long ddp_kernel_launches(const ddp_ctx *ctx) { return ctx ? ctx->launches : 0; }

// Autotuner: time the three inner-loop stencil variants on the domain for every
// admissible number of columns per block (the block shape: 32 sites x columns) and
// every candidate shared-memory carveout of the stencils (the split of the unified
// L1 / shared memory between the staged links of the resident blocks and the L1 that
// serves the neighbour gathers: fewer columns per block means more resident blocks,
// each staging its own links), and keep, for this storage format, the pair with the
// shortest stencil time of one BiCGStab iteration (two PLAIN launches and one of each
// Schur variant).
int ddp_autotune(ddp_ctx *ctx, int domain_id, double kappa, int ncol, int precision, int iters, int *best_cols,
                 float *best_ms) {
    if (!ctx || ncol < 1 || precision < 0 || precision > 3 || iters < 1) return DDP_ERR_INVALID_ARG;
    const int cands[] = {12, 8, 6, 4, 3, 2, 1};
    const int carves[] = {28, 50, 100};
    const int weight[3] = {2, 1, 1};
    const int saved = ctx->prm.CG, saved_cv = ctx->prm.carveout_prec[precision];
    int best = 0, best_cv = carves[0];
    float bms = 0;
    for (int cv : carves) {
        ctx->prm.carveout_prec[precision] = cv;
        for (int c : cands) {
            if (c > ncol) continue;
            ctx->prm.CG = c;
            float tot = 0;
            for (int k = DDP_HOP_PLAIN; k <= DDP_HOP_SCHUR_TS; k++) {
                float ms = 0;
                double by = 0;
                int rc = ddp_time_hop(ctx, domain_id, kappa, ncol, precision, k, iters, &ms, &by);
                if (rc) {
                    ctx->prm.CG = saved;
                    ctx->prm.carveout_prec[precision] = saved_cv;
                    return rc;
                }
                tot += weight[k] * ms;
            }
            if (!best || tot < bms) {
                best = c;
                best_cv = cv;
                bms = tot;
            }
        }
    }
    ctx->prm.CG = saved;
    ctx->prm.CG_prec[precision] = best;
    ctx->prm.carveout_prec[precision] = best_cv;
    if (best_cols) *best_cols = best;
    if (best_ms) *best_ms = bms;
    return DDP_OK;
}

}  // extern "C"
