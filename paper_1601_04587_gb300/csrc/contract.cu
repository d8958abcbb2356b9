// Wick contractions of domain propagators (FP64; the nucleon, the one ALU-heavy
// contraction, in double-FP32 arithmetic unless "contraction_double_fp32" is 0):
//   - local disconnected trace tr{g5 S(x,x)} (Sec. 3, Eq. W0),
//   - stochastic time-slice trace sum_{x vec} sum_c eta_c^+ g5 psi_c (Sec. 5),
//   - pion sum_{y vec} tr{S S^+} (Sec. 4, Eq. W0pc with the exact S),
//   - nucleon sum_{y vec} [W_N1 - W_N2](y,x) (Sec. 4).
// Per time slice: blocks reduce a chunk of the slice to a partial (warp
// shuffles, fixed order), a second kernel adds a slice's partials in order.
#include <cstring>

#include "ddfloat.cuh"
#include "ddp_host.h"

namespace ddp {

// Chiral basis: g5 = diag(-1,-1,1,1); C g5 = diag(s2, s2) with s2 = [[0,-i],[i,0]];
// P- = (1 - g0)/2 with g0 = [[0,1],[1,0]] (2x2 blocks).

struct Cplx {
    double re, im;
};
__device__ __forceinline__ Cplx cadd(Cplx a, Cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ Cplx csub(Cplx a, Cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ Cplx cmulc(Cplx a, Cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ Cplx cscale(double s, Cplx a) { return {s * a.re, s * a.im}; }

struct ContractArgs {
    Item it;
    const double2 *S;    // [ncol][n][12]
    const double2 *eta;  // [ncol][n][12] (noise kind)
    int ncol;
    int kind;
    int nchunk;          // blocks per local time slice
    double2 *part;       // [e0][nchunk]
};

__device__ __forceinline__ Cplx ld(const double2 *p) {
    double2 v = __ldg(p);
    return {v.x, v.y};
}

__constant__ int kPerm[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
__constant__ double kSign[6] = {1, 1, 1, -1, -1, -1};

// Nucleon W_N1 - W_N2 at one sink site with u = d = S:
//   W_N1 = eps^{abc} eps^{feg} tr[S^{ag T} C g5 S^{bf} C g5] tr[S^{ce} P-]
//   W_N2 = eps^{abc} eps^{feg} tr[S^{ag T} C g5 S^{be} P- S^{cf} C g5].
// With Gamma = C g5, which maps
// spin rho to rho^1 with a phase, (Gamma M Gamma)_{rho sigma} = (-1)^(rho+sigma)
// M_{rho^1, sigma^1}; with P- = (1 - g0)/2 of rank 2,
//   (S^{be} P- S^{cf})_{alpha beta} = sum_{lambda=0,1} E_{alpha lambda} F_{lambda beta},
//   E_{alpha lambda} = (S^{be}_{alpha lambda} - S^{be}_{alpha, lambda^2}) / 2,
//   F_{lambda beta}  =  S^{cf}_{lambda beta} - S^{cf}_{lambda^2, beta},
// so that with t_rho the row-rho parts of the traces,
//   W_N1 = sum eps eps [sum_rho sum_sigma S^{ag}_{rho sigma} (-1)^(rho+sigma) S^{bf}_{rho^1 sigma^1}] tr[S^{ce} P-],
//   W_N2 = sum eps eps  sum_rho sum_sigma S^{ag}_{rho sigma} (-1)^(rho+sigma) (E F)_{rho^1 sigma^1}.
template <class C>
__device__ __forceinline__ C sel(const C *site, int rho, int a, int sigma, int b) {
    return site[(3 * sigma + b) * 12 + 3 * rho + a];  // S(y,x)_{rho a, sigma b}
}

// The nucleon is computed in FP64 (Cplx) or in double-FP32 (Cdd, the default: GB300's
// FP64 rate is about 1/64 of its FP32 rate); the conversions of the loaded entries and of
// the per-lane sums are the only FP64 arithmetic of the double-FP32 form.
template <class C>
__device__ __forceinline__ C czero();
template <>
__device__ __forceinline__ Cplx czero<Cplx>() { return {0, 0}; }
template <>
__device__ __forceinline__ Cdd czero<Cdd>() { return {dd(0.f, 0.f), dd(0.f, 0.f)}; }
template <class C>
__device__ __forceinline__ C cfrom(Cplx v);
template <>
__device__ __forceinline__ Cplx cfrom<Cplx>(Cplx v) { return v; }
template <>
__device__ __forceinline__ Cdd cfrom<Cdd>(Cplx v) { return {dd_of(v.re), dd_of(v.im)}; }
__device__ __forceinline__ Cplx cto(Cplx v) { return v; }
__device__ __forceinline__ Cplx cto(Cdd v) { return {dd_to_double(v.re), dd_to_double(v.im)}; }

// grid (nchunk, e0), 128 threads: 4 warps x 8 sites = 32 sites of a time slice per block.
// A warp takes its sites two at a time.  The factors that do not depend on the
// row rho or on the whole epsilon pair are formed once per site in shared
// memory: t2[c][e] = tr[S^{ce} P-], E[rho][b][e][lambda] and F[c][sigma][f][lambda]
// above.  Then every lane evaluates 9 of the 2 x 144 (pair, rho) units as
//   t1 = sum_sigma g S^{bf}_{rho^1 sigma^1},  X_lambda = sum_sigma g F[c][sigma^1][f][lambda],
//   g = (-1)^(rho+sigma) S^{ag}_{rho sigma},
//   unit = sign (t1 t2[c][e] - E[rho^1][b][e][0] X_0 - E[rho^1][b][e][1] X_1).
constexpr int NUC_WARPS = 4, NUC_SITES_PER_WARP = 8;

template <class C>
struct NucSite {
    C S[144];
    C t2[9];   // [c][e]
    C E[72];   // [rho][b][e][lambda]
    C F[72];   // [c][sigma][f][lambda]
};

template <class C>
__device__ __forceinline__ C nucleon_unit(const NucSite<C> &q, int unit) {
    const int pr = unit >> 2, rho = unit & 3;
    const int p1 = pr / 6, p2 = pr - 6 * (pr / 6);
    const int a = kPerm[p1][0], b = kPerm[p1][1], c = kPerm[p1][2];
    const int f = kPerm[p2][0], e = kPerm[p2][1], g = kPerm[p2][2];
    const double sg = kSign[p1] * kSign[p2];
    const int r1 = rho ^ 1;
    C t1 = czero<C>(), x0 = czero<C>(), x1 = czero<C>();
#pragma unroll
    for (int sigma = 0; sigma < 4; sigma++) {
        const int s1 = sigma ^ 1;
        const double ph = ((rho + sigma) & 1) ? -1.0 : 1.0;
        const C sag = cscale(ph, sel(q.S, rho, a, sigma, g));
        t1 = cadd(t1, cmulc(sag, sel(q.S, r1, b, s1, f)));
        x0 = cadd(x0, cmulc(sag, q.F[((c * 4 + s1) * 3 + f) * 2 + 0]));
        x1 = cadd(x1, cmulc(sag, q.F[((c * 4 + s1) * 3 + f) * 2 + 1]));
    }
    const C t3 = cadd(cmulc(q.E[((r1 * 3 + b) * 3 + e) * 2 + 0], x0), cmulc(q.E[((r1 * 3 + b) * 3 + e) * 2 + 1], x1));
    return cscale(sg, csub(cmulc(t1, q.t2[c * 3 + e]), t3));
}

// t2, E and F of a site from its 144 entries (item k of the 153 per site).
template <class C>
__device__ __forceinline__ void nucleon_factor(NucSite<C> &q, int k) {
    if (k < 9) {
        const int c = k / 3, e = k - 3 * (k / 3);
        C t = czero<C>();
#pragma unroll
        for (int r = 0; r < 4; r++) t = cadd(t, csub(sel(q.S, r, c, r, e), sel(q.S, r, c, r ^ 2, e)));
        q.t2[k] = cscale(0.5, t);
    } else if (k < 81) {
        const int m = k - 9, lam = m & 1, e = (m >> 1) % 3, b = ((m >> 1) / 3) % 3, rho = (m >> 1) / 9;
        q.E[m] = cscale(0.5, csub(sel(q.S, rho, b, lam, e), sel(q.S, rho, b, lam + 2, e)));
    } else {
        const int m = k - 81, lam = m & 1, f = (m >> 1) % 3, sigma = ((m >> 1) / 3) % 4, c = (m >> 1) / 12;
        q.F[m] = csub(sel(q.S, lam, c, sigma, f), sel(q.S, lam + 2, c, sigma, f));
    }
}

template <class C>
__global__ void __launch_bounds__(128) k_contract_nucleon(ContractArgs a) {
    __shared__ NucSite<C> s_q[NUC_WARPS][2];
    __shared__ double s_re[NUC_WARPS], s_im[NUC_WARPS];
    const Item &it = a.it;
    const int slice_n = it.e[1] * it.e[2] * it.e[3];
    const int n = 2 * it.nh;
    const int t = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = blockIdx.x * (NUC_WARPS * NUC_SITES_PER_WARP) + warp * NUC_SITES_PER_WARP;
    C acc = czero<C>();
    for (int j = 0; j < NUC_SITES_PER_WARP; j += 2) {
        const int nsite = min(2, slice_n - (r0 + j));
        if (nsite <= 0) break;
        for (int q = lane; q < 144 * nsite; q += 32) {
            const int s = q / 144, m = q - 144 * s;
            const int col = m / 12, k = m - 12 * (m / 12);
            s_q[warp][s].S[m] = cfrom<C>(ld(a.S + ((int64_t)col * n + t * slice_n + r0 + j + s) * 12 + k));
        }
        __syncwarp();
        for (int k = lane; k < 153 * nsite; k += 32) nucleon_factor(s_q[warp][k / 153], k % 153);
        __syncwarp();
        C v = czero<C>();
        for (int u = lane; u < 144 * nsite; u += 32) v = cadd(v, nucleon_unit(s_q[warp][u / 144], u % 144));
        acc = cadd(acc, v);
        __syncwarp();
    }
    const Cplx acc64 = cto(acc);
    double re = warp_sum(acc64.re), im = warp_sum(acc64.im);
    if (lane == 0) {
        s_re[warp] = re;
        s_im[warp] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0;
        for (int w = 0; w < NUC_WARPS; w++) {
            x += s_re[w];
            y += s_im[w];
        }
        a.part[(int64_t)t * a.nchunk + blockIdx.x] = make_double2(x, y);
    }
}

__device__ __forceinline__ void block_sum_to(double2 *dst, Cplx v) {
    __shared__ double sre[32], sim[32];
    double re = warp_sum(v.re), im = warp_sum(v.im);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sre[w] = re;
        sim[w] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; i++) {
            a += sre[i];
            b += sim[i];
        }
        *dst = make_double2(a, b);
    }
}

// Pion and noise traces: grid (nchunk, e0), one thread per site of the slice.
__global__ void k_contract_slice(ContractArgs a) {
    const Item &it = a.it;
    int slice_n = it.e[1] * it.e[2] * it.e[3];
    int n = 2 * it.nh;
    int t = blockIdx.y;
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = r < slice_n;
    int l = t * slice_n + (ok ? r : 0);
    Cplx v = {0, 0};
    if (ok) {
        for (int c = 0; c < a.ncol; c++) {
            const double2 *ps = a.S + ((int64_t)c * n + l) * 12;
            if (a.kind == DDP_CONTRACT_PION) {
                for (int j = 0; j < 12; j++) {
                    Cplx s = ld(ps + j);
                    v.re += s.re * s.re + s.im * s.im;
                }
            } else {  // noise trace: eta^+ g5 psi, g5 = diag(-1,-1,1,1) on spin
                const double2 *pe = a.eta + ((int64_t)c * n + l) * 12;
                for (int j = 0; j < 12; j++) {
                    Cplx e = ld(pe + j), s = ld(ps + j);
                    double g5 = (j < 6) ? -1.0 : 1.0;
                    v.re += g5 * (e.re * s.re + e.im * s.im);
                    v.im += g5 * (e.re * s.im - e.im * s.re);
                }
            }
        }
    }
    block_sum_to(a.part + (int64_t)t * a.nchunk + blockIdx.x, v);
}

// One block per global time slice: fixed-order sum of the slice's partials.
__global__ void k_contract_final(Item it, const double2 *part, int nchunk, double2 *out) {
    int y0 = blockIdx.x;
    int t = y0 - it.o[0];
    if (t < 0) t += it.L[0];
    __shared__ double sre[256], sim[256];
    double re = 0, im = 0;
    if (t < it.e[0]) {
        for (int i = threadIdx.x; i < nchunk; i += blockDim.x) {
            double2 p = part[(int64_t)t * nchunk + i];
            re += p.x;
            im += p.y;
        }
    }
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sre[threadIdx.x] += sre[threadIdx.x + o];
            sim[threadIdx.x] += sim[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[y0] = make_double2(sre[0], sim[0]);
}

// tr{g5 S(x,x)} = sum_{alpha a} g5_alpha S(x,x)_{alpha a, alpha a}
__global__ void k_local_trace(const double2 *S, int64_t n, int l, double2 *out) {
    double re = 0, im = 0;
    for (int al = 0; al < 4; al++)
        for (int a = 0; a < 3; a++) {
            int c = 3 * al + a;
            double2 v = S[((int64_t)c * n + l) * 12 + c];
            double g5 = (al < 2) ? -1.0 : 1.0;
            re += g5 * v.x;
            im += g5 * v.y;
        }
    *out = make_double2(re, im);
}

}  // namespace ddp

using namespace ddp;

namespace {

bool dev_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int ddp_contract(ddp_ctx *ctx, int kind, int domain_id, const double *S, const double *eta, int ncol,
                            const int src[4], double *C_out) {
    if (!ctx || !S || !C_out) return DDP_ERR_INVALID_ARG;
    if (kind < 0 || kind > 3) return DDP_ERR_INVALID_ARG;
    auto di = ctx->domains.find(domain_id);
    if (di == ctx->domains.end()) return DDP_ERR_NOT_FOUND;
    const DomainDev &d = di->second;
    auto gi = ctx->gauges.find(d.gauge_id);
    if (gi == ctx->gauges.end()) return DDP_ERR_NOT_FOUND;
    const GaugeDev &g = *gi->second;
    if (kind == DDP_CONTRACT_PSEUDO_NOISE) {
        if (!eta || ncol < 1) return DDP_ERR_INVALID_ARG;
    } else if (kind == DDP_CONTRACT_PION) {
        if (ncol < 1) return DDP_ERR_INVALID_ARG;
    } else {
        ncol = 12;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    cudaStream_t st = ctx->stream;
    StreamJoin sj(ctx);
    size_t sbytes = (size_t)ncol * d.n * 12 * sizeof(double2);
    int rc = DDP_OK;
    void *dS = const_cast<double *>(S), *dE = const_cast<double *>(eta);
    bool ownS = false, ownE = false;
    void *dOut = nullptr, *dPart = nullptr;
    int nout = (kind == DDP_CONTRACT_PSEUDO_LOCAL) ? 1 : g.L[0];
    bool outdev = dev_ptr(C_out);
    Item it;
    memset(&it, 0, sizeof(it));
    int par = 0;
    for (int m = 0; m < 4; m++) {
        it.o[m] = d.o[m];
        it.e[m] = d.e[m];
        it.L[m] = g.L[m];
        par += d.o[m];
    }
    it.par_o = par & 1;
    it.nh = (int)(d.n / 2);
    it.ncol = ncol;
    int slice_n = d.e[1] * d.e[2] * d.e[3];
    int threads = (kind == DDP_CONTRACT_NUCLEON) ? 32 : 128;
    int nchunk = (slice_n + threads - 1) / threads;
    cudaError_t e = cudaSuccess;
    do {
        int l_src = 0;
        if (kind == DDP_CONTRACT_PSEUDO_LOCAL) {
            if (!src) {
                rc = DDP_ERR_INVALID_ARG;
                break;
            }
            int k[4];
            bool inside = true;
            for (int m = 0; m < 4; m++) {
                if (src[m] < 0 || src[m] >= g.L[m]) inside = false;
                k[m] = ((src[m] - d.o[m]) % g.L[m] + g.L[m]) % g.L[m];
                if (k[m] >= d.e[m]) inside = false;
            }
            if (!inside) {
                rc = DDP_ERR_INVALID_ARG;
                break;
            }
            l_src = ((k[0] * d.e[1] + k[1]) * d.e[2] + k[2]) * d.e[3] + k[3];
        }
        // the local trace reads one site of every column: from host memory only
        // those 12 rows of 12 complex numbers are copied, not the whole propagator
        const bool rows_only = kind == DDP_CONTRACT_PSEUDO_LOCAL && !dev_ptr(S);
        if (rows_only) {
            const size_t row = 12 * sizeof(double2);
            if ((e = cudaMallocAsync(&dS, (size_t)ncol * row, st)) != cudaSuccess) break;
            ownS = true;
            if ((e = cudaMemcpy2DAsync(dS, row, reinterpret_cast<const double2 *>(S) + (size_t)l_src * 12,
                                       (size_t)d.n * row, row, ncol, cudaMemcpyHostToDevice, st)) != cudaSuccess)
                break;
        } else if (!dev_ptr(S)) {
            if ((e = cudaMallocAsync(&dS, sbytes, st)) != cudaSuccess) break;
            ownS = true;
            if ((e = cudaMemcpyAsync(dS, S, sbytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
        }
        if (kind == DDP_CONTRACT_PSEUDO_NOISE && !dev_ptr(eta)) {
            if ((e = cudaMallocAsync(&dE, sbytes, st)) != cudaSuccess) break;
            ownE = true;
            if ((e = cudaMemcpyAsync(dE, eta, sbytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
        }
        if (outdev)
            dOut = C_out;
        else if ((e = cudaMallocAsync(&dOut, nout * sizeof(double2), st)) != cudaSuccess)
            break;
        if (kind == DDP_CONTRACT_PSEUDO_LOCAL) {
            k_local_trace<<<1, 1, 0, st>>>((const double2 *)dS, rows_only ? 1 : d.n, rows_only ? 0 : l_src,
                                           (double2 *)dOut);
            ctx->launches++;
        } else {
            if ((e = cudaMallocAsync(&dPart, (size_t)d.e[0] * nchunk * sizeof(double2), st)) != cudaSuccess) break;
            ContractArgs a;
            a.it = it;
            a.S = (const double2 *)dS;
            a.eta = (const double2 *)dE;
            a.ncol = ncol;
            a.kind = kind;
            a.nchunk = nchunk;
            a.part = (double2 *)dPart;
            dim3 grid(nchunk, d.e[0]);
            if (kind == DDP_CONTRACT_NUCLEON) {
                if (ctx->prm.contract_dd)
                    k_contract_nucleon<Cdd><<<grid, NUC_WARPS * 32, 0, st>>>(a);
                else
                    k_contract_nucleon<Cplx><<<grid, NUC_WARPS * 32, 0, st>>>(a);
            }
            else
                k_contract_slice<<<grid, threads, 0, st>>>(a);
            k_contract_final<<<g.L[0], 256, 0, st>>>(it, (const double2 *)dPart, nchunk, (double2 *)dOut);
            ctx->launches += 2;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if (!outdev) {
            if ((e = cudaMemcpyAsync(C_out, dOut, nout * sizeof(double2), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                break;
        }
        e = cudaStreamSynchronize(st);
    } while (0);
    if (ownS) cudaFreeAsync(dS, st);
    if (ownE) cudaFreeAsync(dE, st);
    if (dOut && !outdev) cudaFreeAsync(dOut, st);
    if (dPart) cudaFreeAsync(dPart, st);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    if (rc) return rc;
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "contraction");
    return DDP_OK;
}

// ------------------------------------------------ allocation-free contraction
//
// Same kernels as ddp_contract, but the per-time-slice partial sums live in a
// fixed array in this file instead of memory the library allocates.  Every
// partial a call reads is first written by the same call, so the array needs
// no clearing; calls that overlap on the GPU share it and race.

#include <mutex>

#define DDP_STATIC_PARTIALS DDP_STATIC_PARTIALS_MAX

static __device__ __align__(256) double2 g_contract_partials[DDP_STATIC_PARTIALS];

namespace {

std::mutex g_static_mu;
double2 *g_static_ptr[64] = {nullptr};  // per device: device address of g_contract_partials

// Device (or managed) memory that the current device can address in kernels.
bool on_current_device(const void *p, int dev) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" int ddp_contract_static(int kind, const int L[4], const int origin[4], const int extent[4],
                                   const double *S, const double *eta, int ncol, const int src[4], double *C_out,
                                   void *cuda_stream) {
    if (!L || !origin || !extent || !S || !C_out) return DDP_ERR_INVALID_ARG;
    if (kind < 0 || kind > 3) return DDP_ERR_INVALID_ARG;
    int64_t n = 1;
    for (int m = 0; m < 4; m++) {
        if (L[m] < 2 || extent[m] < 1 || extent[m] > L[m]) return DDP_ERR_INVALID_ARG;
        n *= extent[m];
    }
    // the same geometry ddp_load_gauge and ddp_set_domain accept
    for (int m = 0; m < 4; m++)
        if (L[m] % 2) return DDP_ERR_UNSUPPORTED;
    if (extent[3] % 2) return DDP_ERR_UNSUPPORTED;
    if (kind == DDP_CONTRACT_PSEUDO_NOISE) {
        if (!eta || ncol < 1) return DDP_ERR_INVALID_ARG;
    } else if (kind == DDP_CONTRACT_PION) {
        if (ncol < 1) return DDP_ERR_INVALID_ARG;
    } else {
        ncol = 12;
    }
    // an error left by earlier, unrelated work is the caller's: report it without touching it
    if (cudaPeekAtLastError() != cudaSuccess) return DDP_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DDP_ERR_CUDA;
    // kernels are launched on these buffers directly: host memory, or memory of another
    // device, is refused before anything is enqueued
    if (!on_current_device(S, dev) || !on_current_device(C_out, dev)) return DDP_ERR_INVALID_ARG;
    if (kind == DDP_CONTRACT_PSEUDO_NOISE && !on_current_device(eta, dev)) return DDP_ERR_INVALID_ARG;
    double2 *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_ptr[dev]) {
            // host code only holds a stand-in for the device array: fetch its device address once per device
            double2 *p = nullptr;
            if (cudaGetSymbolAddress((void **)&p, g_contract_partials) != cudaSuccess || !p) {
                cudaGetLastError();
                return DDP_ERR_CUDA;
            }
            g_static_ptr[dev] = p;
        }
        scratch = g_static_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Item it;
    memset(&it, 0, sizeof(it));
    int par = 0;
    for (int m = 0; m < 4; m++) {
        it.o[m] = ((origin[m] % L[m]) + L[m]) % L[m];
        it.e[m] = extent[m];
        it.L[m] = L[m];
        par += it.o[m];
    }
    it.par_o = par & 1;
    it.nh = (int)(n / 2);
    it.ncol = ncol;
    if (kind == DDP_CONTRACT_PSEUDO_LOCAL) {
        if (!src) return DDP_ERR_INVALID_ARG;
        int k[4];
        for (int m = 0; m < 4; m++) {
            if (src[m] < 0 || src[m] >= L[m]) return DDP_ERR_INVALID_ARG;
            k[m] = ((src[m] - it.o[m]) % L[m] + L[m]) % L[m];
            if (k[m] >= extent[m]) return DDP_ERR_INVALID_ARG;
        }
        int l = ((k[0] * extent[1] + k[1]) * extent[2] + k[2]) * extent[3] + k[3];
        k_local_trace<<<1, 1, 0, st>>>((const double2 *)S, n, l, (double2 *)C_out);
        return cudaPeekAtLastError() == cudaSuccess ? DDP_OK : DDP_ERR_CUDA;
    }
    int slice_n = extent[1] * extent[2] * extent[3];
    int threads = (kind == DDP_CONTRACT_NUCLEON) ? 32 : 128;
    int nchunk = (slice_n + threads - 1) / threads;
    if ((int64_t)extent[0] * nchunk > DDP_STATIC_PARTIALS) return DDP_ERR_INVALID_ARG;
    ContractArgs a;
    a.it = it;
    a.S = (const double2 *)S;
    a.eta = (const double2 *)eta;
    a.ncol = ncol;
    a.kind = kind;
    a.nchunk = nchunk;
    a.part = scratch;
    dim3 grid(nchunk, extent[0]);
    if (kind == DDP_CONTRACT_NUCLEON)
        k_contract_nucleon<Cdd><<<grid, NUC_WARPS * 32, 0, st>>>(a);  // the default form of ddp_contract
    else
        k_contract_slice<<<grid, threads, 0, st>>>(a);
    if (cudaPeekAtLastError() != cudaSuccess) return DDP_ERR_CUDA;
    k_contract_final<<<L[0], 256, 0, st>>>(it, scratch, nchunk, (double2 *)C_out);
    return cudaPeekAtLastError() == cudaSuccess ? DDP_OK : DDP_ERR_CUDA;
}

// ------------------------------------------- two-level factorized correlator
//
// Sec. 3 / Sec. 5 (Eq. factsing): with the spatial links at the cut frozen, the
// factorized part of the disconnected correlator is the product of the two
// regions' level-1 averages of the time-slice traces,
//   C^(f)(y0, x0) = (1/L^3) [mean_v T_A^v(x0)] [mean_w T_B^w(y0)].
// One thread per (y0, x0); the means are summed in variant order (FP64).

namespace ddp {

__global__ void k_factorized(const double2 *TA, int nA, const double2 *TB, int nB, int L0, double inv_vol,
                             double2 *C) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= L0 * L0) return;
    int y0 = g / L0, x0 = g - y0 * L0;
    double ar = 0, ai = 0, br = 0, bi = 0;
    for (int v = 0; v < nA; v++) {
        double2 t = TA[(int64_t)v * L0 + x0];
        ar += t.x;
        ai += t.y;
    }
    for (int v = 0; v < nB; v++) {
        double2 t = TB[(int64_t)v * L0 + y0];
        br += t.x;
        bi += t.y;
    }
    ar /= nA;
    ai /= nA;
    br /= nB;
    bi /= nB;
    C[g] = make_double2(inv_vol * (ar * br - ai * bi), inv_vol * (ar * bi + ai * br));
}

}  // namespace ddp

extern "C" int ddp_factorized_correlator(ddp_ctx *ctx, const double *T_A, int nvar_A, const double *T_B, int nvar_B,
                                         int L0, double spatial_volume, double *C_out) {
    if (!ctx || !T_A || !T_B || !C_out || nvar_A < 1 || nvar_B < 1 || L0 < 1 || !(spatial_volume > 0))
        return DDP_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    cudaStream_t st = ctx->stream;
    StreamJoin sj(ctx);
    size_t ba = (size_t)nvar_A * L0 * sizeof(double2), bb = (size_t)nvar_B * L0 * sizeof(double2);
    size_t bc = (size_t)L0 * L0 * sizeof(double2);
    void *dA = const_cast<double *>(T_A), *dB = const_cast<double *>(T_B), *dC = C_out;
    bool oA = !dev_ptr(T_A), oB = !dev_ptr(T_B), oC = !dev_ptr(C_out);
    cudaError_t e = cudaSuccess;
    do {
        if (oA && ((e = cudaMallocAsync(&dA, ba, st)) != cudaSuccess ||
                   (e = cudaMemcpyAsync(dA, T_A, ba, cudaMemcpyHostToDevice, st)) != cudaSuccess))
            break;
        if (oB && ((e = cudaMallocAsync(&dB, bb, st)) != cudaSuccess ||
                   (e = cudaMemcpyAsync(dB, T_B, bb, cudaMemcpyHostToDevice, st)) != cudaSuccess))
            break;
        if (oC && (e = cudaMallocAsync(&dC, bc, st)) != cudaSuccess) break;
        int n = L0 * L0;
        k_factorized<<<(n + 255) / 256, 256, 0, st>>>((const double2 *)dA, nvar_A, (const double2 *)dB, nvar_B, L0,
                                                    1.0 / spatial_volume, (double2 *)dC);
        ctx->launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if (oC && (e = cudaMemcpyAsync(C_out, dC, bc, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        e = cudaStreamSynchronize(st);
    } while (0);
    if (oA && dA) cudaFreeAsync(dA, st);
    if (oB && dB) cudaFreeAsync(dB, st);
    if (oC && dC) cudaFreeAsync(dC, st);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "factorized correlator");
    return DDP_OK;
}
