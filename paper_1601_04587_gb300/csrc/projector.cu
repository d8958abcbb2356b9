// Projector-cut factorization of the pion and nucleon propagators (Sec. 5):
// orthonormal vectors from inverse iteration (Eq. proj), time-slice Gram blocks
// of Eq. Bpions and the product of Eq. fullfactpi, the colourless spinors and the
// nucleon contractions of Eq. W0tbary.
//
// All arithmetic is FP64.  Fields are in the user layout [m][n][4][3] complex of
// a domain (domain-local lexicographic sites, so the sites of one time slice of
// the domain are contiguous).
#include <cmath>
#include <cstring>
#include <vector>

#include "ddfloat.cuh"
#include "ddp_host.h"

using namespace ddp;

namespace {

// ------------------------------------------------------------ Gram blocks
//
// G_z[i][j] = sum over rows r of segment z of conj(A_i[r]) A_j[r], A_i[r] the
// complex component r of column i (column stride cs complex numbers).  Segment
// z covers rows [z * seg, (z + 1) * seg).  Tiles of 32 x 32 outputs per block of
// 256 threads (2 x 2 outputs each), split over the rows in kchunk pieces; the
// pieces are added in a fixed order by k_gram_reduce.

constexpr int GT = 32;   // output tile
constexpr int GK = 16;   // rows per shared-memory stage

struct GramArgs {
    const double2 *A;
    int64_t cs;     // column stride (complex)
    int m;
    int64_t seg;    // rows per segment
    int64_t kchunk; // rows per block
    int nks;        // pieces per segment
    int ntile;      // ceil(m / GT)
    double2 *part;  // [nseg][nks][m][m]
};

__global__ void __launch_bounds__(256) k_gram(GramArgs a) {
    __shared__ double2 sa[GK][GT + 1], sb[GK][GT + 1];
    const int ti = blockIdx.x / a.ntile, tj = blockIdx.x % a.ntile;
    const int ks = blockIdx.y, z = blockIdx.z;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t r0 = (int64_t)z * a.seg + (int64_t)ks * a.kchunk;
    const int64_t r1 = min((int64_t)z * a.seg + a.seg, r0 + a.kchunk);
    double2 acc[2][2];
    for (int p = 0; p < 2; p++)
        for (int q = 0; q < 2; q++) acc[p][q] = make_double2(0.0, 0.0);
    for (int64_t rb = r0; rb < r1; rb += GK) {
        // stage GK rows of the 32 i-columns and the 32 j-columns
        for (int e = threadIdx.x; e < GK * GT; e += blockDim.x) {
            const int c = e / GK, rr = e % GK;  // consecutive threads: consecutive rows of one column
            const int64_t r = rb + rr;
            const int ci = ti * GT + c, cj = tj * GT + c;
            sa[rr][c] = (r < r1 && ci < a.m) ? a.A[(int64_t)ci * a.cs + r] : make_double2(0.0, 0.0);
            sb[rr][c] = (r < r1 && cj < a.m) ? a.A[(int64_t)cj * a.cs + r] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < GK; rr++) {
            double2 x[2], y[2];
            for (int p = 0; p < 2; p++) x[p] = sa[rr][ty + 16 * p];
            for (int q = 0; q < 2; q++) y[q] = sb[rr][tx + 16 * q];
            for (int p = 0; p < 2; p++)
                for (int q = 0; q < 2; q++) {
                    // conj(x) y
                    acc[p][q].x = fma(x[p].x, y[q].x, fma(x[p].y, y[q].y, acc[p][q].x));
                    acc[p][q].y = fma(x[p].x, y[q].y, fma(-x[p].y, y[q].x, acc[p][q].y));
                }
        }
        __syncthreads();
    }
    for (int p = 0; p < 2; p++)
        for (int q = 0; q < 2; q++) {
            const int i = ti * GT + ty + 16 * p, j = tj * GT + tx + 16 * q;
            if (i < a.m && j < a.m) a.part[(((int64_t)z * a.nks + ks) * a.m + i) * a.m + j] = acc[p][q];
        }
}

__global__ void k_gram_reduce(const double2 *part, int nks, int m, int nseg, double2 *out) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t mm = (int64_t)m * m;
    if (g >= nseg * mm) return;
    const int64_t z = g / mm, ij = g - z * mm;
    double re = 0, im = 0;
    for (int s = 0; s < nks; s++) {
        const double2 v = part[(z * nks + s) * mm + ij];
        re += v.x;
        im += v.y;
    }
    out[g] = make_double2(re, im);
}

// Gram blocks of nseg consecutive row segments of seg rows each; out [nseg][m][m].
// On the tensor cores (gram_tc) unless the context asks for the FP64 kernel or m > TC_MMAX.
int gram(ddp_ctx *ctx, const double2 *A, int64_t cs, int m, int64_t seg, int nseg, double2 *out, Arena &ar) {
    if (ctx->prm.proj_tc && m <= TC_MMAX) return gram_tc(ctx, A, cs, m, seg, nseg, out);
    const int ntile = (m + GT - 1) / GT;
    // enough blocks to fill the GPU: split each segment into pieces of >= 512 rows
    int64_t want = std::max<int64_t>(1, 1200 / std::max<int64_t>(1, (int64_t)ntile * ntile * nseg));
    int64_t kchunk = std::max<int64_t>(512, (seg + want - 1) / want);
    kchunk = ((kchunk + GK - 1) / GK) * GK;
    const int nks = (int)((seg + kchunk - 1) / kchunk);
    const size_t pb = (size_t)nseg * nks * m * m * sizeof(double2);
    ar.reset();
    DDP_CUDA(ctx, ar.reserve(pb + 1024));
    double2 *part = (double2 *)ar.take(pb);
    GramArgs g;
    g.A = A;
    g.cs = cs;
    g.m = m;
    g.seg = seg;
    g.kchunk = kchunk;
    g.nks = nks;
    g.ntile = ntile;
    g.part = part;
    dim3 grid(ntile * ntile, nks, nseg);
    k_gram<<<grid, 256, 0, ctx->stream>>>(g);
    const int64_t n = (int64_t)nseg * m * m;
    k_gram_reduce<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(part, nks, m, nseg, out);
    ctx->launches += 2;
    DDP_CUDA(ctx, cudaGetLastError());
    return DDP_OK;
}

// -------------------------------------------------------- orthonormalization
//
// Cholesky QR applied twice: G = A^+ A = R^+ R (R upper triangular with a positive
// diagonal), A <- A R^-1.  The result is the unique Q of A = QR with a positive
// real diagonal of R (the basis that Gram-Schmidt in column order produces).

// A_j <- sum_{i <= j} A_i Rinv[i][j] in place, for every row; columns written from
// the highest tile down so that the columns still read are the original ones.
__global__ void k_apply_rinv(double2 *A, int64_t cs, int m, const double2 *Rinv) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= cs) return;
    constexpr int TJ = 8;
    for (int j0 = ((m - 1) / TJ) * TJ; j0 >= 0; j0 -= TJ) {
        double2 acc[TJ];
        for (int t = 0; t < TJ; t++) acc[t] = make_double2(0.0, 0.0);
        const int jmax = min(m, j0 + TJ);
        for (int i = 0; i < jmax; i++) {
            const double2 v = A[(int64_t)i * cs + r];
            for (int t = 0; t < TJ; t++) {
                const int j = j0 + t;
                if (j >= m || i > j) continue;
                const double2 c = __ldg(Rinv + (int64_t)i * m + j);
                acc[t].x = fma(v.x, c.x, fma(-v.y, c.y, acc[t].x));
                acc[t].y = fma(v.x, c.y, fma(v.y, c.x, acc[t].y));
            }
        }
        for (int t = 0; t < TJ; t++)
            if (j0 + t < m) A[(int64_t)(j0 + t) * cs + r] = acc[t];
    }
}

// The same update in double-FP32 arithmetic (the A entries split from their bits,
// R^-1 staged in shared memory): GB300's FP64 rate is about 1/64 of its FP32 rate.
// Up to RINV_MMAX_ALL columns R^-1 is staged whole; beyond, the TJ columns of each
// output tile are staged in turn (the same products in the same order).
constexpr int RINV_MMAX_ALL = 32, RINV_MMAX = TC_MMAX, RINV_TJ = 8;
__global__ void __launch_bounds__(128) k_apply_rinv_dd(double2 *A, int64_t cs, int m, const double2 *Rinv) {
    constexpr int TJ = RINV_TJ;
    constexpr int SR = RINV_MMAX_ALL * RINV_MMAX_ALL > RINV_MMAX * TJ ? RINV_MMAX_ALL * RINV_MMAX_ALL : RINV_MMAX * TJ;
    __shared__ Cdd sR[SR];
    const bool whole = m <= RINV_MMAX_ALL;
    if (whole) {
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const double2 c = Rinv[e];
            sR[e] = {dd_of(c.x), dd_of(c.y)};
        }
        __syncthreads();
    }
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // rows beyond the field still take part in the staging barriers of the tiles
    const bool row = r < cs;
    if (whole && !row) return;
    for (int j0 = ((m - 1) / TJ) * TJ; j0 >= 0; j0 -= TJ) {
        const int jmax = min(m, j0 + TJ);
        if (!whole) {
            // R^-1 [i][j0 .. jmax) for i < jmax, at sR[i * TJ + (j - j0)]
            __syncthreads();  // the previous tile's reads are done
            for (int e = threadIdx.x; e < jmax * TJ; e += blockDim.x) {
                const int i = e / TJ, j = j0 + e % TJ;
                const double2 c = j < m ? Rinv[(int64_t)i * m + j] : make_double2(0.0, 0.0);
                sR[e] = {dd_of(c.x), dd_of(c.y)};
            }
            __syncthreads();
        }
        if (!row) continue;
        Cdd acc[TJ];
#pragma unroll
        for (int t = 0; t < TJ; t++) acc[t] = {dd(0.f, 0.f), dd(0.f, 0.f)};
        for (int i = 0; i < jmax; i++) {
            const double2 a = A[(int64_t)i * cs + r];
            const Cdd v = {dd_of_bits(a.x), dd_of_bits(a.y)};
#pragma unroll
            for (int t = 0; t < TJ; t++) {
                const int j = j0 + t;
                if (j >= m || i > j) continue;
                acc[t] = cadd(acc[t], cmulc(v, whole ? sR[i * m + j] : sR[i * TJ + t]));
            }
        }
#pragma unroll
        for (int t = 0; t < TJ; t++)
            if (j0 + t < m) A[(int64_t)(j0 + t) * cs + r] = make_double2(dd_to_double(acc[t].re), dd_to_double(acc[t].im));
    }
}

// Upper-triangular R with G = R^+ R and its inverse (host, m x m complex).
bool cholesky_upper_inverse(const std::vector<double2> &G, int m, std::vector<double2> &Rinv) {
    std::vector<double> Rr((size_t)m * m, 0.0), Ri((size_t)m * m, 0.0);
    for (int j = 0; j < m; j++) {
        double d = G[(size_t)j * m + j].x;
        for (int k = 0; k < j; k++) d -= Rr[(size_t)k * m + j] * Rr[(size_t)k * m + j] + Ri[(size_t)k * m + j] * Ri[(size_t)k * m + j];
        if (!(d > 0)) return false;
        const double rjj = std::sqrt(d);
        Rr[(size_t)j * m + j] = rjj;
        for (int i = j + 1; i < m; i++) {
            // R_ji = (G_ji - sum_{k<j} conj(R_kj) R_ki) / R_jj
            double sr = G[(size_t)j * m + i].x, si = G[(size_t)j * m + i].y;
            for (int k = 0; k < j; k++) {
                const double ar = Rr[(size_t)k * m + j], ai = -Ri[(size_t)k * m + j];
                const double br = Rr[(size_t)k * m + i], bi = Ri[(size_t)k * m + i];
                sr -= ar * br - ai * bi;
                si -= ar * bi + ai * br;
            }
            Rr[(size_t)j * m + i] = sr / rjj;
            Ri[(size_t)j * m + i] = si / rjj;
        }
    }
    // back substitution: Rinv upper triangular, R Rinv = 1
    Rinv.assign((size_t)m * m, make_double2(0.0, 0.0));
    for (int c = 0; c < m; c++) {
        for (int i = c; i >= 0; i--) {
            double sr = (i == c) ? 1.0 : 0.0, si = 0.0;
            for (int k = i + 1; k <= c; k++) {
                const double ar = Rr[(size_t)i * m + k], ai = Ri[(size_t)i * m + k];
                const double2 b = Rinv[(size_t)k * m + c];
                sr -= ar * b.x - ai * b.y;
                si -= ar * b.y + ai * b.x;
            }
            const double d = Rr[(size_t)i * m + i];
            Rinv[(size_t)i * m + c] = make_double2(sr / d, si / d);
        }
    }
    return true;
}

int orthonormalize(ddp_ctx *ctx, double2 *A, int64_t cs, int m, Arena &ar) {
    std::vector<double2> G((size_t)m * m), Rinv;
    for (int pass = 0; pass < 2; pass++) {
        // the Gram matrix lives after the partials in the arena: keep it separate
        double2 *dG = nullptr;
        DDP_CUDA(ctx, cudaMallocAsync((void **)&dG, (size_t)m * m * sizeof(double2) * 2, ctx->stream));
        int rc = gram(ctx, A, cs, m, cs, 1, dG, ar);
        if (rc) {
            cudaFreeAsync(dG, ctx->stream);
            return rc;
        }
        DDP_CUDA(ctx, cudaMemcpyAsync(G.data(), dG, (size_t)m * m * sizeof(double2), cudaMemcpyDeviceToHost,
                                      ctx->stream));
        DDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (!cholesky_upper_inverse(G, m, Rinv)) {
            cudaFreeAsync(dG, ctx->stream);
            snprintf(ctx->last_error, sizeof(ctx->last_error), "orthonormalization: columns linearly dependent");
            return DDP_ERR_INVALID_ARG;
        }
        double2 *dR = dG + (size_t)m * m;
        DDP_CUDA(ctx, cudaMemcpyAsync(dR, Rinv.data(), (size_t)m * m * sizeof(double2), cudaMemcpyHostToDevice,
                                      ctx->stream));
        if (ctx->prm.proj_tc && m <= RINV_MMAX)
            k_apply_rinv_dd<<<(unsigned)((cs + 127) / 128), 128, 0, ctx->stream>>>(A, cs, m, dR);
        else
            k_apply_rinv<<<(unsigned)((cs + 127) / 128), 128, 0, ctx->stream>>>(A, cs, m, dR);
        ctx->launches++;
        DDP_CUDA(ctx, cudaGetLastError());
        DDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        cudaFreeAsync(dG, ctx->stream);
    }
    return DDP_OK;
}

// ---------------------------------------------------------------- embedding

struct EmbedArgs {
    Item from, to;
    const double2 *src;  // [ncol][n_from][12]
    double2 *dst;        // [ncol][n_to][12]
    int ncol;
    int g5;
};

// dst = E (g5^g5 src): the field of the `from` box extended by zero to the `to` box.
__global__ void k_embed(EmbedArgs a) {
    const int64_t nt = 2 * (int64_t)a.to.nh, nf = 2 * (int64_t)a.from.nh;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nt * a.ncol) return;
    const int col = (int)(g / nt);
    const int l = (int)(g - (int64_t)col * nt);
    int k[4], kf[4];
    local_coords(a.to, l, k);
    bool inside = true;
    for (int m = 0; m < 4; m++) {
        const int x = (a.to.o[m] + k[m]) % a.to.L[m];
        int d = x - a.from.o[m];
        if (d < 0) d += a.to.L[m];
        kf[m] = d;
        inside = inside && (d < a.from.e[m]);
    }
    double2 *o = a.dst + ((int64_t)col * nt + l) * 12;
    if (!inside) {
        for (int c = 0; c < 12; c++) o[c] = make_double2(0.0, 0.0);
        return;
    }
    const double2 *s = a.src + ((int64_t)col * nf + local_lex(a.from, kf)) * 12;
    for (int c = 0; c < 12; c++) {
        // gamma_5 = diag(-1, -1, 1, 1) in the chiral basis: spins 0, 1 change sign
        const double f = (a.g5 && c < 6) ? -1.0 : 1.0;
        o[c] = make_double2(f * s[c].x, f * s[c].y);
    }
}

// -------------------------------------------------------- colourless spinors
//
// X[t][i][j][k][alpha] = sum_{x vec at t} eps^{abc} (s_i^a)^T C g5 s_j^b (s_k^c)_alpha,
// C = i g0 g2.  In the chiral basis C g5 has the entries (0,1) = -i, (1,0) = i,
// (2,3) = -i, (3,2) = i, so the diquark is
//   (s_i^a)^T C g5 s_j^b = i [s_i(1,a) s_j(0,b) - s_i(0,a) s_j(1,b) + s_i(3,a) s_j(2,b) - s_i(2,a) s_j(3,b)].
// form: 0 s = A, 1 s = g5 conj(A) (the spinor of phi^+ D^-1), 2 s = -A.
// One block per (slice z, chunk of sites, i); its threads own (j, k, alpha) outputs.

constexpr int CB_SITES = 32;   // sites staged per pass
constexpr int CB_MMAX = 32;    // largest number of columns

struct BaryArgs {
    const double2 *A;
    int64_t n;        // sites of the domain
    int m;
    int form;
    int64_t slice_n;  // sites per time slice of the domain
    int nslice;       // time slices of the domain
    int nchunk;       // site chunks per slice
    int64_t chunk;    // sites per chunk
    double2 *part;    // [nslice][nchunk][m][m][m][4]
};

__device__ __forceinline__ double2 cmul2(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

__global__ void __launch_bounds__(256) k_colourless(BaryArgs a) {
    __shared__ double2 s_s[CB_MMAX][12];   // s_k(x) of the current site, all k
    __shared__ double2 s_d[CB_MMAX][9];    // diquark D_ij^{ab}(x) of this block's i, all j
    const int i = blockIdx.x;
    const int ch = blockIdx.y, z = blockIdx.z;
    const int m = a.m;
    const int nout = m * m * 4;
    // outputs of this thread: o = threadIdx.x + q * blockDim.x
    constexpr int QMAX = (CB_MMAX * CB_MMAX * 4 + 255) / 256;
    double2 acc[QMAX];
    for (int q = 0; q < QMAX; q++) acc[q] = make_double2(0.0, 0.0);
    const int64_t s0 = (int64_t)z * a.slice_n + (int64_t)ch * a.chunk;
    const int64_t s1 = min((int64_t)z * a.slice_n + a.slice_n, s0 + a.chunk);
    const double sgn = (a.form == 2) ? -1.0 : 1.0;
    for (int64_t site = s0; site < s1; site++) {
        __syncthreads();
        for (int e = threadIdx.x; e < m * 12; e += blockDim.x) {
            const int k = e / 12, c = e % 12;
            double2 v = a.A[((int64_t)k * a.n + site) * 12 + c];
            if (a.form == 1) {
                v.y = -v.y;                       // conj
                if (c < 6) v = make_double2(-v.x, -v.y);  // g5
            }
            s_s[k][c] = make_double2(sgn * v.x, sgn * v.y);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < m * 9; e += blockDim.x) {
            const int j = e / 9, ab = e % 9, ca = ab / 3, cb = ab % 3;
            // component (spin s, colour c) is 3 s + c
            const double2 i0 = s_s[i][ca], i1 = s_s[i][3 + ca], i2 = s_s[i][6 + ca], i3 = s_s[i][9 + ca];
            const double2 j0 = s_s[j][cb], j1 = s_s[j][3 + cb], j2 = s_s[j][6 + cb], j3 = s_s[j][9 + cb];
            const double2 t1 = cmul2(i1, j0), t2 = cmul2(i0, j1), t3 = cmul2(i3, j2), t4 = cmul2(i2, j3);
            const double2 s = make_double2(t1.x - t2.x + t3.x - t4.x, t1.y - t2.y + t3.y - t4.y);
            s_d[j][ab] = make_double2(-s.y, s.x);  // times i
        }
        __syncthreads();
        for (int q = 0; q < QMAX; q++) {
            const int o = threadIdx.x + q * blockDim.x;
            if (o >= nout) break;
            const int j = o / (m * 4), k = (o / 4) % m, al = o % 4;
            // eps^{abc} D^{ab} s^c: (0,1,2) (1,2,0) (2,0,1) +, (0,2,1) (2,1,0) (1,0,2) -
            const double2 *d = s_d[j];
            const double2 *sk = &s_s[k][3 * al];
            double2 t = cmul2(d[0 * 3 + 1], sk[2]);
            double2 u = cmul2(d[1 * 3 + 2], sk[0]);
            t.x += u.x, t.y += u.y;
            u = cmul2(d[2 * 3 + 0], sk[1]);
            t.x += u.x, t.y += u.y;
            u = cmul2(d[0 * 3 + 2], sk[1]);
            t.x -= u.x, t.y -= u.y;
            u = cmul2(d[2 * 3 + 1], sk[0]);
            t.x -= u.x, t.y -= u.y;
            u = cmul2(d[1 * 3 + 0], sk[2]);
            t.x -= u.x, t.y -= u.y;
            acc[q].x += t.x;
            acc[q].y += t.y;
        }
    }
    for (int q = 0; q < QMAX; q++) {
        const int o = threadIdx.x + q * blockDim.x;
        if (o >= nout) break;
        const int j = o / (m * 4), k = (o / 4) % m, al = o % 4;
        a.part[(((((int64_t)z * a.nchunk + ch) * m + i) * m + j) * m + k) * 4 + al] = acc[q];
    }
}

// X[t] = sum over chunks (fixed order); global slice t of local slice z is (o0 + z) mod L0.
__global__ void k_colourless_reduce(const double2 *part, int nchunk, int64_t per, int nslice, int o0, int L0,
                                    double2 *X) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)nslice * per) return;
    const int z = (int)(g / per);
    const int64_t e = g - (int64_t)z * per;
    double re = 0, im = 0;
    for (int c = 0; c < nchunk; c++) {
        const double2 v = part[((int64_t)z * nchunk + c) * per + e];
        re += v.x;
        im += v.y;
    }
    X[(int64_t)((o0 + z) % L0) * per + e] = make_double2(re, im);
}

// ---------------------------------------------------- projected correlators

// C(y0, x0) = (1/vol3) sum_ij Mt[y0][i][j] M[x0][j][i]  (complex)
__global__ void k_proj_pion(const double2 *Mt, const double2 *M, int L0, int m, double inv_vol, double2 *C) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= L0 * L0) return;
    const int y0 = g / L0, x0 = g - y0 * L0;
    double re = 0, im = 0;
    for (int i = 0; i < m; i++)
        for (int j = 0; j < m; j++) {
            const double2 p = Mt[((int64_t)y0 * m + i) * m + j], q = M[((int64_t)x0 * m + j) * m + i];
            re += p.x * q.x - p.y * q.y;
            im += p.x * q.y + p.y * q.x;
        }
    C[g] = make_double2(inv_vol * re, inv_vol * im);
}

// C(y0, x0) = sum_ijk [X_{jik}(x0) - X_{kij}(x0)]^T P- Y_{ijk}(y0), P- = (1 - g0)/2,
// i.e. (P- v)_a = (v_a - v_{a^2}) / 2 with a^2 the spin two places away.  Written as the
// product C = P D^T over the index K = ((i m + j) m + k) 4 + alpha of length 4 m^3, with
// P[y0][K] = (P- Y_{ijk}(y0))_alpha and D[x0][K] = (X_{jik}(x0) - X_{kij}(x0))_alpha.

// D, formed once (K-major rows, one per time slice).
__global__ void k_nucleon_d(const double2 *X, int L0, int m, double2 *D) {
    const int64_t m3 = (int64_t)m * m * m, nk = 4 * m3;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)L0 * nk) return;
    const int64_t t = g / nk, K = g % nk, e = K / 4;
    const int al = (int)(K % 4);
    const int i = (int)(e / ((int64_t)m * m)), j = (int)((e / m) % m), k = (int)(e % m);
    const double2 a = X[(t * m3 + ((int64_t)j * m + i) * m + k) * 4 + al];
    const double2 b = X[(t * m3 + ((int64_t)k * m + i) * m + j) * 4 + al];
    D[g] = make_double2(a.x - b.x, a.y - b.y);
}

// Partial products over K chunks: block (chunk, 16 x 16 output tile) sums
// P[y0][K] D[x0][K] over its K range in steps of NK_STEP staged in shared memory (P- of Y
// applied while staging), one output per thread, written to part[chunk][y0][x0].
constexpr int NK_TILE = 16, NK_STEP = 64;
__global__ void __launch_bounds__(NK_TILE *NK_TILE) k_nucleon_gemm(const double2 *Y, const double2 *D, int L0,
                                                                   int64_t nk, int64_t kchunk, double2 *part) {
    // rows padded by one element: the 16 rows a quarter-warp reads fall in distinct banks
    __shared__ double2 sP[NK_TILE][NK_STEP + 1], sD[NK_TILE][NK_STEP + 1];
    const int ntx = (L0 + NK_TILE - 1) / NK_TILE;
    const int ty = blockIdx.y / ntx, tx = blockIdx.y % ntx;
    const int ly = threadIdx.x / NK_TILE, lx = threadIdx.x % NK_TILE;
    const int y0 = ty * NK_TILE + ly, x0 = tx * NK_TILE + lx;
    const int64_t k0 = blockIdx.x * kchunk, k1 = min(nk, k0 + kchunk);
    double re = 0, im = 0;
    for (int64_t kb = k0; kb < k1; kb += NK_STEP) {
        for (int e = threadIdx.x; e < NK_TILE * NK_STEP; e += blockDim.x) {
            const int r = e / NK_STEP, c = e % NK_STEP;
            const int64_t K = kb + c;
            const int yr = ty * NK_TILE + r, xr = tx * NK_TILE + r;
            double2 pv = make_double2(0.0, 0.0), dv = make_double2(0.0, 0.0);
            if (K < k1 && yr < L0) {
                const double2 u = Y[(int64_t)yr * nk + K], w = Y[(int64_t)yr * nk + (K ^ 2)];
                pv = make_double2(0.5 * (u.x - w.x), 0.5 * (u.y - w.y));
            }
            if (K < k1 && xr < L0) dv = D[(int64_t)xr * nk + K];
            sP[r][c] = pv;
            sD[r][c] = dv;
        }
        __syncthreads();
#pragma unroll 8
        for (int c = 0; c < NK_STEP; c++) {
            const double2 p = sP[ly][c], d = sD[lx][c];
            re = fma(p.x, d.x, fma(-p.y, d.y, re));
            im = fma(p.x, d.y, fma(p.y, d.x, im));
        }
        __syncthreads();
    }
    if (y0 < L0 && x0 < L0) part[((int64_t)blockIdx.x * L0 + y0) * L0 + x0] = make_double2(re, im);
}

// C[y0][x0] = the chunk partials summed in chunk order.
__global__ void k_nucleon_sum(const double2 *part, int nchunk, int L0, double2 *C) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= L0 * L0) return;
    double re = 0, im = 0;
    for (int c = 0; c < nchunk; c++) {
        const double2 v = part[(int64_t)c * L0 * L0 + g];
        re += v.x;
        im += v.y;
    }
    C[g] = make_double2(re, im);
}

bool dptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A host or device buffer as device memory for the duration of a call.
struct DevBuf {
    ddp_ctx *ctx = nullptr;
    void *user = nullptr;
    void *dev = nullptr;
    size_t bytes = 0;
    bool owned = false;
    int init(ddp_ctx *c, const void *u, size_t b, bool copy_in) {
        ctx = c;
        user = const_cast<void *>(u);
        bytes = b;
        if (!u) return DDP_ERR_INVALID_ARG;
        if (dptr(u)) {
            dev = user;
            return DDP_OK;
        }
        DDP_CUDA(c, cudaMallocAsync(&dev, b, c->stream));
        owned = true;
        if (copy_in) DDP_CUDA(c, cudaMemcpyAsync(dev, u, b, cudaMemcpyHostToDevice, c->stream));
        return DDP_OK;
    }
    int copy_out() {
        if (owned) DDP_CUDA(ctx, cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        DDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        return DDP_OK;
    }
    ~DevBuf() {
        if (owned && dev) cudaFreeAsync(dev, ctx->stream);
    }
};

int domain_of(ddp_ctx *ctx, int id, const DomainDev **d, const GaugeDev **g) {
    auto it = ctx->domains.find(id);
    if (it == ctx->domains.end()) return DDP_ERR_NOT_FOUND;
    auto gi = ctx->gauges.find(it->second.gauge_id);
    if (gi == ctx->gauges.end()) return DDP_ERR_NOT_FOUND;
    *d = &it->second;
    *g = gi->second.get();
    return DDP_OK;
}

Item box_item(const GaugeDev &g, const DomainDev &d) {
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
    return it;
}

struct Guard {
    int prev = -1;
    explicit Guard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~Guard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

int ddp_solve_sources(ddp_ctx *ctx, int domain_id, double kappa, double csw, const double *eta, int ncol, double tol,
                      int precision, double *psi_out, ddp_solve_info *info);

int ddp_orthonormalize(ddp_ctx *ctx, int domain_id, double *V, int m) {
    if (!ctx || !V || m < 1) return DDP_ERR_INVALID_ARG;
    const DomainDev *d;
    const GaugeDev *g;
    int rc = domain_of(ctx, domain_id, &d, &g);
    if (rc) return rc;
    if ((int64_t)m > d->n * 12) return DDP_ERR_INVALID_ARG;
    Guard gd(ctx->device);
    StreamJoin sj(ctx);
    DevBuf b;
    if ((rc = b.init(ctx, V, (size_t)m * d->n * 12 * sizeof(double2), true))) return rc;
    if ((rc = orthonormalize(ctx, (double2 *)b.dev, d->n * 12, m, ctx->aux))) return rc;
    return b.copy_out();
}

int ddp_inverse_iteration(ddp_ctx *ctx, int domain_id, double kappa, double csw, double *V, int m, int iters,
                          double tol, int precision, ddp_solve_info *info) {
    if (!ctx || !V || m < 1 || iters < 0 || !(tol > 0)) return DDP_ERR_INVALID_ARG;
    const DomainDev *d;
    const GaugeDev *g;
    int rc = domain_of(ctx, domain_id, &d, &g);
    if (rc) return rc;
    if ((int64_t)m > d->n * 12) return DDP_ERR_INVALID_ARG;
    Guard gd(ctx->device);
    StreamJoin sj(ctx);
    const size_t bytes = (size_t)m * d->n * 12 * sizeof(double2);
    DevBuf b;
    if ((rc = b.init(ctx, V, bytes, true))) return rc;
    double2 *X = nullptr;
    DDP_CUDA(ctx, cudaMallocAsync((void **)&X, bytes, ctx->stream));
    double2 *cur = (double2 *)b.dev, *nxt = X;
    rc = orthonormalize(ctx, cur, d->n * 12, m, ctx->aux);
    int worst = DDP_OK;
    for (int it = 0; it < iters && !rc; it++) {
        int s = ddp_solve_sources(ctx, domain_id, kappa, csw, (const double *)cur, m, tol, precision, (double *)nxt,
                                  info);
        if (s != DDP_OK && s != DDP_ERR_NOT_CONVERGED) {
            rc = s;
            break;
        }
        if (s) worst = s;
        if ((rc = orthonormalize(ctx, nxt, d->n * 12, m, ctx->aux))) break;
        std::swap(cur, nxt);
    }
    if (!rc && cur != (double2 *)b.dev) {
        cudaError_t e = cudaMemcpyAsync(b.dev, cur, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess) rc = set_cuda_error(ctx, e, "copy of the modes");
    }
    cudaFreeAsync(X, ctx->stream);
    if (rc) return rc;
    if ((rc = b.copy_out())) return rc;
    return worst;
}

int ddp_embed(ddp_ctx *ctx, int domain_from, const double *psi, int domain_to, double *out, int ncol, int gamma5) {
    if (!ctx || !psi || !out || ncol < 1) return DDP_ERR_INVALID_ARG;
    const DomainDev *df, *dt;
    const GaugeDev *gf, *gt;
    int rc = domain_of(ctx, domain_from, &df, &gf);
    if (rc) return rc;
    if ((rc = domain_of(ctx, domain_to, &dt, &gt))) return rc;
    if (gf->L[0] != gt->L[0] || gf->L[1] != gt->L[1] || gf->L[2] != gt->L[2] || gf->L[3] != gt->L[3])
        return DDP_ERR_INVALID_ARG;
    for (int m = 0; m < 4; m++) {
        if (dt->e[m] == gt->L[m]) continue;
        const int d0 = ((df->o[m] - dt->o[m]) % gt->L[m] + gt->L[m]) % gt->L[m];
        if (df->e[m] > dt->e[m] || d0 + df->e[m] > dt->e[m]) return DDP_ERR_INVALID_ARG;
    }
    Guard gd(ctx->device);
    StreamJoin sj(ctx);
    DevBuf bi, bo;
    if ((rc = bi.init(ctx, psi, (size_t)ncol * df->n * 12 * sizeof(double2), true))) return rc;
    if ((rc = bo.init(ctx, out, (size_t)ncol * dt->n * 12 * sizeof(double2), false))) return rc;
    EmbedArgs a;
    a.from = box_item(*gf, *df);
    a.to = box_item(*gt, *dt);
    a.src = (const double2 *)bi.dev;
    a.dst = (double2 *)bo.dev;
    a.ncol = ncol;
    a.g5 = gamma5 ? 1 : 0;
    const int64_t nt = (int64_t)ncol * dt->n;
    k_embed<<<(unsigned)((nt + 255) / 256), 256, 0, ctx->stream>>>(a);
    ctx->launches++;
    DDP_CUDA(ctx, cudaGetLastError());
    return bo.copy_out();
}

int ddp_gram_slices(ddp_ctx *ctx, int domain_id, const double *A, int m, double *M_out) {
    if (!ctx || !A || !M_out || m < 1) return DDP_ERR_INVALID_ARG;
    const DomainDev *d;
    const GaugeDev *g;
    int rc = domain_of(ctx, domain_id, &d, &g);
    if (rc) return rc;
    Guard gd(ctx->device);
    StreamJoin sj(ctx);
    const int L0 = g->L[0];
    const int64_t slice_n = (int64_t)d->e[1] * d->e[2] * d->e[3];
    const size_t mm = (size_t)m * m * sizeof(double2);
    DevBuf ba, bo;
    if ((rc = ba.init(ctx, A, (size_t)m * d->n * 12 * sizeof(double2), true))) return rc;
    if ((rc = bo.init(ctx, M_out, (size_t)L0 * mm, false))) return rc;
    double2 *loc = nullptr;
    DDP_CUDA(ctx, cudaMallocAsync((void **)&loc, (size_t)d->e[0] * mm, ctx->stream));
    // local slice z of the domain is global slice (o0 + z) mod L0; the rest are zero
    rc = gram(ctx, (const double2 *)ba.dev, d->n * 12, m, slice_n * 12, d->e[0], loc, ctx->aux);
    if (!rc) {
        cudaError_t e = cudaMemsetAsync(bo.dev, 0, (size_t)L0 * mm, ctx->stream);
        for (int z = 0; z < d->e[0] && e == cudaSuccess; z++)
            e = cudaMemcpyAsync((char *)bo.dev + (size_t)((d->o[0] + z) % L0) * mm, loc + (size_t)z * m * m, mm,
                                cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess) rc = set_cuda_error(ctx, e, "slice placement");
    }
    cudaFreeAsync(loc, ctx->stream);
    if (rc) return rc;
    return bo.copy_out();
}

int ddp_colourless_slices(ddp_ctx *ctx, int domain_id, const double *A, int m, int form, double *X_out) {
    if (!ctx || !A || !X_out || m < 1 || form < 0 || form > 2) return DDP_ERR_INVALID_ARG;
    // the tensor-core sums take up to TC_MMAX columns, the direct FP64 kernel CB_MMAX
    if (m > (ctx->prm.proj_tc ? TC_MMAX : CB_MMAX)) return DDP_ERR_UNSUPPORTED;
    const DomainDev *d;
    const GaugeDev *g;
    int rc = domain_of(ctx, domain_id, &d, &g);
    if (rc) return rc;
    Guard gd(ctx->device);
    StreamJoin sj(ctx);
    const int L0 = g->L[0];
    const int64_t slice_n = (int64_t)d->e[1] * d->e[2] * d->e[3];
    const int64_t per = (int64_t)m * m * m * 4;
    DevBuf ba, bo;
    if ((rc = ba.init(ctx, A, (size_t)m * d->n * 12 * sizeof(double2), true))) return rc;
    if ((rc = bo.init(ctx, X_out, (size_t)L0 * per * sizeof(double2), false))) return rc;
    DDP_CUDA(ctx, cudaMemsetAsync(bo.dev, 0, (size_t)L0 * per * sizeof(double2), ctx->stream));
    if (ctx->prm.proj_tc) {
        rc = colourless_tc(ctx, (const double2 *)ba.dev, d->n, m, form, slice_n, d->e[0], d->o[0], L0,
                           (double2 *)bo.dev);
        if (rc) return rc;
        return bo.copy_out();
    }
    BaryArgs a;
    a.A = (const double2 *)ba.dev;
    a.n = d->n;
    a.m = m;
    a.form = form;
    a.slice_n = slice_n;
    a.nslice = d->e[0];
    // enough blocks: chunks of at least 64 sites
    const int64_t want = std::max<int64_t>(1, 2400 / std::max<int64_t>(1, (int64_t)m * d->e[0]));
    a.chunk = std::max<int64_t>(64, (slice_n + want - 1) / want);
    a.nchunk = (int)((slice_n + a.chunk - 1) / a.chunk);
    const size_t pb = (size_t)a.nslice * a.nchunk * per * sizeof(double2);
    Arena &ar = ctx->aux;
    ar.reset();
    DDP_CUDA(ctx, ar.reserve(pb + 1024));
    a.part = (double2 *)ar.take(pb);
    dim3 grid(m, a.nchunk, a.nslice);
    k_colourless<<<grid, 256, 0, ctx->stream>>>(a);
    const int64_t n = (int64_t)a.nslice * per;
    k_colourless_reduce<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(a.part, a.nchunk, per, a.nslice,
                                                                             d->o[0], L0, (double2 *)bo.dev);
    ctx->launches += 2;
    DDP_CUDA(ctx, cudaGetLastError());
    return bo.copy_out();
}

int ddp_projected_pion(ddp_ctx *ctx, int L0, int m, const double *Mt, const double *M, double spatial_volume,
                       double *C_out) {
    if (!ctx || L0 < 1 || m < 1 || !Mt || !M || !C_out || !(spatial_volume > 0)) return DDP_ERR_INVALID_ARG;
    Guard gd(ctx->device);
    StreamJoin sj(ctx);
    const size_t mb = (size_t)L0 * m * m * sizeof(double2);
    DevBuf a, b, c;
    int rc;
    if ((rc = a.init(ctx, Mt, mb, true)) || (rc = b.init(ctx, M, mb, true)) ||
        (rc = c.init(ctx, C_out, (size_t)L0 * L0 * sizeof(double2), false)))
        return rc;
    const int n = L0 * L0;
    k_proj_pion<<<(n + 127) / 128, 128, 0, ctx->stream>>>((const double2 *)a.dev, (const double2 *)b.dev, L0, m,
                                                          1.0 / spatial_volume, (double2 *)c.dev);
    ctx->launches++;
    DDP_CUDA(ctx, cudaGetLastError());
    return c.copy_out();
}

int ddp_projected_nucleon(ddp_ctx *ctx, int L0, int m, const double *X, const double *Y, double *C_out) {
    if (!ctx || L0 < 1 || m < 1 || !X || !Y || !C_out) return DDP_ERR_INVALID_ARG;
    Guard gd(ctx->device);
    StreamJoin sj(ctx);
    const size_t xb = (size_t)L0 * m * m * m * 4 * sizeof(double2);
    DevBuf a, b, c;
    int rc;
    if ((rc = a.init(ctx, X, xb, true)) || (rc = b.init(ctx, Y, xb, true)) ||
        (rc = c.init(ctx, C_out, (size_t)L0 * L0 * sizeof(double2), false)))
        return rc;
    const int64_t nk = 4 * (int64_t)m * m * m;
    const int ntx = (L0 + NK_TILE - 1) / NK_TILE, ntile = ntx * ntx;
    // K chunks: about four blocks per SM over all tiles, whole staging steps each
    int64_t nchunk = std::max<int64_t>(1, std::min<int64_t>(4 * 152 / ntile + 1, (nk + NK_STEP - 1) / NK_STEP));
    int64_t kchunk = (nk + nchunk - 1) / nchunk;
    kchunk = ((kchunk + NK_STEP - 1) / NK_STEP) * NK_STEP;
    nchunk = (nk + kchunk - 1) / kchunk;
    const size_t db = (size_t)L0 * nk * sizeof(double2), pb = (size_t)nchunk * L0 * L0 * sizeof(double2);
    Arena &ar = ctx->aux;
    ar.reset();
    DDP_CUDA(ctx, ar.reserve(db + pb + 512));
    double2 *D = (double2 *)ar.take(db);
    double2 *part = (double2 *)ar.take(pb);
    const int64_t nd = (int64_t)L0 * nk;
    k_nucleon_d<<<(unsigned)((nd + 255) / 256), 256, 0, ctx->stream>>>((const double2 *)a.dev, L0, m, D);
    k_nucleon_gemm<<<dim3((unsigned)nchunk, (unsigned)ntile), NK_TILE * NK_TILE, 0, ctx->stream>>>(
        (const double2 *)b.dev, D, L0, nk, kchunk, part);
    k_nucleon_sum<<<(L0 * L0 + 255) / 256, 256, 0, ctx->stream>>>(part, (int)nchunk, L0, (double2 *)c.dev);
    ctx->launches += 3;
    DDP_CUDA(ctx, cudaGetLastError());
    return c.copy_out();
}

}  // extern "C"
