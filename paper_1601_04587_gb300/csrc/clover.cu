// Clover fields T = 1 + 2 kappa C and T^-1 of a resident gauge field, built on
// the device in FP64 (see clover.cuh for the term and its storage).
#include <cmath>
#include <cstring>

#include "ddp_host.h"

namespace ddp {

namespace {

struct CloverArgs {
    const double2 *u;  // FP64 links [mu][9][V], even-odd site rows
    int L[4];
    int64_t V;
    double kappa, csw;
    double2 *t64, *ti64;  // [36][V]
    float4 *t32, *ti32;   // [18][V]
    int *singular;        // set when a block cannot be inverted
};

struct M3 {
    cx<double> m[3][3];
};

__device__ M3 m3_link(const CloverArgs &a, int mu, const int x[4]) {
    const int64_t lex = (((int64_t)x[0] * a.L[1] + x[1]) * a.L[2] + x[2]) * a.L[3] + x[3];
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    const int64_t row = (par ? a.V / 2 : 0) + (lex >> 1);
    M3 r;
    for (int j = 0; j < 9; j++) {
        const double2 c = a.u[((int64_t)mu * 9 + j) * a.V + row];
        r.m[j / 3][j % 3] = mk(c.x, c.y);
    }
    return r;
}

__device__ M3 m3_mul(const M3 &p, const M3 &q) {
    M3 r;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cx<double> s = mk(0.0, 0.0);
            for (int k = 0; k < 3; k++) s = s + p.m[i][k] * q.m[k][j];
            r.m[i][j] = s;
        }
    return r;
}

__device__ M3 m3_adj(const M3 &p) {
    M3 r;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) r.m[i][j] = conj(p.m[j][i]);
    return r;
}

__device__ void shift(const CloverArgs &a, const int x[4], int mu, int dmu, int nu, int dnu, int y[4]) {
    for (int m = 0; m < 4; m++) y[m] = x[m];
    y[mu] = (y[mu] + dmu + a.L[mu]) % a.L[mu];
    y[nu] = (y[nu] + dnu + a.L[nu]) % a.L[nu];
}

// F_{mu nu}(x) = (Q - Q^+)/8, Q = the four plaquettes of the (mu, nu) plane through x,
// each traversed mu-direction first.
__device__ M3 field_strength(const CloverArgs &a, const int x[4], int mu, int nu) {
    int y[4];
    M3 q;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) q.m[i][j] = mk(0.0, 0.0);
    // leaf in the (+mu, +nu) quadrant
    shift(a, x, mu, 1, nu, 0, y);
    M3 b = m3_link(a, nu, y);
    shift(a, x, mu, 0, nu, 1, y);
    M3 c = m3_adj(m3_link(a, mu, y));
    M3 l = m3_mul(m3_mul(m3_link(a, mu, x), b), m3_mul(c, m3_adj(m3_link(a, nu, x))));
    // (-mu, +nu)
    shift(a, x, mu, -1, nu, 1, y);
    M3 b2 = m3_adj(m3_link(a, mu, y));
    shift(a, x, mu, -1, nu, 0, y);
    M3 c2 = m3_adj(m3_link(a, nu, y));
    M3 d2 = m3_link(a, mu, y);
    M3 l2 = m3_mul(m3_mul(m3_link(a, nu, x), b2), m3_mul(c2, d2));
    // (-mu, -nu)
    shift(a, x, mu, -1, nu, 0, y);
    M3 a3 = m3_adj(m3_link(a, mu, y));
    shift(a, x, mu, -1, nu, -1, y);
    M3 b3 = m3_adj(m3_link(a, nu, y));
    M3 c3 = m3_link(a, mu, y);
    shift(a, x, mu, 0, nu, -1, y);
    M3 d3 = m3_link(a, nu, y);
    M3 l3 = m3_mul(m3_mul(a3, b3), m3_mul(c3, d3));
    // (+mu, -nu)
    shift(a, x, mu, 0, nu, -1, y);
    M3 a4 = m3_adj(m3_link(a, nu, y));
    M3 b4 = m3_link(a, mu, y);
    shift(a, x, mu, 1, nu, -1, y);
    M3 c4 = m3_link(a, nu, y);
    M3 l4 = m3_mul(m3_mul(a4, b4), m3_mul(c4, m3_adj(m3_link(a, mu, x))));
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) q.m[i][j] = l.m[i][j] + l2.m[i][j] + l3.m[i][j] + l4.m[i][j];
    M3 f;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            const cx<double> d = q.m[i][j] - conj(q.m[j][i]);
            f.m[i][j] = mk(d.re / 8.0, d.im / 8.0);
        }
    return f;
}

// In-place inverse of a 6x6 complex matrix (Gauss-Jordan, partial pivoting).
__device__ bool invert6(cx<double> m[6][6]) {
    cx<double> inv[6][6];
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) inv[i][j] = mk(i == j ? 1.0 : 0.0, 0.0);
    for (int c = 0; c < 6; c++) {
        int piv = c;
        double best = 0;
        for (int r = c; r < 6; r++) {
            const double v = m[r][c].re * m[r][c].re + m[r][c].im * m[r][c].im;
            if (v > best) {
                best = v;
                piv = r;
            }
        }
        if (!(best > 0)) return false;
        if (piv != c)
            for (int j = 0; j < 6; j++) {
                cx<double> t = m[c][j];
                m[c][j] = m[piv][j];
                m[piv][j] = t;
                t = inv[c][j];
                inv[c][j] = inv[piv][j];
                inv[piv][j] = t;
            }
        const cx<double> p = m[c][c];
        const double pn = p.re * p.re + p.im * p.im;
        const cx<double> ip = mk(p.re / pn, -p.im / pn);
        for (int j = 0; j < 6; j++) {
            m[c][j] = ip * m[c][j];
            inv[c][j] = ip * inv[c][j];
        }
        for (int r = 0; r < 6; r++) {
            if (r == c) continue;
            const cx<double> f = m[r][c];
            for (int j = 0; j < 6; j++) {
                m[r][j] = m[r][j] - f * m[c][j];
                inv[r][j] = inv[r][j] - f * inv[c][j];
            }
        }
    }
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) m[i][j] = inv[i][j];
    return true;
}

// Pack a (numerically) Hermitian 6x6 matrix: real diagonal, upper triangle
// averaged with the conjugate of the lower one.
__device__ void pack6(const cx<double> m[6][6], double out[36]) {
    for (int i = 0; i < 6; i++) out[i] = m[i][i].re;
    for (int i = 0; i < 6; i++)
        for (int j = i + 1; j < 6; j++) {
            const int o = herm_off(i, j);
            out[o] = 0.5 * (m[i][j].re + m[j][i].re);
            out[o + 1] = 0.5 * (m[i][j].im - m[j][i].im);
        }
}

// One thread per global site: F_{mu nu} of the six planes, the two chiral blocks
//   C_+- = -(i/2) c_sw sum_l sigma_l (x) G_l,  G_l = B_l +- F_{0 l},
//   B_1 = F_23, B_2 = F_31, B_3 = F_12
// (sigma_{0k} = -+sigma_k and sigma_{jk} = -eps_jkl sigma_l on the two blocks of the
// chiral basis), T = 1 + 2 kappa C and T^-1.
__global__ void k_clover(CloverArgs a) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= a.V) return;
    int x[4];
    int64_t r = g;
    for (int m = 3; m >= 0; m--) {
        x[m] = (int)(r % a.L[m]);
        r /= a.L[m];
    }
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    const int64_t row = (par ? a.V / 2 : 0) + (g >> 1);
    const M3 F01 = field_strength(a, x, 0, 1), F02 = field_strength(a, x, 0, 2), F03 = field_strength(a, x, 0, 3);
    const M3 F12 = field_strength(a, x, 1, 2), F13 = field_strength(a, x, 1, 3), F23 = field_strength(a, x, 2, 3);
    double tp[2][36], ip[2][36];
    for (int blk = 0; blk < 2; blk++) {
        const double s0 = blk ? -1.0 : 1.0;  // sign of F_{0 l} in G_l
        M3 G[3];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                G[0].m[i][j] = F23.m[i][j] + mk(s0 * F01.m[i][j].re, s0 * F01.m[i][j].im);
                G[1].m[i][j] = mk(-F13.m[i][j].re, -F13.m[i][j].im) + mk(s0 * F02.m[i][j].re, s0 * F02.m[i][j].im);
                G[2].m[i][j] = F12.m[i][j] + mk(s0 * F03.m[i][j].re, s0 * F03.m[i][j].im);
            }
        // sum_l sigma_l (x) G_l = [[G3, G1 - i G2], [G1 + i G2, -G3]] over (spin mod 2, colour)
        cx<double> T[6][6];
        const double f = -0.5 * a.csw * 2.0 * a.kappa;  // 2 kappa times -(1/2) c_sw, times i below
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                const cx<double> g1 = G[0].m[i][j], g2 = G[1].m[i][j], g3 = G[2].m[i][j];
                const cx<double> e00 = g3, e11 = mk(-g3.re, -g3.im);
                const cx<double> e01 = g1 - mul_i(g2), e10 = g1 + mul_i(g2);
                // T = 1 + i f M
                T[i][j] = mul_i(e00);
                T[i][3 + j] = mul_i(e01);
                T[3 + i][j] = mul_i(e10);
                T[3 + i][3 + j] = mul_i(e11);
            }
        for (int i = 0; i < 6; i++)
            for (int j = 0; j < 6; j++) {
                T[i][j] = mk(f * T[i][j].re, f * T[i][j].im);
                if (i == j) T[i][j].re += 1.0;
            }
        pack6(T, tp[blk]);
        if (!invert6(T)) atomicExch(a.singular, 1);
        pack6(T, ip[blk]);
    }
    for (int j = 0; j < 36; j++) {
        const int blk = (2 * j) / 36, k = (2 * j) % 36;
        a.t64[(int64_t)j * a.V + row] = make_double2(tp[blk][k], tp[blk][k + 1]);
        a.ti64[(int64_t)j * a.V + row] = make_double2(ip[blk][k], ip[blk][k + 1]);
    }
    for (int j = 0; j < 18; j++) {
        const int blk = (4 * j) / 36, k = (4 * j) % 36;
        a.t32[(int64_t)j * a.V + row] = make_float4((float)tp[blk][k], (float)tp[blk][k + 1], (float)tp[blk][k + 2],
                                                    (float)tp[blk][k + 3]);
        a.ti32[(int64_t)j * a.V + row] = make_float4((float)ip[blk][k], (float)ip[blk][k + 1],
                                                     (float)ip[blk][k + 2], (float)ip[blk][k + 3]);
    }
}

}  // namespace

// The clover fields of (gauge, kappa, c_sw), built on first use and kept with the
// gauge field: the CLOVER_CACHE most recently used pairs (a call that uses at most
// that many pairs never evicts one of its own).
int clover_for(ddp_ctx *ctx, GaugeDev &g, double kappa, double csw, const CloverDev **out) {
    for (size_t i = 0; i < g.clov.size(); i++)
        if (g.clov[i]->kappa == kappa && g.clov[i]->csw == csw) {
            std::unique_ptr<CloverDev> c = std::move(g.clov[i]);
            g.clov.erase(g.clov.begin() + i);
            *out = c.get();
            g.clov.push_back(std::move(c));
            return DDP_OK;
        }
    auto c = std::make_unique<CloverDev>();
    c->kappa = kappa;
    c->csw = csw;
    cudaError_t e = cudaMalloc((void **)&c->t64, (size_t)36 * g.V * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->ti64, (size_t)36 * g.V * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->t32, (size_t)18 * g.V * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->ti32, (size_t)18 * g.V * sizeof(float4));
    int *flag = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void **)&flag, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(flag);
        return set_cuda_error(ctx, e, "clover field allocation");
    }
    DDP_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
    CloverArgs a;
    a.u = g.u64;
    memcpy(a.L, g.L, sizeof(a.L));
    a.V = g.V;
    a.kappa = kappa;
    a.csw = csw;
    a.t64 = c->t64;
    a.ti64 = c->ti64;
    a.t32 = c->t32;
    a.ti32 = c->ti32;
    a.singular = flag;
    k_clover<<<(unsigned)((g.V + 127) / 128), 128, 0, ctx->stream>>>(a);
    ctx->launches++;
    int h = 0;
    DDP_CUDA(ctx, cudaGetLastError());
    DDP_CUDA(ctx, cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    DDP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(flag);
    if (h) {
        snprintf(ctx->last_error, sizeof(ctx->last_error), "1 + 2 kappa C is singular at some site");
        return DDP_ERR_INVALID_ARG;
    }
    if ((int)g.clov.size() >= CLOVER_CACHE) g.clov.erase(g.clov.begin());
    *out = c.get();
    g.clov.push_back(std::move(c));
    return DDP_OK;
}

CloverDev::~CloverDev() {
    cudaFree(t64);
    cudaFree(ti64);
    cudaFree(t32);
    cudaFree(ti32);
}

}  // namespace ddp
