// Kernels of the domain solver: the masked even-odd hopping term with fused
// epilogues and dot products, BiCGStab vector updates, per-solve scalar
// updates, FP64 defect-correction steps and layout conversions.
#pragma once

#include <type_traits>

#include "ddp_device.cuh"
#include "clover.cuh"

namespace ddp {

// ------------------------------------------------------------ solver state

// Per solve (one column of one request).  Complex scalars as double2.
struct SolveState {
    double2 rho, alpha, omega, beta;
    double rr;       // inner recursive |r|^2
    double target2;  // inner stopping threshold on |r|^2
    double bnorm2;   // |eta|^2 (FP64)
    double rr64;     // |eta - D_Gamma x|^2 of the current outer cycle (FP64)
    double sigma;    // |r64| of the current cycle (0: nothing to do)
    double scale;    // 2 kappa / sigma
    double delta;    // inner relative tolerance of the cycle
    double tol;      // requested relative tolerance
    double floor_delta;  // smallest useful inner tolerance of the storage format
    int active;      // inner iteration running
    int iters;       // inner iterations of the current cycle
    int total_iters; // inner iterations over all cycles
    int status;      // inner: 0 running, 1 converged, 2 breakdown, 3 iteration cap, 4 skipped
    int outer_done;  // 1 once |eta - D x| <= tol |eta|
    int item, col;
    int maxit;       // inner iteration cap per cycle
};

struct LoopCtl {
    int n_active;
    int iter;
    int maxit;
    int pad;          // host-polled loop: 1 while the loop continues
    int done_blocks;  // blocks of k_fin<FIN_RHO> finished in this iteration
};

// Reduction partial buffers: complex and real, per (item, column, tile).
struct Partials {
    double2 *c;
    double *n;
};

// Epilogues of the hopping kernel (acc = the hopping sum, v1, v2 operands at the
// output site; T / T^-1 the clover matrices of the output site, identity without
// the clover term):
//   PLAIN  T^-1 acc                 MHAT  v1 - kappa^2 T^-1 acc
//   AXPY_K v1 + kappa T^-1 acc      RHS   T^-1 (v1 + kappa acc)
//   DIRAC  T v1 / (2 kappa) - acc/2 RESID v2 - T v1 / (2 kappa) + acc/2
enum Epi { EPI_PLAIN = 0, EPI_MHAT = 1, EPI_AXPY_K = 2, EPI_DIRAC = 3, EPI_RESID = 4, EPI_RHS = 5 };
enum Dot { DOT_NONE = 0, DOT_RHAT = 1, DOT_TS = 2, DOT_NORM = 3 };

struct HopArgs {
    Launch L;
    int p;          // parity of the output sites
    FieldView in;   // opposite-parity input
    FieldView out;  // output (parity p)
    FieldView v1;   // same-parity operand of the epilogue
    FieldView v2;   // second same-parity operand (EPI_RESID: eta)
    FieldView rh;   // shadow residual for DOT_RHAT
    Partials part;
    const SolveState *st;  // skip 1: leave columns whose inner solve is not active untouched;
    int skip;              // skip 2: leave columns whose outer solve has converged untouched
};

// Tiles are exactly HOP_TS = 32 sites (one warp per column of a tile); a
// block holds at most HOP_MAX_CG = 12 columns.  The kernels use the tile size
// as a compile-time constant.
// Storage of the BiCGStab shadow residual rh: any fixed vector serves as rh, so with
// FP32 storage it is kept as a BF16 copy of r_0 (same exponent range, half the bytes
// of the two reads per iteration); the other formats keep their own.
template <class P>
struct ShadowOf {
    using type = P;
};
template <>
struct ShadowOf<PF32> {
    using type = PBF16;
};

constexpr int HOP_TS = 32;
constexpr int HOP_MAX_CG = 12;

// Map a block/thread of a tile-structured launch to (item, column, site).
struct TileCoord {
    int col, h, tile;
    bool valid;
    int64_t cb;  // column base in the fields
};

__device__ __forceinline__ TileCoord tile_coord(const Item &it, const Launch &L) {
    TileCoord t;
    int lb = blockIdx.x - it.blk0;
    t.tile = lb % it.ntiles;
    int cg = lb / it.ntiles;
    int cl = threadIdx.x / HOP_TS;
    int sl = threadIdx.x - cl * HOP_TS;
    t.col = cg * L.CG + cl;
    t.h = t.tile * HOP_TS + sl;
    t.valid = (t.col < it.ncol) && (t.h < it.nh) && (cl < L.CG);
    t.cb = it.fbase + (int64_t)t.col * it.nh;
    return t;
}

// Block reduction of (complex, real) per column.  Each thread's products and
// the 32-lane warp sums are formed in the compute precision R (FP32 for the
// low-precision formats: FP64 arithmetic is a small fraction of GB300's FP32
// rate); the sums across warps and, in the scalar kernels, across blocks are
// FP64.  Lanes of a warp share one column (TS = 32); warps of the same
// column are added in warp order.  Fixed order: results do not depend on
// the batch around them.
template <typename R>
__device__ __forceinline__ void block_partials(const Item &it, const Launch &L, const TileCoord &tc, R cre, R cim,
                                               R nn, Partials part, bool want_c, bool want_n, int blk = -1) {
    __shared__ double s_re[32], s_im[32], s_nn[32];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (want_c) {
        cre = warp_sum(cre);
        cim = warp_sum(cim);
    }
    if (want_n) nn = warp_sum(nn);
    if (lane == 0) {
        s_re[warp] = (double)cre;
        s_im[warp] = (double)cim;
        s_nn[warp] = (double)nn;
    }
    __syncthreads();
    constexpr int wpc = HOP_TS >> 5;  // warps per column
    if ((int)threadIdx.x < L.CG) {
        int cl = threadIdx.x;
        int lb = (blk < 0 ? (int)blockIdx.x : blk) - it.blk0;
        int cg = lb / it.ntiles;
        int col = cg * L.CG + cl;
        if (col < it.ncol) {
            double a = 0, b = 0, c = 0;
            for (int w = cl * wpc; w < (cl + 1) * wpc; w++) {
                a += s_re[w];
                b += s_im[w];
                c += s_nn[w];
            }
            int64_t idx = it.pbase + (int64_t)col * it.ntiles + tc.tile;
            if (want_c) part.c[idx] = make_double2(a, b);
            if (want_n) part.n[idx] = c;
        }
    }
}

__device__ __forceinline__ void load_item(const Launch &L, Item &dst) {
    if (threadIdx.x == 0) dst = L.items[find_item(L.items, L.nitems, blockIdx.x)];
    __syncthreads();
}

// ------------------------------------------------------------ hopping kernel

// Tiles of TS sites: the links (oriented, boundary sign folded in, row 2
// rebuilt) and neighbour indices of the tile's 8 TS hops are staged in shared
// memory once and shared by the CG column-threads of every site.
// Epilogue of the hopping kernels: out = combination of acc and same-parity
// operands, stored in the storage format, plus the requested dot products.
template <class P, int EPI, int DOT, bool CLOV>
__device__ __forceinline__ void hop_store_epilogue(const HopArgs &a, const Item &it, const TileCoord &tc,
                                                   const cx<typename P::real> acc[4][3], typename P::real &cre,
                                                   typename P::real &cim, typename P::real &nn) {
    using R = typename P::real;
    R o[24];
    int64_t i = tc.cb + tc.h;
    const R kap = (R)it.kappa;
    // clover matrices of the output site (T^-1 on the hopping sum, T on v1)
    const bool clov = CLOV && it.clovinv;
    int64_t row = 0;
    if (clov) row = site_row(it, tc.h, a.p);
    R h[24];
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            h[2 * (3 * s + c)] = acc[s][c].re;
            h[2 * (3 * s + c) + 1] = acc[s][c].im;
        }
    if (clov && (EPI == EPI_PLAIN || EPI == EPI_MHAT || EPI == EPI_AXPY_K)) clover_apply<R>(it.clovinv, it.gV, row, h);
    if (EPI == EPI_PLAIN) {
#pragma unroll
        for (int j = 0; j < 24; j++) o[j] = h[j];
    } else {
        R w[24];
        load_spinor<P>(a.v1, i, w);
        if (clov && (EPI == EPI_DIRAC || EPI == EPI_RESID))
            clover_apply<R>(EPI == EPI_RESID ? it.clov64 : it.clov, it.gV, row, w);
        R cw, ca;
        if (EPI == EPI_MHAT) {
            cw = R(1);
            ca = -kap * kap;
        } else if (EPI == EPI_AXPY_K || EPI == EPI_RHS) {
            cw = R(1);
            ca = kap;
        } else if (EPI == EPI_DIRAC) {
            cw = R(1) / (R(2) * kap);
            ca = R(-0.5);
        } else {  // EPI_RESID: eta - T x/(2 kappa) + acc/2
            cw = -R(1) / (R(2) * kap);
            ca = R(0.5);
        }
#pragma unroll
        for (int j = 0; j < 24; j++) o[j] = cw * w[j] + ca * h[j];
        if (clov && EPI == EPI_RHS) clover_apply<R>(it.clovinv, it.gV, row, o);
        if (EPI == EPI_RESID) {
            load_spinor<P>(a.v2, i, w);
#pragma unroll
            for (int j = 0; j < 24; j++) o[j] += w[j];
        }
        if (DOT == DOT_TS) {
            // (t, s) = sum conj(t) s with t = out, s = v1 (reload v1: w was reused)
            R s1[24];
            load_spinor<P>(a.v1, i, s1);
#pragma unroll
            for (int j = 0; j < 12; j++) {
                cre += o[2 * j] * s1[2 * j] + o[2 * j + 1] * s1[2 * j + 1];
                cim += o[2 * j] * s1[2 * j + 1] - o[2 * j + 1] * s1[2 * j];
            }
        }
    }
    store_spinor<P>(a.out, i, o);
    if (DOT == DOT_RHAT) {
        R r[24];
        load_spinor<typename ShadowOf<P>::type>(a.rh, i, r);
#pragma unroll
        for (int j = 0; j < 12; j++) {
            cre += r[2 * j] * o[2 * j] + r[2 * j + 1] * o[2 * j + 1];
            cim += r[2 * j] * o[2 * j + 1] - r[2 * j + 1] * o[2 * j];
        }
    }
    if (DOT == DOT_TS || DOT == DOT_NORM) {
        R s = 0;
#pragma unroll
        for (int j = 0; j < 24; j++) s += o[j] * o[j];
        nn = s;
    }
}

// A staged link in shared memory: 9 complex, one 8-byte (FP32 compute) or
// 16-byte (FP64) access each.
template <typename R>
__device__ __forceinline__ void put_link(R *d, const cx<R> u[3][3]) {
    using V2 = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    V2 *q = reinterpret_cast<V2 *>(d);
#pragma unroll
    for (int k = 0; k < 9; k++) q[k] = V2{u[k / 3][k % 3].re, u[k / 3][k % 3].im};
}
template <typename R>
__device__ __forceinline__ void get_link(const R *d, cx<R> u[3][3]) {
    using V2 = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const V2 *q = reinterpret_cast<const V2 *>(d);
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const V2 c = q[k];
        u[k / 3][k % 3] = mk(c.x, c.y);
    }
}


template <class P, int EPI, int DOT, bool CLOV = false>
// Resident blocks per SM the register budget of the 32- and 16-bit stencils is fitted to
// (3: 56 registers a thread; 2: 80).
#ifndef DDP_HOP_MINB
#define DDP_HOP_MINB 3
#endif

__global__ void __launch_bounds__(384, sizeof(typename P::real) == 8 ? 1 : DDP_HOP_MINB) k_hop(HopArgs a) {
    using R = typename P::real;
    constexpr int TSMAX = HOP_TS;
    __shared__ Item it;
    // oriented link of hop slot q at s_u[q * 18]: 9 complex; vector reads of
    // consecutive slots by a warp fall in distinct banks
    constexpr int LP = 18;
    __shared__ int s_nb[8 * TSMAX];
    __shared__ __align__(16) R s_u[8 * TSMAX * LP];
    load_item(a.L, it);
    constexpr int TS = HOP_TS;
    if (a.skip) {
        // a block whose columns are all finished has nothing to stage or compute
        const int cg = (blockIdx.x - it.blk0) / it.ntiles;
        const int col = cg * a.L.CG + (int)threadIdx.x;
        int live = 0;
        if ((int)threadIdx.x < a.L.CG && col < it.ncol) {
            const SolveState &S = a.st[it.solve0 + col];
            live = (a.skip == 1) ? S.active : !S.outer_done;
        }
        if (!__syncthreads_or(live)) return;
    }
    if (std::is_same<P, PF32>::value) {
        // FP32 storage: the forward time-direction neighbour of this thread's site-column is
        // requested into L1 before the links are staged, so that its latency overlaps the
        // staging (measured on 48x24^3, 12 columns: 2.7-3.3% off each inner-loop stencil;
        // with the backward one too, or with 16-bit storage, less or nothing)
        const TileCoord t0 = tile_coord(it, a.L);
        if (t0.valid) {
            const int v3h = it.nh / it.e[0];  // sites of one parity in a time slice
            int nbf = t0.h + v3h;
            if (nbf >= it.nh) nbf -= it.nh;
            const float4 *base = reinterpret_cast<const float4 *>(a.in.p) + t0.cb + nbf;
#pragma unroll
            for (int j = 0; j < P::NCH; j++) asm volatile("prefetch.global.L1 [%0];" ::"l"(base + j * a.in.stride));
        }
    }
    {
        const int tile = (blockIdx.x - it.blk0) % it.ntiles;
        for (int q = threadIdx.x; q < 8 * TS; q += blockDim.x) {
            const int d = q / TS, sidx = q - d * TS, h = tile * TS + sidx;
            int nb = -1;
            cx<R> u[3][3];
            if (h < it.nh) nb = stage_hop<P>(it, h, a.p, d, u);
            s_nb[q] = nb;
            if (nb >= 0) put_link(s_u + q * LP, u);
        }
    }
    __syncthreads();
    TileCoord tc = tile_coord(it, a.L);
    if (a.skip && tc.valid) {
        const SolveState &S = a.st[it.solve0 + tc.col];
        if ((a.skip == 1) ? !S.active : S.outer_done) tc.valid = false;
    }
    R cre = 0, cim = 0, nn = 0;
    if (tc.valid) {
        cx<R> acc[4][3];
#pragma unroll
        for (int s2 = 0; s2 < 4; s2++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc[s2][c] = mk<R>(0, 0);
        const int sl = tc.h - tc.tile * TS;
#define DDP_HOP_STEP(D)                                                   \
        {                                                                 \
            const int q = (D) * TS + sl;                                  \
            const int nb = s_nb[q];                                       \
            if (nb >= 0) {                                                \
                R v[24], f;                                               \
                load_spinor_raw<P>(a.in, tc.cb + nb, v, &f);              \
                cx<R> u[3][3];                                            \
                get_link(s_u + q * LP, u);                                \
                hop_step<D, P::NCH != 6>(v, u, acc, f);                   \
            }                                                             \
        }
        DDP_HOP_STEP(0)
        DDP_HOP_STEP(1)
        DDP_HOP_STEP(2)
        DDP_HOP_STEP(3)
        DDP_HOP_STEP(4)
        DDP_HOP_STEP(5)
        DDP_HOP_STEP(6)
        DDP_HOP_STEP(7)
#undef DDP_HOP_STEP
        hop_store_epilogue<P, EPI, DOT, CLOV>(a, it, tc, acc, cre, cim, nn);
    }
    if (DOT != DOT_NONE) block_partials(it, a.L, tc, cre, cim, nn, a.part, DOT == DOT_RHAT || DOT == DOT_TS,
                                        DOT == DOT_TS || DOT == DOT_NORM);
}

// ------------------------------------------------------------ vector updates

// The reals of one storage chunk of an unscaled format, and back.
template <class P>
__device__ __forceinline__ void chunk_to_reals(const typename P::chunk &c, typename P::real *v);
template <>
__device__ __forceinline__ void chunk_to_reals<PF64>(const double2 &c, double *v) {
    v[0] = c.x;
    v[1] = c.y;
}
template <>
__device__ __forceinline__ void chunk_to_reals<PF32>(const float4 &c, float *v) {
    v[0] = c.x;
    v[1] = c.y;
    v[2] = c.z;
    v[3] = c.w;
}
template <>
__device__ __forceinline__ void chunk_to_reals<PBF16>(const uint4 &c, float *v) {
    const float2 a0 = b2f(c.x), a1 = b2f(c.y), a2 = b2f(c.z), a3 = b2f(c.w);
    v[0] = a0.x;
    v[1] = a0.y;
    v[2] = a1.x;
    v[3] = a1.y;
    v[4] = a2.x;
    v[5] = a2.y;
    v[6] = a3.x;
    v[7] = a3.y;
}
template <>
__device__ __forceinline__ void chunk_to_reals<PF16>(const uint4 &, float *) {}  // scaled: not chunk-local
template <class P>
__device__ __forceinline__ typename P::chunk reals_to_chunk(const typename P::real *v);
template <>
__device__ __forceinline__ double2 reals_to_chunk<PF64>(const double *v) {
    return make_double2(v[0], v[1]);
}
template <>
__device__ __forceinline__ float4 reals_to_chunk<PF32>(const float *v) {
    return make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ uint4 reals_to_chunk<PBF16>(const float *v) {
    uint4 c;
    c.x = f2b(v[0], v[1]);
    c.y = f2b(v[2], v[3]);
    c.z = f2b(v[4], v[5]);
    c.w = f2b(v[6], v[7]);
    return c;
}
template <>
__device__ __forceinline__ uint4 reals_to_chunk<PF16>(const float *) {
    return make_uint4(0, 0, 0, 0);
}

// The reals of storage chunk j (of format P) of site-column i of the shadow residual,
// stored in ShadowOf<P>.
template <class P>
__device__ __forceinline__ void shadow_reals(const FieldView &f, int j, int64_t i, typename P::real *v) {
    chunk_to_reals<P>(__ldg(reinterpret_cast<const typename P::chunk *>(f.p) + j * f.stride + i), v);
}
template <>
__device__ __forceinline__ void shadow_reals<PF32>(const FieldView &f, int j, int64_t i, float *v) {
    // FP32 chunk j (reals 4j .. 4j+3) is half j % 2 of BF16 chunk j / 2
    const uint2 c = __ldg(reinterpret_cast<const uint2 *>(reinterpret_cast<const uint4 *>(f.p) +
                                                          (int64_t)(j >> 1) * f.stride + i) + (j & 1));
    const float2 a0 = b2f(c.x), a1 = b2f(c.y);
    v[0] = a0.x;
    v[1] = a0.y;
    v[2] = a1.x;
    v[3] = a1.y;
}

enum BlasOp { OP_P_UPDATE = 0, OP_S_UPDATE = 1, OP_XR_UPDATE = 2, OP_INIT = 3, OP_NORM = 4 };

struct BlasArgs {
    Launch L;
    FieldView x, r, rh, p, v, s, t;
    const SolveState *st;
    Partials part;
    int skip;
};

template <class P, int OP>
__global__ void __launch_bounds__(512) k_blas(BlasArgs a) {
    using R = typename P::real;
    __shared__ Item it;
    load_item(a.L, it);
    TileCoord tc = tile_coord(it, a.L);
    if (a.skip && tc.valid && !a.st[it.solve0 + tc.col].active) tc.valid = false;
    R cre = 0, cim = 0, nn = 0;
    if (tc.valid) {
        int64_t i = tc.cb + tc.h;
        const SolveState &S = a.st[it.solve0 + tc.col];
        if (OP == OP_P_UPDATE) {  // p = r + beta (p - omega v)
            R r[24], p[24], v[24];
            load_spinor<P>(a.r, i, r);
            load_spinor<P>(a.p, i, p);
            load_spinor<P>(a.v, i, v);
            const R br = (R)S.beta.x, bi = (R)S.beta.y, wr = (R)S.omega.x, wi = (R)S.omega.y;
#pragma unroll
            for (int j = 0; j < 12; j++) {
                R qr = p[2 * j] - (wr * v[2 * j] - wi * v[2 * j + 1]);
                R qi = p[2 * j + 1] - (wr * v[2 * j + 1] + wi * v[2 * j]);
                p[2 * j] = r[2 * j] + (br * qr - bi * qi);
                p[2 * j + 1] = r[2 * j + 1] + (br * qi + bi * qr);
            }
            store_spinor<P>(a.p, i, p);
        } else if (OP == OP_S_UPDATE) {  // s = r - alpha v
            R r[24], v[24];
            load_spinor<P>(a.r, i, r);
            load_spinor<P>(a.v, i, v);
            const R ar = (R)S.alpha.x, ai = (R)S.alpha.y;
#pragma unroll
            for (int j = 0; j < 12; j++) {
                r[2 * j] -= ar * v[2 * j] - ai * v[2 * j + 1];
                r[2 * j + 1] -= ar * v[2 * j + 1] + ai * v[2 * j];
            }
            store_spinor<P>(a.s, i, r);
        } else if (OP == OP_XR_UPDATE && !P::SCALED) {
            // x += alpha p + omega s ; r = s - omega t ; dots -- one storage chunk at a
            // time (the fields do not alias), so few registers and many loads in flight
            using C = typename P::chunk;
            constexpr int NR = 24 / P::NCH;
            const C *__restrict__ cx_ = reinterpret_cast<const C *>(a.x.p);
            const C *__restrict__ cp_ = reinterpret_cast<const C *>(a.p.p);
            const C *__restrict__ cs_ = reinterpret_cast<const C *>(a.s.p);
            const C *__restrict__ ct_ = reinterpret_cast<const C *>(a.t.p);

            C *__restrict__ ox = reinterpret_cast<C *>(a.x.p);
            C *__restrict__ orr = reinterpret_cast<C *>(a.r.p);
            const R ar = (R)S.alpha.x, ai = (R)S.alpha.y, wr = (R)S.omega.x, wi = (R)S.omega.y;
            R n2 = 0;
#pragma unroll
            for (int j = 0; j < P::NCH; j++) {
                const int64_t o = j * a.x.stride + i;
                R x[NR], p[NR], s[NR], t[NR], rh[NR];
                chunk_to_reals<P>(__ldg(cx_ + o), x);
                chunk_to_reals<P>(__ldg(cp_ + o), p);
                chunk_to_reals<P>(__ldg(cs_ + o), s);
                chunk_to_reals<P>(__ldg(ct_ + o), t);
                shadow_reals<P>(a.rh, j, i, rh);
#pragma unroll
                for (int k = 0; k < NR / 2; k++) {
                    x[2 * k] += (ar * p[2 * k] - ai * p[2 * k + 1]) + (wr * s[2 * k] - wi * s[2 * k + 1]);
                    x[2 * k + 1] += (ar * p[2 * k + 1] + ai * p[2 * k]) + (wr * s[2 * k + 1] + wi * s[2 * k]);
                    s[2 * k] -= wr * t[2 * k] - wi * t[2 * k + 1];
                    s[2 * k + 1] -= wr * t[2 * k + 1] + wi * t[2 * k];
                }
                ox[o] = reals_to_chunk<P>(x);
                orr[o] = reals_to_chunk<P>(s);
#pragma unroll
                for (int k = 0; k < NR / 2; k++) {
                    cre += rh[2 * k] * s[2 * k] + rh[2 * k + 1] * s[2 * k + 1];
                    cim += rh[2 * k] * s[2 * k + 1] - rh[2 * k + 1] * s[2 * k];
                    n2 += s[2 * k] * s[2 * k] + s[2 * k + 1] * s[2 * k + 1];
                }
            }
            nn = n2;
        } else if (OP == OP_XR_UPDATE) {  // x += alpha p + omega s ; r = s - omega t ; dots
            R x[24], p[24], s[24], t[24];
            load_spinor<P>(a.x, i, x);
            load_spinor<P>(a.p, i, p);
            load_spinor<P>(a.s, i, s);
            load_spinor<P>(a.t, i, t);
            const R ar = (R)S.alpha.x, ai = (R)S.alpha.y, wr = (R)S.omega.x, wi = (R)S.omega.y;
#pragma unroll
            for (int j = 0; j < 12; j++) {
                x[2 * j] += (ar * p[2 * j] - ai * p[2 * j + 1]) + (wr * s[2 * j] - wi * s[2 * j + 1]);
                x[2 * j + 1] += (ar * p[2 * j + 1] + ai * p[2 * j]) + (wr * s[2 * j + 1] + wi * s[2 * j]);
                s[2 * j] -= wr * t[2 * j] - wi * t[2 * j + 1];
                s[2 * j + 1] -= wr * t[2 * j + 1] + wi * t[2 * j];
            }
            store_spinor<P>(a.x, i, x);
            store_spinor<P>(a.r, i, s);
            R rh[24];
            load_spinor<typename ShadowOf<P>::type>(a.rh, i, rh);
            R n2 = 0;
#pragma unroll
            for (int j = 0; j < 12; j++) {
                cre += rh[2 * j] * s[2 * j] + rh[2 * j + 1] * s[2 * j + 1];
                cim += rh[2 * j] * s[2 * j + 1] - rh[2 * j + 1] * s[2 * j];
                n2 += s[2 * j] * s[2 * j] + s[2 * j + 1] * s[2 * j + 1];
            }
            nn = n2;
        } else if (OP == OP_INIT) {  // rh = r ; p = r ; x = 0
            R r[24], z[24];
            load_spinor<P>(a.r, i, r);
            store_spinor<typename ShadowOf<P>::type>(a.rh, i, r);
            store_spinor<P>(a.p, i, r);
#pragma unroll
            for (int j = 0; j < 24; j++) z[j] = R(0);
            store_spinor<P>(a.x, i, z);
        } else if (OP == OP_NORM) {  // |x|^2
            R x[24];
            load_spinor<P>(a.x, i, x);
            R n2 = 0;
#pragma unroll
            for (int j = 0; j < 24; j++) n2 += x[j] * x[j];
            nn = n2;
        }
    }
    if (OP == OP_XR_UPDATE || OP == OP_NORM)
        block_partials(it, a.L, tc, cre, cim, nn, a.part, OP == OP_XR_UPDATE, true);
}

// ---------------------------------------------------- FP64 <-> storage format

struct ConvArgs {
    Launch L;
    FieldView lo;   // storage-format field
    FieldView hi;   // FP64 field
    const SolveState *st;
    int p;          // parity of the sites
    int clov;       // k_to_low: apply the clover T^-1 of the site (items that have one)
};

// lo = scale * hi  (scale = 2 kappa / sigma: the normalised defect), times T^-1
// of the site when a.clov is set
template <class P>
__global__ void __launch_bounds__(512) k_to_low(ConvArgs a) {
    using R = typename P::real;
    __shared__ Item it;
    load_item(a.L, it);
    TileCoord tc = tile_coord(it, a.L);
    if (!tc.valid) return;
    int64_t i = tc.cb + tc.h;
    const double sc = a.st[it.solve0 + tc.col].scale;
    double v[24];
    load_spinor<PF64>(a.hi, i, v);
    R w[24];
#pragma unroll
    for (int j = 0; j < 24; j++) w[j] = (R)(sc * v[j]);
    if (a.clov && it.clovinv) clover_apply<R>(it.clovinv, it.gV, site_row(it, tc.h, a.p), w);
    store_spinor<P>(a.lo, i, w);
}

// hi += sigma * lo  (FP64 accumulation of the correction)
template <class P>
__global__ void __launch_bounds__(512) k_accum(ConvArgs a) {
    using R = typename P::real;
    __shared__ Item it;
    load_item(a.L, it);
    TileCoord tc = tile_coord(it, a.L);
    if (!tc.valid) return;
    int64_t i = tc.cb + tc.h;
    const double sg = a.st[it.solve0 + tc.col].sigma;
    if (sg == 0.0) return;
    R w[24];
    load_spinor<P>(a.lo, i, w);
    double v[24];
    load_spinor<PF64>(a.hi, i, v);
#pragma unroll
    for (int j = 0; j < 24; j++) v[j] += sg * (double)w[j];
    store_spinor<PF64>(a.hi, i, v);
}

// ------------------------------------------------------------ scalar updates

enum FinOp { FIN_BNORM = 0, FIN_RESID = 1, FIN_INIT = 2, FIN_ALPHA = 3, FIN_OMEGA = 4, FIN_RHO = 5 };

struct FinArgs {
    const Item *items;
    SolveState *st;
    int nsolve;
    Partials A, B;  // B used by FIN_BNORM / FIN_RESID (odd parity)
    LoopCtl *ctl;
    // FIN_RHO ends an inner-loop iteration: its last block to finish also runs the loop
    // control (0: not in a loop; 1: sets the graph's WHILE condition; 2: host-polled)
    int loop_mode;
    cudaGraphConditionalHandle loop;
};

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cmuld(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One block per solve: fixed-order sum of the solve's tile partials, then the
// scalar recurrences of BiCGStab (van der Vorst) or of the defect correction.
template <int FIN>
__global__ void __launch_bounds__(256) k_fin(FinArgs a) {
    int s = blockIdx.x;
    if (s >= a.nsolve) return;
    SolveState &S = a.st[s];
    const Item &it = a.items[S.item];
    int64_t base = it.pbase + (int64_t)S.col * it.ntiles;
    const bool want_c = (FIN == FIN_ALPHA || FIN == FIN_OMEGA || FIN == FIN_RHO);
    const bool two = (FIN == FIN_BNORM || FIN == FIN_RESID);
    double cr = 0, ci = 0, nn = 0;
    for (int t = threadIdx.x; t < it.ntiles; t += blockDim.x) {
        if (want_c) {
            double2 c = a.A.c[base + t];
            cr += c.x;
            ci += c.y;
        }
        if (FIN != FIN_ALPHA) nn += a.A.n[base + t];
        if (two) nn += a.B.n[base + t];
    }
    __shared__ double sr[256], si[256], sn[256];
    sr[threadIdx.x] = cr;
    si[threadIdx.x] = ci;
    sn[threadIdx.x] = nn;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sr[threadIdx.x] += sr[threadIdx.x + o];
            si[threadIdx.x] += si[threadIdx.x + o];
            sn[threadIdx.x] += sn[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double2 c = make_double2(sr[0], si[0]);
    double n = sn[0];
    const double2 zero = make_double2(0, 0), one = make_double2(1, 0);
    if (FIN == FIN_BNORM) {
        S.bnorm2 = n;
        S.outer_done = S.outer_done || (n == 0.0);
    } else if (FIN == FIN_RESID) {
        if (S.outer_done) {  // converged earlier: its residual was not recomputed
            S.sigma = 0;
            S.scale = 0;
            return;
        }
        S.rr64 = n;
        bool done = (n <= S.tol * S.tol * S.bnorm2) || !(n == n);
        S.outer_done = done ? 1 : 0;
        if (done) {
            S.sigma = 0;
            S.scale = 0;
        } else {
            S.sigma = sqrt(n);
            S.scale = 2.0 * it.kappa / S.sigma;
            double d = 0.5 * S.tol * sqrt(S.bnorm2 / n);
            d = fmax(d, S.floor_delta);
            S.delta = fmin(d, 0.1);
        }
    } else if (FIN == FIN_INIT) {
        S.rr = n;
        S.rho = make_double2(n, 0);
        S.target2 = S.delta * S.delta * n;
        S.iters = 0;
        bool act = (S.sigma > 0) && (n > 0);
        S.active = act ? 1 : 0;
        S.status = act ? 0 : 4;
        S.alpha = act ? one : zero;
        S.omega = act ? one : zero;
        S.beta = zero;
        if (act) atomicAdd(&a.ctl->n_active, 1);
    } else if (FIN == FIN_ALPHA) {
        if (S.active) {
            if (!(c.x * c.x + c.y * c.y > 0) || !isfinite(c.x) || !isfinite(c.y)) {
                S.active = 0;
                S.status = 2;
                S.alpha = zero;
                S.omega = zero;
                S.beta = zero;
            } else {
                S.alpha = cdiv(S.rho, c);
            }
        }
    } else if (FIN == FIN_OMEGA) {
        if (S.active) S.omega = (n > 0) ? cdiv(c, make_double2(n, 0)) : zero;
    } else if (FIN == FIN_RHO) {
        if (S.active) {
            S.iters++;
            S.total_iters++;
            S.rr = n;
            bool w0 = (S.omega.x == 0.0 && S.omega.y == 0.0);
            if (n <= S.target2) {
                S.active = 0;
                S.status = 1;
            } else if (!(c.x * c.x + c.y * c.y > 0) || w0 || !isfinite(n)) {
                S.active = 0;
                S.status = 2;
            } else if (S.iters >= S.maxit) {
                S.active = 0;
                S.status = 3;
            } else {
                S.beta = cmuld(cdiv(c, S.rho), cdiv(S.alpha, S.omega));
                S.rho = c;
            }
            if (!S.active) {
                S.alpha = zero;
                S.omega = zero;
                S.beta = zero;
            } else {
                atomicAdd(&a.ctl->n_active, 1);
            }
        }
        if (a.loop_mode) {
            // the last solve's block decides whether the loop goes on (every block's
            // n_active increment is ordered before its arrival by the fence)
            __threadfence();
            if (atomicAdd(&a.ctl->done_blocks, 1) == a.nsolve - 1) {
                __threadfence();
                LoopCtl *c = a.ctl;
                const int cont = (atomicAdd(&c->n_active, 0) > 0) && (++c->iter < c->maxit);
                c->n_active = 0;
                c->done_blocks = 0;
                if (a.loop_mode == 1)
                    cudaGraphSetConditional(a.loop, cont ? 1u : 0u);
                else
                    c->pad = cont;
            }
        }
    }
}

// ---------------------------------------------- user layout <-> even-odd fields
//
// User spinors: [ncol][n][4][3] complex, domain-local lexicographic order.
// One launch per item; thread per (column, site).

struct PackArgs {
    Item it;
    const double2 *user;  // eta (pack) or NULL for a point source
    double2 *uout;        // unpack target
    FieldView fe, fo;     // FP64 even / odd fields
    FieldView xe, xo;     // pack: solution fields zeroed at the same sites (p == NULL: untouched)
    int src_l;            // point source local index (pack with user == NULL)
};

__device__ __forceinline__ void local_coords(const Item &it, int l, int k[4]) {
    k[3] = l % it.e[3];
    l /= it.e[3];
    k[2] = l % it.e[2];
    l /= it.e[2];
    k[1] = l % it.e[1];
    k[0] = l / it.e[1];
}

static __global__ void k_pack(PackArgs a) {
    int64_t n = 2 * (int64_t)a.it.nh;
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n * a.it.ncol) return;
    int col = (int)(g / n);
    int l = (int)(g - (int64_t)col * n);
    int k[4];
    local_coords(a.it, l, k);
    int par = (a.it.par_o + k[0] + k[1] + k[2] + k[3]) & 1;
    int64_t i = a.it.fbase + (int64_t)col * a.it.nh + (l >> 1);
    double v[24];
    if (a.user) {
        const double2 *u = a.user + ((int64_t)col * n + l) * 12;
#pragma unroll
        for (int j = 0; j < 12; j++) {
            double2 c = u[j];
            v[2 * j] = c.x;
            v[2 * j + 1] = c.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 24; j++) v[j] = 0.0;
        if (l == a.src_l) v[2 * col] = 1.0;  // column c = 3 spin + colour is component c
    }
    store_spinor<PF64>(par ? a.fo : a.fe, i, v);
    if (a.xe.p) {
#pragma unroll
        for (int j = 0; j < 24; j++) v[j] = 0.0;
        store_spinor<PF64>(par ? a.xo : a.xe, i, v);
    }
}

static __global__ void k_unpack(PackArgs a) {
    int64_t n = 2 * (int64_t)a.it.nh;
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n * a.it.ncol) return;
    int col = (int)(g / n);
    int l = (int)(g - (int64_t)col * n);
    int k[4];
    local_coords(a.it, l, k);
    int par = (a.it.par_o + k[0] + k[1] + k[2] + k[3]) & 1;
    int64_t i = a.it.fbase + (int64_t)col * a.it.nh + (l >> 1);
    double v[24];
    load_spinor<PF64>(par ? a.fo : a.fe, i, v);
    double2 *u = a.uout + ((int64_t)col * n + l) * 12;
#pragma unroll
    for (int j = 0; j < 12; j++) u[j] = make_double2(v[2 * j], v[2 * j + 1]);
}

// Low-precision pack/unpack (for applying the low-precision stencil alone).
template <class P>
__global__ void k_pack_low(PackArgs a, FieldView le, FieldView lo) {
    using R = typename P::real;
    int64_t n = 2 * (int64_t)a.it.nh;
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n * a.it.ncol) return;
    int col = (int)(g / n);
    int l = (int)(g - (int64_t)col * n);
    int k[4];
    local_coords(a.it, l, k);
    int par = (a.it.par_o + k[0] + k[1] + k[2] + k[3]) & 1;
    int64_t i = a.it.fbase + (int64_t)col * a.it.nh + (l >> 1);
    const double2 *u = a.user + ((int64_t)col * n + l) * 12;
    R v[24];
#pragma unroll
    for (int j = 0; j < 12; j++) {
        double2 c = u[j];
        v[2 * j] = (R)c.x;
        v[2 * j + 1] = (R)c.y;
    }
    store_spinor<P>(par ? lo : le, i, v);
}

template <class P>
__global__ void k_unpack_low(PackArgs a, FieldView le, FieldView lo) {
    using R = typename P::real;
    int64_t n = 2 * (int64_t)a.it.nh;
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n * a.it.ncol) return;
    int col = (int)(g / n);
    int l = (int)(g - (int64_t)col * n);
    int k[4];
    local_coords(a.it, l, k);
    int par = (a.it.par_o + k[0] + k[1] + k[2] + k[3]) & 1;
    int64_t i = a.it.fbase + (int64_t)col * a.it.nh + (l >> 1);
    R v[24];
    load_spinor<P>(par ? lo : le, i, v);
    double2 *u = a.uout + ((int64_t)col * n + l) * 12;
#pragma unroll
    for (int j = 0; j < 12; j++) u[j] = make_double2((double)v[2 * j], (double)v[2 * j + 1]);
}

}  // namespace ddp
