// Column-pair kernels of the low-precision inner solver.
//
// The inner BiCGStab fields of the mixed-precision solves (FP32, FP16 and BF16
// storage) hold the columns of a request two by two: a "pair-site" stores the
// same site of columns 2m and 2m+1 with every real component of the two
// columns side by side, so that each arithmetic step of the hopping term
// (App. A; spin projection, SU(3) products, accumulation) and of the vector
// updates is one packed two-lane FP32 instruction (FFMA2 / FADD2 / FMUL2) for
// two columns at once, with the link of the site loaded once for both.
//
//   FP32 : 12 chunks of float4 per pair-site; chunk k is spin-colour
//          component k = 3 s + a: (re col0, re col1, im col0, im col1).
//   FP16 : 6 chunks of 4 half2; chunk j holds components 2j and 2j+1 as
//          (re, im, re, im) half2 pairs (low half col0, high half col1) and a
//          float2 scale (max |v| of each column) per pair-site.
//   BF16 : as FP16 without scales.
//
// Pair-site index of (pair m, even-odd site h) of an item: qbase + m nh + h.
// A request with an odd number of columns carries one padding column, which
// is kept at zero on entry and never read back.
#pragma once

#include "ddp_kernels.cuh"

namespace ddp {

struct QF32 {
    using chunk = float4;
    using LinkP = PF32;
    static constexpr int NCH = 12;
    static constexpr bool SCALED = false;
    static constexpr bool BF = false;
    static constexpr int NSCALE = 0;
    static constexpr bool IS64 = false;
};
struct QF16 {
    using chunk = uint4;
    using LinkP = PF16;
    static constexpr int NCH = 6;
    static constexpr bool SCALED = true;
    static constexpr bool BF = false;
    static constexpr int NSCALE = 2;
    static constexpr bool IS64 = false;
};
struct QBF16 {
    using chunk = uint4;
    using LinkP = PBF16;
    static constexpr int NCH = 6;
    static constexpr bool SCALED = false;
    static constexpr bool BF = true;
    static constexpr int NSCALE = 0;
    static constexpr bool IS64 = false;
};

template <class P>
struct PairOf;
template <>
struct PairOf<PF32> {
    using type = QF32;
};
template <>
struct PairOf<PF16> {
    using type = QF16;
};
template <>
struct PairOf<PBF16> {
    using type = QBF16;
};

// ------------------------------------------------------- packed arithmetic

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as one fused multiply-add by -1 (exact product, one rounding)
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pneg(float2 a) { return make_float2(-a.x, -a.y); }

// A complex number of two columns: real parts of both, imaginary parts of both.
struct cp {
    float2 re, im;
};

__device__ __forceinline__ float2 hh2f(unsigned int u) {
    __half2 h = *reinterpret_cast<__half2 *>(&u);
    return __half22float2(h);
}
__device__ __forceinline__ float2 bb2f(unsigned int u) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&u);
    return __bfloat1622float2(h);
}

// -------------------------------------------------- pair-site load / store
//
// v[k] = spin-colour component k of both columns.  qload returns the values
// (FP16: scale applied), qload_raw the stored values and the scale.

template <class Q>
__device__ __forceinline__ void qload_raw(const FieldView &f, int64_t i, cp v[12], float2 *s) {
    if constexpr (Q::NCH == 12) {
        const float4 *b = reinterpret_cast<const float4 *>(f.p);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            const float4 c = __ldg(b + k * f.stride + i);
            v[k].re = f2(c.x, c.y);
            v[k].im = f2(c.z, c.w);
        }
        *s = f2(1.f, 1.f);
    } else {
        const uint4 *b = reinterpret_cast<const uint4 *>(f.p);
#pragma unroll
        for (int j = 0; j < 6; j++) {
            const uint4 c = __ldg(b + j * f.stride + i);
            if constexpr (Q::BF) {
                v[2 * j].re = bb2f(c.x);
                v[2 * j].im = bb2f(c.y);
                v[2 * j + 1].re = bb2f(c.z);
                v[2 * j + 1].im = bb2f(c.w);
            } else {
                v[2 * j].re = hh2f(c.x);
                v[2 * j].im = hh2f(c.y);
                v[2 * j + 1].re = hh2f(c.z);
                v[2 * j + 1].im = hh2f(c.w);
            }
        }
        if constexpr (Q::SCALED)
            *s = __ldg(reinterpret_cast<const float2 *>(f.scale) + i);
        else
            *s = f2(1.f, 1.f);
    }
}

template <class Q>
__device__ __forceinline__ void qload(const FieldView &f, int64_t i, cp v[12]) {
    float2 s;
    qload_raw<Q>(f, i, v, &s);
    if constexpr (Q::SCALED) {
#pragma unroll
        for (int k = 0; k < 12; k++) {
            v[k].re = pmul(v[k].re, s);
            v[k].im = pmul(v[k].im, s);
        }
    }
}

__device__ __forceinline__ unsigned int f2h2(float2 v) {
    __half2 h = __float22half2_rn(v);
    return *reinterpret_cast<unsigned int *>(&h);
}
__device__ __forceinline__ unsigned int f2b2(float2 v) {
    __nv_bfloat162 h = __float22bfloat162_rn(v);
    return *reinterpret_cast<unsigned int *>(&h);
}

template <class Q>
__device__ __forceinline__ void qstore(const FieldView &f, int64_t i, const cp v[12]) {
    if constexpr (Q::NCH == 12) {
        float4 *b = reinterpret_cast<float4 *>(f.p);
#pragma unroll
        for (int k = 0; k < 12; k++) b[k * f.stride + i] = make_float4(v[k].re.x, v[k].re.y, v[k].im.x, v[k].im.y);
    } else {
        uint4 *b = reinterpret_cast<uint4 *>(f.p);
        if constexpr (Q::SCALED) {
            // per column: stored values are v / max|v|
            float mx = 0.f, my = 0.f;
#pragma unroll
            for (int k = 0; k < 12; k++) {
                mx = fmaxf(mx, fmaxf(fabsf(v[k].re.x), fabsf(v[k].im.x)));
                my = fmaxf(my, fmaxf(fabsf(v[k].re.y), fabsf(v[k].im.y)));
            }
            const float2 inv = f2(mx > 0.f ? 1.0f / mx : 0.f, my > 0.f ? 1.0f / my : 0.f);
            reinterpret_cast<float2 *>(f.scale)[i] = f2(mx, my);
#pragma unroll
            for (int j = 0; j < 6; j++) {
                uint4 c;
                c.x = f2h2(pmul(v[2 * j].re, inv));
                c.y = f2h2(pmul(v[2 * j].im, inv));
                c.z = f2h2(pmul(v[2 * j + 1].re, inv));
                c.w = f2h2(pmul(v[2 * j + 1].im, inv));
                b[j * f.stride + i] = c;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 6; j++) {
                uint4 c;
                c.x = f2b2(v[2 * j].re);
                c.y = f2b2(v[2 * j].im);
                c.z = f2b2(v[2 * j + 1].re);
                c.w = f2b2(v[2 * j + 1].im);
                b[j * f.stride + i] = c;
            }
        }
    }
}

// ----------------------------------------------------------- pair hopping
//
// Same hop as hop_step (ddp_device.cuh), for two columns at once.  Spin
// projection (1 -/+ g_mu) in the chiral basis leaves two spin rows h0, h1;
// only they are multiplied by the link; the lower spins of the result are
// +/- h or +/- i h of the upper ones.

// h0, h1 of colour a from the four spins p0..p3 of that colour.
template <int MU, bool FWD>
__device__ __forceinline__ void qproject(const cp &p0, const cp &p1, const cp &p2, const cp &p3, cp &h0, cp &h1) {
    if (MU == 0) {
        h0.re = FWD ? psub(p0.re, p2.re) : padd(p0.re, p2.re);
        h0.im = FWD ? psub(p0.im, p2.im) : padd(p0.im, p2.im);
        h1.re = FWD ? psub(p1.re, p3.re) : padd(p1.re, p3.re);
        h1.im = FWD ? psub(p1.im, p3.im) : padd(p1.im, p3.im);
    } else if (MU == 1) {  // h0 = p0 +/- i p3, h1 = p1 +/- i p2
        h0.re = FWD ? psub(p0.re, p3.im) : padd(p0.re, p3.im);
        h0.im = FWD ? padd(p0.im, p3.re) : psub(p0.im, p3.re);
        h1.re = FWD ? psub(p1.re, p2.im) : padd(p1.re, p2.im);
        h1.im = FWD ? padd(p1.im, p2.re) : psub(p1.im, p2.re);
    } else if (MU == 2) {  // h0 = p0 +/- p3, h1 = p1 -/+ p2
        h0.re = FWD ? padd(p0.re, p3.re) : psub(p0.re, p3.re);
        h0.im = FWD ? padd(p0.im, p3.im) : psub(p0.im, p3.im);
        h1.re = FWD ? psub(p1.re, p2.re) : padd(p1.re, p2.re);
        h1.im = FWD ? psub(p1.im, p2.im) : padd(p1.im, p2.im);
    } else {  // h0 = p0 +/- i p2, h1 = p1 -/+ i p3
        h0.re = FWD ? psub(p0.re, p2.im) : padd(p0.re, p2.im);
        h0.im = FWD ? padd(p0.im, p2.re) : psub(p0.im, p2.re);
        h1.re = FWD ? padd(p1.re, p3.im) : psub(p1.re, p3.im);
        h1.im = FWD ? psub(p1.im, p3.re) : padd(p1.im, p3.re);
    }
}

// acc += f w  (f = (1,1) for unscaled storage: plain additions)
template <bool SC>
__device__ __forceinline__ void qacc(float2 &acc, float2 f, float2 w) {
    acc = SC ? pfma(f, w, acc) : padd(acc, w);
}
template <bool SC>
__device__ __forceinline__ void qdec(float2 &acc, float2 nf, float2 w) {
    acc = SC ? pfma(nf, w, acc) : psub(acc, w);
}

// acc[component 3 s + a] += lower/upper spins of w0 = (u h0)_a, w1 = (u h1)_a.
template <int MU, bool FWD, bool SC>
__device__ __forceinline__ void qaccumulate(cp acc[12], int a, const cp &w0, const cp &w1, float2 f, float2 nf) {
    qacc<SC>(acc[a].re, f, w0.re);
    qacc<SC>(acc[a].im, f, w0.im);
    qacc<SC>(acc[3 + a].re, f, w1.re);
    qacc<SC>(acc[3 + a].im, f, w1.im);
    cp &a2 = acc[6 + a];
    cp &a3 = acc[9 + a];
    if (MU == 0) {  // lower = -/+ upper
        if (FWD) {
            qdec<SC>(a2.re, nf, w0.re);
            qdec<SC>(a2.im, nf, w0.im);
            qdec<SC>(a3.re, nf, w1.re);
            qdec<SC>(a3.im, nf, w1.im);
        } else {
            qacc<SC>(a2.re, f, w0.re);
            qacc<SC>(a2.im, f, w0.im);
            qacc<SC>(a3.re, f, w1.re);
            qacc<SC>(a3.im, f, w1.im);
        }
    } else if (MU == 1) {  // a2 += -/+ i w1, a3 += -/+ i w0;  -i w = (w.im, -w.re)
        if (FWD) {
            qacc<SC>(a2.re, f, w1.im);
            qdec<SC>(a2.im, nf, w1.re);
            qacc<SC>(a3.re, f, w0.im);
            qdec<SC>(a3.im, nf, w0.re);
        } else {
            qdec<SC>(a2.re, nf, w1.im);
            qacc<SC>(a2.im, f, w1.re);
            qdec<SC>(a3.re, nf, w0.im);
            qacc<SC>(a3.im, f, w0.re);
        }
    } else if (MU == 2) {  // a2 += -/+ w1, a3 += +/- w0
        if (FWD) {
            qdec<SC>(a2.re, nf, w1.re);
            qdec<SC>(a2.im, nf, w1.im);
            qacc<SC>(a3.re, f, w0.re);
            qacc<SC>(a3.im, f, w0.im);
        } else {
            qacc<SC>(a2.re, f, w1.re);
            qacc<SC>(a2.im, f, w1.im);
            qdec<SC>(a3.re, nf, w0.re);
            qdec<SC>(a3.im, nf, w0.im);
        }
    } else {  // a2 += -/+ i w0, a3 += +/- i w1
        if (FWD) {
            qacc<SC>(a2.re, f, w0.im);
            qdec<SC>(a2.im, nf, w0.re);
            qdec<SC>(a3.re, nf, w1.im);
            qacc<SC>(a3.im, f, w1.re);
        } else {
            qdec<SC>(a2.re, nf, w0.im);
            qacc<SC>(a2.im, f, w0.re);
            qacc<SC>(a3.re, f, w1.im);
            qdec<SC>(a3.im, nf, w1.re);
        }
    }
}

// A staged link: 9 complex entries, each as (re, re, im, im) so that one
// 16-byte shared-memory read gives both operands of the packed products.
__device__ __forceinline__ void put_link_dup(float4 *d, const cx<float> u[3][3]) {
#pragma unroll
    for (int k = 0; k < 9; k++) d[k] = make_float4(u[k / 3][k % 3].re, u[k / 3][k % 3].re, u[k / 3][k % 3].im,
                                                   u[k / 3][k % 3].im);
}

// w_s = (u h_s)_a for both rows s of the half spinor, row a of the link.
__device__ __forceinline__ void qsu3_row(const float4 *urow, const cp h0[3], const cp h1[3], cp &w0, cp &w1) {
    float2 A0, B0, C0, A1, B1, C1;
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const float4 u = urow[b];
        const float2 ur = f2(u.x, u.y), ui = f2(u.z, u.w);
        if (b == 0) {
            A0 = pmul(ur, h0[0].re);
            B0 = pmul(ui, h0[0].im);
            C0 = pmul(ur, h0[0].im);
            A1 = pmul(ur, h1[0].re);
            B1 = pmul(ui, h1[0].im);
            C1 = pmul(ur, h1[0].im);
        } else {
            A0 = pfma(ur, h0[b].re, A0);
            B0 = pfma(ui, h0[b].im, B0);
            C0 = pfma(ur, h0[b].im, C0);
            A1 = pfma(ur, h1[b].re, A1);
            B1 = pfma(ui, h1[b].im, B1);
            C1 = pfma(ur, h1[b].im, C1);
        }
        C0 = pfma(ui, h0[b].re, C0);
        C1 = pfma(ui, h1[b].re, C1);
    }
    w0.re = psub(A0, B0);
    w0.im = C0;
    w1.re = psub(A1, B1);
    w1.im = C1;
}

// acc += f (1 -/+ g_mu) u psi for hop D of both columns; link u staged at s_u.
template <int D, class Q>
__device__ __forceinline__ void qhop(const FieldView &in, int64_t i, const float4 *s_u, cp acc[12]) {
    constexpr int MU = D >> 1;
    constexpr bool FWD = !(D & 1);
    constexpr bool SC = Q::SCALED;
    cp v[12];
    float2 f;
    qload_raw<Q>(in, i, v, &f);
    const float2 nf = pneg(f);
    cp h0[3], h1[3];
#pragma unroll
    for (int a = 0; a < 3; a++) qproject<MU, FWD>(v[a], v[3 + a], v[6 + a], v[9 + a], h0[a], h1[a]);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        cp w0, w1;
        qsu3_row(s_u + 3 * a, h0, h1, w0, w1);
        qaccumulate<MU, FWD, SC>(acc, a, w0, w1, f, nf);
    }
}

// ------------------------------------------------------ pair launch table

__device__ __forceinline__ int find_item_q(const Item *items, int nitems, int b) {
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (items[mid].blk0q <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void load_item_q(const Launch &L, Item &dst) {
    if (threadIdx.x == 0) dst = L.items[find_item_q(L.items, L.nitems, blockIdx.x)];
    __syncthreads();
}

// Block = HOP_TS sites (one warp) x L.PG pairs; warp w handles pair pg*PG + w.
struct QCoord {
    int pair, h, tile;
    bool valid;
    int64_t i;  // pair-site index
};

__device__ __forceinline__ QCoord qcoord(const Item &it, const Launch &L) {
    QCoord q;
    const int lb = blockIdx.x - it.blk0q;
    q.tile = lb % it.ntiles;
    const int pg = lb / it.ntiles;
    const int w = threadIdx.x >> 5;
    q.pair = pg * L.PG + w;
    q.h = q.tile * HOP_TS + (threadIdx.x & 31);
    q.valid = (w < L.PG) && (q.pair < it.npair) && (q.h < it.nh);
    q.i = it.qbase + (int64_t)q.pair * it.nh + q.h;
    return q;
}

// Per-column partial sums of one warp (= one pair of one tile): lanes of the
// warp hold the products of their sites; the sums over the warp are formed
// in FP32 and stored in FP64 at (column, tile), fixed order.
__device__ __forceinline__ void qpartials(const Item &it, const QCoord &q, float2 cre, float2 cim, float2 nn,
                                          Partials part, bool want_c, bool want_n) {
    const bool lane0 = (threadIdx.x & 31) == 0;
    if (want_c) {
        cre.x = warp_sum(cre.x);
        cre.y = warp_sum(cre.y);
        cim.x = warp_sum(cim.x);
        cim.y = warp_sum(cim.y);
    }
    if (want_n) {
        nn.x = warp_sum(nn.x);
        nn.y = warp_sum(nn.y);
    }
    if (!lane0 || q.pair >= it.npair) return;
#pragma unroll
    for (int l = 0; l < 2; l++) {
        const int col = 2 * q.pair + l;
        if (col >= it.ncol) break;
        const int64_t idx = it.pbase + (int64_t)col * it.ntiles + q.tile;
        if (want_c) part.c[idx] = make_double2((double)(l ? cre.y : cre.x), (double)(l ? cim.y : cim.x));
        if (want_n) part.n[idx] = (double)(l ? nn.y : nn.x);
    }
}

// Column activity of the pair (columns beyond ncol count as inactive).
__device__ __forceinline__ void pair_live(const Item &it, const SolveState *st, int pair, int skip, bool &l0,
                                          bool &l1) {
    l0 = l1 = false;
    const int c0 = 2 * pair, c1 = c0 + 1;
    if (c0 < it.ncol) {
        const SolveState &S = st[it.solve0 + c0];
        l0 = (skip == 1) ? S.active != 0 : !S.outer_done;
    }
    if (c1 < it.ncol) {
        const SolveState &S = st[it.solve0 + c1];
        l1 = (skip == 1) ? S.active != 0 : !S.outer_done;
    }
}

// ----------------------------------------------------------- pair stencil

constexpr int HOP_MAX_PG = 6;

template <class Q, int EPI, int DOT>
__device__ __forceinline__ void qhop_epilogue(const HopArgs &a, const Item &it, const QCoord &q, const cp acc[12],
                                              float2 &cre, float2 &cim, float2 &nn) {
    cp o[12];
    const float kap = (float)it.kappa;
    if (EPI == EPI_PLAIN) {
#pragma unroll
        for (int k = 0; k < 12; k++) o[k] = acc[k];
    } else {
        cp w[12];
        qload<Q>(a.v1, q.i, w);
        float cw, ca;
        if (EPI == EPI_MHAT) {
            cw = 1.f;
            ca = -kap * kap;
        } else if (EPI == EPI_AXPY_K) {
            cw = 1.f;
            ca = kap;
        } else {  // EPI_DIRAC
            cw = 1.f / (2.f * kap);
            ca = -0.5f;
        }
        const float2 CW = f2(cw, cw), CA = f2(ca, ca);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            if (EPI == EPI_DIRAC) {
                o[k].re = pfma(CA, acc[k].re, pmul(CW, w[k].re));
                o[k].im = pfma(CA, acc[k].im, pmul(CW, w[k].im));
            } else {
                o[k].re = pfma(CA, acc[k].re, w[k].re);
                o[k].im = pfma(CA, acc[k].im, w[k].im);
            }
        }
        if (DOT == DOT_TS) {  // (t, s) = sum conj(t) s with t = out, s = v1
            float2 r = f2(0.f, 0.f), m = f2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 12; k++) {
                r = pfma(o[k].re, w[k].re, r);
                r = pfma(o[k].im, w[k].im, r);
                m = pfma(o[k].re, w[k].im, m);
                m = pfma(pneg(o[k].im), w[k].re, m);
            }
            cre = r;
            cim = m;
        }
    }
    qstore<Q>(a.out, q.i, o);
    if (DOT == DOT_RHAT) {  // (rh, v) = sum conj(rh) v
        cp r[12];
        qload<Q>(a.rh, q.i, r);
        float2 x = f2(0.f, 0.f), y = f2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            x = pfma(r[k].re, o[k].re, x);
            x = pfma(r[k].im, o[k].im, x);
            y = pfma(r[k].re, o[k].im, y);
            y = pfma(pneg(r[k].im), o[k].re, y);
        }
        cre = x;
        cim = y;
    }
    if (DOT == DOT_TS || DOT == DOT_NORM) {
        float2 s = f2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            s = pfma(o[k].re, o[k].re, s);
            s = pfma(o[k].im, o[k].im, s);
        }
        nn = s;
    }
}

// out(p) = epilogue(acc = sum over the 8 hops of (1 -/+ g) U in(p^1)) for every
// pair-site of the launch: the oriented links (row 2 rebuilt, boundary sign
// folded in) and the neighbour indices of a tile's 8 x 32 hops are staged in
// shared memory once and shared by the tile's pair-warps.
template <class Q, int EPI, int DOT>
__global__ void __launch_bounds__(HOP_TS *HOP_MAX_PG, 2) k_qhop(HopArgs a) {
    using LP = typename Q::LinkP;
    constexpr int TS = HOP_TS;
    __shared__ Item it;
    __shared__ int s_nb[8 * TS];
    __shared__ float4 s_u[8 * TS * 9];
    load_item_q(a.L, it);
    const int pg = (blockIdx.x - it.blk0q) / it.ntiles;
    if (a.skip) {
        // a block whose columns are all finished has nothing to stage or compute
        int live = 0;
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0 && w < a.L.PG) {
            bool l0, l1;
            pair_live(it, a.st, pg * a.L.PG + w, a.skip, l0, l1);
            live = l0 || l1;
        }
        if (!__syncthreads_or(live)) return;
    }
    {
        const int tile = (blockIdx.x - it.blk0q) % it.ntiles;
        for (int q = threadIdx.x; q < 8 * TS; q += blockDim.x) {
            const int d = q / TS, sidx = q - d * TS, h = tile * TS + sidx;
            int nb = -1;
            cx<float> u[3][3];
            if (h < it.nh) nb = stage_hop<LP>(it, h, a.p, d, u);
            s_nb[q] = nb;
            if (nb >= 0) put_link_dup(s_u + q * 9, u);
        }
    }
    __syncthreads();
    QCoord q = qcoord(it, a.L);
    if (a.skip && q.valid) {
        bool l0, l1;
        pair_live(it, a.st, q.pair, a.skip, l0, l1);
        if (!l0 && !l1) q.valid = false;
    }
    float2 cre = f2(0.f, 0.f), cim = f2(0.f, 0.f), nn = f2(0.f, 0.f);
    if (q.valid) {
        cp acc[12];
#pragma unroll
        for (int k = 0; k < 12; k++) acc[k].re = acc[k].im = f2(0.f, 0.f);
        const int sl = q.h - q.tile * TS;
        const int64_t cb = it.qbase + (int64_t)q.pair * it.nh;
#define DDP_QHOP_STEP(D)                                        \
        {                                                       \
            const int qs = (D) * TS + sl;                       \
            const int nb = s_nb[qs];                            \
            if (nb >= 0) qhop<D, Q>(a.in, cb + nb, s_u + qs * 9, acc); \
        }
        DDP_QHOP_STEP(0)
        DDP_QHOP_STEP(1)
        DDP_QHOP_STEP(2)
        DDP_QHOP_STEP(3)
        DDP_QHOP_STEP(4)
        DDP_QHOP_STEP(5)
        DDP_QHOP_STEP(6)
        DDP_QHOP_STEP(7)
#undef DDP_QHOP_STEP
        qhop_epilogue<Q, EPI, DOT>(a, it, q, acc, cre, cim, nn);
    }
    if (DOT != DOT_NONE)
        qpartials(it, q, cre, cim, nn, a.part, DOT == DOT_RHAT || DOT == DOT_TS, DOT == DOT_TS || DOT == DOT_NORM);
}

// ------------------------------------------------------ pair vector updates

// Scalars of the two columns of a pair as packed pairs (inactive or padding
// columns: zeros, which leave their fields as they are).
struct PairScalars {
    float2 ar, ai, wr, wi, br, bi;
};

__device__ __forceinline__ PairScalars pair_scalars(const Item &it, const SolveState *st, int pair) {
    PairScalars p;
    float v[2][6];
#pragma unroll
    for (int l = 0; l < 2; l++) {
        const int col = 2 * pair + l;
#pragma unroll
        for (int j = 0; j < 6; j++) v[l][j] = 0.f;
        if (col < it.ncol) {
            const SolveState &S = st[it.solve0 + col];
            v[l][0] = (float)S.alpha.x;
            v[l][1] = (float)S.alpha.y;
            v[l][2] = (float)S.omega.x;
            v[l][3] = (float)S.omega.y;
            v[l][4] = (float)S.beta.x;
            v[l][5] = (float)S.beta.y;
        }
    }
    p.ar = f2(v[0][0], v[1][0]);
    p.ai = f2(v[0][1], v[1][1]);
    p.wr = f2(v[0][2], v[1][2]);
    p.wi = f2(v[0][3], v[1][3]);
    p.br = f2(v[0][4], v[1][4]);
    p.bi = f2(v[0][5], v[1][5]);
    return p;
}

// a -= z b (complex pairs)
__device__ __forceinline__ void cp_sub_mul(cp &a, float2 zr, float2 zi, const cp &b) {
    a.re = pfma(pneg(zr), b.re, a.re);
    a.re = pfma(zi, b.im, a.re);
    a.im = pfma(pneg(zr), b.im, a.im);
    a.im = pfma(pneg(zi), b.re, a.im);
}
// a += z b
__device__ __forceinline__ void cp_add_mul(cp &a, float2 zr, float2 zi, const cp &b) {
    a.re = pfma(zr, b.re, a.re);
    a.re = pfma(pneg(zi), b.im, a.re);
    a.im = pfma(zr, b.im, a.im);
    a.im = pfma(zi, b.re, a.im);
}

struct QBlasArgs {
    Launch L;
    FieldView x, r, rh, p, v, s, t;
    const SolveState *st;
    Partials part;
    int skip;
};

template <class Q, int OP>
__global__ void __launch_bounds__(HOP_TS *HOP_MAX_PG) k_qblas(QBlasArgs a) {
    __shared__ Item it;
    load_item_q(a.L, it);
    QCoord q = qcoord(it, a.L);
    bool l0 = true, l1 = true;
    if (q.valid && a.skip) {
        pair_live(it, a.st, q.pair, 1, l0, l1);
        if (!l0 && !l1) q.valid = false;
    }
    float2 cre = f2(0.f, 0.f), cim = f2(0.f, 0.f), nn = f2(0.f, 0.f);
    if (q.valid) {
        const int64_t i = q.i;
        const PairScalars S = pair_scalars(it, a.st, q.pair);
        if (OP == OP_P_UPDATE) {  // p = r + beta (p - omega v)
            cp r[12], p[12], v[12];
            qload<Q>(a.r, i, r);
            qload<Q>(a.p, i, p);
            qload<Q>(a.v, i, v);
#pragma unroll
            for (int k = 0; k < 12; k++) {
                cp_sub_mul(p[k], S.wr, S.wi, v[k]);
                cp t = r[k];
                cp_add_mul(t, S.br, S.bi, p[k]);
                p[k] = t;
            }
            qstore<Q>(a.p, i, p);
        } else if (OP == OP_S_UPDATE) {  // s = r - alpha v
            cp r[12], v[12];
            qload<Q>(a.r, i, r);
            qload<Q>(a.v, i, v);
#pragma unroll
            for (int k = 0; k < 12; k++) cp_sub_mul(r[k], S.ar, S.ai, v[k]);
            qstore<Q>(a.s, i, r);
        } else if (OP == OP_XR_UPDATE) {
            // x += alpha p + omega s ; r = s - omega t ; (rh, r), (r, r).  Columns of the
            // pair that are not iterating keep x and r (their scalars are zero, but their
            // other fields may hold anything).
            cp x[12], p[12], s[12], t[12];
            qload<Q>(a.x, i, x);
            qload<Q>(a.p, i, p);
            qload<Q>(a.s, i, s);
            qload<Q>(a.t, i, t);
            const bool both = l0 && l1;
            cp x0[12], s0[12];
            if (!both) {
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    x0[k] = x[k];
                    s0[k] = s[k];
                }
            }
#pragma unroll
            for (int k = 0; k < 12; k++) {
                cp_add_mul(x[k], S.ar, S.ai, p[k]);
                cp_add_mul(x[k], S.wr, S.wi, s[k]);
                cp_sub_mul(s[k], S.wr, S.wi, t[k]);
            }
            if (!both) {
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    if (!l0) {
                        x[k].re.x = x0[k].re.x;
                        x[k].im.x = x0[k].im.x;
                        s[k].re.x = s0[k].re.x;
                        s[k].im.x = s0[k].im.x;
                    }
                    if (!l1) {
                        x[k].re.y = x0[k].re.y;
                        x[k].im.y = x0[k].im.y;
                        s[k].re.y = s0[k].re.y;
                        s[k].im.y = s0[k].im.y;
                    }
                }
            }
            qstore<Q>(a.x, i, x);
            qstore<Q>(a.r, i, s);
            cp rh[12];
            qload<Q>(a.rh, i, rh);
#pragma unroll
            for (int k = 0; k < 12; k++) {
                cre = pfma(rh[k].re, s[k].re, cre);
                cre = pfma(rh[k].im, s[k].im, cre);
                cim = pfma(rh[k].re, s[k].im, cim);
                cim = pfma(pneg(rh[k].im), s[k].re, cim);
                nn = pfma(s[k].re, s[k].re, nn);
                nn = pfma(s[k].im, s[k].im, nn);
            }
        } else if (OP == OP_INIT) {  // rh = r ; p = r ; x = 0
            cp r[12];
            qload<Q>(a.r, i, r);
            qstore<Q>(a.rh, i, r);
            qstore<Q>(a.p, i, r);
#pragma unroll
            for (int k = 0; k < 12; k++) r[k].re = r[k].im = f2(0.f, 0.f);
            qstore<Q>(a.x, i, r);
        }
    }
    if (OP == OP_XR_UPDATE) qpartials(it, q, cre, cim, nn, a.part, true, true);
}

// ------------------------------------------- FP64 per-column <-> pair fields

struct QConvArgs {
    Launch L;
    FieldView lo;   // pair field
    FieldView hi;   // FP64 per-column field
    const SolveState *st;
};

// lo = scale * hi per column (scale = 2 kappa / sigma: the normalised defect);
// a padding column is zero.
template <class Q>
__global__ void __launch_bounds__(HOP_TS *HOP_MAX_PG) k_to_pair(QConvArgs a) {
    __shared__ Item it;
    load_item_q(a.L, it);
    const QCoord q = qcoord(it, a.L);
    if (!q.valid) return;
    cp v[12];
    double sc[2] = {0.0, 0.0};
    int64_t base[2] = {0, 0};
#pragma unroll
    for (int l = 0; l < 2; l++) {
        const int col = 2 * q.pair + l;
        if (col < it.ncol) {
            sc[l] = a.st[it.solve0 + col].scale;
            base[l] = it.fbase + (int64_t)col * it.nh + q.h;
        }
    }
    const double2 *b = reinterpret_cast<const double2 *>(a.hi.p);
#pragma unroll
    for (int k = 0; k < 12; k++) {
        double2 c0 = make_double2(0.0, 0.0), c1 = make_double2(0.0, 0.0);
        if (sc[0] != 0.0) c0 = b[k * a.hi.stride + base[0]];
        if (sc[1] != 0.0) c1 = b[k * a.hi.stride + base[1]];
        v[k].re = f2((float)(sc[0] * c0.x), (float)(sc[1] * c1.x));
        v[k].im = f2((float)(sc[0] * c0.y), (float)(sc[1] * c1.y));
    }
    qstore<Q>(a.lo, q.i, v);
}

// hi += sigma * lo per column (FP64 accumulation of the correction)
template <class Q>
__global__ void __launch_bounds__(HOP_TS *HOP_MAX_PG) k_accum_pair(QConvArgs a) {
    __shared__ Item it;
    load_item_q(a.L, it);
    const QCoord q = qcoord(it, a.L);
    if (!q.valid) return;
    double sg[2] = {0.0, 0.0};
    int64_t base[2] = {0, 0};
#pragma unroll
    for (int l = 0; l < 2; l++) {
        const int col = 2 * q.pair + l;
        if (col < it.ncol) {
            sg[l] = a.st[it.solve0 + col].sigma;
            base[l] = it.fbase + (int64_t)col * it.nh + q.h;
        }
    }
    if (sg[0] == 0.0 && sg[1] == 0.0) return;
    cp v[12];
    qload<Q>(a.lo, q.i, v);
    double2 *b = reinterpret_cast<double2 *>(a.hi.p);
#pragma unroll
    for (int k = 0; k < 12; k++) {
        if (sg[0] != 0.0) {
            double2 &c = b[k * a.hi.stride + base[0]];
            c = make_double2(c.x + sg[0] * (double)v[k].re.x, c.y + sg[0] * (double)v[k].im.x);
        }
        if (sg[1] != 0.0) {
            double2 &c = b[k * a.hi.stride + base[1]];
            c = make_double2(c.x + sg[1] * (double)v[k].re.y, c.y + sg[1] * (double)v[k].im.y);
        }
    }
}

// User layout [ncol][n][4][3] complex128 <-> pair fields of one item (for
// applying the low-precision stencil alone).  Thread per (pair, local site).
template <class Q>
__global__ void k_pack_pair(PackArgs a, FieldView le, FieldView lo) {
    const int64_t n = 2 * (int64_t)a.it.nh;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n * a.it.npair) return;
    const int pair = (int)(g / n);
    const int l = (int)(g - (int64_t)pair * n);
    int k[4];
    local_coords(a.it, l, k);
    const int par = (a.it.par_o + k[0] + k[1] + k[2] + k[3]) & 1;
    const int64_t i = a.it.qbase + (int64_t)pair * a.it.nh + (l >> 1);
    const double2 *u0 = a.user + ((int64_t)(2 * pair) * n + l) * 12;
    const bool has1 = 2 * pair + 1 < a.it.ncol;
    const double2 *u1 = a.user + ((int64_t)(2 * pair + 1) * n + l) * 12;
    cp v[12];
#pragma unroll
    for (int c = 0; c < 12; c++) {
        const double2 x0 = u0[c];
        const double2 x1 = has1 ? u1[c] : make_double2(0.0, 0.0);
        v[c].re = f2((float)x0.x, (float)x1.x);
        v[c].im = f2((float)x0.y, (float)x1.y);
    }
    qstore<Q>(par ? lo : le, i, v);
}

template <class Q>
__global__ void k_unpack_pair(PackArgs a, FieldView le, FieldView lo) {
    const int64_t n = 2 * (int64_t)a.it.nh;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n * a.it.npair) return;
    const int pair = (int)(g / n);
    const int l = (int)(g - (int64_t)pair * n);
    int k[4];
    local_coords(a.it, l, k);
    const int par = (a.it.par_o + k[0] + k[1] + k[2] + k[3]) & 1;
    const int64_t i = a.it.qbase + (int64_t)pair * a.it.nh + (l >> 1);
    cp v[12];
    qload<Q>(par ? lo : le, i, v);
    double2 *u0 = a.uout + ((int64_t)(2 * pair) * n + l) * 12;
    const bool has1 = 2 * pair + 1 < a.it.ncol;
    double2 *u1 = a.uout + ((int64_t)(2 * pair + 1) * n + l) * 12;
#pragma unroll
    for (int c = 0; c < 12; c++) {
        u0[c] = make_double2((double)v[c].re.x, (double)v[c].im.x);
        if (has1) u1[c] = make_double2((double)v[c].re.y, (double)v[c].im.y);
    }
}

}  // namespace ddp
