// Device-side building blocks of libddp: complex arithmetic, storage formats of
// spinor and link fields, the batch work table and the Dirichlet-masked
// even-odd hopping term of the Wilson-Dirac operator (App. A, Sec. 2).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace ddp {

// ---------------------------------------------------------------- complex

template <typename T>
struct cx {
    T re, im;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T r, T i) {
    cx<T> c;
    c.re = r;
    c.im = i;
    return c;
}
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a) { return mk(-a.re, -a.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mk(s * a.re, s * a.im); }
// i * a and -i * a
template <typename T>
__device__ __forceinline__ cx<T> mul_i(cx<T> a) { return mk(-a.im, a.re); }
template <typename T>
__device__ __forceinline__ cx<T> mul_mi(cx<T> a) { return mk(a.im, -a.re); }
template <typename T>
__device__ __forceinline__ cx<T> conj(cx<T> a) { return mk(a.re, -a.im); }
// conj(a) * b
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
    return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}

// ------------------------------------------------------- storage formats
//
// A spinor field holds one parity of ncol columns of several domains.  Site
// component (spin s, colour a) is complex number 3 s + a, i.e. reals
// 2(3s+a), 2(3s+a)+1 of a 24-real site vector.  The field is chunk-major:
// chunk j of site-column i lives at base[j * stride + i], so that a warp
// reading 32 consecutive site-columns issues fully coalesced 16-byte loads.
//
//   FP64 : 12 chunks of double2  (one complex each)
//   FP32 :  6 chunks of float4   (two complex each)
//   FP16 :  3 chunks of 8 halves (uint4) + one float scale per site-column;
//           stored values are v / max|v| so the site's largest component is
//           exactly representable and small sites keep 11 significant bits.
//   BF16 :  3 chunks of 8 bfloat16 (uint4), no scale (FP32 exponent range).
//
// Links: FP64 keeps all 9 complex entries (9 double2 chunks per link); the
// low-precision copies keep rows 0 and 1 (6 complex) and rebuild row 2 as
// the conjugated cross product, exact for SU(3).
//   FP32 : 3 float4 chunks; FP16 / BF16 : 3 uint2 chunks (4 halves each).
// Link field layout [mu][chunk][V], sites in the global even-odd order
// parity * V/2 + (lex >> 1).

struct PF64 {
    using real = double;
    using chunk = double2;
    static constexpr int NCH = 12;
    static constexpr bool SCALED = false;
    static constexpr int LCH = 9;
    static constexpr bool IS64 = true;
};
struct PF32 {
    using real = float;
    using chunk = float4;
    static constexpr int NCH = 6;
    static constexpr bool SCALED = false;
    static constexpr int LCH = 3;
    static constexpr bool IS64 = false;
};
struct PF16 {
    using real = float;
    using chunk = uint4;
    static constexpr int NCH = 3;
    static constexpr bool SCALED = true;
    static constexpr int LCH = 3;
    static constexpr bool IS64 = false;
};
struct PBF16 {
    using real = float;
    using chunk = uint4;
    static constexpr int NCH = 3;
    static constexpr bool SCALED = false;
    static constexpr int LCH = 3;
    static constexpr bool IS64 = false;
};

struct FieldView {
    void *p;        // chunk array
    float *scale;   // per-site-column scale (FP16 only)
    int64_t stride; // chunks between consecutive chunk rows
};

__device__ __forceinline__ float2 h2f(unsigned int u) {
    __half2 h = *reinterpret_cast<__half2 *>(&u);
    return __half22float2(h);
}
__device__ __forceinline__ unsigned int f2h(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<unsigned int *>(&h);
}
__device__ __forceinline__ float2 b2f(unsigned int u) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&u);
    return __bfloat1622float2(h);
}
__device__ __forceinline__ unsigned int f2b(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<unsigned int *>(&h);
}

template <class P>
__device__ __forceinline__ void load_spinor(const FieldView &f, int64_t i, typename P::real v[24]);

template <>
__device__ __forceinline__ void load_spinor<PF64>(const FieldView &f, int64_t i, double v[24]) {
    const double2 *b = reinterpret_cast<const double2 *>(f.p);
#pragma unroll
    for (int j = 0; j < 12; j++) {
        double2 c = __ldg(b + j * f.stride + i);
        v[2 * j] = c.x;
        v[2 * j + 1] = c.y;
    }
}
template <>
__device__ __forceinline__ void load_spinor<PF32>(const FieldView &f, int64_t i, float v[24]) {
    const float4 *b = reinterpret_cast<const float4 *>(f.p);
#pragma unroll
    for (int j = 0; j < 6; j++) {
        float4 c = __ldg(b + j * f.stride + i);
        v[4 * j] = c.x;
        v[4 * j + 1] = c.y;
        v[4 * j + 2] = c.z;
        v[4 * j + 3] = c.w;
    }
}
template <>
__device__ __forceinline__ void load_spinor<PF16>(const FieldView &f, int64_t i, float v[24]) {
    const uint4 *b = reinterpret_cast<const uint4 *>(f.p);
    float s = __ldg(f.scale + i);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        uint4 c = __ldg(b + j * f.stride + i);
        float2 a0 = h2f(c.x), a1 = h2f(c.y), a2 = h2f(c.z), a3 = h2f(c.w);
        v[8 * j + 0] = s * a0.x;
        v[8 * j + 1] = s * a0.y;
        v[8 * j + 2] = s * a1.x;
        v[8 * j + 3] = s * a1.y;
        v[8 * j + 4] = s * a2.x;
        v[8 * j + 5] = s * a2.y;
        v[8 * j + 6] = s * a3.x;
        v[8 * j + 7] = s * a3.y;
    }
}
template <>
__device__ __forceinline__ void load_spinor<PBF16>(const FieldView &f, int64_t i, float v[24]) {
    const uint4 *b = reinterpret_cast<const uint4 *>(f.p);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        uint4 c = __ldg(b + j * f.stride + i);
        float2 a0 = b2f(c.x), a1 = b2f(c.y), a2 = b2f(c.z), a3 = b2f(c.w);
        v[8 * j + 0] = a0.x;
        v[8 * j + 1] = a0.y;
        v[8 * j + 2] = a1.x;
        v[8 * j + 3] = a1.y;
        v[8 * j + 4] = a2.x;
        v[8 * j + 5] = a2.y;
        v[8 * j + 6] = a3.x;
        v[8 * j + 7] = a3.y;
    }
}

// Spinor as stored: FP16 values without their site-column scale, which is
// returned in *s (1 for the other formats).
template <class P>
__device__ __forceinline__ void load_spinor_raw(const FieldView &f, int64_t i, typename P::real v[24],
                                                typename P::real *s) {
    load_spinor<P>(f, i, v);
    *s = typename P::real(1);
}
template <>
__device__ __forceinline__ void load_spinor_raw<PF16>(const FieldView &f, int64_t i, float v[24], float *s) {
    const uint4 *b = reinterpret_cast<const uint4 *>(f.p);
    *s = __ldg(f.scale + i);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        uint4 c = __ldg(b + j * f.stride + i);
        float2 a0 = h2f(c.x), a1 = h2f(c.y), a2 = h2f(c.z), a3 = h2f(c.w);
        v[8 * j + 0] = a0.x;
        v[8 * j + 1] = a0.y;
        v[8 * j + 2] = a1.x;
        v[8 * j + 3] = a1.y;
        v[8 * j + 4] = a2.x;
        v[8 * j + 5] = a2.y;
        v[8 * j + 6] = a3.x;
        v[8 * j + 7] = a3.y;
    }
}

template <class P>
__device__ __forceinline__ void store_spinor(const FieldView &f, int64_t i, const typename P::real v[24]);

template <>
__device__ __forceinline__ void store_spinor<PF64>(const FieldView &f, int64_t i, const double v[24]) {
    double2 *b = reinterpret_cast<double2 *>(f.p);
#pragma unroll
    for (int j = 0; j < 12; j++) b[j * f.stride + i] = make_double2(v[2 * j], v[2 * j + 1]);
}
template <>
__device__ __forceinline__ void store_spinor<PF32>(const FieldView &f, int64_t i, const float v[24]) {
    float4 *b = reinterpret_cast<float4 *>(f.p);
#pragma unroll
    for (int j = 0; j < 6; j++) b[j * f.stride + i] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
}
template <>
__device__ __forceinline__ void store_spinor<PF16>(const FieldView &f, int64_t i, const float v[24]) {
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < 24; j++) m = fmaxf(m, fabsf(v[j]));
    float inv = (m > 0.f) ? 1.0f / m : 0.f;
    f.scale[i] = m;
    uint4 *b = reinterpret_cast<uint4 *>(f.p);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        uint4 c;
        c.x = f2h(v[8 * j + 0] * inv, v[8 * j + 1] * inv);
        c.y = f2h(v[8 * j + 2] * inv, v[8 * j + 3] * inv);
        c.z = f2h(v[8 * j + 4] * inv, v[8 * j + 5] * inv);
        c.w = f2h(v[8 * j + 6] * inv, v[8 * j + 7] * inv);
        b[j * f.stride + i] = c;
    }
}
template <>
__device__ __forceinline__ void store_spinor<PBF16>(const FieldView &f, int64_t i, const float v[24]) {
    uint4 *b = reinterpret_cast<uint4 *>(f.p);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        uint4 c;
        c.x = f2b(v[8 * j + 0], v[8 * j + 1]);
        c.y = f2b(v[8 * j + 2], v[8 * j + 3]);
        c.z = f2b(v[8 * j + 4], v[8 * j + 5]);
        c.w = f2b(v[8 * j + 6], v[8 * j + 7]);
        b[j * f.stride + i] = c;
    }
}

// -------------------------------------------------------------- links

template <typename T>
__device__ __forceinline__ void reconstruct_row2(cx<T> u[3][3]) {
    // row2 = conj(row0 x row1), exact for SU(3)
    u[2][0] = conj(u[0][1] * u[1][2] - u[0][2] * u[1][1]);
    u[2][1] = conj(u[0][2] * u[1][0] - u[0][0] * u[1][2]);
    u[2][2] = conj(u[0][0] * u[1][1] - u[0][1] * u[1][0]);
}

template <class P>
__device__ __forceinline__ void load_link(const void *L, int64_t V, int mu, int64_t g, cx<typename P::real> u[3][3]);

template <>
__device__ __forceinline__ void load_link<PF64>(const void *L, int64_t V, int mu, int64_t g, cx<double> u[3][3]) {
    const double2 *b = reinterpret_cast<const double2 *>(L) + (int64_t)mu * 9 * V + g;
#pragma unroll
    for (int j = 0; j < 9; j++) {
        double2 c = __ldg(b + j * V);
        u[j / 3][j % 3] = mk(c.x, c.y);
    }
}
template <>
__device__ __forceinline__ void load_link<PF32>(const void *L, int64_t V, int mu, int64_t g, cx<float> u[3][3]) {
    const float4 *b = reinterpret_cast<const float4 *>(L) + (int64_t)mu * 3 * V + g;
    float4 c0 = __ldg(b), c1 = __ldg(b + V), c2 = __ldg(b + 2 * V);
    u[0][0] = mk(c0.x, c0.y);
    u[0][1] = mk(c0.z, c0.w);
    u[0][2] = mk(c1.x, c1.y);
    u[1][0] = mk(c1.z, c1.w);
    u[1][1] = mk(c2.x, c2.y);
    u[1][2] = mk(c2.z, c2.w);
    reconstruct_row2(u);
}
template <>
__device__ __forceinline__ void load_link<PF16>(const void *L, int64_t V, int mu, int64_t g, cx<float> u[3][3]) {
    const uint2 *b = reinterpret_cast<const uint2 *>(L) + (int64_t)mu * 3 * V + g;
    uint2 c0 = __ldg(b), c1 = __ldg(b + V), c2 = __ldg(b + 2 * V);
    float2 a;
    a = h2f(c0.x); u[0][0] = mk(a.x, a.y);
    a = h2f(c0.y); u[0][1] = mk(a.x, a.y);
    a = h2f(c1.x); u[0][2] = mk(a.x, a.y);
    a = h2f(c1.y); u[1][0] = mk(a.x, a.y);
    a = h2f(c2.x); u[1][1] = mk(a.x, a.y);
    a = h2f(c2.y); u[1][2] = mk(a.x, a.y);
    reconstruct_row2(u);
}
template <>
__device__ __forceinline__ void load_link<PBF16>(const void *L, int64_t V, int mu, int64_t g, cx<float> u[3][3]) {
    const uint2 *b = reinterpret_cast<const uint2 *>(L) + (int64_t)mu * 3 * V + g;
    uint2 c0 = __ldg(b), c1 = __ldg(b + V), c2 = __ldg(b + 2 * V);
    float2 a;
    a = b2f(c0.x); u[0][0] = mk(a.x, a.y);
    a = b2f(c0.y); u[0][1] = mk(a.x, a.y);
    a = b2f(c1.x); u[0][2] = mk(a.x, a.y);
    a = b2f(c1.y); u[1][0] = mk(a.x, a.y);
    a = b2f(c2.x); u[1][1] = mk(a.x, a.y);
    a = b2f(c2.y); u[1][2] = mk(a.x, a.y);
    reconstruct_row2(u);
}

// ------------------------------------------------------ batch work table
//
// One Item per (domain, request) of a launch.  All spinor fields of a launch
// are concatenations of the items' column segments: column c of item it
// occupies site-columns [fbase + c*nh, fbase + (c+1)*nh) of each parity field.
// Hop-style kernels use blocks of TS sites x CG columns; item it owns blocks
// [blk0, blk0 + ntiles*ncg).  Reduction partials of (column c, tile t) live at
// pbase + c*ntiles + t.

struct Item {
    int o[4];        // origin (global coordinates, reduced mod L)
    int e[4];        // extent
    int L[4];        // lattice
    int rmask;       // bit mu set: direction mu restricted (Dirichlet faces)
    int bc;          // time boundary: 0 periodic, 1 antiperiodic, 2 open
    int par_o;       // (o0+o1+o2+o3) & 1
    int nh;          // sites per parity = n/2
    int ntiles;      // ceil(nh / TS)
    int ncol;
    int ncg;         // ceil(ncol / CG)
    int blk0;
    int solve0;      // first solve (column) index
    int64_t fbase;
    int64_t pbase;
    double kappa;
    const void *links;    // links of the launch's storage precision
    const void *links64;  // FP64 links
    int64_t gV;           // lattice volume (link field row length)
    // clover term (clover.cuh), NULL without it: T and T^-1 in the launch's arithmetic
    // (FP64 packed for the FP64 path, FP32 packed otherwise) and T in FP64
    const void *clov;
    const void *clovinv;
    const void *clov64;
};

struct Launch {
    const Item *items;
    int nitems;
    int TS, CG;          // sites per tile (multiple of 32), columns per block
};

// Locate the item owning block b (items sorted by blk0).
__device__ __forceinline__ int find_item(const Item *items, int nitems, int b) {
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (items[mid].blk0 <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Domain-local coordinates of the even-odd index h of parity p (requires e3 even):
// the local lexicographic index l = ((k0 e1 + k1) e2 + k2) e3 + k3 satisfies h = l >> 1.
__device__ __forceinline__ void decode_site(const Item &it, int h, int p, int k[4]) {
    int hx = it.e[3] >> 1;
    int row = h / hx;
    int j = h - row * hx;
    k[2] = row % it.e[2];
    row /= it.e[2];
    k[1] = row % it.e[1];
    k[0] = row / it.e[1];
    k[3] = 2 * j + ((p + it.par_o + k[0] + k[1] + k[2]) & 1);
}

__device__ __forceinline__ int local_lex(const Item &it, const int k[4]) {
    return ((k[0] * it.e[1] + k[1]) * it.e[2] + k[2]) * it.e[3] + k[3];
}

__device__ __forceinline__ int64_t global_lex(const Item &it, const int x[4]) {
    return (((int64_t)x[0] * it.L[1] + x[1]) * it.L[2] + x[2]) * it.L[3] + x[3];
}

// Link-field row of global site x with parity p.
__device__ __forceinline__ int64_t link_row(const Item &it, const int x[4], int p) {
    return (p ? (it.gV >> 1) : 0) + (global_lex(it, x) >> 1);
}

// ------------------------------------------------------------ hopping
//
// acc(y) = sum_mu [ f+ (1 - g_mu) U_mu(y) psi(y+mu) + f- (1 + g_mu) U_mu(y-mu)^+ psi(y-mu) ]
// restricted to the item's box: f = 0 for hops leaving a restricted direction
// or crossing an open time boundary, -1 across an antiperiodic one.  The spin
// projectors (1 -/+ g_mu) have rank 2 in the chiral basis
// g_mu = [[0, A_mu], [A_mu^+, 0]]: (1 - g)psi = [h; -A^+ h] with h = psi_up - A psi_dn
// and (1 + g)psi = [h; A^+ h] with h = psi_up + A psi_dn, so only the two
// rows of h are multiplied by the link.

// w = u h.  FMA: one multiply-add chain per real component (6 instructions
// instead of 8); it saves issue slots where the kernel is issue-bound (16-bit
// storage) but holds more registers live, so the FP32-storage stencil keeps
// the plain form.
template <bool FMA, typename R>
__device__ __forceinline__ void su3_mul_half(const cx<R> u[3][3], const cx<R> h[2][3], cx<R> w[2][3]) {
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (FMA) {
                R re = u[a][0].re * h[s][0].re;
                R im = u[a][0].re * h[s][0].im;
                re = fma(-u[a][0].im, h[s][0].im, re);
                im = fma(u[a][0].im, h[s][0].re, im);
#pragma unroll
                for (int b = 1; b < 3; b++) {
                    re = fma(u[a][b].re, h[s][b].re, re);
                    im = fma(u[a][b].re, h[s][b].im, im);
                    re = fma(-u[a][b].im, h[s][b].im, re);
                    im = fma(u[a][b].im, h[s][b].re, im);
                }
                w[s][a] = mk(re, im);
            } else {
                w[s][a] = u[a][0] * h[s][0] + u[a][1] * h[s][1] + u[a][2] * h[s][2];
            }
        }
}
template <typename R>
__device__ __forceinline__ void su3_adj_mul_half(const cx<R> u[3][3], const cx<R> h[2][3], cx<R> w[2][3]) {
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int a = 0; a < 3; a++)
            w[s][a] = cmul(u[0][a], h[s][0]) + cmul(u[1][a], h[s][1]) + cmul(u[2][a], h[s][2]);
}

// Spin projection of direction MU, FWD = forward hop (1 - g_mu), else (1 + g_mu).
template <int MU, bool FWD, typename R>
__device__ __forceinline__ void project(const R v[24], cx<R> h[2][3]) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        cx<R> p0 = mk(v[2 * a], v[2 * a + 1]);
        cx<R> p1 = mk(v[6 + 2 * a], v[6 + 2 * a + 1]);
        cx<R> p2 = mk(v[12 + 2 * a], v[12 + 2 * a + 1]);
        cx<R> p3 = mk(v[18 + 2 * a], v[18 + 2 * a + 1]);
        if (MU == 0) {
            h[0][a] = FWD ? p0 - p2 : p0 + p2;
            h[1][a] = FWD ? p1 - p3 : p1 + p3;
        } else if (MU == 1) {
            h[0][a] = FWD ? p0 + mul_i(p3) : p0 - mul_i(p3);
            h[1][a] = FWD ? p1 + mul_i(p2) : p1 - mul_i(p2);
        } else if (MU == 2) {
            h[0][a] = FWD ? p0 + p3 : p0 - p3;
            h[1][a] = FWD ? p1 - p2 : p1 + p2;
        } else {
            h[0][a] = FWD ? p0 + mul_i(p2) : p0 - mul_i(p2);
            h[1][a] = FWD ? p1 - mul_i(p3) : p1 + mul_i(p3);
        }
    }
}

// acc += f * [w; lower(w)] for direction MU and hop sense FWD, each real
// component one multiply-add (f is 1 for unscaled storage, the site-column
// scale for FP16).
template <typename R>
__device__ __forceinline__ void cfma(cx<R> &acc, R f, cx<R> w) {
    acc.re = fma(f, w.re, acc.re);
    acc.im = fma(f, w.im, acc.im);
}
template <int MU, bool FWD, typename R>
__device__ __forceinline__ void accumulate(cx<R> acc[4][3], const cx<R> w[2][3], R f) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const cx<R> w0 = w[0][a], w1 = w[1][a];
        cfma(acc[0][a], f, w0);
        cfma(acc[1][a], f, w1);
        if (MU == 0) {
            cfma(acc[2][a], FWD ? -f : f, w0);
            cfma(acc[3][a], FWD ? -f : f, w1);
        } else if (MU == 1) {
            cfma(acc[2][a], f, FWD ? mul_mi(w1) : mul_i(w1));
            cfma(acc[3][a], f, FWD ? mul_mi(w0) : mul_i(w0));
        } else if (MU == 2) {
            cfma(acc[2][a], FWD ? -f : f, w1);
            cfma(acc[3][a], FWD ? f : -f, w0);
        } else {
            cfma(acc[2][a], f, FWD ? mul_mi(w0) : mul_i(w0));
            cfma(acc[3][a], f, FWD ? mul_i(w1) : mul_mi(w1));
        }
    }
}

// Geometry of one hop d = 2 mu + (backward ? 1 : 0) from even-odd site h of
// parity p: the neighbour's even-odd index (or -1 when the hop is dropped)
// and the link the neighbour is transported with, U_mu(x) forward and
// U_mu(x - mu)^+ backward, multiplied by the boundary factor of the hop
// (-1 across an antiperiodic time boundary).
template <class P>
__device__ __forceinline__ int stage_hop(const Item &it, int h, int p, int d, cx<typename P::real> u[3][3]) {
    using R = typename P::real;
    int k[4], x[4];
    decode_site(it, h, p, k);
#pragma unroll
    for (int m = 0; m < 4; m++) {
        int t = it.o[m] + k[m];
        x[m] = (t >= it.L[m]) ? t - it.L[m] : t;
    }
    const int mu = d >> 1;
    const bool fwd = !(d & 1);
    int kn[4] = {k[0], k[1], k[2], k[3]};
    bool ok = true;
    const bool restricted = (it.rmask >> mu) & 1;
    if (fwd) {
        kn[mu] += 1;
        if (restricted)
            ok = kn[mu] < it.e[mu];
        else if (kn[mu] == it.e[mu])
            kn[mu] = 0;
    } else {
        kn[mu] -= 1;
        if (restricted)
            ok = kn[mu] >= 0;
        else if (kn[mu] < 0)
            kn[mu] = it.e[mu] - 1;
    }
    R f = R(1);
    if (mu == 0 && x[0] == (fwd ? it.L[0] - 1 : 0)) {
        if (it.bc == 1) f = R(-1);
        if (it.bc == 2) ok = false;
    }
    if (!ok) return -1;
    const void *lk = P::IS64 ? it.links64 : it.links;
    if (fwd) {
        load_link<P>(lk, it.gV, mu, link_row(it, x, p), u);
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) u[i][j] = f * u[i][j];
    } else {
        int xm[4] = {x[0], x[1], x[2], x[3]};
        xm[mu] = (xm[mu] == 0) ? it.L[mu] - 1 : xm[mu] - 1;
        cx<R> v[3][3];
        load_link<P>(lk, it.gV, mu, link_row(it, xm, p ^ 1), v);
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) u[i][j] = f * conj(v[j][i]);
    }
    return local_lex(it, kn) >> 1;
}

// acc += f (1 -/+ g_mu) u psi for hop D (compile-time), link u already
// oriented; f is the FP16 site-column scale of psi, else 1.
template <int D, bool FMA, typename R>
__device__ __forceinline__ void hop_step(const R v[24], const cx<R> u[3][3], cx<R> acc[4][3], R f) {
    constexpr int MU = D >> 1;
    constexpr bool FWD = !(D & 1);
    cx<R> h[2][3], w[2][3];
    project<MU, FWD>(v, h);
    su3_mul_half<FMA>(u, h, w);
    accumulate<MU, FWD>(acc, w, f);
}

// --------------------------------------------------------- reductions

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace ddp
