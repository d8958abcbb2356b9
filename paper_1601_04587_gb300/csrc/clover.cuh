// The O(a)-improvement (clover) term of the Wilson-Dirac operator on the
// device.  With 2 kappa D = T - kappa D_hop, T(x) = 1 + 2 kappa C(x) and
//   C(x) = c_sw (i/4) sum_{mu,nu} sigma_{mu nu} F_{mu nu}(x)
// (clover-leaf field strength F = (Q_{mu nu} - Q_{nu mu}) / 8; the paper refers
// to this improved operator in the footnotes of Sec. 4 and Sec. 5).
//
// In the chiral basis sigma_{mu nu} commutes with gamma_5, so T is block
// diagonal: spins {0, 1} and spins {2, 3}, each a Hermitian 6x6 matrix over
// (spin mod 2, colour), index 3 (s mod 2) + a.  A block is stored packed:
// 6 real diagonal entries, then the 15 entries above the diagonal row by row
// (complex) - 36 reals; a site holds block 0 then block 1 (72 reals).  Fields
// are chunk-major over the global even-odd site order of the links:
// FP64 36 double2 chunks, FP32 18 float4 chunks per site.
#pragma once

#include "ddp_device.cuh"

namespace ddp {

constexpr int CLOV_REALS = 72;  // per site

// Index of the packed upper-triangle entry (i < j) of a 6x6 block.
__host__ __device__ constexpr int herm_off(int i, int j) {
    // rows 0..i-1 hold 5, 4, ... entries
    return 6 + 2 * (i * 5 - i * (i - 1) / 2 + (j - i - 1));
}

// y = A x for a packed Hermitian 6x6 block A (reals a[36]).
template <typename R>
__device__ __forceinline__ void herm6_mul(const R *a, const cx<R> x[6], cx<R> y[6]) {
#pragma unroll
    for (int i = 0; i < 6; i++) y[i] = mk(a[i] * x[i].re, a[i] * x[i].im);
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
        for (int j = i + 1; j < 6; j++) {
            const int o = herm_off(i, j);
            const cx<R> h = mk(a[o], a[o + 1]);
            y[i] = y[i] + h * x[j];
            y[j] = y[j] + cmul(h, x[i]);  // conj(h) x_i
        }
}

// Load the 72 reals of a site (FP64 or FP32 clover field, chunk-major).
template <typename R>
__device__ __forceinline__ void load_clover(const void *f, int64_t V, int64_t row, R a[CLOV_REALS]);
template <>
__device__ __forceinline__ void load_clover<double>(const void *f, int64_t V, int64_t row, double a[CLOV_REALS]) {
    const double2 *b = reinterpret_cast<const double2 *>(f);
#pragma unroll
    for (int j = 0; j < 36; j++) {
        const double2 c = __ldg(b + j * V + row);
        a[2 * j] = c.x;
        a[2 * j + 1] = c.y;
    }
}
template <>
__device__ __forceinline__ void load_clover<float>(const void *f, int64_t V, int64_t row, float a[CLOV_REALS]) {
    const float4 *b = reinterpret_cast<const float4 *>(f);
#pragma unroll
    for (int j = 0; j < 18; j++) {
        const float4 c = __ldg(b + j * V + row);
        a[4 * j] = c.x;
        a[4 * j + 1] = c.y;
        a[4 * j + 2] = c.z;
        a[4 * j + 3] = c.w;
    }
}

// v <- T v (or T^-1 v) at one site: spinor v[24] reals, component 3 s + a.
template <typename R>
__device__ __forceinline__ void clover_apply(const void *f, int64_t V, int64_t row, R v[24]) {
    R a[CLOV_REALS];
    load_clover<R>(f, V, row, a);
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        cx<R> x[6], y[6];
#pragma unroll
        for (int i = 0; i < 6; i++) x[i] = mk(v[2 * (6 * blk + i)], v[2 * (6 * blk + i) + 1]);
        herm6_mul(a + 36 * blk, x, y);
#pragma unroll
        for (int i = 0; i < 6; i++) {
            v[2 * (6 * blk + i)] = y[i].re;
            v[2 * (6 * blk + i) + 1] = y[i].im;
        }
    }
}

// Link-field row of the output site h (parity p) of an item.
__device__ __forceinline__ int64_t site_row(const Item &it, int h, int p) {
    int k[4], x[4];
    decode_site(it, h, p, k);
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const int t = it.o[m] + k[m];
        x[m] = (t >= it.L[m]) ? t - it.L[m] : t;
    }
    return link_row(it, x, p);
}

}  // namespace ddp
