// The two contraction-shaped steps of the projector-cut factorization (Sec. 5) on the
// tensor cores with FP64-level accuracy: the time-slice sums of the colourless spinors
// (Eq. W0tbary) and the Gram blocks conj(A_i) . A_j (the pion blocks of Eq. Bpions and
// the Cholesky QR of the inverse iteration), both as one emulated-FP64 product kernel.
//
// Colourless spinors.  Per time slice the sum is a complex matrix product
//   X[(i,j)][(k,alpha)] = sum_{(x,c)} E[(i,j)][(x,c)] s_k(x)_{alpha c},
//   E[(i,j)][(x,c)] = sum_{ab} eps_abc (s_i^a)^T C g5 s_j^b          (the diquark, FP64).
// C g5 is antisymmetric, so E is symmetric in (i, j): only the m(m+1)/2 rows i <= j
// are formed and X[j][i] = X[i][j].  The complex product is one real product
// C' = A' B'^T with A' = [Re E | Im E] and the rows of B' = [Re s | -Im s] (real-part
// columns) and [Im s | Re s] (imaginary-part columns).
//
// Every row of A' and every column of B' is split into S integer slices of 7 bits
// under a shared power-of-two exponent (the splitting of Ozaki, Ogita, Oishi and Rump,
// 2012): with |a| < 2^e over the row (column), N = round(a 2^(49-e)) is written in
// balanced base 128, a = 2^(e-7) sum_p q_p 2^(-7p) + O(2^(e-50)), q_0 in [-128, 128],
// q_p in [-64, 63] for p > 0, each exact in BF16.  For every d < S the products of slices
// p + q = d are summed on the tensor cores (tcgen05.mma kind::f16, BF16 operands,
// FP32 accumulators in tensor memory, one per d).  Over KC = 448 reduction terms
// every such sum is an integer of magnitude below 9 * 2^12 * 448 < 2^24, hence
// exact in FP32; after each chunk the seven sums are converted to integers and
// added exactly into two 64-bit fixed-point accumulators per output.  Products of
// slices with p + q >= S are dropped: each term of the sum is exact to about
// 2^-47 of its row maximum times its column maximum.
//
// Operands reach the tensor cores through a four-stage pipeline of bulk copies
// (cp.async.bulk, completion on an mbarrier): the split kernels write every
// (slice, 128- or 64-row tile, 16-deep K step) block contiguously in the
// shared-memory layout the MMA descriptor describes (K-major, no swizzle: 8-row x
// 16-byte core matrices, 128 bytes apart along K, 256 bytes apart between 8-row
// groups), so that one copy per block stages it.
#include <cmath>
#include <cstring>

#include "ddp_host.h"

using namespace ddp;

namespace {

constexpr int S = 7;          // slices per operand; accumulator groups d = p + q < S
constexpr int TM = 128;       // rows of A' per tile (the MMA's M)
constexpr int TN = 64;        // rows of B' (output columns) per tile (the MMA's N)
constexpr int KSTEP = 16;     // reduction depth per pipeline stage (one MMA of K = 16 per slice pair)
constexpr int CS = 28;        // stages per exact chunk: KC = 448
constexpr int SBO = 16 * KSTEP, LBO = 128;  // bytes between 8-row groups; between K core matrices
constexpr int TILE_A = TM * KSTEP * 2, TILE_B = TN * KSTEP * 2;  // bytes
constexpr int STAGE = S * (TILE_A + TILE_B);
constexpr int NSTAGE = 4;   // operand buffers in flight
constexpr int GEMM_THREADS = 512;   // thread 0 streams the operands and issues the MMAs; all drain
constexpr int GEMM_BLOCK = GEMM_THREADS;
constexpr int DCOLS = TN / (GEMM_THREADS / 128);  // accumulator columns a thread drains
constexpr int TMEM_COLS = 512;  // S * TN = 448 used
constexpr int MAX_STEPS_PER_BLOCK = 1 << 16;  // keeps the fixed-point sums far below 2^63
constexpr int MMAX = TC_MMAX; // largest number of columns (the paper's 120 modes fit)
// sites per block of the diquark kernel: all m spinors of the block's sites are staged in
// shared memory, m * ES * 192 bytes (16 sites up to 32 columns, 4 beyond, plus 64 bytes
// of padding per column)
constexpr int ES_SMALL = 16, ES_LARGE = 4, ES_SMALL_MMAX = 32;
// float4 elements between the staged spinors of consecutive columns k
__host__ __device__ constexpr int colour_kstride(int es) { return 12 * es + (es == 4 ? 4 : 0); }
constexpr unsigned long long WAIT_NS = 2000000000ull;  // a wait gives up after 2 s

static_assert(S * TN <= TMEM_COLS, "accumulators exceed the tensor memory");
static_assert(4 * TN <= 256, "one MMA spans at most four B slices (N <= 256)");
static_assert(DCOLS == 16, "the drain loads 16 columns per thread");
static_assert(CS * KSTEP * 9 * 4096 < (1 << 24), "chunk sums must stay exact in FP32");

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t mma_desc(uint32_t saddr) {
    return ((uint64_t)(saddr >> 4) & 0x3FFF) | ((uint64_t)((LBO >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((SBO >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M = TM.
__host__ __device__ constexpr uint32_t idesc_n(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the completion of the mbarrier phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 0;; it++) {
        uint32_t ok;
        asm volatile("{\n .reg .pred pw;\n mbarrier.try_wait.parity.shared::cta.b64 pw, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, pw;\n}\n"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (ok) return true;
        if ((it & 255u) == 255u && globaltimer() - t0 > WAIT_NS) return false;
    }
}

__device__ __forceinline__ void atomic_max_pos(double *a, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long *>(a), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ int exponent_of(double mx) {
    if (!(mx > 0)) return 0;
    int e;
    frexp(mx, &e);  // mx < 2^e
    return e;
}

// The shared exponent of every row or column: e with max < 2^e, or NONFINITE for a
// row or column that holds a NaN or an infinity (its slices are zero and its outputs NaN).
constexpr int NONFINITE = -100000;
__global__ void k_exponents(const double *mx, int n, int *ex) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) ex[i] = isfinite(mx[i]) ? exponent_of(mx[i]) : NONFINITE;
}

// (i, j), i <= j, of the symmetric row r (rows ordered i-major).
__device__ __forceinline__ void pair_of(int r, int m, int &i, int &j) {
    i = 0;
    while (r >= m - i) {
        r -= m - i;
        i++;
    }
    j = i + r;
}

// spinor component of the source field in the requested form: 0 s = A,
// 1 s = g5 conj(A), 2 s = -A (g5 = diag(-1, -1, 1, 1) in the chiral basis)
__device__ __forceinline__ double2 form_of(double2 v, int form, int spin) {
    if (form == 1) {
        v.y = -v.y;
        if (spin < 2) v = make_double2(-v.x, -v.y);
    } else if (form == 2) {
        v = make_double2(-v.x, -v.y);
    }
    return v;
}

// ------------------------------------------------------------- pre-passes
//
// GB300 runs FP64 arithmetic at a small fraction of its FP32 rate, so the pre-passes
// avoid it: the diquarks are formed in double-FP32 arithmetic (each value an unevaluated
// sum hi + lo of two floats, 48 significant bits; Dekker's product with fused
// multiply-adds and Knuth's two-sum), and the 7-bit slices are cut from the integer
// round(v 2^(49-e)) obtained from the bit pattern of v by shifts.

// Magnitude used for the shared exponents: +inf for a non-finite value, so that a NaN or
// an infinity in the input turns the affected outputs into NaN (see k_ozaki_finish).
__device__ __forceinline__ double mag(double v) { return isfinite(v) ? fabs(v) : (double)INFINITY; }

__device__ __forceinline__ float magf(float v) { return isfinite(v) ? fabsf(v) : INFINITY; }

// 2^k as a float, -126 <= k <= 127.
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

// hi + lo = v 2^-f to 48 significant bits, from the bits of v by integer operations
// (|v| < 2^f; parts below 2^-100 of 2^f, irrelevant at the 2^-49 precision of the
// slices, are dropped; a non-finite v gives NaN).
__device__ __forceinline__ float2 df_scaled(double v, int f) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ev = (int)((b >> 52) & 0x7FF);
    if (ev == 0x7FF) return make_float2(NAN, NAN);
    const int e = ev - 1023 - f;  // v 2^-f = 1.m 2^e
    if (ev == 0 || e < -100) return make_float2(0.f, 0.f);
    const unsigned long long m = (b & ((1ull << 52) - 1)) | (1ull << 52);
    const unsigned long long mh = (m + (1ull << 28)) >> 29;  // the significand rounded to 24 bits
    const long long rem = (long long)m - (long long)(mh << 29);  // |rem| <= 2^28
    const float sc = pow2f(e - 23);
    float hi = __uint2float_rn((unsigned)mh) * sc;                    // exact
    float lo = (__ll2float_rn(rem) * 3.7252902984619140625e-9f) * sc;  // rem 2^-28 2^(e-23) ... 2^-1
    lo *= 0.5f;                                                          // rem 2^(e-52)
    if (b >> 63) {
        hi = -hi;
        lo = -lo;
    }
    return make_float2(hi, lo);
}

// (S, E) += sg * a * b for double-float a, b; (S, E) is an unnormalized sum.
__device__ __forceinline__ void df_mac(float &S, float &E, float2 a, float2 b, float sg) {
    const float ah = sg * a.x, al = sg * a.y;
    const float p = __fmul_rn(ah, b.x);
    float e = __fmaf_rn(ah, b.x, -p);
    e = __fmaf_rn(ah, b.y, e);
    e = __fmaf_rn(al, b.x, e);
    const float s = __fadd_rn(S, p);
    const float bb = __fsub_rn(s, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    E = __fadd_rn(E, __fadd_rn(err, e));
    S = s;
}

__device__ __forceinline__ float2 df_norm(float S, float E) {
    const float h = __fadd_rn(S, E);
    return make_float2(h, __fsub_rn(E, __fsub_rn(h, S)));
}

// (S_re, E_re, S_im, E_im) += sg * a * b for double-float complex a, b (float4: re h, re l,
// im h, im l).
__device__ __forceinline__ void dfc_mac(float acc[4], float4 a, float4 b, float sg) {
    const float2 ar = make_float2(a.x, a.y), ai = make_float2(a.z, a.w);
    const float2 br = make_float2(b.x, b.y), bi = make_float2(b.z, b.w);
    df_mac(acc[0], acc[1], ar, br, sg);
    df_mac(acc[0], acc[1], ai, bi, -sg);
    df_mac(acc[2], acc[3], ar, bi, sg);
    df_mac(acc[2], acc[3], ai, br, sg);
}

// Column maxima of the spinors over one time slice: colmax[q], q = (k, alpha), the
// largest |Re|, |Im| of s_k(x)_{alpha c} over x and c.
__global__ void __launch_bounds__(256) k_colour_max(const double2 *A, int64_t n, int64_t site0, int64_t slice_n,
                                                    int m, double *colmax) {
    __shared__ double bm[4 * MMAX];
    const int Q = 4 * m, per = blockDim.x / Q;
    for (int q = threadIdx.x; q < Q; q += blockDim.x) bm[q] = 0;
    __syncthreads();
    if (per == 0) {
        // more columns than threads: each thread takes columns q, q + blockDim.x, ...
        // over the block's share of the sites
        for (int q = threadIdx.x; q < Q; q += blockDim.x) {
            const int k = q / 4, al = q % 4;
            double mx = 0;
            for (int64_t x = blockIdx.x; x < slice_n; x += gridDim.x)
                for (int c = 0; c < 3; c++) {
                    const double2 v = A[((int64_t)k * n + site0 + x) * 12 + 3 * al + c];
                    mx = fmax(mx, fmax(mag(v.x), mag(v.y)));
                }
            bm[q] = mx;
        }
    } else if ((int)threadIdx.x < per * Q) {
        const int q = threadIdx.x % Q, k = q / 4, al = q % 4;
        double mx = 0;
        for (int64_t x = blockIdx.x * (int64_t)per + threadIdx.x / Q; x < slice_n; x += (int64_t)gridDim.x * per)
            for (int c = 0; c < 3; c++) {
                const double2 v = A[((int64_t)k * n + site0 + x) * 12 + 3 * al + c];
                mx = fmax(mx, fmax(mag(v.x), mag(v.y)));
            }
        if (mx > 0) atomic_max_pos(bm + q, mx);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < Q; q += blockDim.x)
        if (bm[q] > 0) atomic_max_pos(colmax + q, bm[q]);
}

// f_k: |s_k(x)| < 2^f_k over the slice (the exponent of the spinor column k).
__device__ __forceinline__ int column_exponent(const double *colmax, int k) {
    return exponent_of(fmax(fmax(colmax[4 * k], colmax[4 * k + 1]), fmax(colmax[4 * k + 2], colmax[4 * k + 3])));
}

struct EArgs {
    const double2 *A;   // [m][n][12]
    int64_t n, site0, slice_n;
    int m, form, rows;  // rows = m (m + 1) / 2
    float4 *E;          // [rows][3 slice_n]: Re hi, Re lo, Im hi, Im lo of E 2^-(f_i + f_j)
    double *rowmax;     // [rows]   max |Re|, |Im| (hi parts) of the row of E 2^-(f_i + f_j)
    const double *colmax;
};

// The diquarks E^c_ij(x) = i sum over the spin pairs of Eq. W0tbary for i <= j, formed
// from the spinors scaled by 2^-f_k (so that double-FP32 arithmetic keeps its range),
// with the row maxima.  Block: ESITES sites, all rows; ESITES consecutive threads share a row.
template <int ESITES>
__global__ void __launch_bounds__(256) k_colour_E(EArgs a) {
    static_assert(ESITES >= 1 && ESITES <= 32 && (ESITES & (ESITES - 1)) == 0, "row groups within a warp");
    // [m][12][ESITES] with the site index fastest; with 4 sites the spinors of consecutive
    // k start 16 banks apart, so that the two rows a quarter-warp reads do not collide
    constexpr int KSTR = colour_kstride(ESITES);
    extern __shared__ float4 sh[];
    __shared__ int fexp[MMAX];
    const int m = a.m;
    const int64_t x0 = (int64_t)blockIdx.x * ESITES;
    const int ns = (int)min((int64_t)ESITES, a.slice_n - x0);
    for (int k = threadIdx.x; k < m; k += blockDim.x) fexp[k] = column_exponent(a.colmax, k);
    __syncthreads();
    for (int e = threadIdx.x; e < m * ns * 12; e += blockDim.x) {
        const int c = e % 12, xs = (e / 12) % ns, k = e / (12 * ns);
        const double2 v = a.A[((int64_t)k * a.n + a.site0 + x0 + xs) * 12 + c];
        float2 re = df_scaled(v.x, fexp[k]), im = df_scaled(v.y, fexp[k]);
        // the form, exactly on the parts: 1 conj then g5 (spins 0, 1 negated), 2 negation
        if (a.form == 1) im = make_float2(-im.x, -im.y);
        if ((a.form == 1 && c < 6) || a.form == 2) {
            re = make_float2(-re.x, -re.y);
            im = make_float2(-im.x, -im.y);
        }
        sh[k * KSTR + c * ESITES + xs] = make_float4(re.x, re.y, im.x, im.y);
    }
    __syncthreads();
    const int nit = a.rows * ESITES;
    for (int it0 = 0; it0 < nit; it0 += blockDim.x) {
        const int it = it0 + threadIdx.x;
        const int r = it / ESITES, xs = it % ESITES;
        float mx = 0.f;
        if (r < a.rows && xs < ns) {
            int i, j;
            pair_of(r, m, i, j);
            const float4 *si = sh + i * KSTR + xs, *sj = sh + j * KSTR + xs;
            float4 *o = a.E + (int64_t)r * 3 * a.slice_n + (x0 + xs) * 3;
            for (int c = 0; c < 3; c++) {
                const int ca = (c + 1) % 3, cb = (c + 2) % 3;
                // f(a, b) = s_i(1,a) s_j(0,b) - s_i(0,a) s_j(1,b) + s_i(3,a) s_j(2,b) - s_i(2,a) s_j(3,b);
                // E^c = i [f(ca, cb) - f(cb, ca)]
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
                for (int t = 0; t < 2; t++) {
                    const float sg = t ? -1.f : 1.f;
                    const int p = t ? cb : ca, q = t ? ca : cb;
                    dfc_mac(acc, si[(3 + p) * ESITES], sj[q * ESITES], sg);
                    dfc_mac(acc, si[p * ESITES], sj[(3 + q) * ESITES], -sg);
                    dfc_mac(acc, si[(9 + p) * ESITES], sj[(6 + q) * ESITES], sg);
                    dfc_mac(acc, si[(6 + p) * ESITES], sj[(9 + q) * ESITES], -sg);
                }
                const float2 R = df_norm(acc[0], acc[1]), I = df_norm(acc[2], acc[3]);
                o[c] = make_float4(-I.x, -I.y, R.x, R.y);  // times i
                mx = fmaxf(mx, fmaxf(magf(R.x), magf(I.x)));
            }
        }
        for (int off = ESITES / 2; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        if ((threadIdx.x & (ESITES - 1)) == 0 && r < a.rows && mx > 0.f) atomic_max_pos(a.rowmax + r, (double)mx);
    }
}

// round(mant 2^(ee + k)), |result| < 2^62 by the caller's choice of k (half away from zero).
__device__ __forceinline__ long long fixed_round(unsigned long long mant, int sh, bool neg) {
    unsigned long long n;
    if (sh >= 0)
        n = mant << sh;
    else if (sh > -64)
        n = (mant + (1ull << (-sh - 1))) >> (-sh);
    else
        n = 0;
    return neg ? -(long long)n : (long long)n;
}

// round(v 2^k) from the bits of a finite double (subnormals included).
__device__ __forceinline__ long long fixed_of(double v, int k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ev = (int)((b >> 52) & 0x7FF);
    const unsigned long long mant = (b & ((1ull << 52) - 1)) | (ev ? 1ull << 52 : 0ull);
    return fixed_round(mant, (ev ? ev : 1) - 1075 + k, b >> 63);
}

// round(f 2^k) from the bits of a finite float.
__device__ __forceinline__ long long fixed_of(float f, int k) {
    const unsigned b = __float_as_uint(f);
    const int ev = (int)((b >> 23) & 0xFF);
    const unsigned long long mant = (b & 0x7FFFFFu) | (ev ? 0x800000u : 0u);
    return fixed_round(mant, (ev ? ev : 1) - 150 + k, b >> 31);
}

// The S balanced base-128 digits of N (|N| <= 2^49 + 1): N = sum_p q_p 128^(S-1-p),
// q_p in [-64, 63] for p > 0 and |q_0| <= 128; each exact in BF16.
__device__ __forceinline__ void digits7(long long N, __nv_bfloat16 out[S]) {
#pragma unroll
    for (int p = S - 1; p > 0; p--) {
        int d = (int)(N & 127);
        if (d >= 64) d -= 128;
        N = (N - d) >> 7;  // exact: N - d is a multiple of 128
        out[p] = __int2bfloat16_rn(d);
    }
    out[0] = __int2bfloat16_rn((int)N);
}

// (row rl, depth kl) of element e of one tile block in the MMA's shared-memory layout.
__device__ __forceinline__ void tile_pos(int e, int &rl, int &kl) {
    constexpr int KC8 = KSTEP / 8;  // core matrices along K
    rl = ((e >> 3) & 7) + 8 * (e / (64 * KC8));
    kl = (e & 7) + 8 * ((e >> 6) % KC8);
}

struct SplitArgs {
    const float4 *E;
    const double2 *A;
    int64_t n, site0, K;  // K = 3 slice_n
    int m, form, rows;
    int MT, NT, KSh;      // tiles; K steps of one half (Re / Im) of the reduction
    const int *rexp, *cexp;  // exponents of the rows of A' and of the spinor columns (k, alpha)
    __nv_bfloat16 *Aq, *Bq;  // [MT][2 KSh][S][128 x KSTEP], [NT][2 KSh][S][64 x KSTEP]
};

// A' = [Re E | Im E]: thread per (row, kx), writes the slices of both halves.  With
// |v| < 2^e for the row, v = 2^(e-49) round(v 2^(49-e)) to within half a unit.
__global__ void k_split_A(SplitArgs a) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)a.MT * a.KSh * (TM * KSTEP);
    if (g >= total) return;
    const int e = (int)(g % (TM * KSTEP));
    const int64_t t = g / (TM * KSTEP);
    const int ksr = (int)(t % a.KSh), mt = (int)(t / a.KSh);
    int rl, kl;
    tile_pos(e, rl, kl);
    const int r = mt * TM + rl;
    const int64_t kx = (int64_t)ksr * KSTEP + kl;
    __nv_bfloat16 re[S], im[S];
    const int er = r < a.rows ? a.rexp[r] : NONFINITE;
    if (kx < a.K && er != NONFINITE) {
        const float4 v = a.E[(int64_t)r * a.K + kx];
        const int k = 49 - er;
        digits7(fixed_of(v.x, k) + fixed_of(v.y, k), re);
        digits7(fixed_of(v.z, k) + fixed_of(v.w, k), im);
    } else {
        for (int p = 0; p < S; p++) re[p] = im[p] = __double2bfloat16(0.0);
    }
    // tile block (mt, K step, slice): the S slices of one step lie contiguously
    const int KS = 2 * a.KSh;
    const int64_t bre = ((int64_t)mt * KS + ksr) * S, bim = ((int64_t)mt * KS + a.KSh + ksr) * S;
    for (int p = 0; p < S; p++) {
        a.Aq[(bre + p) * (TM * KSTEP) + e] = re[p];
        a.Aq[(bim + p) * (TM * KSTEP) + e] = im[p];
    }
}

// B' rows: col < 4m: [Re s | -Im s]; 4m <= col < 8m: [Im s | Re s]; beyond: zero.
__global__ void k_split_B(SplitArgs a) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)a.NT * a.KSh * (TN * KSTEP);
    if (g >= total) return;
    const int e = (int)(g % (TN * KSTEP));
    const int64_t t = g / (TN * KSTEP);
    const int ksr = (int)(t % a.KSh), nt = (int)(t / a.KSh);
    int rl, kl;
    tile_pos(e, rl, kl);
    const int col = nt * TN + rl;
    const int64_t kx = (int64_t)ksr * KSTEP + kl;
    const int Q = 4 * a.m;
    const int q = col < Q ? col : col - Q;
    __nv_bfloat16 lo[S], hi[S];
    const int eq = col < 2 * Q ? a.cexp[q] : NONFINITE;
    if (kx < a.K && eq != NONFINITE) {
        const int k = q / 4, al = q % 4;
        const int64_t x = kx / 3;
        const int c = (int)(kx % 3);
        const double2 v = form_of(a.A[((int64_t)k * a.n + a.site0 + x) * 12 + 3 * al + c], a.form, al);
        const int sc = 49 - eq;
        digits7(fixed_of(col < Q ? v.x : v.y, sc), lo);
        digits7(fixed_of(col < Q ? -v.y : v.x, sc), hi);
    } else {
        for (int p = 0; p < S; p++) lo[p] = hi[p] = __double2bfloat16(0.0);
    }
    const int KS = 2 * a.KSh;
    const int64_t blo = ((int64_t)nt * KS + ksr) * S, bhi = ((int64_t)nt * KS + a.KSh + ksr) * S;
    for (int p = 0; p < S; p++) {
        a.Bq[(blo + p) * (TN * KSTEP) + e] = lo[p];
        a.Bq[(bhi + p) * (TN * KSTEP) + e] = hi[p];
    }
}

// -------------------------------------------------------------- the product

struct GemmArgs {
    const uint8_t *Aq, *Bq;
    int a_bytes;      // bytes of one A slice block per K step: TILE_A, or fewer rows (see gram_tc)
    int MT, NT, KS, ksplit;
    int ncols;        // NT * TN
    double *part;     // [ksplit][MT * TM][ncols]: sum_d 2^-7d G_d of this block's K range
    int *err;         // set when a wait gave up
};

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Barrier 1 over the GEMM_THREADS threads; returns the OR of v over them.
__device__ __forceinline__ bool drain_barrier_or(bool v) {
    uint32_t r;
    asm volatile("{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n"
                 " barrier.cta.red.or.pred po, 1, %2, pi;\n selp.u32 %0, 1, 0, po;\n}\n"
                 : "=r"(r)
                 : "r"((uint32_t)v), "n"(GEMM_THREADS)
                 : "memory");
    return r != 0;
}

// One CTA per (64-column tile, 128-row tile, K range): the column tiles of one row tile
// are neighbours in the launch order, so that the CTAs streaming the same A blocks run at
// the same time and share them through L2.  Thread 0 streams the operand
// blocks of each K step into NSTAGE buffers (two bulk copies per step) and issues the
// MMAs; after every CS steps the sixteen warps drain the seven accumulators (warp w: lanes 32 (w % 4) .. + 31, columns DCOLS (w / 4) .. + DCOLS - 1)
// into exact 64-bit fixed point.
__global__ void __launch_bounds__(GEMM_BLOCK, 1) k_ozaki_gemm(GemmArgs a) {
    extern __shared__ __align__(128) uint8_t dsm[];
    __shared__ __align__(8) uint64_t full[NSTAGE], empty[NSTAGE];
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nt = blockIdx.x, mt = blockIdx.y, z = blockIdx.z;
    const int s0 = (int)((int64_t)a.KS * z / a.ksplit), s1 = (int)((int64_t)a.KS * (z + 1) / a.ksplit);
    const int nsteps = s1 - s0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)),
                     "n"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < NSTAGE; s++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tbase;

    auto load = [&](int q) {  // thread 0: K step s0 + q into buffer q % NSTAGE (two bulk copies)
        const int st = q % NSTAGE;
        const uint32_t sa = smem_u32(dsm + st * STAGE), fb = smem_u32(&full[st]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                     "r"((uint32_t)(S * (a.a_bytes + TILE_B)))
                     : "memory");
        bulk_copy(sa, a.Aq + (((int64_t)mt * a.KS + s0 + q) * S) * a.a_bytes, S * a.a_bytes, fb);
        bulk_copy(sa + S * a.a_bytes, a.Bq + (((int64_t)nt * a.KS + s0 + q) * S) * TILE_B, S * TILE_B, fb);
    };
    {
        // ---- MMA issue (thread 0) and accumulator drain (GEMM_THREADS threads)
        // 2^14 sum_{d<=2} 2^-7d G_d and 2^42 sum_{d>=3} 2^-7d G_d in two's complement (unsigned
        // arithmetic: exact for every accumulator row that holds a result, and defined
        // modulo 2^64 for the padding rows, whose values are discarded)
        uint64_t acc_hi[DCOLS], acc_lo[DCOLS];
#pragma unroll
        for (int c = 0; c < DCOLS; c++) acc_hi[c] = acc_lo[c] = 0;
        bool ok = true, aborted = false;
        // thread 0: the last step loaded, the last step whose operands arrived, the last
        // step whose MMAs were committed
        int loaded = -1, consumed = -1, pend_mma = -1;
        if (tid == 0)
            for (int q = 0; q < NSTAGE - 1 && q < nsteps; q++) {
                load(q);
                loaded = q;
            }
        for (int j = 0; j < nsteps; j++) {
            const int st = j % NSTAGE;
            if (tid == 0 && ok) {
                ok = mbar_wait(smem_u32(&full[st]), (j / NSTAGE) & 1);
                if (ok) {
                    consumed = j;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    // A slices a_bytes apart: with fewer than 128 rows stored, the MMA's
                    // remaining rows read whatever follows and only feed accumulator rows
                    // that are never drained into results
                    const uint32_t sa = smem_u32(dsm + st * STAGE), sb = sa + S * a.a_bytes;
                    const uint64_t da0 = mma_desc(sa), db0 = mma_desc(sb);
                    // The B slices of a stage lie one after another along N, so one MMA of
                    // A slice p against B slices q0 .. q0 + nq - 1 (N = 64 nq <= 256) writes the
                    // adjacent accumulators of the groups p + q0 .. p + q0 + nq - 1.
#pragma unroll
                    for (int p = 0; p < S; p++) {
#pragma unroll
                        for (int q0 = 0; q0 < S - p; q0 += 4) {
                            const int nq = (S - p - q0) < 4 ? (S - p - q0) : 4;
                            const uint32_t dcol = tmem + (uint32_t)((p + q0) * TN);
                            const uint64_t da = da0 + (uint64_t)((p * a.a_bytes) >> 4);
                            const uint64_t db = db0 + (uint64_t)((q0 * TILE_B) >> 4);
                            // the first products of a chunk (p = 0 covers every group) overwrite
                            const uint32_t accum = (j % CS == 0 && p == 0) ? 0u : 1u;
                            asm volatile("{\n .reg .pred pa;\n setp.ne.b32 pa, %4, 0;\n"
                                         " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n}\n"
                                         ::"r"(dcol), "l"(da), "l"(db), "r"(idesc_n(TN * nq)), "r"(accum)
                                         : "memory");
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 ::"r"(smem_u32(&empty[st]))
                                 : "memory");
                    pend_mma = j;
                    const int nxt = j + NSTAGE - 1;
                    if (nxt < nsteps) {
                        // its buffer is free once the MMAs of step j - 1 have read it
                        if (j >= 1) ok = mbar_wait(smem_u32(&empty[(j - 1) % NSTAGE]), ((j - 1) / NSTAGE) & 1);
                        if (ok) {
                            load(nxt);
                            loaded = nxt;
                        }
                    }
                }
                if (!ok) atomicExch(a.err, 1);
            }
            if (j % CS == CS - 1 || j == nsteps - 1) {
                // every draining thread takes the same branch: the barrier returns the OR
                if (drain_barrier_or(tid == 0 && !ok)) {
                    aborted = true;
                    break;
                }
                const bool done = mbar_wait(smem_u32(&empty[st]), (j / NSTAGE) & 1);
                if (!done) atomicExch(a.err, 1);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (done) {
                    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
                    const int cbase = DCOLS * (warp >> 2);
#pragma unroll
                    for (int d = 0; d < S; d++) {
                        uint32_t r[DCOLS];
                        const uint32_t taddr = tmem + lane_base + (uint32_t)(d * TN + cbase);
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                            "%15}, [%16];"
                            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                              "=r"(r[14]), "=r"(r[15])
                            : "r"(taddr)
                            : "memory");
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        // G_d is an integer below 2^24: the conversion is exact
                        const int sh = d <= 2 ? 14 - 7 * d : 42 - 7 * d;
#pragma unroll
                        for (int c = 0; c < DCOLS; c++) {
                            const uint64_t v = (uint64_t)(int64_t)__float2int_rn(__uint_as_float(r[c])) << sh;
                            if (d <= 2)
                                acc_hi[c] += v;
                            else
                                acc_lo[c] += v;
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                if (drain_barrier_or(!done)) {
                    aborted = true;
                    break;
                }
            }
        }
        if (tid == 0) {
            // after a failed wait: give the copies and MMAs in flight a bounded time to land
            if (pend_mma >= 0) mbar_wait(smem_u32(&empty[pend_mma % NSTAGE]), (pend_mma / NSTAGE) & 1);
            for (int q = consumed + 1; q <= loaded; q++) mbar_wait(smem_u32(&full[q % NSTAGE]), (q / NSTAGE) & 1);
        }
        if (!aborted) {
            const int row = mt * TM + 32 * (warp & 3) + lane;
            double *o = a.part + ((int64_t)z * a.MT * TM + row) * a.ncols + nt * TN + DCOLS * (warp >> 2);
#pragma unroll
            for (int c = 0; c < DCOLS; c++)
                o[c] = ldexp((double)(int64_t)acc_hi[c], -14) + ldexp((double)(int64_t)acc_lo[c], -42);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TMEM_COLS) : "memory");
}

// Number of K ranges per output tile.  The product runs one CTA per SM: up to one wave,
// as many ranges as fill it; where that leaves the last wave poorly filled (few tiles
// per wave, or a ragged tail), more ranges of at least 8 chunks each are taken if they
// fill the waves better by more than 5%.  Every range stays below MAX_STEPS_PER_BLOCK.
int pick_ksplit(int tiles, int KS) {
    constexpr int NSM = 152;
    auto fill = [&](int k) {
        const int64_t ctas = (int64_t)tiles * k;
        return (double)ctas / (double)(((ctas + NSM - 1) / NSM) * NSM);
    };
    int best = std::max(1, std::min(KS, NSM / tiles));
    for (int k = best + 1; k <= 256 && k <= KS / (8 * CS); k++)
        if (fill(k) > fill(best) + 0.05) best = k;
    return std::max(best, (KS + MAX_STEPS_PER_BLOCK - 1) / MAX_STEPS_PER_BLOCK);
}

// X[i][j][k][alpha] = X[j][i][k][alpha] = 2^(e_row + e_col - 14) sum over the K-range
// partials (fixed order).
__global__ void k_ozaki_finish(const double *part, int ksplit, int prow, int ncols, int m, int rows,
                               const double *rowmax, const double *colmax, double2 *X) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int Q = 4 * m;
    if (g >= (int64_t)rows * Q) return;
    const int r = (int)(g / Q), q = (int)(g % Q);
    double re = 0, im = 0;
    for (int s = 0; s < ksplit; s++) {
        const double *p = part + ((int64_t)s * prow + r) * ncols;
        re += p[q];
        im += p[Q + q];
    }
    // the splits carried v = 2^(e - 49) N = 2^(e - 7) sum_p q_p 2^(-7p) for each operand
    int i, j;
    pair_of(r, m, i, j);
    const int sc = exponent_of(rowmax[r]) + column_exponent(colmax, i) + column_exponent(colmax, j) +
                   exponent_of(colmax[q]) - 14;
    double2 v = make_double2(ldexp(re, sc), ldexp(im, sc));
    if (!isfinite(rowmax[r]) || !isfinite(colmax[q])) v = make_double2(NAN, NAN);  // a non-finite input
    X[((int64_t)i * m + j) * Q + q] = v;
    if (i != j) X[((int64_t)j * m + i) * Q + q] = v;
}

}  // namespace

namespace ddp {

// Colourless-spinor slice sums of a domain on the tensor cores (fields and forms as
// ddp_colourless_slices).  A: [m][n][12] on the device; X: L0 x m^3 x 4 complex on the
// device, slices outside the domain left untouched.
int colourless_tc(ddp_ctx *ctx, const double2 *A, int64_t n, int m, int form, int64_t slice_n, int nslice, int o0,
                  int L0, double2 *X) {
    if (m < 1 || m > MMAX) return DDP_ERR_UNSUPPORTED;
    const int rows = m * (m + 1) / 2, Q = 4 * m;
    const int MT = (rows + TM - 1) / TM;
    const int NT = (2 * Q + TN - 1) / TN;
    const int64_t K = 3 * slice_n;
    const int64_t KSh64 = (K + KSTEP - 1) / KSTEP;
    if (KSh64 > (1 << 28)) return DDP_ERR_UNSUPPORTED;
    const int KSh = (int)KSh64, KS = 2 * KSh;
    const int ksplit = pick_ksplit(MT * NT, KS);
    const int ncols = NT * TN, prow = MT * TM;
    const size_t bE = (size_t)rows * K * sizeof(float4);
    const size_t bA = (size_t)S * MT * KS * TILE_A, bB = (size_t)S * NT * KS * TILE_B;
    const size_t bP = (size_t)ksplit * prow * ncols * sizeof(double);
    Arena &ar = ctx->aux;
    ar.reset();
    DDP_CUDA(ctx, ar.reserve(bE + bA + bB + bP + (size_t)(rows + Q) * 12 + 64 + 10 * 256));
    float4 *E = (float4 *)ar.take(bE);
    uint8_t *Aq = (uint8_t *)ar.take(bA);
    uint8_t *Bq = (uint8_t *)ar.take(bB);
    double *part = (double *)ar.take(bP);
    double *rowmax = (double *)ar.take((size_t)rows * 8);
    double *colmax = (double *)ar.take((size_t)Q * 8);
    int *rexp = (int *)ar.take((size_t)rows * 4);
    int *cexp = (int *)ar.take((size_t)Q * 4);
    int *err = (int *)ar.take(64);
    const int es = m <= ES_SMALL_MMAX ? ES_SMALL : ES_LARGE;
    const size_t esm = (size_t)m * colour_kstride(es) * sizeof(float4);
    const size_t gsm = (size_t)NSTAGE * STAGE;
    DDP_CUDA(ctx, cudaFuncSetAttribute(es == ES_SMALL ? k_colour_E<ES_SMALL> : k_colour_E<ES_LARGE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)esm));
    DDP_CUDA(ctx, cudaFuncSetAttribute(k_ozaki_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
    cudaStream_t st = ctx->stream;
    DDP_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), st));
    for (int z = 0; z < nslice; z++) {
        const int64_t site0 = (int64_t)z * slice_n;
        DDP_CUDA(ctx, cudaMemsetAsync(rowmax, 0, (size_t)rows * 8, st));
        DDP_CUDA(ctx, cudaMemsetAsync(colmax, 0, (size_t)Q * 8, st));
        EArgs ea;
        ea.A = A;
        ea.n = n;
        ea.site0 = site0;
        ea.slice_n = slice_n;
        ea.m = m;
        ea.form = form;
        ea.rows = rows;
        ea.E = E;
        ea.rowmax = rowmax;
        ea.colmax = colmax;
        k_colour_max<<<(unsigned)std::min<int64_t>(2 * 152, (slice_n + 1) / 2), 256, 0, st>>>(A, n, site0, slice_n,
                                                                                          m, colmax);
        if (es == ES_SMALL)
            k_colour_E<ES_SMALL><<<(unsigned)((slice_n + ES_SMALL - 1) / ES_SMALL), 256, esm, st>>>(ea);
        else
            k_colour_E<ES_LARGE><<<(unsigned)((slice_n + ES_LARGE - 1) / ES_LARGE), 256, esm, st>>>(ea);
        SplitArgs sa;
        sa.E = E;
        sa.A = A;
        sa.n = n;
        sa.site0 = site0;
        sa.K = K;
        sa.m = m;
        sa.form = form;
        sa.rows = rows;
        sa.MT = MT;
        sa.NT = NT;
        sa.KSh = KSh;
        k_exponents<<<(rows + 255) / 256, 256, 0, st>>>(rowmax, rows, rexp);
        k_exponents<<<(Q + 255) / 256, 256, 0, st>>>(colmax, Q, cexp);
        sa.rexp = rexp;
        sa.cexp = cexp;
        sa.Aq = (__nv_bfloat16 *)Aq;
        sa.Bq = (__nv_bfloat16 *)Bq;
        const int64_t na = (int64_t)MT * KSh * TM * KSTEP, nb = (int64_t)NT * KSh * TN * KSTEP;
        k_split_A<<<(unsigned)((na + 255) / 256), 256, 0, st>>>(sa);
        k_split_B<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(sa);
        GemmArgs g;
        g.Aq = Aq;
        g.Bq = Bq;
        g.a_bytes = TILE_A;
        g.MT = MT;
        g.NT = NT;
        g.KS = KS;
        g.ksplit = ksplit;
        g.ncols = ncols;
        g.part = part;
        g.err = err;
        k_ozaki_gemm<<<dim3(NT, MT, ksplit), GEMM_BLOCK, gsm, st>>>(g);
        const int64_t nx = (int64_t)rows * Q;
        k_ozaki_finish<<<(unsigned)((nx + 255) / 256), 256, 0, st>>>(
            part, ksplit, prow, ncols, m, rows, rowmax, colmax, X + (int64_t)((o0 + z) % L0) * m * m * Q);
        ctx->launches += 8;
        DDP_CUDA(ctx, cudaGetLastError());
    }
    int h = 0;
    DDP_CUDA(ctx, cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    DDP_CUDA(ctx, cudaStreamSynchronize(st));
    if (h) {
        snprintf(ctx->last_error, sizeof(ctx->last_error), "colourless spinors: a wait for the tensor cores gave up");
        return DDP_ERR_CUDA;
    }
    return DDP_OK;
}

}  // namespace ddp

// ------------------------------------------------------------ Gram blocks
//
// G[i][j] = sum_r conj(A_i[r]) A_j[r] over the rows r of one segment, on the same
// emulated-FP64 product: A' rows i = [Re A_i | Im A_i], B' rows = [Re A_j | Im A_j]
// (the real parts, columns j < m) and [Im A_j | -Re A_j] (the imaginary parts,
// m <= c < 2m), every row and column with its own power-of-two exponent.  The m <= 128
// rows of A' are stored as R8 = 8 ceil(m / 8) rows per block (the MMA's other rows read
// whatever follows in shared memory and feed accumulator rows that are never used); the
// 2m columns of B' span ceil(2m / 64) column tiles.

namespace {

// colmax[i] = max over the segment's rows of |Re A_i|, |Im A_i|
__global__ void __launch_bounds__(256) k_gram_max(const double2 *A, int64_t cs, int m, int64_t r0, int64_t nrow,
                                                  double *colmax) {
    const int i = blockIdx.y;
    double mx = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrow; r += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = A[(int64_t)i * cs + r0 + r];
        mx = fmax(mx, fmax(mag(v.x), mag(v.y)));
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0 && mx > 0) atomic_max_pos(colmax + i, mx);
    (void)m;
}

struct GramSplitArgs {
    const double2 *A;
    int64_t cs, r0, nrow;  // column stride; the segment's rows
    int m, R8, KSh, NT;
    const int *cexp;       // exponents of the columns
    __nv_bfloat16 *Aq, *Bq;  // [2 KSh][S][R8 x KSTEP], [NT][2 KSh][S][64 x KSTEP]
};

__global__ void k_gram_split_A(GramSplitArgs a) {
    const int tile = a.R8 * KSTEP;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)a.KSh * tile) return;
    const int e = (int)(g % tile);
    const int ksr = (int)(g / tile);
    int rl, kl;
    tile_pos(e, rl, kl);
    const int64_t kx = (int64_t)ksr * KSTEP + kl;
    __nv_bfloat16 re[S], im[S];
    const int er = rl < a.m ? a.cexp[rl] : NONFINITE;
    if (kx < a.nrow && er != NONFINITE) {
        const double2 v = a.A[(int64_t)rl * a.cs + a.r0 + kx];
        const int k = 49 - er;
        digits7(fixed_of(v.x, k), re);
        digits7(fixed_of(v.y, k), im);
    } else {
        for (int p = 0; p < S; p++) re[p] = im[p] = __double2bfloat16(0.0);
    }
    const int64_t bre = (int64_t)ksr * S, bim = (int64_t)(a.KSh + ksr) * S;
    for (int p = 0; p < S; p++) {
        a.Aq[(bre + p) * tile + e] = re[p];
        a.Aq[(bim + p) * tile + e] = im[p];
    }
}

__global__ void k_gram_split_B(GramSplitArgs a) {
    const int tile = TN * KSTEP;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)a.NT * a.KSh * tile) return;
    const int e = (int)(g % tile);
    const int64_t t = g / tile;
    const int ksr = (int)(t % a.KSh), nt = (int)(t / a.KSh);
    int col, kl;
    tile_pos(e, col, kl);
    col += nt * TN;
    const int64_t kx = (int64_t)ksr * KSTEP + kl;
    const int j = col < a.m ? col : col - a.m;
    __nv_bfloat16 lo[S], hi[S];
    const int ej = col < 2 * a.m ? a.cexp[j] : NONFINITE;
    if (kx < a.nrow && ej != NONFINITE) {
        const double2 v = a.A[(int64_t)j * a.cs + a.r0 + kx];
        const int k = 49 - ej;
        digits7(fixed_of(col < a.m ? v.x : v.y, k), lo);
        digits7(fixed_of(col < a.m ? v.y : -v.x, k), hi);
    } else {
        for (int p = 0; p < S; p++) lo[p] = hi[p] = __double2bfloat16(0.0);
    }
    // tile block (nt, K step, slice), as k_ozaki_gemm reads it
    const int64_t KS = 2 * (int64_t)a.KSh;
    const int64_t blo = (nt * KS + ksr) * S, bhi = (nt * KS + a.KSh + ksr) * S;
    for (int p = 0; p < S; p++) {
        a.Bq[(blo + p) * tile + e] = lo[p];
        a.Bq[(bhi + p) * tile + e] = hi[p];
    }
}

// G[i][j] = 2^(e_i + e_j - 14) (sum of the K-range partials of the real and the
// imaginary column), fixed order.
__global__ void k_gram_finish(const double *part, int ksplit, int ncols, int m, const double *colmax, double2 *G) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= m * m) return;
    const int i = g / m, j = g % m;
    double re = 0, im = 0;
    for (int s = 0; s < ksplit; s++) {
        const double *p = part + ((int64_t)s * TM + i) * ncols;
        re += p[j];
        im += p[m + j];
    }
    const int sc = exponent_of(colmax[i]) + exponent_of(colmax[j]) - 14;
    double2 v = make_double2(ldexp(re, sc), ldexp(im, sc));
    if (!isfinite(colmax[i]) || !isfinite(colmax[j])) v = make_double2(NAN, NAN);
    G[g] = v;
}

}  // namespace

namespace ddp {

// Gram blocks of nseg consecutive row segments of seg rows each on the tensor cores:
// out[z][i][j] = sum over the rows r of segment z of conj(A_i[r]) A_j[r], A_i[r] the
// complex component r of column i (column stride cs); A and out on the device, m <= 128.
int gram_tc(ddp_ctx *ctx, const double2 *A, int64_t cs, int m, int64_t seg, int nseg, double2 *out) {
    if (m < 1 || m > TM) return DDP_ERR_UNSUPPORTED;
    const int R8 = 8 * ((m + 7) / 8);
    const int a_bytes = R8 * KSTEP * 2;
    const int NT = (2 * m + TN - 1) / TN, ncols = NT * TN;
    const int64_t KSh64 = (seg + KSTEP - 1) / KSTEP;
    if (KSh64 > (1 << 28)) return DDP_ERR_UNSUPPORTED;
    const int KSh = (int)KSh64, KS = 2 * KSh;
    const int ksplit = pick_ksplit(NT, KS);
    const size_t bA = (size_t)S * KS * a_bytes, bB = (size_t)S * NT * KS * TILE_B;
    const size_t bP = (size_t)ksplit * TM * ncols * sizeof(double);
    Arena &ar = ctx->aux;
    ar.reset();
    DDP_CUDA(ctx, ar.reserve(bA + bB + bP + (size_t)m * 12 + 64 + 7 * 256));
    uint8_t *Aq = (uint8_t *)ar.take(bA);
    uint8_t *Bq = (uint8_t *)ar.take(bB);
    double *part = (double *)ar.take(bP);
    double *colmax = (double *)ar.take((size_t)m * 8);
    int *cexp = (int *)ar.take((size_t)m * 4);
    int *err = (int *)ar.take(64);
    const size_t gsm = (size_t)NSTAGE * STAGE;
    DDP_CUDA(ctx, cudaFuncSetAttribute(k_ozaki_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
    cudaStream_t st = ctx->stream;
    DDP_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), st));
    for (int z = 0; z < nseg; z++) {
        DDP_CUDA(ctx, cudaMemsetAsync(colmax, 0, (size_t)m * 8, st));
        const int64_t r0 = (int64_t)z * seg;
        k_gram_max<<<dim3((unsigned)std::min<int64_t>(64, (seg + 255) / 256), m), 256, 0, st>>>(A, cs, m, r0, seg,
                                                                                            colmax);
        GramSplitArgs sa;
        sa.A = A;
        sa.cs = cs;
        sa.r0 = r0;
        sa.nrow = seg;
        sa.m = m;
        sa.R8 = R8;
        sa.KSh = KSh;
        sa.NT = NT;
        k_exponents<<<(m + 255) / 256, 256, 0, st>>>(colmax, m, cexp);
        sa.cexp = cexp;
        sa.Aq = (__nv_bfloat16 *)Aq;
        sa.Bq = (__nv_bfloat16 *)Bq;
        const int64_t na = (int64_t)KSh * R8 * KSTEP, nb = (int64_t)NT * KSh * TN * KSTEP;
        k_gram_split_A<<<(unsigned)((na + 255) / 256), 256, 0, st>>>(sa);
        k_gram_split_B<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(sa);
        GemmArgs g;
        g.Aq = Aq;
        g.Bq = Bq;
        g.a_bytes = a_bytes;
        g.MT = 1;
        g.NT = NT;
        g.KS = KS;
        g.ksplit = ksplit;
        g.ncols = ncols;
        g.part = part;
        g.err = err;
        k_ozaki_gemm<<<dim3(NT, 1, ksplit), GEMM_BLOCK, gsm, st>>>(g);
        k_gram_finish<<<(unsigned)((m * m + 255) / 256), 256, 0, st>>>(part, ksplit, ncols, m, colmax,
                                                                       out + (int64_t)z * m * m);
        ctx->launches += 6;
        DDP_CUDA(ctx, cudaGetLastError());
    }
    int h = 0;
    DDP_CUDA(ctx, cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    DDP_CUDA(ctx, cudaStreamSynchronize(st));
    if (h) {
        snprintf(ctx->last_error, sizeof(ctx->last_error), "Gram blocks: a wait for the tensor cores gave up");
        return DDP_ERR_CUDA;
    }
    return DDP_OK;
}

}  // namespace ddp
