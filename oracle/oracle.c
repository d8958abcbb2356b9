/*
 * FP64 CPU oracle for domain-restricted Wilson-Dirac propagators.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * statement of what the CUDA library computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the library
 * never calls it and shares no code, header or table with it.
 *
 * Everything is double precision, round-to-nearest, with fixed-order sums
 * (one OpenMP partition per call, partial sums added in thread order).
 *
 * Conventions (the paper leaves them open; each reading is stated here):
 *  - lattice L0 x L1 x L2 x L3, direction 0 is time; global site index
 *    ((x0*L1 + x1)*L2 + x2)*L3 + x3;
 *  - gauge field U[mu][site][row][col], complex interleaved (re, im);
 *  - spinor fields psi[col][site][spin][colour], complex interleaved;
 *  - Euclidean chiral gamma basis: gamma_0 = [[0,1],[1,0]],
 *    gamma_k = [[0,-i sigma_k],[i sigma_k,0]], gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3,
 *    so that gamma_0, gamma_2 are symmetric and C = i gamma_0 gamma_2 obeys
 *    C gamma_mu C^-1 = -gamma_mu^T;
 *  - time boundary: 0 periodic, 1 antiperiodic, 2 open (hop across T-1 <-> 0
 *    dropped); space is periodic.
 *  - a domain is a box {(o_mu + k_mu) mod L_mu : 0 <= k_mu < e_mu}; when
 *    e_mu == L_mu the direction is not restricted and the global boundary
 *    condition holds, otherwise every hop leaving the box is dropped;
 *  - domain-local order is lexicographic in k with the same nesting as the
 *    global index.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    int L[4];
    int64_t V;
    int bc;
} lat_t;

typedef struct {
    int o[4];
    int e[4];
    int64_t n;
} box_t;

/* ------------------------------------------------------------------ gamma */

static void matmul4(const cplx a[4][4], const cplx b[4][4], cplx c[4][4]) {
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            cplx s = 0;
            for (int k = 0; k < 4; k++) s += a[i][k] * b[k][j];
            c[i][j] = s;
        }
}

/* gamma[0..3] = gamma_mu, gamma[4] = gamma_5 (Euclidean, Hermitian). */
static void make_gamma(cplx g[5][4][4]) {
    memset(g, 0, sizeof(cplx) * 5 * 16);
    /* Pauli matrices */
    cplx s[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
    for (int i = 0; i < 2; i++) {
        g[0][i][2 + i] = 1;
        g[0][2 + i][i] = 1;
    }
    for (int k = 0; k < 3; k++)
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) {
                g[1 + k][i][2 + j] = -I * s[k][i][j];
                g[1 + k][2 + i][j] = I * s[k][i][j];
            }
    cplx t1[4][4], t2[4][4];
    matmul4(g[0], g[1], t1);
    matmul4(t1, g[2], t2);
    matmul4(t2, g[3], g[4]);
}

int orc_gamma(double *out /* [5][4][4] complex */) {
    cplx g[5][4][4];
    make_gamma(g);
    memcpy(out, g, sizeof(g));
    return 0;
}

/* -------------------------------------------------------------- geometry */

static int set_lat(lat_t *lat, const int L[4], int bc) {
    lat->V = 1;
    for (int m = 0; m < 4; m++) {
        if (L[m] < 1) return 1;
        lat->L[m] = L[m];
        lat->V *= L[m];
    }
    if (bc < 0 || bc > 2) return 1;
    lat->bc = bc;
    return 0;
}

static int set_box(box_t *b, const lat_t *lat, const int o[4], const int e[4]) {
    b->n = 1;
    for (int m = 0; m < 4; m++) {
        if (e[m] < 1 || e[m] > lat->L[m]) return 1;
        b->o[m] = ((o[m] % lat->L[m]) + lat->L[m]) % lat->L[m];
        b->e[m] = e[m];
        b->n *= e[m];
    }
    return 0;
}

static int64_t glob_index(const lat_t *lat, const int x[4]) {
    return (((int64_t)x[0] * lat->L[1] + x[1]) * lat->L[2] + x[2]) * lat->L[3] + x[3];
}

static int64_t loc_index(const box_t *b, const int k[4]) {
    return (((int64_t)k[0] * b->e[1] + k[1]) * b->e[2] + k[2]) * b->e[3] + k[3];
}

static void loc_coords(const box_t *b, int64_t l, int k[4]) {
    for (int m = 3; m >= 0; m--) {
        k[m] = (int)(l % b->e[m]);
        l /= b->e[m];
    }
}

static void glob_coords(const lat_t *lat, const box_t *b, const int k[4], int x[4]) {
    for (int m = 0; m < 4; m++) x[m] = (b->o[m] + k[m]) % lat->L[m];
}

/* Neighbour of local site k in direction mu (dir=+1 forward, -1 backward).
 * Returns the boundary factor of the hop: 0 when the hop is dropped (it leaves
 * a restricted box, or crosses an open time boundary), -1 across the
 * antiperiodic time boundary, otherwise +1.  kn receives the neighbour. */
static double hop_factor(const lat_t *lat, const box_t *b, const int k[4], int mu, int dir, int kn[4]) {
    int x[4];
    glob_coords(lat, b, k, x);
    memcpy(kn, k, sizeof(int) * 4);
    kn[mu] += dir;
    if (b->e[mu] < lat->L[mu]) {
        if (kn[mu] < 0 || kn[mu] >= b->e[mu]) return 0.0; /* Dirichlet: outside the box */
    } else {
        kn[mu] = (kn[mu] + lat->L[mu]) % lat->L[mu];
    }
    if (mu == 0) {
        int crosses = (dir > 0) ? (x[0] == lat->L[0] - 1) : (x[0] == 0);
        if (crosses) {
            if (lat->bc == 1) return -1.0;
            if (lat->bc == 2) return 0.0;
        }
    }
    return 1.0;
}

static int local_of_global(const lat_t *lat, const box_t *b, const int x[4], int k[4]) {
    for (int m = 0; m < 4; m++) {
        k[m] = ((x[m] - b->o[m]) % lat->L[m] + lat->L[m]) % lat->L[m];
        if (k[m] >= b->e[m]) return 0;
    }
    return 1;
}

/* Domain-local lexicographic order -> global site index, even-odd rank and
 * parity.  Parity is (x0+x1+x2+x3) mod 2 of the global coordinates; the
 * even-odd rank is the position among the domain's sites of the same parity,
 * counted in domain-local lexicographic order.  Any pointer may be NULL. */
int orc_domain_maps(const int L[4], const int o[4], const int e[4], int64_t *global_index,
                    int64_t *eo_index, int8_t *parity) {
    lat_t lat;
    box_t b;
    if (set_lat(&lat, L, 1) || set_box(&b, &lat, o, e)) return 1;
    int64_t cnt[2] = {0, 0};
    for (int64_t l = 0; l < b.n; l++) {
        int k[4], x[4];
        loc_coords(&b, l, k);
        glob_coords(&lat, &b, k, x);
        int p = (x[0] + x[1] + x[2] + x[3]) & 1;
        if (global_index) global_index[l] = glob_index(&lat, x);
        if (parity) parity[l] = (int8_t)p;
        if (eo_index) eo_index[l] = cnt[p];
        cnt[p]++;
    }
    return 0;
}

/* ---------------------------------------------------------- the operator */

static inline const cplx *link(const lat_t *lat, const cplx *U, int mu, int64_t site) {
    return U + ((int64_t)mu * lat->V + site) * 9;
}

/* Hopping term of App. A, restricted to the box (Sec. 2):
 *   (Hop psi)(y) = sum_mu [ f+ (1 - gamma_mu) U_mu(y) psi(y+mu)
 *                         + f- (1 + gamma_mu) U_mu(y-mu)^+ psi(y-mu) ]
 * with f the boundary factor of each hop (0 for hops leaving the box). */
static void hop_site(const lat_t *lat, const box_t *b, const cplx g[5][4][4], const cplx *U,
                     const cplx *in, int64_t l, cplx acc[4][3]) {
    int k[4], x[4];
    loc_coords(b, l, k);
    glob_coords(lat, b, k, x);
    memset(acc, 0, sizeof(cplx) * 12);
    for (int mu = 0; mu < 4; mu++) {
        for (int dir = 1; dir >= -1; dir -= 2) {
            int kn[4];
            double f = hop_factor(lat, b, k, mu, dir, kn);
            if (f == 0.0) continue;
            const cplx *nb = in + loc_index(b, kn) * 12;
            cplx Uv[3][3];
            if (dir > 0) {
                const cplx *u = link(lat, U, mu, glob_index(lat, x));
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) Uv[i][j] = u[i * 3 + j];
            } else {
                int xm[4];
                memcpy(xm, x, sizeof(xm));
                xm[mu] = (xm[mu] - 1 + lat->L[mu]) % lat->L[mu];
                const cplx *u = link(lat, U, mu, glob_index(lat, xm));
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) Uv[i][j] = conj(u[j * 3 + i]);
            }
            /* colour: w[s][a] = sum_b Uv[a][b] nb[s][b] */
            cplx w[4][3];
            for (int s = 0; s < 4; s++)
                for (int a = 0; a < 3; a++) {
                    cplx t = 0;
                    for (int c = 0; c < 3; c++) t += Uv[a][c] * nb[s * 3 + c];
                    w[s][a] = t;
                }
            /* spin: (1 -/+ gamma_mu) w */
            double sg = (dir > 0) ? -1.0 : 1.0;
            for (int s = 0; s < 4; s++)
                for (int a = 0; a < 3; a++) {
                    cplx t = w[s][a];
                    for (int r = 0; r < 4; r++) t += sg * g[mu][s][r] * w[r][a];
                    acc[s][a] += f * t;
                }
        }
    }
}

/* out = Hop_Gamma in, i.e. the Dirichlet-restricted D_hop of Sec. 5 (2 kappa D = 1 - kappa D_hop). */
int orc_apply_hop(const int L[4], int bc, const double *Ud, const int o[4], const int e[4],
                  const double *ind, double *outd, int ncol) {
    lat_t lat;
    box_t b;
    if (set_lat(&lat, L, bc) || set_box(&b, &lat, o, e)) return 1;
    cplx g[5][4][4];
    make_gamma(g);
    const cplx *U = (const cplx *)Ud;
    for (int c = 0; c < ncol; c++) {
        const cplx *in = (const cplx *)ind + (int64_t)c * b.n * 12;
        cplx *out = (cplx *)outd + (int64_t)c * b.n * 12;
#pragma omp parallel for schedule(static)
        for (int64_t l = 0; l < b.n; l++) {
            cplx acc[4][3];
            hop_site(&lat, &b, g, U, in, l, acc);
            memcpy(out + l * 12, acc, sizeof(acc));
        }
    }
    return 0;
}

/* ------------------------------------------------------ the clover term */

/* 3x3 complex products for the clover leaves. */
static void m3mul(const cplx a[9], const cplx b[9], cplx c[9]) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx t = 0;
            for (int k = 0; k < 3; k++) t += a[i * 3 + k] * b[k * 3 + j];
            c[i * 3 + j] = t;
        }
}
static void m3dag(const cplx a[9], cplx c[9]) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) c[i * 3 + j] = conj(a[j * 3 + i]);
}
static void m3copy(const cplx *a, cplx c[9]) { memcpy(c, a, 9 * sizeof(cplx)); }

/* Global site index of x + s_mu mu + s_nu nu (periodic gauge field). */
static int64_t shifted(const lat_t *lat, const int x[4], int mu, int smu, int nu, int snu) {
    int y[4];
    memcpy(y, x, sizeof(y));
    y[mu] = (y[mu] + smu + lat->L[mu]) % lat->L[mu];
    y[nu] = (y[nu] + snu + lat->L[nu]) % lat->L[nu];
    return glob_index(lat, y);
}

/* Q_{mu nu}(x): the four plaquettes in the (mu, nu) plane that start and end at x,
 * each traversed mu first (counterclockwise): the clover leaves. */
static void clover_leaves(const lat_t *lat, const cplx *U, const int x[4], int mu, int nu, cplx Q[9]) {
    cplx a[9], b[9], c[9], d[9], t1[9], t2[9], t3[9];
    memset(Q, 0, 9 * sizeof(cplx));
    /* x -> x+mu -> x+mu+nu -> x+nu -> x */
    m3copy(link(lat, U, mu, shifted(lat, x, mu, 0, nu, 0)), a);
    m3copy(link(lat, U, nu, shifted(lat, x, mu, 1, nu, 0)), b);
    m3dag(link(lat, U, mu, shifted(lat, x, mu, 0, nu, 1)), c);
    m3dag(link(lat, U, nu, shifted(lat, x, mu, 0, nu, 0)), d);
    m3mul(a, b, t1), m3mul(t1, c, t2), m3mul(t2, d, t3);
    for (int i = 0; i < 9; i++) Q[i] += t3[i];
    /* x -> x+nu -> x+nu-mu -> x-mu -> x */
    m3copy(link(lat, U, nu, shifted(lat, x, mu, 0, nu, 0)), a);
    m3dag(link(lat, U, mu, shifted(lat, x, mu, -1, nu, 1)), b);
    m3dag(link(lat, U, nu, shifted(lat, x, mu, -1, nu, 0)), c);
    m3copy(link(lat, U, mu, shifted(lat, x, mu, -1, nu, 0)), d);
    m3mul(a, b, t1), m3mul(t1, c, t2), m3mul(t2, d, t3);
    for (int i = 0; i < 9; i++) Q[i] += t3[i];
    /* x -> x-mu -> x-mu-nu -> x-nu -> x */
    m3dag(link(lat, U, mu, shifted(lat, x, mu, -1, nu, 0)), a);
    m3dag(link(lat, U, nu, shifted(lat, x, mu, -1, nu, -1)), b);
    m3copy(link(lat, U, mu, shifted(lat, x, mu, -1, nu, -1)), c);
    m3copy(link(lat, U, nu, shifted(lat, x, mu, 0, nu, -1)), d);
    m3mul(a, b, t1), m3mul(t1, c, t2), m3mul(t2, d, t3);
    for (int i = 0; i < 9; i++) Q[i] += t3[i];
    /* x -> x-nu -> x-nu+mu -> x+mu -> x */
    m3dag(link(lat, U, nu, shifted(lat, x, mu, 0, nu, -1)), a);
    m3copy(link(lat, U, mu, shifted(lat, x, mu, 0, nu, -1)), b);
    m3copy(link(lat, U, nu, shifted(lat, x, mu, 1, nu, -1)), c);
    m3dag(link(lat, U, mu, shifted(lat, x, mu, 0, nu, 0)), d);
    m3mul(a, b, t1), m3mul(t1, c, t2), m3mul(t2, d, t3);
    for (int i = 0; i < 9; i++) Q[i] += t3[i];
}

/* The O(a)-improvement (clover) term of the Wilson-Dirac operator, site by site:
 *   C(x) = c_sw (i/4) sum_{mu,nu} sigma_{mu nu} F_{mu nu}(x),
 *   sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu],  F_{mu nu} = (Q_{mu nu} - Q_{nu mu}) / 8,
 * the clover-leaf lattice field strength of the gauge field (periodic in every
 * direction whatever the fermion boundary condition).  The paper names the
 * improved operator (the footnotes of Sec. 4 and Sec. 5) without writing it down;
 * this is the standard Sheikholeslami-Wohlert term.  out: [V][12][12] complex,
 * rows and columns indexed 3 spin + colour. */
static void clover_field(const lat_t *lat, const cplx g[5][4][4], const cplx *U, double csw, cplx *out) {
    cplx sigma[4][4][4][4];
    for (int mu = 0; mu < 4; mu++)
        for (int nu = 0; nu < 4; nu++)
            for (int s = 0; s < 4; s++)
                for (int r = 0; r < 4; r++) {
                    cplx t = 0;
                    for (int q = 0; q < 4; q++) t += g[mu][s][q] * g[nu][q][r] - g[nu][s][q] * g[mu][q][r];
                    sigma[mu][nu][s][r] = 0.5 * I * t;
                }
#pragma omp parallel for schedule(static)
    for (int64_t site = 0; site < lat->V; site++) {
        int x[4];
        int64_t r = site;
        for (int m = 3; m >= 0; m--) {
            x[m] = (int)(r % lat->L[m]);
            r /= lat->L[m];
        }
        cplx *C = out + site * 144;
        memset(C, 0, 144 * sizeof(cplx));
        for (int mu = 0; mu < 4; mu++)
            for (int nu = 0; nu < 4; nu++) {
                if (mu == nu) continue;
                cplx Qa[9], Qb[9], F[9];
                clover_leaves(lat, U, x, mu, nu, Qa);
                clover_leaves(lat, U, x, nu, mu, Qb);
                for (int i = 0; i < 9; i++) F[i] = (Qa[i] - Qb[i]) / 8.0;
                for (int s = 0; s < 4; s++)
                    for (int a = 0; a < 3; a++)
                        for (int q = 0; q < 4; q++)
                            for (int b = 0; b < 3; b++)
                                C[(s * 3 + a) * 12 + q * 3 + b] += csw * 0.25 * I * sigma[mu][nu][s][q] * F[a * 3 + b];
            }
    }
}

int orc_clover_field(const int L[4], const double *Ud, double csw, double *outd) {
    lat_t lat;
    if (set_lat(&lat, L, 1)) return 1;
    cplx g[5][4][4];
    make_gamma(g);
    clover_field(&lat, g, (const cplx *)Ud, csw, (cplx *)outd);
    return 0;
}

/* D_Gamma of Sec. 2 applied to the box: D = D_w + m0 (App. A) written as
 *   (D psi)(y) = (4 + m0) psi(y) - 1/2 (Hop psi)(y),   4 + m0 = 1/(2 kappa),
 * with every term that involves a site outside the box set to zero. */
static void apply_D(const lat_t *lat, const box_t *b, const cplx g[5][4][4], const cplx *U, const cplx *clov,
                    double kappa, const cplx *in, cplx *out) {
    double diag = 1.0 / (2.0 * kappa);
#pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < b->n; l++) {
        cplx acc[4][3];
        hop_site(lat, b, g, U, in, l, acc);
        for (int s = 0; s < 4; s++)
            for (int a = 0; a < 3; a++) out[l * 12 + s * 3 + a] = diag * in[l * 12 + s * 3 + a] - 0.5 * acc[s][a];
        if (clov) {
            /* the clover term is site-local: D[Gamma, Gamma] keeps it at every site of the box */
            int k[4], x[4];
            loc_coords(b, l, k);
            glob_coords(lat, b, k, x);
            const cplx *C = clov + glob_index(lat, x) * 144;
            for (int i = 0; i < 12; i++) {
                cplx t = 0;
                for (int j = 0; j < 12; j++) t += C[i * 12 + j] * in[l * 12 + j];
                out[l * 12 + i] += t;
            }
        }
    }
}

/* csw != 0 adds the clover term (clover_field). */
int orc_apply_dirac(const int L[4], int bc, const double *Ud, const int o[4], const int e[4], double kappa,
                    double csw, const double *ind, double *outd, int ncol) {
    lat_t lat;
    box_t b;
    if (set_lat(&lat, L, bc) || set_box(&b, &lat, o, e) || !(kappa > 0)) return 1;
    cplx g[5][4][4];
    make_gamma(g);
    cplx *clov = NULL;
    if (csw != 0.0) {
        clov = (cplx *)malloc((size_t)lat.V * 144 * sizeof(cplx));
        if (!clov) return 1;
        clover_field(&lat, g, (const cplx *)Ud, csw, clov);
    }
    for (int c = 0; c < ncol; c++)
        apply_D(&lat, &b, g, (const cplx *)Ud, clov, kappa, (const cplx *)ind + (int64_t)c * b.n * 12,
                (cplx *)outd + (int64_t)c * b.n * 12);
    free(clov);
    return 0;
}

/* ------------------------------------------------------------- the solver */

/* <a, b> = sum conj(a) b with a fixed-order reduction: per-thread partial sums
 * over a static partition, added in thread order. */
static cplx dot(const cplx *a, const cplx *b, int64_t n) {
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    cplx *part = (cplx *)calloc((size_t)nt, sizeof(cplx));
#pragma omp parallel num_threads(nt)
    {
        int t = 0, nth = 1;
#ifdef _OPENMP
        t = omp_get_thread_num();
        nth = omp_get_num_threads();
#endif
        int64_t lo = n * t / nth, hi = n * (t + 1) / nth;
        cplx s = 0;
        for (int64_t i = lo; i < hi; i++) s += conj(a[i]) * b[i];
        part[t] = s;
    }
    cplx s = 0;
    for (int t = 0; t < nt; t++) s += part[t];
    free(part);
    return s;
}

static double norm2(const cplx *a, int64_t n) { return creal(dot(a, a, n)); }

/* BiCGStab (van der Vorst 1992) on the unpreconditioned D_Gamma, one column.
 * The paper does not name its solver; the propagator is by definition the
 * unique solution of D_Gamma psi = eta (Sec. 2, Eq. diric).  Stops when the
 * recomputed true residual |eta - D psi| / |eta| <= tol; the recursion is
 * restarted from the true residual whenever the recursive residual reaches
 * tol without the true one doing so. */
static int bicgstab(const lat_t *lat, const box_t *b, const cplx g[5][4][4], const cplx *U, const cplx *clov,
                    double kappa, const cplx *eta, cplx *x, double tol, int maxit, int *iters, double *relres) {
    int64_t N = b->n * 12;
    cplx *r = calloc(N, sizeof(cplx)), *rh = calloc(N, sizeof(cplx)), *p = calloc(N, sizeof(cplx));
    cplx *v = calloc(N, sizeof(cplx)), *s = calloc(N, sizeof(cplx)), *t = calloc(N, sizeof(cplx));
    double bn = sqrt(norm2(eta, N));
    int it = 0, status = 1;
    memset(x, 0, N * sizeof(cplx));
    if (bn == 0.0) {
        *iters = 0;
        *relres = 0.0;
        status = 0;
        goto done;
    }
    for (int restart = 0; restart < 50 && it < maxit; restart++) {
        /* r = eta - D x */
        apply_D(lat, b, g, U, clov, kappa, x, r);
        for (int64_t i = 0; i < N; i++) r[i] = eta[i] - r[i];
        double rn = sqrt(norm2(r, N));
        if (rn <= tol * bn) {
            status = 0;
            break;
        }
        memcpy(rh, r, N * sizeof(cplx));
        memset(p, 0, N * sizeof(cplx));
        memset(v, 0, N * sizeof(cplx));
        cplx rho = 1, alpha = 1, omega = 1;
        while (it < maxit) {
            it++;
            cplx rho1 = dot(rh, r, N);
            if (cabs(rho1) == 0.0) break;
            cplx beta = (rho1 / rho) * (alpha / omega);
            for (int64_t i = 0; i < N; i++) p[i] = r[i] + beta * (p[i] - omega * v[i]);
            apply_D(lat, b, g, U, clov, kappa, p, v);
            cplx rv = dot(rh, v, N);
            if (cabs(rv) == 0.0) break;
            alpha = rho1 / rv;
            for (int64_t i = 0; i < N; i++) s[i] = r[i] - alpha * v[i];
            apply_D(lat, b, g, U, clov, kappa, s, t);
            double tt = norm2(t, N);
            omega = (tt > 0) ? dot(t, s, N) / tt : 0.0;
            for (int64_t i = 0; i < N; i++) {
                x[i] += alpha * p[i] + omega * s[i];
                r[i] = s[i] - omega * t[i];
            }
            rho = rho1;
            if (sqrt(norm2(r, N)) <= 0.5 * tol * bn || omega == 0.0) break;
        }
    }
    /* final true residual */
    apply_D(lat, b, g, U, clov, kappa, x, r);
    for (int64_t i = 0; i < N; i++) r[i] = eta[i] - r[i];
    *relres = (bn > 0) ? sqrt(norm2(r, N)) / bn : 0.0;
    *iters = it;
    status = (*relres <= tol) ? 0 : 2;
done:
    free(r);
    free(rh);
    free(p);
    free(v);
    free(s);
    free(t);
    return status;
}

/* Solve D_Gamma psi_c = eta_c for ncol columns (Sec. 2, Eq. diric).  Returns 0
 * when every column reached tol, 2 if some did not, 1 on bad arguments. */
int orc_solve(const int L[4], int bc, const double *Ud, const int o[4], const int e[4], double kappa, double csw,
              const double *etad, double *psid, int ncol, double tol, int maxit, int *iters, double *relres) {
    lat_t lat;
    box_t b;
    if (set_lat(&lat, L, bc) || set_box(&b, &lat, o, e) || !(kappa > 0)) return 1;
    cplx g[5][4][4];
    make_gamma(g);
    cplx *clov = NULL;
    if (csw != 0.0) {
        clov = (cplx *)malloc((size_t)lat.V * 144 * sizeof(cplx));
        if (!clov) return 1;
        clover_field(&lat, g, (const cplx *)Ud, csw, clov);
    }
    int worst = 0;
    for (int c = 0; c < ncol; c++) {
        int st = bicgstab(&lat, &b, g, (const cplx *)Ud, clov, kappa, (const cplx *)etad + (int64_t)c * b.n * 12,
                          (cplx *)psid + (int64_t)c * b.n * 12, tol, maxit, &iters[c], &relres[c]);
        if (st > worst) worst = st;
    }
    free(clov);
    return worst;
}

/* ---------------------------------------------------------------- series */

/* T = S_big - E S_small on the big box, where E extends the small-box
 * propagator by zero outside the small box (Eq. Dseries, Sec. 1).  The small
 * box must lie inside the big one. */
int orc_series_term(const int L[4], const int os[4], const int es[4], const double *Ssd, const int ob[4],
                    const int eb[4], const double *Sbd, double *Td, int ncol) {
    lat_t lat;
    box_t bs, bb;
    if (set_lat(&lat, L, 1) || set_box(&bs, &lat, os, es) || set_box(&bb, &lat, ob, eb)) return 1;
    for (int64_t l = 0; l < bs.n; l++) { /* containment check */
        int k[4], x[4], kb[4];
        loc_coords(&bs, l, k);
        glob_coords(&lat, &bs, k, x);
        if (!local_of_global(&lat, &bb, x, kb)) return 1;
    }
    const cplx *Ss = (const cplx *)Ssd, *Sb = (const cplx *)Sbd;
    cplx *T = (cplx *)Td;
    for (int c = 0; c < ncol; c++)
        for (int64_t l = 0; l < bb.n; l++) {
            int k[4], x[4], ks[4];
            loc_coords(&bb, l, k);
            glob_coords(&lat, &bb, k, x);
            int in_small = local_of_global(&lat, &bs, x, ks);
            int64_t ls = in_small ? loc_index(&bs, ks) : -1;
            for (int i = 0; i < 12; i++) {
                cplx v = Sb[((int64_t)c * bb.n + l) * 12 + i];
                if (in_small) v -= Ss[((int64_t)c * bs.n + ls) * 12 + i];
                T[((int64_t)c * bb.n + l) * 12 + i] = v;
            }
        }
    return 0;
}

/* ----------------------------------------------------------- contractions */

/* S(y,x)_{rho a, sigma b} from 12 point-source columns: column 3 sigma + b. */
static inline cplx Sel(const cplx *S, int64_t n, int64_t l, int rho, int a, int sigma, int b) {
    return S[((int64_t)(3 * sigma + b) * n + l) * 12 + rho * 3 + a];
}

/* Local disconnected trace t(x) = sum_{alpha a} [gamma_5 S(x,x)]_{alpha a, alpha a}
 * at the point source x (the traces in Eq. W0, Sec. 3).  out: complex. */
int orc_contract_local_trace(const int L[4], const int o[4], const int e[4], const double *Sd, const int src[4],
                             double *out) {
    lat_t lat;
    box_t b;
    if (set_lat(&lat, L, 1) || set_box(&b, &lat, o, e)) return 1;
    int k[4];
    if (!local_of_global(&lat, &b, src, k)) return 1;
    int64_t l = loc_index(&b, k);
    cplx g[5][4][4];
    make_gamma(g);
    const cplx *S = (const cplx *)Sd;
    cplx t = 0;
    for (int al = 0; al < 4; al++)
        for (int a = 0; a < 3; a++)
            for (int r = 0; r < 4; r++) t += g[4][al][r] * Sel(S, b.n, l, r, a, al, a);
    out[0] = creal(t);
    out[1] = cimag(t);
    return 0;
}

/* Connected pseudoscalar contraction with S in place of S^(f) (Eq. W0pc, Sec. 4):
 * C(y0) = sum_{y vec} tr{S(y,x) S(y,x)^+}.  out[L0] real, indexed by global y0;
 * time slices outside the box are 0. */
int orc_contract_pion(const int L[4], const int o[4], const int e[4], const double *Sd, double *out) {
    lat_t lat;
    box_t b;
    if (set_lat(&lat, L, 1) || set_box(&b, &lat, o, e)) return 1;
    const cplx *S = (const cplx *)Sd;
    for (int t = 0; t < lat.L[0]; t++) out[t] = 0;
    for (int64_t l = 0; l < b.n; l++) {
        int k[4], x[4];
        loc_coords(&b, l, k);
        glob_coords(&lat, &b, k, x);
        double s = 0;
        for (int c = 0; c < 12; c++)
            for (int i = 0; i < 12; i++) {
                cplx v = S[((int64_t)c * b.n + l) * 12 + i];
                s += creal(v) * creal(v) + cimag(v) * cimag(v);
            }
        out[x[0]] += s;
    }
    return 0;
}

static const int EPS_PERM[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
static const double EPS_SIGN[6] = {1, 1, 1, -1, -1, -1};

/* Nucleon two-point function of Sec. 4 for one point source with u = d = S:
 *   C_N(y0) = sum_{y vec} [W_N1(y,x) - W_N2(y,x)],
 *   W_N1 = tr[S^{ag T} C g5 S^{bf} C g5] tr[S^{ce} P-] eps^{abc} eps^{feg},
 *   W_N2 = tr[S^{ag T} C g5 S^{be} P- S^{cf} C g5] eps^{abc} eps^{feg},
 * with C = i g0 g2, P- = (1 - g0)/2 and S^{ab} the 4x4 spin block at colours
 * (a, b); both contractions are read with arguments (y,x).  out[L0] complex. */
int orc_contract_nucleon(const int L[4], const int o[4], const int e[4], const double *Sd, double *out) {
    lat_t lat;
    box_t b;
    if (set_lat(&lat, L, 1) || set_box(&b, &lat, o, e)) return 1;
    cplx g[5][4][4], C[4][4], Cg5[4][4], Pm[4][4], t1[4][4];
    make_gamma(g);
    matmul4(g[0], g[2], t1);
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) C[i][j] = I * t1[i][j];
    matmul4(C, g[4], Cg5);
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) Pm[i][j] = 0.5 * ((i == j ? 1.0 : 0.0) - g[0][i][j]);
    const cplx *S = (const cplx *)Sd;
    cplx *acc = calloc(lat.L[0], sizeof(cplx));
    for (int64_t l = 0; l < b.n; l++) {
        int k[4], x[4];
        loc_coords(&b, l, k);
        glob_coords(&lat, &b, k, x);
        cplx blk[3][3][4][4]; /* blk[a][b][rho][sigma] = S(y,x)_{rho a, sigma b} */
        for (int a = 0; a < 3; a++)
            for (int bb = 0; bb < 3; bb++)
                for (int r = 0; r < 4; r++)
                    for (int s = 0; s < 4; s++) blk[a][bb][r][s] = Sel(S, b.n, l, r, a, s, bb);
        cplx W1 = 0, W2 = 0;
        for (int p1 = 0; p1 < 6; p1++)
            for (int p2 = 0; p2 < 6; p2++) {
                int a = EPS_PERM[p1][0], bq = EPS_PERM[p1][1], c = EPS_PERM[p1][2];
                /* eps^{feg}: (f, e, g) runs over the permutations */
                int f = EPS_PERM[p2][0], ee = EPS_PERM[p2][1], gg = EPS_PERM[p2][2];
                double sg = EPS_SIGN[p1] * EPS_SIGN[p2];
                cplx At[4][4], m1[4][4], m2[4][4], m3[4][4], m4[4][4];
                for (int i = 0; i < 4; i++)
                    for (int j = 0; j < 4; j++) At[i][j] = blk[a][gg][j][i]; /* S^{ag T} */
                /* W_N1 */
                matmul4(At, Cg5, m1);
                matmul4(m1, blk[bq][f], m2);
                matmul4(m2, Cg5, m3);
                cplx tr1 = 0, tr2 = 0;
                for (int i = 0; i < 4; i++) tr1 += m3[i][i];
                matmul4(blk[c][ee], Pm, m4);
                for (int i = 0; i < 4; i++) tr2 += m4[i][i];
                W1 += sg * tr1 * tr2;
                /* W_N2 */
                matmul4(m1, blk[bq][ee], m2);
                matmul4(m2, Pm, m3);
                matmul4(m3, blk[c][f], m4);
                matmul4(m4, Cg5, m2);
                cplx tr3 = 0;
                for (int i = 0; i < 4; i++) tr3 += m2[i][i];
                W2 += sg * tr3;
            }
        acc[x[0]] += W1 - W2;
    }
    for (int t = 0; t < lat.L[0]; t++) {
        out[2 * t] = creal(acc[t]);
        out[2 * t + 1] = cimag(acc[t]);
    }
    free(acc);
    return 0;
}

/* Stochastic estimate of the time-slice trace of Sec. 5 (without the hopping
 * expansion): T(x0) = sum_{x vec} sum_c eta_c(x)^+ gamma_5 psi_c(x), with
 * psi_c = D_Gamma^-1 eta_c.  out[L0] complex by global x0. */
int orc_contract_noise_trace(const int L[4], const int o[4], const int e[4], const double *etad, const double *psid,
                             int ncol, double *out) {
    lat_t lat;
    box_t b;
    if (set_lat(&lat, L, 1) || set_box(&b, &lat, o, e)) return 1;
    cplx g[5][4][4];
    make_gamma(g);
    const cplx *eta = (const cplx *)etad, *psi = (const cplx *)psid;
    cplx *acc = calloc(lat.L[0], sizeof(cplx));
    for (int c = 0; c < ncol; c++)
        for (int64_t l = 0; l < b.n; l++) {
            int k[4], x[4];
            loc_coords(&b, l, k);
            glob_coords(&lat, &b, k, x);
            const cplx *et = eta + ((int64_t)c * b.n + l) * 12, *ps = psi + ((int64_t)c * b.n + l) * 12;
            cplx s = 0;
            for (int al = 0; al < 4; al++)
                for (int a = 0; a < 3; a++) {
                    cplx gp = 0;
                    for (int r = 0; r < 4; r++) gp += g[4][al][r] * ps[r * 3 + a];
                    s += conj(et[al * 3 + a]) * gp;
                }
            acc[x[0]] += s;
        }
    for (int t = 0; t < lat.L[0]; t++) {
        out[2 * t] = creal(acc[t]);
        out[2 * t + 1] = cimag(acc[t]);
    }
    free(acc);
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Two-level factorized correlator (Sec. 3, Eq. factsing): the level-1 means of
 * the two regions' time-slice traces, multiplied and divided by L^3:
 *   C[y0][x0] = (1/L^3) (1/nA sum_v TA[v][x0]) (1/nB sum_w TB[w][y0]).
 * TA [nA][L0], TB [nB][L0], C [L0][L0], all complex. */
int orc_factorized_correlator(const double *TAd, int nA, const double *TBd, int nB, int L0, double vol3,
                              double *Cd) {
    if (nA < 1 || nB < 1 || L0 < 1 || !(vol3 > 0)) return 1;
    const cplx *TA = (const cplx *)TAd, *TB = (const cplx *)TBd;
    cplx *C = (cplx *)Cd;
    for (int y0 = 0; y0 < L0; y0++)
        for (int x0 = 0; x0 < L0; x0++) {
            cplx a = 0, b = 0;
            for (int v = 0; v < nA; v++) a += TA[(int64_t)v * L0 + x0];
            for (int w = 0; w < nB; w++) b += TB[(int64_t)w * L0 + y0];
            C[(int64_t)y0 * L0 + x0] = (a / nA) * (b / nB) / vol3;
        }
    return 0;
}
