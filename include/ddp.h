/*
 * ddp.h - C ABI of libddp: domain-restricted Wilson-Dirac quark propagators
 * and their Wick contractions on one NVIDIA GB300 (sm_103a).
 *
 * The library computes the propagators S^(i) = D_{Gamma_i}^{-1} of the
 * Wilson-Dirac operator restricted to a box-shaped domain Gamma_i with
 * Dirichlet faces (Sec. 2, Eq. blkdec and Eq. diric of Ce, Giusti, Schaefer,
 * "Domain decomposition, multi-level integration and exponential noise
 * reduction in lattice QCD"), the terms of the telescoping series
 * S = S^(0) + sum_i [S^(i) - S^(i-1)] (Sec. 1, Eq. Dseries) and the Wick
 * contractions that consume them (Sec. 3 Eq. W0, Sec. 4 Eq. W0pc and the
 * nucleon two-point function, Sec. 5 Eq. factsing).
 *
 * Operator (App. A): D = D_w + m0, 2 kappa D = 1 - kappa D_hop (Sec. 5), i.e.
 *   (D psi)(y) = psi(y)/(2 kappa)
 *              - 1/2 sum_mu [ (1 - g_mu) U_mu(y) psi(y+mu) + (1 + g_mu) U_mu(y-mu)^+ psi(y-mu) ].
 * D_Gamma drops every term that involves a site outside the domain.
 *
 * Conventions shared by every call
 *  - Lattice L0 x L1 x L2 x L3, direction 0 is time, every L_mu even and >= 2.
 *    Global site index ((x0*L1 + x1)*L2 + x2)*L3 + x3.
 *  - Complex numbers are interleaved (re, im) doubles.
 *  - Gauge field U[mu][site][row][col] (4*V*9 complex).  Links must be SU(3)
 *    (unitary, det 1, to 1e-8): the low-precision copies keep two rows and
 *    rebuild the third.
 *  - A domain is a box {(o_mu + k_mu) mod L_mu : 0 <= k_mu < e_mu}.  If
 *    e_mu == L_mu the direction is not restricted and the global boundary
 *    condition holds; otherwise both faces are Dirichlet.  Boxes may wrap
 *    around the lattice.  e_3 must be even.  Domain-local site order is
 *    lexicographic in k with the nesting of the global index.
 *  - Spinor fields are [ncol][n_sites][spin 4][colour 3] complex in
 *    domain-local order.  The 12 columns of a point-source propagator are
 *    ordered c = 3*spin + colour: S(y,x)_{alpha a, beta b} = S_out[3 beta + b][y][alpha][a].
 *  - Gamma matrices (Euclidean, chiral basis): g_0 = [[0,1],[1,0]],
 *    g_k = [[0,-i s_k],[i s_k,0]], g_5 = g_0 g_1 g_2 g_3.
 *  - Ownership: the caller owns every input and output buffer.  Buffers may
 *    be device memory or host memory (detected per pointer); the library never
 *    frees or retains them after a call returns.  ddp_load_gauge copies.
 *  - Calls are ordered on the context's CUDA stream.  Calls that return a
 *    status that depends on device results (solves, contractions to host
 *    memory) synchronise that stream before returning.
 *  - Every call returns a ddp_status.  On error, outputs are unspecified
 *    unless stated otherwise, and the context stays usable.
 */
#ifndef DDP_H
#define DDP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DDP_OK = 0,
    DDP_ERR_INVALID_ARG = 1,   /* bad size, box, source, kappa, id or non-SU(3)/non-finite links */
    DDP_ERR_UNSUPPORTED = 2,   /* odd lattice extent, odd e_3, csw != 0 when serving */
    DDP_ERR_OOM = 3,           /* device allocation failed or over the context's memory budget */
    DDP_ERR_NOT_CONVERGED = 4, /* a solve missed its tolerance within the iteration caps */
    DDP_ERR_CUDA = 5,          /* a CUDA runtime error (message in ddp_last_error) */
    DDP_ERR_BUSY = 6,          /* serving: no slot or memory free now, retry later */
    DDP_ERR_NOT_FOUND = 7      /* unknown gauge, domain or ticket id */
} ddp_status;

typedef enum { DDP_BC_PERIODIC = 0, DDP_BC_ANTIPERIODIC = 1, DDP_BC_OPEN = 2 } ddp_time_bc;

/* Arithmetic of a solve.  FP64: every vector and link in FP64 (the plain
 * path).  MIXED_*: inner Krylov iterations in FP32 arithmetic on FP32 / FP16
 * (per-site scaled spinors) / BF16 storage of spinors and 2-row links; the
 * true residual, the accumulation of the solution and the norms that decide
 * convergence are FP64 (defect correction). */
typedef enum {
    DDP_PREC_FP64 = 0,
    DDP_PREC_MIXED_FP32 = 1,
    DDP_PREC_MIXED_FP16 = 2,
    DDP_PREC_MIXED_BF16 = 3
} ddp_precision;

typedef enum {
    DDP_CONTRACT_PSEUDO_LOCAL = 0, /* tr{g5 S(x,x)} at the point source (Eq. W0), C_out[0] */
    DDP_CONTRACT_PSEUDO_NOISE = 1, /* sum_{x vec} sum_c eta_c^+ g5 psi_c per time slice (Sec. 5) */
    DDP_CONTRACT_NUCLEON = 2,      /* sum_{y vec} [W_N1 - W_N2](y,x) per time slice (Sec. 4) */
    DDP_CONTRACT_PION = 3          /* sum_{y vec} tr{S S^+}(y,x) per time slice (Eq. W0pc) */
} ddp_contract_kind;

#define DDP_INFO_COLS 12

typedef struct {
    int status;             /* DDP_OK or DDP_ERR_NOT_CONVERGED */
    int ncol;
    int outer_cycles;       /* FP64 true-residual recomputations */
    int inner_iters;        /* BiCGStab iterations summed over outer cycles (max over columns) */
    double max_rel_residual;                    /* max over columns of |eta - D_Gamma psi| / |eta| (FP64) */
    double rel_residual[DDP_INFO_COLS];         /* per column, first DDP_INFO_COLS columns */
    double seconds;         /* wall time of the call */
    int64_t column_iters;   /* BiCGStab iterations summed over columns and outer cycles */
} ddp_solve_info;

typedef struct ddp_ctx ddp_ctx;

/* Text of a status code (static storage). */
const char *ddp_error_string(int status);
/* Text of the last CUDA error seen by this context (static per context). */
const char *ddp_last_error(const ddp_ctx *ctx);
int ddp_version(void);

/* Create a context on CUDA device `device`, ordered on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The context owns all
 * internal device memory. */
int ddp_create(ddp_ctx **ctx, int device, void *cuda_stream);
int ddp_destroy(ddp_ctx *ctx);
int ddp_set_stream(ddp_ctx *ctx, void *cuda_stream);

/* Gauge field U_mu(x), the link variables of App. A.  Copies U (host or
 * device, [4][V][3][3] complex) into a resident FP64 copy plus 2-row FP32,
 * FP16 and BF16 copies in an even-odd site order.  time_bc: ddp_time_bc.
 * Rejects non-finite or non-SU(3) links with DDP_ERR_INVALID_ARG. */
int ddp_load_gauge(ddp_ctx *ctx, const double *U, const int L[4], int time_bc, int *gauge_id);

/* A level-1 variant (Sec. 3 two-level integration): a new gauge field equal
 * to base_gauge_id except for the links U_mu(x) with x in the box, which are
 * replaced by U_box[4][n_box][3][3] (box-local order).  Used to re-solve
 * domain propagators for updates of the links inside one region. */
int ddp_load_gauge_region(ddp_ctx *ctx, int base_gauge_id, const int origin[4], const int extent[4],
                          const double *U_box, int *gauge_id);
int ddp_free_gauge(ddp_ctx *ctx, int gauge_id);

/* Domain Gamma (Sec. 2): a box on a loaded gauge field. */
int ddp_set_domain(ddp_ctx *ctx, int gauge_id, const int origin[4], const int extent[4], int *domain_id);
int ddp_free_domain(ddp_ctx *ctx, int domain_id);

/* Index maps of a domain, computed on the device: for each domain-local
 * site, its global site index and its even-odd index (rank among the
 * domain's sites of the same global parity, in domain-local order).  Output
 * pointers may be NULL. */
int ddp_domain_sites(ddp_ctx *ctx, int domain_id, int64_t *n_sites, int64_t *global_index_out,
                     int64_t *eo_index_out);

/* out = D_Gamma psi for ncol columns (App. A, Sec. 2).  precision FP64 uses
 * the FP64 links; the MIXED_* values apply the low-precision stencil of the
 * inner solver (FP32 arithmetic on the stored copies).  csw != 0 adds the
 * O(a)-improvement (clover) term c_sw (i/4) sum_{mu,nu} sigma_{mu nu} F_{mu nu}(x)
 * with the clover-leaf field strength F = (Q_{mu nu} - Q_{nu mu}) / 8 of the whole
 * gauge field (the improved operator the footnotes of Sec. 4 and Sec. 5 refer to);
 * the term is site-local, so D_Gamma keeps it at every site of the domain. */
int ddp_apply_dirac(ddp_ctx *ctx, int domain_id, double kappa, double csw, const double *psi, double *out, int ncol,
                    int precision);

/* out = (kappa D_hop)^p psi on the domain, in FP64: p applications of the
 * hopping term of D_Gamma (the Dirichlet-masked stencil of Sec. 2, with
 * 2 kappa D = 1 - kappa D_hop of Sec. 5), each scaled by kappa.  This is the
 * operator of the hopping-parameter-expanded trace, Eq. HPEtr:
 * tr{g5 D^-1} = kappa^p tr{g5 D_hop^p D^-1} for p <= 8.  With
 * psi = D_Gamma^-1 g5 eta (ddp_solve_sources) and p = 8,
 * ddp_contract(DDP_CONTRACT_PSEUDO_NOISE, out, eta = g5 eta) is the expanded
 * stochastic estimator of sum_x tr{g5 D^-1(x,x)} per time slice, because
 * (g5 eta)^+ g5 v = eta^+ v.
 * psi, out: [ncol][n_sites][4][3] complex, domain-local lexicographic order,
 * host or device memory (may not alias).  p = 0 copies psi.
 * DDP_ERR_INVALID_ARG for kappa <= 0, p < 0, p > 64 or ncol < 1;
 * DDP_ERR_NOT_FOUND for an unknown domain.  Returns when out is complete. */
int ddp_hop_power(ddp_ctx *ctx, int domain_id, double kappa, int p, const double *psi, double *out, int ncol);

/* Domain propagator S^(i)(y,x) = D_Gamma^{-1}(y,x) (Eq. diric) for the 12
 * spin-colour point sources at global site src (which must lie in the
 * domain).  Stops when every column has |eta - D_Gamma psi|_2 / |eta|_2 <= tol
 * (FP64, unpreconditioned operator).  csw != 0 solves with the clover term
 * (see ddp_apply_dirac): the even-odd inner operator becomes
 * 1 - kappa^2 T_ee^-1 H_eo T_oo^-1 H_oe with T = 1 + 2 kappa C the site-local
 * part of 2 kappa D; T and T^-1 are built once per (gauge field, kappa, c_sw) and
 * kept with the gauge field (the 4 most recently used pairs; one call may use at
 * most 4 distinct pairs, else DDP_ERR_UNSUPPORTED).  DDP_ERR_INVALID_ARG if T is
 * singular at some site.
 * S_out: [12][n_sites][4][3].  On DDP_ERR_NOT_CONVERGED S_out holds the best
 * iterate and info the residuals.  info may be NULL. */
int ddp_solve_propagator(ddp_ctx *ctx, int domain_id, double kappa, double csw, const int src[4], double tol,
                         int precision, double *S_out, ddp_solve_info *info);

/* psi_c = D_Gamma^{-1} eta_c for ncol arbitrary sources eta [ncol][n][4][3]. */
int ddp_solve_sources(ddp_ctx *ctx, int domain_id, double kappa, double csw, const double *eta, int ncol,
                      double tol, int precision, double *psi_out, ddp_solve_info *info);

/* One request of a batched solve. */
typedef struct {
    int domain_id;
    double kappa;
    double csw;          /* clover coefficient c_sw (0: plain Wilson; see ddp_apply_dirac) */
    int src[4];          /* point source (used when eta == NULL) */
    const double *eta;   /* NULL: 12 point-source columns at src; else ncol sources */
    int ncol;            /* 12 for point sources */
    double tol;
    double *out;         /* [ncol][n_sites][4][3] */
} ddp_solve_req;

/* Many independent domain solves (different domains, gauge fields, kappas)
 * in one device-driven launch sequence: all columns of all requests iterate
 * together inside a graph-captured loop.  All requests use `precision`.
 * infos: n entries or NULL.  Returns DDP_ERR_NOT_CONVERGED if any request
 * missed its tolerance (its info says which). */
int ddp_solve_batch(ddp_ctx *ctx, const ddp_solve_req *reqs, int n, int precision, ddp_solve_info *infos);

/* Series term T^(i) = S^(i) - E S^(i-1) on the big domain (Eq. Dseries), where
 * E extends S_small by zero outside the small domain; the small domain must
 * lie inside the big one.  S_small [ncol][n_small][4][3], S_big and T_out
 * [ncol][n_big][4][3]. */
int ddp_series_terms(ddp_ctx *ctx, int domain_small, const double *S_small, int domain_big, const double *S_big,
                     double *T_out, int ncol);

/* Boundary coupling of two domains of the same gauge field (Eq. blkdec):
 * sigma = -D[to, from \ to] psi, the terms of D that connect sites of the
 * `from` domain lying outside the `to` domain to sites of `to` -- exactly the
 * hops the Dirichlet boundary of `to` drops, with the gauge field's time
 * boundary condition.  With from = Gamma-bar_0, to = Gamma*_0 and
 * psi = D^{-1}_{Gamma-bar_0} eta (ddp_solve_propagator / ddp_solve_sources),
 * D^{-1}_{Gamma*_0} sigma (ddp_solve_sources) is the factorized propagator
 * S^(f) = -D^{-1}_{Gamma*_0} D_{dGamma*_0} D^{-1}_{Gamma-bar_0} of Eq. approxlong.
 * FP64.  psi [ncol][n_from][4][3], sigma [ncol][n_to][4][3] complex,
 * domain-local lexicographic order, host or device memory; psi and sigma must
 * not overlap.  Returns when sigma is complete.
 * DDP_ERR_INVALID_ARG for ncol < 1 or domains of different gauge fields. */
int ddp_boundary_source(ddp_ctx *ctx, int domain_from, const double *psi, int domain_to, double *sigma, int ncol);

/* The point-source propagators S^(i) = D_{Gamma_i}^{-1}(., x) of nested domains
 * Gamma_0 in Gamma_1 in ... in Gamma_{n-1} (Sec. 2, Eq. diric), solved in one
 * batch, the terms of their series T^(i) = S^(i) - E S^(i-1) (Sec. 1, Eq. Dseries)
 * and the point-source contractions of every S^(i) (Sec. 3 Eq. W0, Sec. 4), in one
 * call that keeps every intermediate on the device.
 *  - domain_ids: n domains of one gauge field, each inside the next (else
 *    DDP_ERR_INVALID_ARG); src must lie in Gamma_0.
 *  - S_out: n pointers (or NULL), entry i receives S^(i) as ddp_solve_propagator
 *    writes it, or is NULL when S^(i) is not wanted.  T_out: n-1 pointers (or
 *    NULL), entry i-1 receives T^(i) in the layout of ddp_series_terms.
 *  - contract_mask: bit k set for ddp_contract_kind k among PSEUDO_LOCAL, NUCLEON,
 *    PION (PSEUDO_NOISE needs sources: DDP_ERR_INVALID_ARG).  C_out holds
 *    n x 4 x 2*L0 doubles: the result of kind k for domain i at offset
 *    (4 i + k) 2 L0, in the layout of ddp_contract; other entries are untouched.
 *  - Outputs may be host or device memory (detected per pointer); host outputs
 *    are copied down on a second stream while the later kernels run, and
 *    nothing the call computed is uploaded again.  Device-resident copies live
 *    in the context until its next call of this function.
 *  - Returns DDP_ERR_NOT_CONVERGED (with every output written) when a solve missed
 *    tol; infos: n entries or NULL.  csw: as in ddp_solve_propagator. */
int ddp_propagator_series(ddp_ctx *ctx, int n, const int *domain_ids, double kappa, double csw, const int src[4],
                          double tol, int precision, double *const *S_out, double *const *T_out, int contract_mask,
                          double *C_out, ddp_solve_info *infos);

/* Wick contractions of a solved propagator on a domain.
 *  PSEUDO_LOCAL: S = 12 point-source columns, src = the source; C_out[2] = tr{g5 S(x,x)}.
 *  PSEUDO_NOISE: S = psi_c = D_Gamma^{-1} eta_c, eta = the ncol sources;
 *                C_out[2*L0] = sum_{x vec} sum_c eta_c^+ g5 psi_c by global time slice.
 *  NUCLEON:      S = 12 point-source columns, u = d = S, C = i g0 g2, P- = (1 - g0)/2;
 *                C_out[2*L0] = sum_{y vec} [W_N1 - W_N2](y, x).
 *  PION:         C_out[2*L0] = sum_{y vec} tr{S(y,x) S(y,x)^+} (imaginary parts 0).
 * Time slices outside the domain are 0.  C_out is host or device memory. */
int ddp_contract(ddp_ctx *ctx, int kind, int domain_id, const double *S, const double *eta, int ncol,
                 const int src[4], double *C_out);

/* Level-1 averaging of the two-level integration (Sec. 3, Eq. factsing): with
 * T_A[v][L0] and T_B[w][L0] the time-slice traces (complex) of region A for
 * nvar_A level-1 variants and of region B for nvar_B variants,
 *   C_out[y0][x0] = (1/L^3) * mean_v T_A^v(x0) * mean_w T_B^w(y0)
 * (complex, L0 x L0).  spatial_volume = L^3.  Buffers host or device. */
int ddp_factorized_correlator(ddp_ctx *ctx, const double *T_A, int nvar_A, const double *T_B, int nvar_B, int L0,
                              double spatial_volume, double *C_out);

/* ---- serving: continuous batching of propagator solves ------------------
 * A server owns a fixed-capacity set of resident solver fields sized by its
 * memory budget.  ddp_submit admits a request at once if an active slot and
 * enough contiguous capacity are free, and returns DDP_ERR_BUSY otherwise
 * (retry after a ddp_serve_step has retired work).  Each ddp_serve_step runs
 * one defect-correction cycle (FP64 residual, inner BiCGStab loop, FP64
 * accumulation) for every active request in one launch sequence, so requests
 * admitted while others are running join them on the device; converged
 * requests are written to their output buffers and retire.  A request's
 * result equals the same request solved alone by ddp_solve_propagator /
 * ddp_solve_sources (bit for bit: per-request fixed-order reductions and
 * stopping criteria).  Gauge fields and domains must stay loaded while their
 * requests are in flight. */

/* Configure (or reconfigure, dropping all requests) the server: memory budget
 * in bytes for its resident fields (0 = 80% of free device memory), the
 * maximum number of active requests and the storage format of the solves.
 * DDP_ERR_OOM if the budget cannot hold a useful capacity. */
int ddp_serve_config(ddp_ctx *ctx, uint64_t mem_budget_bytes, int max_active, int precision);
/* Admit a request (eta and out must be device memory; at most 16 columns).
 * DDP_ERR_BUSY: no slot or capacity free now; DDP_ERR_OOM: larger than the
 * server's whole capacity.  ticket receives an id on DDP_OK. */
int ddp_submit(ddp_ctx *ctx, const ddp_solve_req *req, uint64_t *ticket);
/* Run one cycle for all active requests (blocking until it is done);
 * *in_flight receives the number of requests still active. */
int ddp_serve_step(ddp_ctx *ctx, int *in_flight);
/* done = 1 when the request has retired; its output buffer is then complete
 * and info holds its residuals and latency (seconds from submit to retire).
 * A finished ticket is forgotten after it has been polled once. */
int ddp_poll(ddp_ctx *ctx, uint64_t ticket, int *done, ddp_solve_info *info);

/* ---- tuning and measurement ---------------------------------------------- */

/* Solver knobs: "max_outer" (defect-correction cycles), "max_inner"
 * (BiCGStab iterations per cycle), "delta_fp64" / "delta_fp32" /
 * "delta_fp16" / "delta_bf16" (smallest inner relative tolerance per storage
 * format), "tile_sites" (sites per block tile: 32; 0 = automatic),
 * "tile_cols" (columns per block, 1..12, 0 = automatic), "tuned_cols_fp64" ...
 * "tuned_cols_bf16" (a remembered autotuner choice, 0 = none), "tuned_carveout_fp64" ...
 * "tuned_carveout_bf16" (the autotuner's stencil carveout for that storage format,
 * percent, -1 = the driver's choice, -2 = none: "stencil_carveout" applies), "conditional" (1: the
 * inner loop is a device-driven CUDA-graph WHILE node; 0: host-polled graph
 * chunks), "stencil_carveout" (preferred shared-memory share of the unified L1 /
 * shared memory for the inner-loop stencils, percent; default 28, -1 = the driver's
 * choice), "contraction_double_fp32" (1, the default: the nucleon contraction of
 * ddp_contract in double-FP32 arithmetic, relative error about 1e-13; 0: FP64),
 * "projector_tensor_cores" (1, the default: the Gram blocks and colourless
 * spinor sums of the projector cut, m <= 128, run as an emulated-FP64 product on the
 * tensor cores and the Cholesky-QR update A <- A R^-1 in double-FP32; 0: direct FP64
 * kernels), "overlap_downloads" (1, the default: ddp_propagator_series with host
 * outputs solves the smaller nested domains first and copies their results to the host
 * while the largest domain solves; 0: one batched solve, then the copies).
 * DDP_ERR_INVALID_ARG for unknown names or values. */
int ddp_set_param(ddp_ctx *ctx, const char *name, double value);

/* *value = the current value of a parameter ddp_set_param accepts ("delta_fp64" ...
 * "delta_bf16" for the inner tolerance floors).  DDP_ERR_INVALID_ARG for unknown
 * names. */
int ddp_get_param(const ddp_ctx *ctx, const char *name, double *value);

/* Inner-loop stencil variants, for ddp_time_hop: one BiCGStab iteration on the
 * even-odd Schur complement runs PLAIN twice and each SCHUR variant once. */
typedef enum {
    DDP_HOP_PLAIN = 0,        /* tmp = H_oe p (odd output sites) */
    DDP_HOP_SCHUR_RHAT = 1,   /* v = p - kappa^2 H_eo tmp, with the (rh, v) partial sums */
    DDP_HOP_SCHUR_TS = 2      /* t = s - kappa^2 H_eo tmp, with the (t, s), (t, t) partial sums */
} ddp_hop_kernel;

/* Average duration (ms) of one inner-loop stencil variant (ddp_hop_kernel) on
 * a domain with ncol columns in the given storage format, timed with CUDA
 * events over `iters` launches on the context's stream after 3 warm-up
 * launches; bytes_per_launch receives the variant's algorithmic HBM bytes:
 * the spinors it reads or writes once per output site-column (2 for PLAIN,
 * 4 for SCHUR_RHAT, of which the shadow residual rh is counted in its own
 * storage: BF16 for FP32 storage, 3 for SCHUR_TS) plus the 8 links touching
 * every output site once for all columns. */
int ddp_time_hop(ddp_ctx *ctx, int domain_id, double kappa, int ncol, int precision, int kernel, int iters,
                 float *ms_per_launch, double *bytes_per_launch);

/* Autotuner: times the three inner-loop stencil variants on the domain (ncol
 * columns, the given storage format, iters launches each) for every admissible
 * number of columns per thread block (the block shape, 32 sites x columns) and
 * every candidate shared-memory carveout of the stencils (28, 50, 100 percent of the
 * unified L1 / shared memory), keeps the pair with the shortest stencil time per
 * BiCGStab iteration (2 x PLAIN + SCHUR_RHAT + SCHUR_TS) for that storage format in
 * the context (used by every later solve with that format; ddp_get_param
 * "tuned_cols_<format>" and "tuned_carveout_<format>" read it back) and returns the
 * columns with that time. */
int ddp_autotune(ddp_ctx *ctx, int domain_id, double kappa, int ncol, int precision, int iters, int *best_cols,
                 float *best_ms);

/* Number of kernels this context has launched so far. */
long ddp_kernel_launches(const ddp_ctx *ctx);

/* Clears the serving state (pending and finished requests). */
int ddp_serve_reset(ddp_ctx *ctx);

/* ---- projector-cut factorization (Sec. 5) ------------------------------------
 * The factorized propagator of Eq. approxlong with the projector P = sum_i phi_i
 * phi_i^+ on N_m orthonormal vectors inserted at the cut (Eq. proj, approxlong2):
 *   S~(y, x) = -sum_i [D^-1_{G*} D_dG* phi_i](y) [phi_i^+ D^-1_{Gbar}](x).
 * A caller builds it from these calls and the solves above:
 *   phi  = ddp_inverse_iteration on the thick slice Omega at the cut,
 *   u_i  = D^-1_{Gbar} g5 phi_i      (ddp_embed with gamma5 = 1, ddp_solve_sources),
 *   w_i  = D^-1_{G*} sigma_i,  sigma_i = ddp_boundary_source(Omega -> G*, phi_i),
 *   pion:    M = ddp_gram_slices(Gbar, u), M~ = ddp_gram_slices(G*, w),
 *            ddp_projected_pion(M~, M)                         (Eq. Bpions, fullfactpi),
 *   nucleon: X = ddp_colourless_slices(Gbar, u, form 1), Y = ddp_colourless_slices(G*, w,
 *            form 2), ddp_projected_nucleon(X, Y)              (Eq. W0tbary).
 * Fields: [m][n_sites][4][3] complex in domain-local order, host or device memory
 * (detected per pointer); every call returns when its output is complete.
 * Gram blocks and colourless sums (m <= 128: the paper's N_m = 120 modes fit) run on the
 * tensor cores: every operand is
 * split into seven 7-bit integer slices under a power-of-two exponent per row or
 * column, the slice products are summed exactly, and each term of a sum is exact to
 * about 2^-47 of its row maximum times its column maximum (FP64-level; the parameter
 * "projector_tensor_cores" = 0 selects direct FP64 kernels, the colourless sums for
 * m <= 32 only).  A NaN or infinity in an
 * input makes exactly the outputs of its time slice that depend on it NaN. */

/* V <- the orthonormal basis of span(V) that Gram-Schmidt in column order gives
 * (Cholesky QR, twice, in FP64).  DDP_ERR_INVALID_ARG if the columns are linearly
 * dependent or m > 12 n_sites. */
int ddp_orthonormalize(ddp_ctx *ctx, int domain_id, double *V, int m);

/* Subspace inverse iteration of the Dirichlet operator of the domain (Sec. 5: 10
 * iterations on random vectors): V <- orthonormalize(V), then `iters` times
 * V <- orthonormalize(D_Gamma^-1 V), each solve to the relative residual tol in
 * `precision` (ddp_solve_sources).  V: m columns in, the orthonormal vectors out;
 * info: as ddp_solve_sources for the last solve (may be NULL).  Returns
 * DDP_ERR_NOT_CONVERGED (V still written) if a solve missed tol. */
int ddp_inverse_iteration(ddp_ctx *ctx, int domain_id, double kappa, double csw, double *V, int m, int iters,
                          double tol, int precision, ddp_solve_info *info);

/* out = E psi (times gamma_5 when gamma5 != 0): the ncol columns of the `from`
 * domain extended by zero to the `to` domain, which must contain it. */
int ddp_embed(ddp_ctx *ctx, int domain_from, const double *psi, int domain_to, double *out, int ncol, int gamma5);

/* M[t][i][j] = sum_{x vec at global time t} sum_{spin, colour} conj(A_i(x)) A_j(x)
 * for the m columns of a domain: the time-slice sums of the pion blocks B_ij of
 * Eq. Bpions.  M_out: L0 x m x m complex; slices outside the domain are zero. */
int ddp_gram_slices(ddp_ctx *ctx, int domain_id, const double *A, int m, double *M_out);

/* X[t][i][j][k][alpha] = sum_{x vec at time t} B[s_i, s_j, s_k; x]_alpha, the
 * colourless spinors B[s_i, s_j, s_k; x]_alpha = eps^{abc} (s_i^a)^T C g5 s_j^b (s_k^c)_alpha
 * of Eq. W0tbary (C = i g0 g2) with s_i = A_i (form 0), g5 conj(A_i) (form 1: the
 * spinor of the row phi_i^+ D^-1 when A_i = D^-1 g5 phi_i) or -A_i (form 2).
 * X_out: L0 x m^3 x 4 complex.  m <= 128 on the tensor cores, m <= 32 with the direct
 * FP64 kernel (else DDP_ERR_UNSUPPORTED).  The tensor-core sums need scratch of about
 * (66 m^2 + 700 m) bytes per site of a time slice (14.5 GB at m = 120 on a 24^3 slice),
 * which the context keeps for later calls until ddp_destroy. */
int ddp_colourless_slices(ddp_ctx *ctx, int domain_id, const double *A, int m, int form, double *X_out);

/* C[y0][x0] = (1/L^3) sum_ij Mt[y0][i][j] M[x0][j][i] = (1/L^3) sum_{x vec, y vec} W~(y, x)
 * of Eq. fullfactpi.  Mt, M: L0 x m x m complex; C_out: L0 x L0 complex. */
int ddp_projected_pion(ddp_ctx *ctx, int L0, int m, const double *Mt, const double *M, double spatial_volume,
                       double *C_out);

/* C[y0][x0] = sum_{x vec, y vec} [W~_N1 - W~_N2](y, x) = sum_ijk [X_jik(x0) - X_kij(x0)]^T
 * P- Y_ijk(y0), P- = (1 - g0)/2: the nucleon contractions of Sec. 4 with S~
 * substituted (Eq. W0tbary; the paper prints -g5 P- between the spinors, which
 * corresponds to an x-side spinor with an extra -g5).  X, Y: L0 x m^3 x 4 complex
 * from ddp_colourless_slices; C_out: L0 x L0 complex.  Computed as the FP64 product
 * C = P D^T over the 4 m^3 (i, j, k, alpha) terms, split into chunks summed in a fixed
 * order; needs L0 x 4 m^3 complex of scratch (5.3 GB at m = 120, L0 = 48). */
int ddp_projected_nucleon(ddp_ctx *ctx, int L0, int m, const double *X, const double *Y, double *C_out);

/* ---- allocation-free contraction ------------------------------------------
 * The paper has no counterpart: this entry point exists for callers that
 * must not allocate device memory, for instance code running under another
 * runtime's memory manager (a framework's custom operator whose allocator
 * owns the device), or latency-critical loops where cudaMalloc/cudaFree
 * would synchronise the device.  It computes exactly what ddp_contract computes
 * (same kernels, same reduction order) without a context and without
 * allocating: the per-time-slice partial sums go to one fixed device array
 * of DDP_STATIC_PARTIALS_MAX double2 entries (2 MiB) that lives in the
 * library and stays held on every GPU that loads it until the process exits.
 *
 *  - S, eta (noise kind only) and C_out must be device (or managed) memory of
 *    the current device; host memory, pinned or not, and memory of another
 *    device are refused with DDP_ERR_INVALID_ARG before anything is enqueued.
 *    The caller also guarantees their sizes: S (and eta) hold ncol * n_sites *
 *    12 complex doubles (ncol = 12 except for PION and PSEUDO_NOISE), C_out
 *    2*L[0] doubles (2 for PSEUDO_LOCAL).  Geometry as in ddp_set_domain: an
 *    extent outside [1, L] is DDP_ERR_INVALID_ARG, an odd L[mu] or an odd
 *    extent[3] DDP_ERR_UNSUPPORTED.
 *  - A CUDA error already pending in the calling thread when the call starts
 *    is returned as DDP_ERR_CUDA and left pending (nothing is launched).
 *  - The partial sums need extent[0] * ceil(extent[1]*extent[2]*extent[3] / T)
 *    entries with T = 32 for NUCLEON and 128 otherwise; more than
 *    DDP_STATIC_PARTIALS_MAX returns DDP_ERR_INVALID_ARG and launches nothing.
 *  - The first call on a device looks up the device address of the array
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    before any stream capture.  Later calls only enqueue kernels on
 *    cuda_stream.  The address is kept for the life of the process and is
 *    valid for the device's primary context only: after cudaDeviceReset, or
 *    with another context current, do not call this entry point again.
 *  - All calls share the array.  Each call writes every entry it reads, so
 *    nothing has to be cleared between calls, but calls that may overlap on
 *    the GPU (different streams without ordering between them) race on it.
 *  - Returns DDP_OK once the kernels are enqueued; it does not synchronise. */
#define DDP_STATIC_PARTIALS_MAX (1 << 17)
int ddp_contract_static(int kind, const int L[4], const int origin[4], const int extent[4], const double *S,
                        const double *eta, int ncol, const int src[4], double *C_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* DDP_H */
