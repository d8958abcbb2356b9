"""CUDA path against the FP64 oracle, through the C ABI (GPU required).

Tolerances: index maps and series terms bit-exact; FP64 stencil 1e-13
relative L2 per column (summation order only); low-precision stencils at the
rounding level of their storage (FP32 1e-6, FP16 per-site scaled 4e-3, BF16
3e-2); propagator columns 1e-8 relative L2 at solver residual 1e-10 against
the oracle at 1e-12; correlators 1e-7 relative L2 over time slices.
"""
import numpy as np
import pytest

import oracle
from oracle import dense
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
AP = oracle.BC_ANTIPERIODIC

COL_TOL = 1e-8
CORR_TOL = 1e-7


@pytest.fixture(scope="module")
def ddp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_04587_gb300 import build
    build.build()
    import paper_1601_04587_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(ddp):
    c = ddp.ddp_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    ddp.ddp_destroy(c)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _col_errors(got, ref):
    return [_rel(got[c], ref[c]) for c in range(ref.shape[0])]


LAT = (8, 4, 4, 6)


@pytest.fixture(scope="module")
def field(ddp, ctx):
    U = synth.gauge_field(LAT, seed=1234)
    gid = ddp.ddp_load_gauge(ctx, torch.from_numpy(U).cuda(), LAT, ddp.DDP_BC_ANTIPERIODIC)
    return U, gid


BOXES = [((0, 0, 0, 0), LAT),                    # whole lattice
         ((6, 0, 0, 0), (4, 4, 4, 6)),           # time slab across the antiperiodic boundary
         ((5, 1, 3, 2), (3, 2, 3, 4)),           # Dirichlet in every direction, wrapped, odd extents
         ((2, 3, 0, 5), (5, 4, 2, 2)),
         ((1, 0, 0, 0), (8, 4, 4, 6)),           # full extent, shifted origin
         ((7, 3, 1, 5), (1, 1, 1, 2)),           # two sites: every hop but one dropped
         ((3, 0, 2, 0), (1, 4, 1, 6))]           # extent 1 in two directions


# ------------------------------------------------------------------ index maps

@pytest.mark.parametrize("box", BOXES)
def test_domain_maps_bit_exact(ddp, ctx, field, box):
    U, gid = field
    o, e = box
    did = ddp.ddp_set_domain(ctx, gid, o, e)
    n = int(np.prod(e))
    gi = np.zeros(n, dtype=np.int64)
    eo = np.zeros(n, dtype=np.int64)
    assert ddp.ddp_domain_sites(ctx, did, gi, eo) == n
    rg, reo, _ = oracle.domain_maps(LAT, o, e)
    assert np.array_equal(gi, rg)
    assert np.array_equal(eo, reo)


def test_odd_innermost_extent_rejected(ddp, ctx, field):
    U, gid = field
    with pytest.raises(ddp.DDPError) as ei:
        ddp.ddp_set_domain(ctx, gid, (0, 0, 0, 0), (4, 4, 4, 3))
    assert ei.value.status == ddp.DDP_ERR_UNSUPPORTED


# -------------------------------------------------------------------- stencil

@pytest.mark.parametrize("box", BOXES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 1e-6), (2, 4e-3), (3, 3e-2)])
def test_apply_dirac(ddp, ctx, field, box, prec, tol):
    U, gid = field
    o, e = box
    did = ddp.ddp_set_domain(ctx, gid, o, e)
    n = int(np.prod(e))
    psi = synth.random_spinor(3, n, 17)
    ref = oracle.apply_dirac(U, LAT, AP, o, e, 0.1315, psi)
    out = torch.zeros((3, n, 4, 3), dtype=torch.complex128, device="cuda")
    ddp.ddp_apply_dirac(ctx, did, 0.1315, torch.from_numpy(psi).cuda(), out, 3, prec)
    errs = _col_errors(out.cpu().numpy(), ref)
    assert max(errs) < tol, errs


@pytest.mark.parametrize("bc", [0, 2])
def test_apply_dirac_other_time_boundaries(ddp, ctx, bc):
    U = synth.gauge_field(LAT, seed=77)
    gid = ddp.ddp_load_gauge(ctx, torch.from_numpy(U).cuda(), LAT, bc)
    for o, e in BOXES[:3]:
        did = ddp.ddp_set_domain(ctx, gid, o, e)
        n = int(np.prod(e))
        psi = synth.random_spinor(1, n, 3)
        ref = oracle.apply_dirac(U, LAT, bc, o, e, 0.12, psi)
        out = np.zeros_like(psi)
        ddp.ddp_apply_dirac(ctx, did, 0.12, psi, out, 1, 0)   # host buffers
        assert _rel(out, ref) < 1e-13


# ----------------------------------------------------------------- propagators

@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("box,src", [(BOXES[0], (0, 0, 0, 0)), (BOXES[1], (7, 1, 2, 3)),
                                     (BOXES[2], (6, 2, 0, 5)), (BOXES[3], (4, 3, 1, 0))])
def test_solve_propagator(ddp, ctx, field, prec, box, src):
    U, gid = field
    o, e = box
    kappa = 0.124
    did = ddp.ddp_set_domain(ctx, gid, o, e)
    n = int(np.prod(e))
    ref, _, rr, st = oracle.propagator(U, LAT, AP, o, e, kappa, src, tol=1e-12)
    assert st == 0
    S = torch.zeros((12, n, 4, 3), dtype=torch.complex128, device="cuda")
    rc, info = ddp.ddp_solve_propagator(ctx, did, kappa, 0.0, src, 1e-10, prec, S)
    assert rc == ddp.DDP_OK, ddp.info_dict(info)
    assert info.max_rel_residual <= 1e-10
    errs = _col_errors(S.cpu().numpy(), ref)
    assert max(errs) < COL_TOL, errs


def test_solve_sources_host_buffers(ddp, ctx, field):
    U, gid = field
    o, e = BOXES[1]
    did = ddp.ddp_set_domain(ctx, gid, o, e)
    n = int(np.prod(e))
    eta = synth.random_spinor(5, n, 8)
    ref, _, rr, st = oracle.solve(U, LAT, AP, o, e, 0.125, eta, tol=1e-12)
    out = np.zeros_like(eta)
    rc, info = ddp.ddp_solve_sources(ctx, did, 0.125, 0.0, eta, 5, 1e-10, ddp.DDP_PREC_MIXED_FP32, out)
    assert rc == ddp.DDP_OK
    assert max(_col_errors(out, ref)) < COL_TOL


def test_batch_equals_individual_solves(ddp, ctx, field):
    """One batched launch over uneven domains gives bit-identical columns to the
    same requests solved one by one (fixed-order per-request reductions)."""
    U, gid = field
    reqs, outs, alone = [], [], []
    specs = [(BOXES[1], (7, 1, 2, 3), 0.124), (BOXES[2], (6, 2, 0, 5), 0.12), (BOXES[0], (3, 3, 3, 3), 0.122)]
    for (o, e), src, kappa in specs:
        did = ddp.ddp_set_domain(ctx, gid, o, e)
        n = int(np.prod(e))
        out = torch.zeros((12, n, 4, 3), dtype=torch.complex128, device="cuda")
        outs.append(out)
        reqs.append(ddp.make_req(did, kappa, src, 1e-10, out))
        one = torch.zeros_like(out)
        ddp.ddp_solve_propagator(ctx, did, kappa, 0.0, src, 1e-10, ddp.DDP_PREC_MIXED_FP32, one)
        alone.append(one)
    rc, infos = ddp.ddp_solve_batch(ctx, reqs, ddp.DDP_PREC_MIXED_FP32)
    assert rc == ddp.DDP_OK
    for out, one, ((o, e), src, kappa) in zip(outs, alone, specs):
        ref, *_ = oracle.propagator(U, LAT, AP, o, e, kappa, src, tol=1e-12)
        assert max(_col_errors(out.cpu().numpy(), ref)) < COL_TOL
        # per-request reductions in a fixed order: the batch does not change a bit
        assert torch.equal(out, one)


def test_not_converged_reported(ddp, ctx, field):
    U, gid = field
    did = ddp.ddp_set_domain(ctx, gid, (0, 0, 0, 0), LAT)
    n = int(np.prod(LAT))
    S = torch.zeros((12, n, 4, 3), dtype=torch.complex128, device="cuda")
    ddp.ddp_set_param(ctx, "max_outer", 1)
    ddp.ddp_set_param(ctx, "max_inner", 3)
    try:
        rc, info = ddp.ddp_solve_propagator(ctx, did, 0.124, 0.0, (0, 0, 0, 0), 1e-10, 1, S)
    finally:
        ddp.ddp_set_param(ctx, "max_outer", 40)
        ddp.ddp_set_param(ctx, "max_inner", 30000)
    assert rc == ddp.DDP_ERR_NOT_CONVERGED
    assert info.max_rel_residual > 1e-10
    assert np.isfinite(S.cpu().numpy()).all()


def test_invalid_arguments(ddp, ctx, field):
    U, gid = field
    did = ddp.ddp_set_domain(ctx, gid, BOXES[1][0], BOXES[1][1])
    n = int(np.prod(BOXES[1][1]))
    S = torch.zeros((12, n, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(ddp.DDPError) as ei:
        ddp.ddp_solve_propagator(ctx, did, 0.12, float("nan"), (7, 0, 0, 0), 1e-10, 0, S)
    assert ei.value.status == ddp.DDP_ERR_INVALID_ARG      # clover coefficient not finite
    with pytest.raises(ddp.DDPError) as ei:
        ddp.ddp_solve_propagator(ctx, did, 0.12, 0.0, (3, 0, 0, 0), 1e-10, 0, S)
    assert ei.value.status == ddp.DDP_ERR_INVALID_ARG      # source outside the domain
    bad = U.copy()
    bad[2, 5, 1, 1] = np.nan
    with pytest.raises(ddp.DDPError) as ei:
        ddp.ddp_load_gauge(ctx, bad, LAT, 1)
    assert ei.value.status == ddp.DDP_ERR_INVALID_ARG
    nonunitary = U.copy()
    nonunitary[0, 0] *= 1.01
    with pytest.raises(ddp.DDPError):
        ddp.ddp_load_gauge(ctx, nonunitary, LAT, 1)
    with pytest.raises(ddp.DDPError):
        ddp.ddp_load_gauge(ctx, U, (8, 4, 4, 5), 1)


# ------------------------------------------------------------- series + contractions

def test_series_terms_bit_exact(ddp, ctx, field):
    U, gid = field
    src = (7, 1, 2, 3)
    small, big = ((6, 0, 0, 0), (4, 4, 4, 6)), ((5, 0, 0, 0), (6, 4, 4, 6))
    ds = ddp.ddp_set_domain(ctx, gid, *small)
    db = ddp.ddp_set_domain(ctx, gid, *big)
    Ss, *_ = oracle.propagator(U, LAT, AP, *small, 0.124, src)
    Sb, *_ = oracle.propagator(U, LAT, AP, *big, 0.124, src)
    T = torch.zeros(Sb.shape, dtype=torch.complex128, device="cuda")
    ddp.ddp_series_terms(ctx, ds, torch.from_numpy(Ss).cuda(), db, torch.from_numpy(Sb).cuda(), T, 12)
    ref = oracle.series_term(LAT, small[0], small[1], Ss, big[0], big[1], Sb)
    assert np.array_equal(T.cpu().numpy(), ref)


def test_series_rejects_non_nested(ddp, ctx, field):
    U, gid = field
    ds = ddp.ddp_set_domain(ctx, gid, (0, 0, 0, 0), (4, 4, 4, 6))
    db = ddp.ddp_set_domain(ctx, gid, (2, 0, 0, 0), (4, 4, 4, 6))
    S = np.zeros((12, 384, 4, 3), dtype=np.complex128)
    with pytest.raises(ddp.DDPError):
        ddp.ddp_series_terms(ctx, ds, S, db, S.copy(), S.copy(), 12)


@pytest.mark.parametrize("box,src", [(BOXES[0], (0, 0, 0, 0)), (BOXES[1], (7, 1, 2, 3)), (BOXES[2], (6, 2, 0, 5))])
def test_contractions(ddp, ctx, field, box, src):
    U, gid = field
    o, e = box
    did = ddp.ddp_set_domain(ctx, gid, o, e)
    S, *_ = oracle.propagator(U, LAT, AP, o, e, 0.124, src)
    Sd = torch.from_numpy(S).cuda()
    C = np.zeros(2 * LAT[0])
    ddp.ddp_contract(ctx, ddp.DDP_CONTRACT_NUCLEON, did, Sd, C)
    want = oracle.nucleon(LAT, o, e, S)
    assert _rel(C[0::2] + 1j * C[1::2], want) < CORR_TOL
    ddp.ddp_contract(ctx, ddp.DDP_CONTRACT_PION, did, Sd, C)
    assert _rel(C[0::2], oracle.pion(LAT, o, e, S)) < CORR_TOL
    assert np.all(C[1::2] == 0)
    c1 = np.zeros(2)
    ddp.ddp_contract(ctx, ddp.DDP_CONTRACT_PSEUDO_LOCAL, did, Sd, c1, src=src)
    t = oracle.local_trace(LAT, o, e, S, src)
    assert abs(complex(c1[0], c1[1]) - t) <= CORR_TOL * abs(t)
    n = int(np.prod(e))
    eta = synth.diluted_noise_columns(synth.noise_field(n, 5))
    psi, *_ = oracle.solve(U, LAT, AP, o, e, 0.124, eta)
    Cd = torch.zeros(2 * LAT[0], dtype=torch.float64, device="cuda")
    ddp.ddp_contract(ctx, ddp.DDP_CONTRACT_PSEUDO_NOISE, did, torch.from_numpy(psi).cuda(), Cd,
                     eta=torch.from_numpy(eta).cuda(), ncol=12)
    Cn = Cd.cpu().numpy()
    assert _rel(Cn[0::2] + 1j * Cn[1::2], oracle.noise_trace(LAT, o, e, eta, psi)) < CORR_TOL


@pytest.mark.parametrize("box,src", [(BOXES[0], (0, 0, 0, 0)), (BOXES[2], (6, 2, 0, 5)), (BOXES[3], (4, 3, 1, 0))])
def test_nucleon_double_fp32_against_fp64(ddp, ctx, field, box, src):
    """The nucleon in double-FP32 arithmetic (the default) against the FP64 form and the
    oracle.  Each double-FP32 operation is exact to about 2^-46 of its result, so over the
    ~10^4 products per site the time-slice sums agree with FP64 to ~1e-12 of their norm."""
    U, gid = field
    o, e = box
    did = ddp.ddp_set_domain(ctx, gid, o, e)
    S, *_ = oracle.propagator(U, LAT, AP, o, e, 0.124, src)
    Sd = torch.from_numpy(S).cuda()
    out = {}
    for dd in (1, 0):
        C = np.zeros(2 * LAT[0])
        ddp.ddp_set_param(ctx, "contraction_double_fp32", dd)
        try:
            ddp.ddp_contract(ctx, ddp.DDP_CONTRACT_NUCLEON, did, Sd, C)
        finally:
            ddp.ddp_set_param(ctx, "contraction_double_fp32", 1)
        out[dd] = C[0::2] + 1j * C[1::2]
    ddp.ddp_free_domain(ctx, did)
    assert _rel(out[1], out[0]) < 1e-12
    want = oracle.nucleon(LAT, o, e, S)
    assert _rel(out[1], want) < 1e-12 and _rel(out[0], want) < 1e-12


def test_series_and_contractions_host_buffers(ddp, ctx, field):
    """Host arguments (pinned torch tensors and plain numpy arrays) give the same bits
    as device arguments in the series terms and every contraction: the library stages
    host buffers itself, and the arithmetic is the same."""
    U, gid = field
    src = (7, 1, 2, 3)
    small, big = ((6, 0, 0, 0), (4, 4, 4, 6)), ((5, 0, 0, 0), (6, 4, 4, 6))
    ds = ddp.ddp_set_domain(ctx, gid, *small)
    db = ddp.ddp_set_domain(ctx, gid, *big)
    Ss, *_ = oracle.propagator(U, LAT, AP, *small, 0.124, src)
    Sb, *_ = oracle.propagator(U, LAT, AP, *big, 0.124, src)
    Td = torch.zeros(Sb.shape, dtype=torch.complex128, device="cuda")
    ddp.ddp_series_terms(ctx, ds, torch.from_numpy(Ss).cuda(), db, torch.from_numpy(Sb).cuda(), Td, 12)
    Tp = torch.zeros(Sb.shape, dtype=torch.complex128).pin_memory()
    ddp.ddp_series_terms(ctx, ds, torch.from_numpy(Ss).pin_memory(), db, torch.from_numpy(Sb).pin_memory(), Tp, 12)
    Tn = np.zeros(Sb.shape, dtype=np.complex128)
    ddp.ddp_series_terms(ctx, ds, Ss, db, Sb, Tn, 12)
    assert np.array_equal(Tp.numpy(), Td.cpu().numpy()) and np.array_equal(Tn, Td.cpu().numpy())

    n = Sb.shape[1]
    eta = synth.diluted_noise_columns(synth.noise_field(n, 9))
    cases = [(ddp.DDP_CONTRACT_NUCLEON, {}), (ddp.DDP_CONTRACT_PION, {}),
             (ddp.DDP_CONTRACT_PSEUDO_LOCAL, {"src": src})]
    for kind, kw in cases:
        want = np.zeros(2 * LAT[0])
        ddp.ddp_contract(ctx, kind, db, torch.from_numpy(Sb).cuda(), want, **kw)
        for S_host in (torch.from_numpy(Sb).pin_memory(), Sb):
            got = np.zeros(2 * LAT[0])
            ddp.ddp_contract(ctx, kind, db, S_host, got, **kw)
            assert np.array_equal(got, want), kind
    want = np.zeros(2 * LAT[0])
    ddp.ddp_contract(ctx, ddp.DDP_CONTRACT_PSEUDO_NOISE, db, torch.from_numpy(Sb).cuda(), want,
                     eta=torch.from_numpy(eta).cuda(), ncol=12)
    got = np.zeros(2 * LAT[0])
    ddp.ddp_contract(ctx, ddp.DDP_CONTRACT_PSEUDO_NOISE, db, Sb, got, eta=eta, ncol=12)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("box", BOXES[:4])
def test_hop_power(ddp, ctx, field, box):
    """(kappa D_hop)^p in FP64 against the oracle's p plain applications of the
    restricted hopping term (Eq. HPEtr operator), p = 0, 1, 8; host arguments give
    the same bits as device arguments."""
    U, gid = field
    o, e = box
    did = ddp.ddp_set_domain(ctx, gid, o, e)
    n = int(np.prod(e))
    rng = np.random.default_rng(3)
    psi = rng.standard_normal((3, n, 4, 3)) + 1j * rng.standard_normal((3, n, 4, 3))
    for p in (0, 1, 8):
        want = oracle.hop_power(U, LAT, AP, o, e, 0.124, p, psi)
        out = torch.zeros(psi.shape, dtype=torch.complex128, device="cuda")
        ddp.ddp_hop_power(ctx, did, 0.124, p, torch.from_numpy(psi).cuda(), out, 3)
        got = out.cpu().numpy()
        assert max(_col_errors(got, want)) < 1e-12, p
        host = np.zeros_like(psi)
        ddp.ddp_hop_power(ctx, did, 0.124, p, psi, host, 3)
        assert np.array_equal(host, got)
    for bad in ((-1, 0.124), (65, 0.124), (8, 0.0)):
        with pytest.raises(ddp.DDPError) as ei:
            ddp.ddp_hop_power(ctx, did, bad[1], bad[0], psi, np.zeros_like(psi), 3)
        assert ei.value.status == ddp.DDP_ERR_INVALID_ARG


def test_expanded_noise_trace(ddp, ctx, field):
    """The stochastic trace of Eq. HPEtr with p = 8: psi = D^-1 g5 eta, then
    (kappa D_hop)^8 psi contracted with g5 eta (= eta^+ [kappa^8 D_hop^8 D^-1 g5 eta]
    per time slice), against the oracle's same steps."""
    U, gid = field
    o, e = BOXES[1]
    did = ddp.ddp_set_domain(ctx, gid, o, e)
    n = int(np.prod(e))
    eta = synth.diluted_noise_columns(synth.noise_field(n, 13))
    g5eta = np.ascontiguousarray(np.einsum("ab,cnbk->cnak", oracle.gamma()[4], eta))
    psi, *_ = oracle.solve(U, LAT, AP, o, e, 0.124, g5eta)
    want = oracle.noise_trace(LAT, o, e, g5eta, oracle.hop_power(U, LAT, AP, o, e, 0.124, 8, psi))
    v = torch.zeros(psi.shape, dtype=torch.complex128, device="cuda")
    ddp.ddp_hop_power(ctx, did, 0.124, 8, torch.from_numpy(psi).cuda(), v, 12)
    C = torch.zeros(2 * LAT[0], dtype=torch.float64, device="cuda")
    ddp.ddp_contract(ctx, ddp.DDP_CONTRACT_PSEUDO_NOISE, did, v, C, eta=torch.from_numpy(g5eta).cuda(), ncol=12)
    Cn = C.cpu().numpy()
    assert _rel(Cn[0::2] + 1j * Cn[1::2], want) < CORR_TOL


GB0 = ((0, 0, 0, 0), (4, 4, 4, 6))      # Gamma-bar_0: time slices 0..3
GS0 = ((3, 0, 0, 0), (5, 4, 4, 6))      # Gamma*_0: slices 3..7, overlapping Gamma-bar_0 by one slice


@pytest.mark.parametrize("pair", [(GB0, GS0),
                                  (((0, 0, 0, 0), LAT), ((5, 1, 3, 2), (3, 2, 3, 4))),
                                  (((0, 0, 0, 0), (8, 4, 2, 6)), ((0, 0, 2, 0), (8, 4, 2, 6)))])
def test_boundary_source(ddp, ctx, field, pair):
    """-D[to, from minus to] psi (Eq. blkdec) against the oracle's sparse D built from the
    covariant derivatives: overlapping time slabs, the whole lattice into a wrapped
    Dirichlet box, and two halves of the lattice split in a periodic direction (hops
    across the periodic wrap); host arguments give the same bits."""
    U, gid = field
    fb, tb = pair
    d_from = ddp.ddp_set_domain(ctx, gid, *fb)
    d_to = ddp.ddp_set_domain(ctx, gid, *tb)
    nf, nt = int(np.prod(fb[1])), int(np.prod(tb[1]))
    rng = np.random.default_rng(4)
    psi = rng.standard_normal((3, nf, 4, 3)) + 1j * rng.standard_normal((3, nf, 4, 3))
    want = dense.boundary_source(U, LAT, AP, fb, psi, tb)
    sig = torch.zeros((3, nt, 4, 3), dtype=torch.complex128, device="cuda")
    ddp.ddp_boundary_source(ctx, d_from, torch.from_numpy(psi).cuda(), d_to, sig, 3)
    got = sig.cpu().numpy()
    assert max(_col_errors(got, want)) < 1e-12
    host = np.zeros((3, nt, 4, 3), dtype=np.complex128)
    ddp.ddp_boundary_source(ctx, d_from, psi, d_to, host, 3)
    assert np.array_equal(host, got)


def test_factorized_propagator(ddp, ctx, field):
    """S^(f) = -D^-1_{Gamma*_0} D_{dGamma*_0} D^-1_{Gamma-bar_0} (Eq. approxlong) through the
    C ABI -- mixed-precision solve on Gamma-bar_0, boundary source, solve on Gamma*_0 --
    against the oracle's same three steps; and its pion contraction (Eq. W0pc with S^(f))."""
    U, gid = field
    src = (1, 1, 2, 3)                  # in Gamma-bar_0, outside Gamma*_0
    kappa = 0.124
    d_bar = ddp.ddp_set_domain(ctx, gid, *GB0)
    d_star = ddp.ddp_set_domain(ctx, gid, *GS0)
    nb, ns = int(np.prod(GB0[1])), int(np.prod(GS0[1]))
    Sb = torch.zeros((12, nb, 4, 3), dtype=torch.complex128, device="cuda")
    rc, info = ddp.ddp_solve_propagator(ctx, d_bar, kappa, 0.0, src, 1e-10, ddp.DDP_PREC_MIXED_FP32, Sb)
    assert rc == ddp.DDP_OK
    sig = torch.zeros((12, ns, 4, 3), dtype=torch.complex128, device="cuda")
    ddp.ddp_boundary_source(ctx, d_bar, Sb, d_star, sig, 12)
    Sf = torch.zeros((12, ns, 4, 3), dtype=torch.complex128, device="cuda")
    rc, info = ddp.ddp_solve_sources(ctx, d_star, kappa, 0.0, sig, 12, 1e-10, ddp.DDP_PREC_MIXED_FP32, Sf)
    assert rc == ddp.DDP_OK
    Sbo, *_ = oracle.propagator(U, LAT, AP, *GB0, kappa, src)
    sig_o = dense.boundary_source(U, LAT, AP, GB0, Sbo, GS0)
    Sfo, *_ = oracle.solve(U, LAT, AP, *GS0, kappa, sig_o)
    assert max(_col_errors(Sf.cpu().numpy(), Sfo)) < COL_TOL
    C = np.zeros(2 * LAT[0])
    ddp.ddp_contract(ctx, ddp.DDP_CONTRACT_PION, d_star, Sf, C)
    assert _rel(C[0::2], oracle.pion(LAT, *GS0, Sfo)) < CORR_TOL


def test_gauge_region_variant(ddp, ctx, field):
    """A variant gauge field (links of one region replaced) solves like a
    freshly loaded field with the same links."""
    U, gid = field
    Uv = synth.variant_field(U, LAT, 0, 4, seed=9)
    o, e = (0, 0, 0, 0), (4, 4, 4, 6)
    gi, _, _ = oracle.domain_maps(LAT, o, e)
    Ubox = np.ascontiguousarray(Uv[:, gi])
    vid = ddp.ddp_load_gauge_region(ctx, gid, o, e, torch.from_numpy(Ubox).cuda())
    fid = ddp.ddp_load_gauge(ctx, torch.from_numpy(Uv).cuda(), LAT, 1)
    psi = synth.random_spinor(1, int(np.prod(LAT)), 2)
    outs = []
    for g in (vid, fid):
        did = ddp.ddp_set_domain(ctx, g, (0, 0, 0, 0), LAT)
        out = np.zeros_like(psi)
        ddp.ddp_apply_dirac(ctx, did, 0.12, psi, out, 1, 0)
        outs.append(out)
        ddp.ddp_free_domain(ctx, did)
    assert np.array_equal(outs[0], outs[1])
    ref = oracle.apply_dirac(Uv, LAT, AP, (0, 0, 0, 0), LAT, 0.12, psi)
    assert _rel(outs[0], ref) < 1e-13
    ddp.ddp_free_gauge(ctx, vid)
    ddp.ddp_free_gauge(ctx, fid)


def test_autotune_choice_keeps_results(ddp, ctx, field, tmp_path):
    U, gid = field
    o, e = BOXES[0]
    did = ddp.ddp_set_domain(ctx, gid, o, e)
    n = int(np.prod(e))
    cache = tmp_path / "tune.json"
    cols, ms = ddp.autotune_cached(ctx, did, n, 0.124, 12, ddp.DDP_PREC_MIXED_FP32, str(cache), iters=3)
    assert cols in (12, 8, 6, 4, 3, 2, 1) and ms > 0
    carve = ddp.ddp_get_param(ctx, "tuned_carveout_fp32")
    assert carve in (28, 50, 100) and ddp.ddp_get_param(ctx, "tuned_cols_fp32") == cols
    ddp.ddp_set_param(ctx, "tuned_carveout_fp32", -2)
    again = ddp.autotune_cached(ctx, did, n, 0.124, 12, ddp.DDP_PREC_MIXED_FP32, str(cache))
    assert again[0] == cols and ddp.ddp_get_param(ctx, "tuned_carveout_fp32") == carve
    S = torch.zeros((12, n, 4, 3), dtype=torch.complex128, device="cuda")
    rc, info = ddp.ddp_solve_propagator(ctx, did, 0.124, 0.0, (0, 0, 0, 0), 1e-10, 1, S)
    assert rc == ddp.DDP_OK
    ref, *_ = oracle.propagator(U, LAT, AP, o, e, 0.124, (0, 0, 0, 0), tol=1e-12)
    assert max(_col_errors(S.cpu().numpy(), ref)) < COL_TOL
    ddp.ddp_set_param(ctx, "tuned_cols_fp32", 0)
    ddp.ddp_set_param(ctx, "tuned_carveout_fp32", -2)


@pytest.mark.parametrize("box,src", [(BOXES[5], (7, 3, 1, 5)), (BOXES[6], (3, 2, 2, 4))])
def test_degenerate_boxes_solve(ddp, ctx, field, box, src):
    U, gid = field
    o, e = box
    did = ddp.ddp_set_domain(ctx, gid, o, e)
    n = int(np.prod(e))
    ref, *_ = oracle.propagator(U, LAT, AP, o, e, 0.124, src, tol=1e-12)
    S = torch.zeros((12, n, 4, 3), dtype=torch.complex128, device="cuda")
    rc, info = ddp.ddp_solve_propagator(ctx, did, 0.124, 0.0, src, 1e-10, 1, S)
    assert rc == ddp.DDP_OK
    assert max(_col_errors(S.cpu().numpy(), ref)) < COL_TOL


def test_zero_source_and_bad_kappa(ddp, ctx, field):
    U, gid = field
    o, e = BOXES[1]
    did = ddp.ddp_set_domain(ctx, gid, o, e)
    n = int(np.prod(e))
    eta = torch.zeros((3, n, 4, 3), dtype=torch.complex128, device="cuda")
    eta[1, 5, 2, 1] = 1.0                      # one non-zero column among zero columns
    out = torch.full_like(eta, float("nan"))
    rc, info = ddp.ddp_solve_sources(ctx, did, 0.124, 0.0, eta, 3, 1e-10, 1, out)
    assert rc == ddp.DDP_OK
    got = out.cpu().numpy()
    assert np.all(got[0] == 0) and np.all(got[2] == 0)
    ref, *_ = oracle.solve(U, LAT, AP, o, e, 0.124, eta[1:2].cpu().numpy())
    assert _rel(got[1], ref[0]) < COL_TOL
    for bad in (0.0, -0.1, float("nan")):
        with pytest.raises(ddp.DDPError) as ei:
            ddp.ddp_solve_sources(ctx, did, bad, 0.0, eta, 3, 1e-10, 1, out)
        assert ei.value.status == ddp.DDP_ERR_INVALID_ARG
    with pytest.raises(ddp.DDPError):
        ddp.ddp_solve_sources(ctx, did, 0.124, 0.0, eta, 3, 0.0, 1, out)      # tol must be positive


# ------------------------------------------------- nested propagators in one call

@pytest.mark.parametrize("where,overlap", [("device", 1), ("pinned", 1), ("numpy", 1), ("pinned", 0)])
def test_propagator_series_matches_separate_calls(ddp, ctx, field, where, overlap):
    """ddp_propagator_series gives the same bits as ddp_solve_batch + ddp_series_terms +
    ddp_contract on the same nested domains, whether its outputs are device memory,
    pinned host memory or plain numpy arrays, and with host outputs whether the smaller
    domains are solved first (overlap_downloads 1) or all in one batch (0); the
    propagators also match the oracle."""
    U, gid = field
    ddp.ddp_set_param(ctx, "overlap_downloads", overlap)
    src, kappa = (7, 1, 2, 3), 0.124
    boxes = [((6, 0, 0, 0), (4, 4, 4, 6)), ((5, 0, 0, 0), (6, 4, 4, 6)), ((0, 0, 0, 0), LAT)]
    dids = [ddp.ddp_set_domain(ctx, gid, *b) for b in boxes]
    shapes = [(12, int(np.prod(b[1])), 4, 3) for b in boxes]
    prec = ddp.DDP_PREC_MIXED_FP32
    # separate calls on device buffers
    S = [torch.zeros(sh, dtype=torch.complex128, device="cuda") for sh in shapes]
    reqs = [ddp.make_req(d, kappa, src, 1e-10, o) for d, o in zip(dids, S)]
    rc, _ = ddp.ddp_solve_batch(ctx, reqs, prec)
    assert rc == ddp.DDP_OK
    T = [torch.zeros(sh, dtype=torch.complex128, device="cuda") for sh in shapes[1:]]
    for i in range(1, 3):
        ddp.ddp_series_terms(ctx, dids[i - 1], S[i - 1], dids[i], S[i], T[i - 1], 12)
    mask = (1 << ddp.DDP_CONTRACT_PSEUDO_LOCAL) | (1 << ddp.DDP_CONTRACT_NUCLEON) | (1 << ddp.DDP_CONTRACT_PION)
    C = np.zeros((3, 4, 2 * LAT[0]))
    for i, d in enumerate(dids):
        for k in (ddp.DDP_CONTRACT_PSEUDO_LOCAL, ddp.DDP_CONTRACT_NUCLEON, ddp.DDP_CONTRACT_PION):
            out = np.zeros(2 * LAT[0])
            ddp.ddp_contract(ctx, k, d, S[i], out, src=src)
            C[i, k] = out
    # one call
    if where == "device":
        mk = lambda sh: torch.zeros(sh, dtype=torch.complex128, device="cuda")  # noqa: E731
        Cg = torch.zeros((3, 4, 2 * LAT[0]), dtype=torch.float64, device="cuda")
    elif where == "pinned":
        mk = lambda sh: torch.zeros(sh, dtype=torch.complex128).pin_memory()  # noqa: E731
        Cg = torch.zeros((3, 4, 2 * LAT[0]), dtype=torch.float64).pin_memory()
    else:
        mk = lambda sh: np.zeros(sh, dtype=np.complex128)  # noqa: E731
        Cg = np.zeros((3, 4, 2 * LAT[0]))
    S2 = [mk(sh) for sh in shapes]
    T2 = [mk(sh) for sh in shapes[1:]]
    rc, infos = ddp.ddp_propagator_series(ctx, dids, kappa, src, 1e-10, prec, S_out=S2, T_out=T2,
                                          contract_mask=mask, C_out=Cg)
    assert rc == ddp.DDP_OK
    host = lambda x: x.cpu().numpy() if hasattr(x, "cpu") else x  # noqa: E731
    for a, b in zip(S2, S):
        assert np.array_equal(host(a), b.cpu().numpy())
    for a, b in zip(T2, T):
        assert np.array_equal(host(a), b.cpu().numpy())
    Cg = host(Cg)
    for i in range(3):
        for k in (ddp.DDP_CONTRACT_PSEUDO_LOCAL, ddp.DDP_CONTRACT_NUCLEON, ddp.DDP_CONTRACT_PION):
            n = 2 if k == ddp.DDP_CONTRACT_PSEUDO_LOCAL else 2 * LAT[0]
            assert np.array_equal(Cg[i, k, :n], C[i, k, :n]), (i, k)
    ddp.ddp_set_param(ctx, "overlap_downloads", 1)
    ref, *_ = oracle.propagator(U, LAT, AP, *boxes[0], kappa, src)
    assert max(_col_errors(host(S2[0]), ref)) < 1e-8
    for d in dids:
        ddp.ddp_free_domain(ctx, d)


def test_propagator_series_rejects_non_nested(ddp, ctx, field):
    U, gid = field
    a = ddp.ddp_set_domain(ctx, gid, (6, 0, 0, 0), (4, 4, 4, 6))
    b = ddp.ddp_set_domain(ctx, gid, (0, 0, 0, 0), (4, 4, 4, 6))
    with pytest.raises(ddp.DDPError) as ei:
        ddp.ddp_propagator_series(ctx, [a, b], 0.124, (7, 0, 0, 0), 1e-10, ddp.DDP_PREC_MIXED_FP32)
    assert ei.value.status == ddp.DDP_ERR_INVALID_ARG
    ddp.ddp_free_domain(ctx, a)
    ddp.ddp_free_domain(ctx, b)


# ----------------------------------------------------- clover (O(a)-improved) operator

CSW = 1.7


@pytest.mark.parametrize("box", BOXES[:5])
@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 1e-6), (2, 4e-3), (3, 3e-2)])
def test_apply_dirac_clover(ddp, ctx, field, box, prec, tol):
    """D_Gamma with the clover term against the oracle, every storage format."""
    U, gid = field
    o, e = box
    did = ddp.ddp_set_domain(ctx, gid, o, e)
    n = int(np.prod(e))
    psi = synth.random_spinor(3, n, 19)
    ref = oracle.apply_dirac(U, LAT, AP, o, e, 0.1315, psi, csw=CSW)
    out = torch.zeros((3, n, 4, 3), dtype=torch.complex128, device="cuda")
    ddp.ddp_apply_dirac(ctx, did, 0.1315, torch.from_numpy(psi).cuda(), out, 3, prec, csw=CSW)
    errs = _col_errors(out.cpu().numpy(), ref)
    assert max(errs) < tol, errs
    # the clover part alone (D(c_sw) - D(0)) is right too, not only the total
    plain = torch.zeros_like(out)
    ddp.ddp_apply_dirac(ctx, did, 0.1315, torch.from_numpy(psi).cuda(), plain, 3, prec)
    diff = (out - plain).cpu().numpy()
    want = ref - oracle.apply_dirac(U, LAT, AP, o, e, 0.1315, psi)
    assert max(_col_errors(diff, want)) < 50 * tol
    ddp.ddp_free_domain(ctx, did)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("box,src", [(BOXES[0], (0, 0, 0, 0)), (BOXES[1], (7, 1, 2, 3)), (BOXES[3], (4, 3, 1, 0))])
def test_solve_propagator_clover(ddp, ctx, field, prec, box, src):
    """S^(i) of the O(a)-improved operator (even-odd Schur complement with T^-1 on both
    parities) against the oracle's solve of the unpreconditioned D_Gamma."""
    U, gid = field
    o, e = box
    kappa, csw = 0.12, 1.0
    did = ddp.ddp_set_domain(ctx, gid, o, e)
    n = int(np.prod(e))
    ref, _, rr, st = oracle.propagator(U, LAT, AP, o, e, kappa, src, tol=1e-12, csw=csw)
    assert st == 0
    S = torch.zeros((12, n, 4, 3), dtype=torch.complex128, device="cuda")
    rc, info = ddp.ddp_solve_propagator(ctx, did, kappa, csw, src, 1e-10, prec, S)
    assert rc == ddp.DDP_OK, ddp.info_dict(info)
    assert info.max_rel_residual <= 1e-10
    errs = _col_errors(S.cpu().numpy(), ref)
    assert max(errs) < COL_TOL, errs
    ddp.ddp_free_domain(ctx, did)


def test_batch_mixing_clover_and_plain_requests(ddp, ctx, field):
    """One batch with a plain Wilson request, two clover requests of different kappa
    and one of a different c_sw: every column against the oracle."""
    U, gid = field
    cases = [((6, 0, 0, 0), (4, 4, 4, 6), (7, 1, 2, 3), 0.12, 0.0),
             ((6, 0, 0, 0), (4, 4, 4, 6), (7, 1, 2, 3), 0.12, 1.0),
             ((0, 0, 0, 0), LAT, (3, 2, 2, 4), 0.115, 1.0),
             ((2, 3, 0, 5), (5, 4, 2, 2), (4, 3, 1, 0), 0.12, 1.5)]
    dids, outs, reqs = [], [], []
    for o, e, src, kappa, csw in cases:
        d = ddp.ddp_set_domain(ctx, gid, o, e)
        out = torch.zeros((12, int(np.prod(e)), 4, 3), dtype=torch.complex128, device="cuda")
        dids.append(d)
        outs.append(out)
        reqs.append(ddp.make_req(d, kappa, src, 1e-10, out, csw=csw))
    rc, infos = ddp.ddp_solve_batch(ctx, reqs, ddp.DDP_PREC_MIXED_FP32)
    assert rc == ddp.DDP_OK
    for (o, e, src, kappa, csw), out in zip(cases, outs):
        ref, *_ = oracle.propagator(U, LAT, AP, o, e, kappa, src, tol=1e-12, csw=csw)
        assert max(_col_errors(out.cpu().numpy(), ref)) < COL_TOL, (o, e, kappa, csw)
    for d in dids:
        ddp.ddp_free_domain(ctx, d)
