"""GPU projector-cut factorization (Sec. 5) against the oracle, through the C ABI.

Pieces: orthonormalization, inverse-iteration modes, time-slice Gram blocks
(Eq. Bpions), colourless spinors (Eq. W0tbary), the two projected correlators;
then the whole pion and nucleon pipeline from the modes to C(y0, x0).
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import projector

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

AP = oracle.BC_ANTIPERIODIC
L = (12, 4, 4, 4)
KAPPA = 0.12
GBAR = ((0, 0, 0, 0), (8, 4, 4, 4))    # slices 0..7   (x0cut = 6, Delta = 2)
GSTAR = ((6, 0, 0, 0), (5, 4, 4, 4))   # slices 6..10
OMEGA = ((4, 0, 0, 0), (4, 4, 4, 4))   # slices 4..7
VOL3 = L[1] * L[2] * L[3]
CORR_TOL = 1e-7
# Tensor-core path: every term of a slice sum is exact to ~2^-47 of its row maximum
# times its column maximum (seven 7-bit slices per operand, exact integer
# accumulation), so on random fields the norm-wise error stays near 1e-14; the
# bound 1e-12 leaves the factor ~40 of max/rms of the two operands.  The direct
# FP64 kernel rounds only in FP64.
TC_TOL = 1e-12


@pytest.fixture(scope="module")
def ddp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_04587_gb300 import build
    build.build()
    import paper_1601_04587_gb300 as m
    return m


@pytest.fixture(scope="module")
def env(ddp):
    U = synth.gauge_field(L, seed=41)
    ctx = ddp.ddp_create(0, torch.cuda.current_stream().cuda_stream)
    gid = ddp.ddp_load_gauge(ctx, torch.from_numpy(U).cuda(), L, ddp.DDP_BC_ANTIPERIODIC)
    doms = {name: ddp.ddp_set_domain(ctx, gid, *box) for name, box in
            (("bar", GBAR), ("star", GSTAR), ("omega", OMEGA))}
    doms["gid"] = gid
    yield U, ctx, doms
    ddp.ddp_destroy(ctx)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


class _Path:
    """Selects the tensor-core (1) or the direct FP64 (0) projector-cut kernels for a block."""

    def __init__(self, ddp, ctx, tc):
        self.ddp, self.ctx, self.tc = ddp, ctx, tc

    def __enter__(self):
        self.ddp.ddp_set_param(self.ctx, "projector_tensor_cores", self.tc)

    def __exit__(self, *exc):
        self.ddp.ddp_set_param(self.ctx, "projector_tensor_cores", 1)


@pytest.mark.parametrize("tc", [1, 0])
def test_orthonormalize_matches_oracle(ddp, env, tc):
    U, ctx, doms = env
    n = oracle.box_sites(OMEGA[1])
    V = synth.random_spinor(8, n, 3)
    Vd = _dev(V)
    with _Path(ddp, ctx, tc):
        ddp.ddp_orthonormalize(ctx, doms["omega"], Vd, 8)
    assert np.abs(Vd.cpu().numpy() - projector.orthonormalize(V)).max() < 1e-12


@pytest.mark.parametrize("tc", [1, 0])
@pytest.mark.parametrize("prec", [0, 1])
def test_inverse_iteration_matches_oracle(ddp, env, prec, tc):
    U, ctx, doms = env
    n = oracle.box_sites(OMEGA[1])
    V0 = synth.random_spinor(6, n, 7)
    want = projector.inverse_iteration(U, L, AP, *OMEGA, KAPPA, V0, 3)
    Vd = _dev(V0)
    with _Path(ddp, ctx, tc):
        rc, _ = ddp.ddp_inverse_iteration(ctx, doms["omega"], KAPPA, Vd, 6, 3, 1e-11, prec)
    assert rc == ddp.DDP_OK
    got = Vd.cpu().numpy()
    assert max(_rel(got[c], want[c]) for c in range(6)) < 1e-8


@pytest.mark.parametrize("tc", [1, 0])
def test_gram_slices_matches_oracle(ddp, env, tc):
    U, ctx, doms = env
    n = oracle.box_sites(GBAR[1])
    A = synth.random_spinor(20, n, 11)
    M = torch.zeros((L[0], 20, 20), dtype=torch.complex128, device="cuda")
    with _Path(ddp, ctx, tc):
        ddp.ddp_gram_slices(ctx, doms["bar"], _dev(A), 20, M)
    want = projector.gram_slices(L, *GBAR, A)
    assert _rel(M.cpu().numpy(), want) < (TC_TOL if tc else 1e-13)
    # a domain that wraps in time puts its slices at their global times (host buffers)
    wrap = ((10, 1, 0, 0), (4, 2, 4, 4))
    did = ddp.ddp_set_domain(ctx, doms["gid"], *wrap)
    M2 = np.zeros((L[0], 20, 20), dtype=np.complex128)
    A2 = synth.random_spinor(20, oracle.box_sites(wrap[1]), 12)
    with _Path(ddp, ctx, tc):
        ddp.ddp_gram_slices(ctx, did, A2, 20, M2)
    assert _rel(M2, projector.gram_slices(L, *wrap, A2)) < (TC_TOL if tc else 1e-13)
    ddp.ddp_free_domain(ctx, did)




def _forms(A, form):
    g5 = oracle.gamma()[4]
    return {0: A, 1: np.einsum("ab,mnbc->mnac", g5, np.conj(A)), 2: -A}[form]


@pytest.mark.parametrize("tc", [1, 0])
@pytest.mark.parametrize("form", [0, 1, 2])
def test_colourless_slices_matches_oracle(ddp, env, form, tc):
    U, ctx, doms = env
    n = oracle.box_sites(GSTAR[1])
    A = synth.random_spinor(5, n, 13)
    X = torch.zeros((L[0], 5, 5, 5, 4), dtype=torch.complex128, device="cuda")
    ddp.ddp_set_param(ctx, "projector_tensor_cores", tc)
    try:
        ddp.ddp_colourless_slices(ctx, doms["star"], _dev(A), 5, form, X)
    finally:
        ddp.ddp_set_param(ctx, "projector_tensor_cores", 1)
    want = projector.colourless_spinors(L, *GSTAR, _forms(A, form))
    assert _rel(X.cpu().numpy(), want) < (TC_TOL if tc else 1e-13)


# A lattice whose time slices hold 512 sites: with m = 20 and m = 32 the tensor-core
# product spans several 128-row and 64-column tiles with ragged tails, and (m = 32)
# more than one exact 256-deep chunk per thread block.
L8 = (6, 8, 8, 8)


@pytest.fixture(scope="module")
def env8(ddp):
    U = synth.gauge_field(L8, seed=43)
    ctx = ddp.ddp_create(0, torch.cuda.current_stream().cuda_stream)
    gid = ddp.ddp_load_gauge(ctx, torch.from_numpy(U).cuda(), L8, ddp.DDP_BC_PERIODIC)
    yield ctx, gid
    ddp.ddp_destroy(ctx)


def _colourless_both(ddp, ctx, did, A, m, form, L0):
    out = []
    for tc in (1, 0):
        X = torch.zeros((L0, m, m, m, 4), dtype=torch.complex128, device="cuda")
        ddp.ddp_set_param(ctx, "projector_tensor_cores", tc)
        try:
            ddp.ddp_colourless_slices(ctx, did, _dev(A), m, form, X)
        finally:
            ddp.ddp_set_param(ctx, "projector_tensor_cores", 1)
        out.append(X.cpu().numpy())
    return out


@pytest.mark.parametrize("m,form,box", [(20, 1, ((1, 0, 0, 0), (3, 8, 8, 8))),
                                        (32, 0, ((4, 0, 0, 0), (2, 8, 8, 8))),
                                        (1, 2, ((5, 0, 0, 0), (3, 8, 8, 8)))])
def test_colourless_tensor_cores_several_tiles(ddp, env8, m, form, box):
    ctx, gid = env8
    did = ddp.ddp_set_domain(ctx, gid, *box)
    A = synth.random_spinor(m, oracle.box_sites(box[1]), 50 + m)
    tc, direct = _colourless_both(ddp, ctx, did, A, m, form, L8[0])
    want = projector.colourless_spinors(L8, *box, _forms(A, form))
    ddp.ddp_free_domain(ctx, did)
    assert _rel(direct, want) < 1e-13
    assert _rel(tc, want) < TC_TOL
    # the slices outside the domain stay zero (the box wraps in time for the last case)
    inside = np.zeros(L8[0], bool)
    inside[[(box[0][0] + t) % L8[0] for t in range(box[1][0])]] = True
    assert not np.any(tc[~inside])


def test_colourless_tensor_cores_wide_dynamic_range(ddp, env8):
    """Columns scaled from 1e-30 to 1e6: every (i, j, k) block keeps its relative accuracy,
    because each spinor column, each row of the diquark matrix and each output column
    carries its own power-of-two exponent (the diquarks of 1e-30 columns, 1e-60, are far
    outside the FP32 range that the double-FP32 pre-pass works in)."""
    ctx, gid = env8
    box = ((0, 0, 0, 0), (2, 8, 8, 8))
    did = ddp.ddp_set_domain(ctx, gid, *box)
    m = 6
    A = synth.random_spinor(m, oracle.box_sites(box[1]), 77) * (10.0 ** np.linspace(-30, 6, m))[:, None, None, None]
    tc, _ = _colourless_both(ddp, ctx, did, A, m, 0, L8[0])
    want = projector.colourless_spinors(L8, *box, A)
    ddp.ddp_free_domain(ctx, did)
    for t in range(2):
        for i in range(m):
            for j in range(m):
                for k in range(m):
                    w = want[t, i, j, k]
                    assert np.linalg.norm(tc[t, i, j, k] - w) <= TC_TOL * np.linalg.norm(w) + 1e-300


def test_colourless_tensor_cores_full_slice(ddp):
    """One 24^3 time slice with 24 columns, the size of every slice of the projector
    workload: the tensor-core sums against the oracle and the direct FP64 kernel."""
    L24 = (2, 24, 24, 24)
    box = ((0, 0, 0, 0), (1, 24, 24, 24))
    m = 24
    ctx = ddp.ddp_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        U = synth.gauge_field(L24, seed=44)
        gid = ddp.ddp_load_gauge(ctx, torch.from_numpy(U).cuda(), L24, ddp.DDP_BC_PERIODIC)
        did = ddp.ddp_set_domain(ctx, gid, *box)
        A = synth.random_spinor(m, oracle.box_sites(box[1]), 91)
        tc, direct = _colourless_both(ddp, ctx, did, A, m, 1, L24[0])
    finally:
        ddp.ddp_destroy(ctx)
    want = projector.colourless_spinors(L24, *box, _forms(A, 1))
    assert _rel(direct, want) < 1e-13
    assert _rel(tc, want) < TC_TOL


def test_colourless_slices_rejects_too_many_columns(ddp, env):
    """More than 128 columns on the tensor cores, more than 32 with the direct FP64 kernel."""
    U, ctx, doms = env
    n = oracle.box_sites(OMEGA[1])
    X = torch.zeros(1, dtype=torch.complex128, device="cuda")
    for m, tc in ((129, 1), (33, 0)):
        A = torch.zeros((m, n, 4, 3), dtype=torch.complex128, device="cuda")
        with _Path(ddp, ctx, tc):
            with pytest.raises(ddp.DDPError) as ei:
                ddp.ddp_colourless_slices(ctx, doms["omega"], A, m, 0, X)
        assert ei.value.status == ddp.DDP_ERR_UNSUPPORTED


def test_colourless_tensor_cores_paper_modes(ddp):
    """N_m = 120 columns, the number of modes of the paper's projector (Sec. 5): 7260
    diquark rows (57 row tiles), 960 output columns (15 column tiles), on a 2 x 4^3
    lattice, against the oracle."""
    L2 = (2, 4, 4, 4)
    box = ((0, 0, 0, 0), L2)
    m = 120
    ctx = ddp.ddp_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        U = synth.gauge_field(L2, seed=45)
        gid = ddp.ddp_load_gauge(ctx, torch.from_numpy(U).cuda(), L2, ddp.DDP_BC_PERIODIC)
        did = ddp.ddp_set_domain(ctx, gid, *box)
        A = synth.random_spinor(m, oracle.box_sites(box[1]), 92)
        X = torch.zeros((L2[0], m, m, m, 4), dtype=torch.complex128, device="cuda")
        ddp.ddp_colourless_slices(ctx, did, _dev(A), m, 2, X)
        got = X.cpu().numpy()
        del X
    finally:
        ddp.ddp_destroy(ctx)
    assert _rel(got, projector.colourless_spinors(L2, *box, _forms(A, 2))) < TC_TOL


@pytest.mark.parametrize("m,form,box", [(40, 1, ((1, 0, 0, 0), (2, 8, 8, 8))),
                                        (33, 0, ((5, 0, 0, 0), (2, 8, 8, 8)))])
def test_colourless_tensor_cores_more_than_32_columns(ddp, env8, m, form, box):
    """Beyond 32 columns (4 sites per diquark block, column maxima with more columns
    than threads), on 512-site slices, the second box wrapping in time."""
    ctx, gid = env8
    did = ddp.ddp_set_domain(ctx, gid, *box)
    A = synth.random_spinor(m, oracle.box_sites(box[1]), 150 + m)
    X = torch.zeros((L8[0], m, m, m, 4), dtype=torch.complex128, device="cuda")
    ddp.ddp_colourless_slices(ctx, did, _dev(A), m, form, X)
    ddp.ddp_free_domain(ctx, did)
    got = X.cpu().numpy()
    assert _rel(got, projector.colourless_spinors(L8, *box, _forms(A, form))) < TC_TOL
    inside = np.zeros(L8[0], bool)
    inside[[(box[0][0] + t) % L8[0] for t in range(box[1][0])]] = True
    assert not np.any(got[~inside])


@pytest.mark.parametrize("L0,m", [(12, 5), (20, 7), (3, 40)])
def test_projected_nucleon_matches_oracle(ddp, env, L0, m):
    """The nucleon projection as a product over the 4 m^3 (i, j, k, alpha) terms against
    the oracle's contraction, on random X and Y: time extents inside one 16 x 16 output
    tile, across tiles with ragged edges, and m > 32."""
    U, ctx, doms = env
    rng = np.random.default_rng(300 + m)
    shape = (L0, m, m, m, 4)
    X = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    Y = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    C = torch.zeros((L0, L0), dtype=torch.complex128, device="cuda")
    ddp.ddp_projected_nucleon(ctx, L0, m, _dev(X), _dev(Y), C)
    assert _rel(C.cpu().numpy(), projector.projected_nucleon(X, Y)) < 1e-12


def test_orthonormalize_more_than_32_columns(ddp, env):
    """40 columns: the Gram blocks over two tensor-core column tiles and the double-FP32
    update with R^-1 staged a column tile at a time."""
    U, ctx, doms = env
    n = oracle.box_sites(OMEGA[1])
    m = 40
    V = synth.random_spinor(m, n, 4)
    Vd = _dev(V)
    ddp.ddp_orthonormalize(ctx, doms["omega"], Vd, m)
    assert np.abs(Vd.cpu().numpy() - projector.orthonormalize(V)).max() < 1e-12


@pytest.mark.parametrize("m", [6, 48])
def test_projected_pion_and_nucleon_pipeline(ddp, env, m):
    """Modes on Omega, u_i = D^-1_{Gbar} g5 phi_i, w_i = D^-1_{G*} sigma_i, the pion
    from the Gram blocks and the nucleon from the colourless spinors, all on the GPU,
    against the oracle's route; m = 48 takes every path beyond 32 modes (Gram blocks over
    two column tiles, the tiled Cholesky-QR update, 4-site diquark blocks, the nucleon
    product over 4 m^3 terms)."""
    U, ctx, doms = env
    n_o, n_b, n_s = (oracle.box_sites(b[1]) for b in (OMEGA, GBAR, GSTAR))
    V0 = synth.random_spinor(m, n_o, 21)
    phi = projector.inverse_iteration(U, L, AP, *OMEGA, KAPPA, V0, 2)
    u_ref, w_ref = projector.factorized_vectors(U, L, AP, KAPPA, GBAR, GSTAR, OMEGA, phi)
    M_ref = projector.gram_slices(L, *GBAR, u_ref)
    Mt_ref = projector.gram_slices(L, *GSTAR, w_ref)
    Cpi_ref = projector.projected_pion(Mt_ref, M_ref, VOL3)
    g5 = oracle.gamma()[4]
    X_ref = projector.colourless_spinors(L, *GBAR, np.einsum("ab,mnbc->mnac", g5, np.conj(u_ref)))
    Y_ref = projector.colourless_spinors(L, *GSTAR, -w_ref)
    Cn_ref = projector.projected_nucleon(X_ref, Y_ref)

    dphi = _dev(V0)
    rc, _ = ddp.ddp_inverse_iteration(ctx, doms["omega"], KAPPA, dphi, m, 2, 1e-11, ddp.DDP_PREC_MIXED_FP32)
    assert rc == ddp.DDP_OK
    src = torch.zeros((m, n_b, 4, 3), dtype=torch.complex128, device="cuda")
    ddp.ddp_embed(ctx, doms["omega"], dphi, doms["bar"], src, m, gamma5=True)
    u = torch.zeros_like(src)
    rc, _ = ddp.ddp_solve_sources(ctx, doms["bar"], KAPPA, 0.0, src, m, 1e-11, ddp.DDP_PREC_MIXED_FP32, u)
    assert rc == ddp.DDP_OK
    sigma = torch.zeros((m, n_s, 4, 3), dtype=torch.complex128, device="cuda")
    ddp.ddp_boundary_source(ctx, doms["omega"], dphi, doms["star"], sigma, m)
    w = torch.zeros_like(sigma)
    rc, _ = ddp.ddp_solve_sources(ctx, doms["star"], KAPPA, 0.0, sigma, m, 1e-11, ddp.DDP_PREC_MIXED_FP32, w)
    assert rc == ddp.DDP_OK
    assert _rel(u.cpu().numpy(), u_ref) < 1e-8 and _rel(w.cpu().numpy(), w_ref) < 1e-8
    M = torch.zeros((L[0], m, m), dtype=torch.complex128, device="cuda")
    Mt = torch.zeros_like(M)
    ddp.ddp_gram_slices(ctx, doms["bar"], u, m, M)
    ddp.ddp_gram_slices(ctx, doms["star"], w, m, Mt)
    Cpi = torch.zeros((L[0], L[0]), dtype=torch.complex128, device="cuda")
    ddp.ddp_projected_pion(ctx, L[0], m, Mt, M, VOL3, Cpi)
    assert _rel(Cpi.cpu().numpy(), Cpi_ref) < CORR_TOL
    X = torch.zeros((L[0], m, m, m, 4), dtype=torch.complex128, device="cuda")
    Y = torch.zeros_like(X)
    ddp.ddp_colourless_slices(ctx, doms["bar"], u, m, 1, X)
    ddp.ddp_colourless_slices(ctx, doms["star"], w, m, 2, Y)
    Cn = torch.zeros((L[0], L[0]), dtype=torch.complex128, device="cuda")
    ddp.ddp_projected_nucleon(ctx, L[0], m, X, Y, Cn)
    assert _rel(Cn.cpu().numpy(), Cn_ref) < CORR_TOL


@pytest.mark.parametrize("tc", [1, 0])
def test_colourless_nan_input_stays_local(ddp, env8, tc):
    """A NaN in one spinor component at one site makes exactly the outputs of that time
    slice that depend on it NaN; every other output stays finite and correct."""
    ctx, gid = env8
    box = ((0, 0, 0, 0), (2, 8, 8, 8))
    did = ddp.ddp_set_domain(ctx, gid, *box)
    m, bad = 4, 2
    A = synth.random_spinor(m, oracle.box_sites(box[1]), 78)
    A[bad, 700, 1, 2] = np.nan            # site 700 lies in the second time slice
    X = torch.zeros((L8[0], m, m, m, 4), dtype=torch.complex128, device="cuda")
    ddp.ddp_set_param(ctx, "projector_tensor_cores", tc)
    try:
        ddp.ddp_colourless_slices(ctx, did, _dev(A), m, 0, X)
    finally:
        ddp.ddp_set_param(ctx, "projector_tensor_cores", 1)
        ddp.ddp_free_domain(ctx, did)
    X = X.cpu().numpy()
    clean = A.copy()
    clean[bad, 700, 1, 2] = 0             # the outputs compared below do not depend on it
    want = projector.colourless_spinors(L8, *box, clean)
    # the diquark of a row with i or j = bad carries the NaN into every (k, alpha); an
    # output column (k = bad, alpha) only when alpha is the NaN's spin
    involved = np.zeros((m, m, m, 4), bool)
    involved[bad] = involved[:, bad] = True
    involved[:, :, bad, 1] = True
    assert np.isnan(X[1][involved]).all()
    assert np.isfinite(X[1][~involved]).all() and np.isfinite(X[0]).all()
    assert _rel(X[1][~involved], want[1][~involved]) < TC_TOL
    assert _rel(X[0], want[0]) < TC_TOL


@pytest.mark.parametrize("m,box", [(1, ((0, 0, 0, 0), (3, 8, 8, 8))),
                                   (20, ((1, 0, 0, 0), (2, 8, 8, 8))),
                                   (32, ((4, 0, 0, 0), (3, 8, 8, 8))),
                                   (40, ((2, 0, 0, 0), (2, 8, 8, 8))),
                                   (120, ((5, 0, 0, 0), (2, 8, 8, 8))),
                                   (128, ((0, 0, 0, 0), (1, 8, 8, 8)))])
def test_gram_tensor_cores_sizes(ddp, env8, m, box):
    """m = 1 to 128 (the largest; 120 is the paper's number of modes) columns over
    512-site slices, one to four 64-column tiles, a box wrapping in time; both paths
    against the oracle, slices outside the box zero."""
    ctx, gid = env8
    did = ddp.ddp_set_domain(ctx, gid, *box)
    A = synth.random_spinor(m, oracle.box_sites(box[1]), 60 + m)
    want = projector.gram_slices(L8, *box, A)
    out = {}
    for tc in (1, 0):
        M = torch.zeros((L8[0], m, m), dtype=torch.complex128, device="cuda")
        with _Path(ddp, ctx, tc):
            ddp.ddp_gram_slices(ctx, did, _dev(A), m, M)
        out[tc] = M.cpu().numpy()
    ddp.ddp_free_domain(ctx, did)
    assert _rel(out[0], want) < 1e-13
    assert _rel(out[1], want) < TC_TOL
    inside = np.zeros(L8[0], bool)
    inside[[(box[0][0] + t) % L8[0] for t in range(box[1][0])]] = True
    assert not np.any(out[1][~inside])


def test_gram_tensor_cores_wide_dynamic_range(ddp, env8):
    """Columns scaled from 1e-30 to 1e6: every entry is accurate relative to the norms of
    its two columns (each column carries its own exponent)."""
    ctx, gid = env8
    box = ((0, 0, 0, 0), (2, 8, 8, 8))
    did = ddp.ddp_set_domain(ctx, gid, *box)
    m = 8
    A = synth.random_spinor(m, oracle.box_sites(box[1]), 79) * (10.0 ** np.linspace(-30, 6, m))[:, None, None, None]
    M = torch.zeros((L8[0], m, m), dtype=torch.complex128, device="cuda")
    ddp.ddp_gram_slices(ctx, did, _dev(A), m, M)
    ddp.ddp_free_domain(ctx, did)
    got, want = M.cpu().numpy(), projector.gram_slices(L8, *box, A)
    for t in range(2):
        nrm = np.sqrt(np.abs(np.diagonal(want[t])))
        assert np.all(np.abs(got[t] - want[t]) <= TC_TOL * np.outer(nrm, nrm))


@pytest.mark.parametrize("tc", [1, 0])
def test_gram_nan_input_stays_local(ddp, env8, tc):
    """A NaN in one column at one site makes that slice's row and column of the Gram block
    NaN and nothing else."""
    ctx, gid = env8
    box = ((0, 0, 0, 0), (2, 8, 8, 8))
    did = ddp.ddp_set_domain(ctx, gid, *box)
    m, bad = 5, 3
    A = synth.random_spinor(m, oracle.box_sites(box[1]), 80)
    A[bad, 900, 2, 1] = np.nan            # the second time slice
    M = torch.zeros((L8[0], m, m), dtype=torch.complex128, device="cuda")
    with _Path(ddp, ctx, tc):
        ddp.ddp_gram_slices(ctx, did, _dev(A), m, M)
    ddp.ddp_free_domain(ctx, did)
    got = M.cpu().numpy()
    clean = A.copy()
    clean[bad, 900, 2, 1] = 0
    want = projector.gram_slices(L8, *box, clean)
    involved = np.zeros((m, m), bool)
    involved[bad] = involved[:, bad] = True
    assert np.isnan(got[1][involved]).all()
    assert np.isfinite(got[1][~involved]).all() and np.isfinite(got[0]).all()
    assert _rel(got[1][~involved], want[1][~involved]) < TC_TOL
    assert _rel(got[0], want[0]) < TC_TOL
