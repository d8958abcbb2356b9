"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a second
construction of the operator from the covariant derivatives (App. A), closed
forms of the free propagator, block-inverse identities (Eq. blkdec, bella,
Scmpt), gamma_5-hermiticity (Eq. g5h), gauge covariance, the structure behind
the hopping-parameter expansion of the trace (Eq. HPEtr), the telescoping
series (Eq. Dseries), and a brute-force Wick enumeration of the nucleon
correlator (Sec. 4).
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from oracle import dense, freefield, wick

AP = oracle.BC_ANTIPERIODIC


@pytest.fixture(scope="module")
def field44():
    L = (4, 4, 4, 4)
    return L, synth.gauge_field(L, seed=11)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ----------------------------------------------------------------------------- gamma

def test_gamma_algebra():
    g = oracle.gamma()
    I4 = np.eye(4)
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
        for n in range(4):
            assert np.allclose(g[m] @ g[n] + g[n] @ g[m], 2 * I4 * (m == n))
    assert np.allclose(g[4], g[0] @ g[1] @ g[2] @ g[3])
    assert np.allclose(g[4] @ g[4], I4)
    for m in range(4):
        assert np.allclose(g[4] @ g[m], -g[m] @ g[4])
    # gamma_0, gamma_2 symmetric, gamma_1, gamma_3 antisymmetric
    assert np.allclose(g[0], g[0].T) and np.allclose(g[2], g[2].T)
    assert np.allclose(g[1], -g[1].T) and np.allclose(g[3], -g[3].T)
    C = 1j * g[0] @ g[2]
    Ci = np.linalg.inv(C)
    for m in range(4):
        assert np.allclose(C @ g[m] @ Ci, -g[m].T)


# ------------------------------------------------------------------- the operator

@pytest.mark.parametrize("bc", [0, 1])
def test_full_operator_matches_covariant_derivative_form(field44, bc):
    L, U = field44
    kappa = 0.137
    D = dense.dirac_matrix(U, L, bc, kappa)
    psi = synth.random_spinor(2, 256, 3)
    out = oracle.apply_dirac(U, L, bc, (0, 0, 0, 0), L, kappa, psi)
    ref = (D @ psi.reshape(2, -1).T).T.reshape(psi.shape)
    assert _rel(out, ref) < 1e-14


BOXES = [((0, 0, 0, 0), (2, 4, 4, 4)),
         ((3, 1, 0, 2), (2, 3, 4, 2)),        # wraps across the antiperiodic time boundary
         ((1, 2, 3, 0), (3, 3, 3, 4)),
         ((2, 0, 0, 0), (4, 4, 4, 4))]         # full extent: no restriction, origin shifted


@pytest.mark.parametrize("box", BOXES)
def test_dirichlet_operator_is_sub_block(field44, box):
    L, U = field44
    o, e = box
    kappa = 0.131
    D = dense.dirac_matrix(U, L, AP, kappa)
    DG = dense.restricted(D, L, o, e)
    n = int(np.prod(e))
    psi = synth.random_spinor(1, n, 9)
    out = oracle.apply_dirac(U, L, AP, o, e, kappa, psi)
    ref = (DG @ psi.reshape(-1)).reshape(psi.shape)
    assert _rel(out, ref) < 1e-14


def test_open_boundary_is_dirichlet_embedding():
    """Open time boundary on T slices == Dirichlet box of extent T inside T+2 slices."""
    L = (4, 2, 2, 4)
    Lb = (6, 2, 2, 4)
    Ub = synth.gauge_field(Lb, seed=3)
    x = synth.site_coords(Lb)
    keep = (x[:, 0] >= 1) & (x[:, 0] <= 4)
    U = Ub[:, keep].copy()
    psi = synth.random_spinor(1, int(np.prod(L)), 4)
    a = oracle.apply_dirac(U, L, oracle.BC_OPEN, (0, 0, 0, 0), L, 0.12, psi)
    b = oracle.apply_dirac(Ub, Lb, AP, (1, 0, 0, 0), (4, 2, 2, 4), 0.12, psi)
    assert _rel(a, b) < 1e-15


def test_gamma5_hermiticity(field44):
    """<phi, g5 D g5 psi> = <D phi, psi> on a Dirichlet box (Eq. g5h)."""
    L, U = field44
    o, e = (3, 1, 0, 2), (2, 3, 4, 2)
    n = int(np.prod(e))
    g5 = oracle.gamma()[4]
    phi = synth.random_spinor(1, n, 1)
    psi = synth.random_spinor(1, n, 2)
    g5psi = np.einsum("ab,cnbk->cnak", g5, psi)
    lhs = np.vdot(phi, np.einsum("ab,cnbk->cnak", g5, oracle.apply_dirac(U, L, AP, o, e, 0.13, g5psi)))
    rhs = np.vdot(oracle.apply_dirac(U, L, AP, o, e, 0.13, phi), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


# ------------------------------------------------------------ free-field closed forms

@pytest.mark.parametrize("bc", [0, 1])
def test_free_propagator_momentum_space(bc):
    L = (8, 4, 4, 6)
    U = synth.unit_gauge_field(L)
    S, it, rr, st = oracle.propagator(U, L, bc, (0, 0, 0, 0), L, 0.12, (0, 0, 0, 0))
    assert st == 0
    Sf = freefield.momentum_propagator(L, 0.12, bc).reshape(-1, 4, 4)   # site, alpha, beta
    V = int(np.prod(L))
    Sor = S.reshape(4, 3, V, 4, 3)                                     # beta, b, site, alpha, a
    for a in range(3):
        for b in range(3):
            got = np.transpose(Sor[:, b, :, :, a], (1, 2, 0))
            want = Sf if a == b else 0 * Sf
            assert np.abs(got - want).max() < 1e-11


def test_free_dirichlet_slab():
    L = (8, 4, 4, 4)
    U = synth.unit_gauge_field(L)
    o, e = (6, 0, 0, 0), (4, 4, 4, 4)      # slab t = 6, 7, 0, 1 (wraps)
    S, it, rr, st = oracle.propagator(U, L, AP, o, e, 0.125, (7, 0, 0, 0))
    assert st == 0
    ref = freefield.slab_propagator(L, 0.125, 6, 4, 7)           # (4, 4, 4, 4, alpha, beta), no BC sign inside
    # the hop 7 -> 0 inside the slab crosses the antiperiodic boundary: sites with
    # slab-local t >= 2 (global 0, 1) pick up a factor -1 relative to the source at t=7
    n = int(np.prod(e))
    Sor = S.reshape(4, 3, n, 4, 3)[:, 0, :, :, 0]                  # beta, site, alpha
    got = np.transpose(Sor, (1, 2, 0)).reshape(4, 4, 4, 4, 4, 4)
    sign = np.array([1, 1, -1, -1])[:, None, None, None, None, None]
    assert np.abs(got - sign * ref).max() < 1e-11


# ------------------------------------------------------ propagators and identities

def test_domain_propagator_is_inverse_of_sub_block(field44):
    """S^(i) = D_Gamma^{-1} (Eq. diric) against a dense inverse of D[Gamma, Gamma]."""
    L, U = field44
    o, e = (1, 2, 3, 0), (3, 3, 3, 4)
    kappa = 0.13
    D = dense.dirac_matrix(U, L, AP, kappa)
    DG = dense.restricted(D, L, o, e)
    src = (2, 3, 0, 1)
    S, it, rr, st = oracle.propagator(U, L, AP, o, e, kappa, src)
    assert st == 0 and rr.max() <= 1e-12
    l = oracle.local_index(L, o, e, src)
    Sinv = np.linalg.inv(DG)
    for c in range(12):
        ref = Sinv[:, l * 12 + c]
        assert _rel(S[c].reshape(-1), ref) < 1e-10


def test_schur_identity_bella(field44):
    """Eq. bella: S = S^(i) + S^(i) D_{dGamma} D^{-1} D_{dGamma*} S^(i) on the box."""
    L, U = field44
    kappa = 0.128
    o, e = (0, 0, 0, 0), (2, 4, 4, 4)
    D = dense.dirac_matrix(U, L, AP, kappa).toarray()
    idx = dense.box_component_index(L, o, e)
    comp = np.setdiff1d(np.arange(D.shape[0]), idx)
    src = (1, 2, 1, 3)
    l = oracle.local_index(L, o, e, src)
    Si, *_ = oracle.propagator(U, L, AP, o, e, kappa, src)
    Sfull, *_ = oracle.propagator(U, L, AP, (0, 0, 0, 0), L, kappa, src)
    B = D[np.ix_(idx, comp)]
    C = D[np.ix_(comp, idx)]
    Dinv = np.linalg.inv(D)
    DG_inv = np.linalg.inv(D[np.ix_(idx, idx)])
    # S^(i)(., x) columns and the full S restricted to the box
    Si_cols = Si.reshape(12, -1).T
    rhs = Si_cols + DG_inv @ B @ Dinv[np.ix_(comp, comp)] @ C @ Si_cols
    gi, _, _ = oracle.domain_maps(L, o, e)
    full_on_box = Sfull.reshape(12, 256, 12)[:, gi, :].reshape(12, -1).T
    assert _rel(rhs, full_on_box) < 1e-10
    # the exact (Gamma, Gamma) block of D^{-1} (Eq. Scmpt)
    assert _rel(Dinv[np.ix_(idx, idx)][:, l * 12:(l + 1) * 12], full_on_box) < 1e-10


def test_propagator_gamma5_hermiticity(field44):
    """S(x,y) = g5 S(y,x)^+ g5 with two point sources in one box."""
    L, U = field44
    o, e = (1, 0, 0, 0), (3, 4, 4, 4)
    x, y = (1, 0, 0, 0), (3, 2, 1, 3)
    Sx, *_ = oracle.propagator(U, L, AP, o, e, 0.13, x)
    Sy, *_ = oracle.propagator(U, L, AP, o, e, 0.13, y)
    lx = oracle.local_index(L, o, e, x)
    ly = oracle.local_index(L, o, e, y)
    g5 = oracle.gamma()[4]
    # S(y,x)_{alpha a, beta b} = Sx[3 beta + b, ly, alpha, a]
    Syx = Sx[:, ly].reshape(4, 3, 4, 3).transpose(2, 3, 0, 1).reshape(12, 12)
    Sxy = Sy[:, lx].reshape(4, 3, 4, 3).transpose(2, 3, 0, 1).reshape(12, 12)
    G5 = np.kron(g5, np.eye(3))
    assert _rel(Sxy, G5 @ Syx.conj().T @ G5) < 1e-10


def test_gauge_covariance(field44):
    L, U = field44
    V = 256
    Lam = synth.random_gauge_transform(V, 77)
    Lr = Lam.reshape(L + (3, 3))
    Up = np.empty_like(U)
    for mu in range(4):
        Ur = U[mu].reshape(L + (3, 3))
        Lp = np.roll(Lr, -1, axis=mu)
        Up[mu] = (Lr @ Ur @ np.conj(np.swapaxes(Lp, -1, -2))).reshape(V, 3, 3)
    o, e = (3, 0, 1, 0), (3, 4, 2, 4)
    src = (3, 1, 1, 2)
    S, *_ = oracle.propagator(U, L, AP, o, e, 0.13, src)
    Sp, *_ = oracle.propagator(Up, L, AP, o, e, 0.13, src)
    gi, _, _ = oracle.domain_maps(L, o, e)
    n = gi.size
    xs = np.ravel_multi_index(src, L)
    # S'(y,x) = Lam(y) S(y,x) Lam(x)^+ ; arrays [beta b][y][alpha a]
    A = S.reshape(4, 3, n, 4, 3)
    Ap = Sp.reshape(4, 3, n, 4, 3)
    # explicit loops keep the index bookkeeping readable
    want = np.zeros_like(Ap)
    Lx = Lam[xs]
    for beta in range(4):
        for alpha in range(4):
            M = A[beta, :, :, alpha, :]          # [b][y][a]: S(y,x)_{alpha a, beta b}
            Mt = np.transpose(M, (1, 2, 0))     # [y][a][b]
            R = Lam[gi] @ Mt @ np.conj(Lx.T)    # [y][a][b]
            want[beta, :, :, alpha, :] = np.transpose(R, (2, 0, 1))
    assert _rel(Ap, want) < 1e-10
    # gauge-invariant contractions are unchanged
    assert _rel(oracle.pion(L, o, e, Sp), oracle.pion(L, o, e, S)) < 1e-10
    assert _rel(oracle.nucleon(L, o, e, Sp), oracle.nucleon(L, o, e, S)) < 1e-9


def test_hopping_expansion_trace_structure(field44):
    """tr[g5 D_hop^k](x,x) = 0 for k < 8 at every site, also in a Dirichlet box
    (the structure behind Eq. HPEtr); k = 8 is generically non-zero."""
    L, U = field44
    o, e = (0, 0, 0, 0), (3, 4, 4, 4)
    n = int(np.prod(e))
    g5 = oracle.gamma()[4]
    sites = [0, 17, n - 1]
    for site in sites:
        eta = np.zeros((12, n, 4, 3), dtype=np.complex128)
        for c in range(12):
            eta[c, site, c // 3, c % 3] = 1
        v = eta
        for k in range(1, 9):
            v = oracle.apply_hop(U, L, AP, o, e, v)
            blk = v[:, site].reshape(4, 3, 4, 3)           # [beta b][alpha a]
            tr = sum(g5[al, r] * blk[al, a, r, a] for al in range(4) for r in range(4) for a in range(3))
            if k < 8:
                assert abs(tr) < 1e-11, (site, k, tr)
            else:
                assert abs(tr) > 1e-6


def test_hopping_expansion_trace_identity(field44):
    """Eq. HPEtr site by site: tr[g5 D^-1](x,x) = tr[g5 (kappa D_hop)^p D^-1](x,x) for
    p <= 8, with D^-1 the dense inverse of D[Gamma, Gamma] built from the covariant
    derivatives (independent of the oracle's hopping code), in a Dirichlet box with an
    antiperiodic wrapped time direction; p = 9 breaks it."""
    L, U = field44
    kappa = 0.124
    o, e = (0, 1, 0, 0), (4, 2, 2, 4)
    n = int(np.prod(e))
    DG = dense.restricted(dense.dirac_matrix(U, L, AP, kappa), L, o, e)
    Dinv = np.linalg.inv(DG)
    cols = np.ascontiguousarray(Dinv.T.reshape(12 * n, n, 4, 3))   # column j of D^-1 as a field
    g5 = np.kron(oracle.gamma()[4], np.eye(3))

    def site_traces(M):
        return np.array([np.trace(g5 @ M[12 * s:12 * s + 12, 12 * s:12 * s + 12]) for s in range(n)])

    want = site_traces(Dinv)
    for p in (4, 8, 9):
        hp = oracle.hop_power(U, L, AP, o, e, kappa, p, cols)        # [j] = (k D_hop)^p D^-1 e_j
        M = hp.reshape(12 * n, 12 * n).T
        got = site_traces(M)
        err = np.max(np.abs(got - want)) / np.max(np.abs(want))
        if p <= 8:
            assert err < 1e-10, (p, err)   # rounding of the dense inverse; a wrong power of kappa is O(1)
        else:
            assert err > 1e-6, (p, err)


def test_boundary_source_block_row(field44):
    """Row block Gamma_to of D S = eta (Eq. blkdec): D_{Gamma_to} S|to = eta|to + sigma with
    sigma the dropped couplings from the rest of the lattice (from = whole lattice),
    for a Dirichlet box and for a time slab wrapped across the antiperiodic boundary."""
    L, U = field44
    kappa = 0.124
    src = (1, 2, 0, 3)
    S, *_ = oracle.propagator(U, L, AP, (0, 0, 0, 0), L, kappa, src)
    gi_full = oracle.domain_maps(L, (0, 0, 0, 0), L)[0]
    for to in [((3, 0, 0, 0), (2, 4, 4, 4)), ((1, 1, 0, 2), (2, 3, 4, 2))]:
        gi = oracle.domain_maps(L, *to)[0]
        full = np.zeros((12, 256, 4, 3), dtype=np.complex128)
        full[:, gi_full] = S
        S_to = np.ascontiguousarray(full[:, gi])
        sigma = dense.boundary_source(U, L, AP, ((0, 0, 0, 0), L), S, to)
        eta_to = np.zeros_like(S_to)
        try:                                        # the source, where it lies in the box
            k = oracle.local_index(L, to[0], to[1], src)
            for c in range(12):
                eta_to[c, k, c // 3, c % 3] = 1
        except ValueError:
            pass
        lhs = oracle.apply_dirac(U, L, AP, to[0], to[1], kappa, S_to)
        assert _rel(lhs, eta_to + sigma) < 1e-10


def test_factorized_propagator_exact_limit(field44):
    """Eq. approxlong with Gamma-bar_0 = the whole lattice is exact: for a source outside
    Gamma*_0, D^-1_{Gamma*_0} sigma(D^-1 eta) = S on Gamma*_0; with a thinner Gamma-bar_0
    it is only an approximation (differs)."""
    L, U = field44
    kappa = 0.124
    src = (0, 1, 2, 3)
    star = ((2, 0, 0, 0), (2, 4, 4, 4))            # Gamma*_0: slices 2, 3
    S, *_ = oracle.propagator(U, L, AP, (0, 0, 0, 0), L, kappa, src)
    gi_full = oracle.domain_maps(L, (0, 0, 0, 0), L)[0]
    gi = oracle.domain_maps(L, *star)[0]
    full = np.zeros((12, 256, 4, 3), dtype=np.complex128)
    full[:, gi_full] = S
    sigma = dense.boundary_source(U, L, AP, ((0, 0, 0, 0), L), S, star)
    Sf, *_ = oracle.solve(U, L, AP, *star, kappa, sigma)
    assert _rel(Sf, full[:, gi]) < 1e-9
    bar = ((0, 0, 0, 0), (3, 4, 4, 4))             # Gamma-bar_0: slices 0..2, overlapping Gamma*_0 by one
    Sb, *_ = oracle.propagator(U, L, AP, *bar, kappa, src)
    sigma_b = dense.boundary_source(U, L, AP, bar, Sb, star)
    Sfb, *_ = oracle.solve(U, L, AP, *star, kappa, sigma_b)
    assert _rel(Sfb, full[:, gi]) > 1e-6


def test_telescoping_series(field44):
    """S^(0) + sum_i [S^(i) - S^(i-1)] = S on the full lattice (Eq. Dseries)."""
    L, U = field44
    src = (0, 1, 2, 3)
    boxes = [((3, 0, 0, 0), (2, 4, 4, 4)), ((3, 0, 0, 0), (3, 4, 4, 4)), ((0, 0, 0, 0), L)]
    Ss = [oracle.propagator(U, L, AP, o, e, 0.125, src)[0] for o, e in boxes]
    gis = [oracle.domain_maps(L, o, e)[0] for o, e in boxes]
    V = 256
    total = np.zeros((12, V, 4, 3), dtype=np.complex128)
    total[:, gis[0]] = Ss[0]
    for i in range(1, len(boxes)):
        T = oracle.series_term(L, boxes[i - 1][0], boxes[i - 1][1], Ss[i - 1], boxes[i][0], boxes[i][1], Ss[i])
        total[:, gis[i]] += T
    assert _rel(total, Ss[-1][:, np.argsort(gis[-1])]) < 1e-14
    # the embedding itself: T^(1) on sites outside Gamma_0 equals S^(1)
    T1 = oracle.series_term(L, boxes[0][0], boxes[0][1], Ss[0], boxes[1][0], boxes[1][1], Ss[1])
    inside = np.isin(gis[1], gis[0])
    assert np.array_equal(T1[:, ~inside], Ss[1][:, ~inside])
    pos = {g: i for i, g in enumerate(gis[0])}
    for l1 in np.nonzero(inside)[0][:20]:
        assert np.array_equal(T1[:, l1], Ss[1][:, l1] - Ss[0][:, pos[gis[1][l1]]])


def test_series_terms_decay():
    """|S^(i) - S^(i-1)| falls as the slab grows (Eq. error), at a distance from the source."""
    L = (16, 4, 4, 4)
    U = synth.gauge_field(L, seed=21)
    src = (0, 0, 0, 0)
    slabs = [synth.centered_time_slab(L, d, 0) for d in (4, 8, 12)]
    Ss = [oracle.propagator(U, L, AP, b.origin, b.extent, 0.12, src)[0] for b in slabs]
    norms = []
    for i in range(1, len(slabs)):
        T = oracle.series_term(L, slabs[i - 1].origin, slabs[i - 1].extent, Ss[i - 1],
                               slabs[i].origin, slabs[i].extent, Ss[i])
        norms.append(np.linalg.norm(T))
    assert norms[1] < 0.5 * norms[0]


# ------------------------------------------------------------------ contractions

def test_local_trace_is_real(field44):
    L, U = field44
    o, e = (3, 1, 0, 2), (2, 3, 4, 2)
    src = (0, 2, 1, 3)
    S, *_ = oracle.propagator(U, L, AP, o, e, 0.13, src)
    t = oracle.local_trace(L, o, e, S, src)
    l = oracle.local_index(L, o, e, src)
    # the imaginary part vanishes up to round-off on the scale of S(x,x)
    assert abs(t.imag) <= 1e-12 * np.linalg.norm(S[:, l])
    g5 = oracle.gamma()[4]
    blk = S[:, l].reshape(4, 3, 4, 3)         # [beta b][alpha a]
    Sxx = blk.transpose(2, 3, 0, 1).reshape(12, 12)
    assert abs(np.trace(np.kron(g5, np.eye(3)) @ Sxx) - t) < 1e-13


def test_pion_positive_and_sum_of_squares(field44):
    L, U = field44
    o, e = (0, 0, 0, 0), L
    S, *_ = oracle.propagator(U, L, AP, o, e, 0.13, (0, 0, 0, 0))
    C = oracle.pion(L, o, e, S)
    assert np.all(C > 0)
    assert abs(C.sum() - np.sum(np.abs(S) ** 2)) < 1e-12 * C.sum()


def _site_blocks(S, n):
    """(n, 4, 3, 4, 3) = S(y,x)_{rho a, sigma b} from 12 columns."""
    return S.reshape(4, 3, n, 4, 3).transpose(2, 3, 4, 0, 1)


def test_nucleon_matches_wick_enumeration(field44):
    L, U = field44
    o, e = (1, 0, 0, 0), (3, 4, 4, 4)
    S, *_ = oracle.propagator(U, L, AP, o, e, 0.13, (2, 1, 0, 3))
    n = int(np.prod(e))
    gi, _, _ = oracle.domain_maps(L, o, e)
    y0 = gi // (L[1] * L[2] * L[3])
    ref = wick.nucleon_correlator(_site_blocks(S, n), y0, L[0])
    got = oracle.nucleon(L, o, e, S)
    assert _rel(got, ref) < 1e-12
    # a random (non-propagator) S also agrees: the identity is algebraic
    R = synth.random_spinor(12, n, 5)
    assert _rel(oracle.nucleon(L, o, e, R), wick.nucleon_correlator(_site_blocks(R, n), y0, L[0])) < 1e-12


def test_nucleon_free_field_closed_form():
    L = (8, 4, 4, 4)
    U = synth.unit_gauge_field(L)
    S, *_ = oracle.propagator(U, L, AP, (0, 0, 0, 0), L, 0.12, (0, 0, 0, 0))
    Sf = freefield.momentum_propagator(L, 0.12, 1).reshape(-1, 4, 4)
    V = int(np.prod(L))
    blocks = np.einsum("yrs,ab->yrasb", Sf, np.eye(3))
    y0 = np.arange(V) // 64
    ref = wick.nucleon_correlator(blocks, y0, L[0])
    got = oracle.nucleon(L, (0, 0, 0, 0), L, S)
    assert _rel(got, ref) < 1e-10
    assert np.abs(ref).max() > 0


def test_noise_trace_against_dense_inverse(field44):
    L, U = field44
    o, e = (1, 0, 0, 0), (2, 4, 4, 4)
    kappa = 0.13
    n = int(np.prod(e))
    z = synth.noise_field(n, 4)
    eta = synth.diluted_noise_columns(z)
    psi, it, rr, st = oracle.solve(U, L, AP, o, e, kappa, eta)
    T = oracle.noise_trace(L, o, e, eta, psi)
    D = dense.dirac_matrix(U, L, AP, kappa)
    Sinv = np.linalg.inv(dense.restricted(D, L, o, e)).reshape(n, 12, n, 12)
    g5 = np.kron(oracle.gamma()[4], np.eye(3))
    # sum_x conj(z_x) sum_y z_y tr[g5 S(x,y)], grouped by x0
    tr = np.einsum("ij,xjyi->xy", g5, Sinv)
    per_x = np.conj(z) * (tr @ z)
    gi, _, _ = oracle.domain_maps(L, o, e)
    ref = np.zeros(L[0], dtype=complex)
    np.add.at(ref, gi // 64, per_x)
    assert _rel(T, ref) < 1e-10


# ----------------------------------------------------------------------- maps

def test_domain_maps_bruteforce():
    L = (6, 4, 4, 8)
    for o, e in [((5, 3, 0, 6), (3, 2, 4, 4)), ((0, 0, 0, 0), L), ((2, 1, 3, 7), (4, 4, 1, 8))]:
        gi, eo, par = oracle.domain_maps(L, o, e)
        cnt = [0, 0]
        l = 0
        for k in itertools.product(*[range(x) for x in e]):
            x = [(o[m] + k[m]) % L[m] for m in range(4)]
            assert gi[l] == ((x[0] * L[1] + x[1]) * L[2] + x[2]) * L[3] + x[3]
            p = sum(x) % 2
            assert par[l] == p and eo[l] == cnt[p]
            cnt[p] += 1
            l += 1
        if e[3] % 2 == 0:
            assert np.array_equal(eo, np.arange(gi.size) // 2)


# -------------------------------------------------------------- synthetic field

def test_synthetic_links_are_su3():
    U = synth.gauge_field((4, 2, 2, 2), seed=8).reshape(-1, 3, 3)
    I3 = np.eye(3)
    assert np.abs(np.conj(np.swapaxes(U, 1, 2)) @ U - I3).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14


def test_plaquette_equals_mean_link_to_the_fourth():
    """E[P] = c^4 for independent conjugation-invariant links; the tuned eps gives 0.59."""
    eps = synth.tune_eps()
    c = synth.mean_link_trace(eps, n=200_000, seed=99)
    assert abs(c ** 4 - 0.59) < 0.002
    L = (8, 8, 8, 8)
    P = synth.plaquette(synth.gauge_field(L, seed=synth.SEED_GAUGE), L)
    # 6 V plaquettes with single-plaquette std ~0.2: standard error ~0.0013
    assert abs(P - 0.59) < 0.005


# ------------------------------------------------------------ two-level averaging

def test_factorized_correlator_is_product_of_level1_means():
    """Eq. factsing: the two traces are averaged separately over the level-1
    variants and then multiplied (not the mean of the products)."""
    rng = np.random.default_rng(3)
    L0, vol3 = 6, 27.0
    TA = rng.standard_normal((4, L0)) + 1j * rng.standard_normal((4, L0))
    TB = rng.standard_normal((5, L0)) + 1j * rng.standard_normal((5, L0))
    C = oracle.factorized_correlator(TA, TB, L0, vol3)
    # identical variants reduce to the single-configuration product
    C1 = oracle.factorized_correlator(TA[:1].repeat(3, 0), TB[:1].repeat(2, 0), L0, vol3)
    assert np.allclose(C1, np.outer(TB[0], TA[0]) / vol3, rtol=1e-14, atol=0)
    # order of the variants does not matter; bilinear in the two means
    Cp = oracle.factorized_correlator(TA[::-1], TB[[2, 0, 4, 1, 3]], L0, vol3)
    assert np.allclose(Cp, C, rtol=1e-13, atol=0)
    C2 = oracle.factorized_correlator(2 * TA, TB, L0, vol3)
    assert np.allclose(C2, 2 * C, rtol=1e-14, atol=0)
    # it differs from the mean over variant pairs of the products when the regions correlate
    pair_mean = np.mean([np.outer(TB[w], TA[v]) for v, w in zip(range(4), range(4))], axis=0) / vol3
    assert not np.allclose(pair_mean, C)


def test_noise_estimator_converges_to_trace():
    """The diluted-noise time-slice trace averages to sum_x tr{g5 S(x,x)} (Sec. 5):
    the off-diagonal terms carry random phases."""
    L = (4, 2, 2, 2)
    U = synth.gauge_field(L, seed=12)
    o, e = (0, 0, 0, 0), L
    n = int(np.prod(e))
    D = dense.dirac_matrix(U, L, AP, 0.12)
    Sinv = np.linalg.inv(D.toarray()).reshape(n, 12, n, 12)
    g5 = np.kron(oracle.gamma()[4], np.eye(3))
    exact = np.zeros(L[0], dtype=complex)
    gi, _, _ = oracle.domain_maps(L, o, e)
    for x in range(n):
        exact[gi[x] // 8] += np.trace(g5 @ Sinv[x, :, x, :])
    # Z2 x Z2 noise (|z| = 1) has no diagonal fluctuation: the estimate differs from the
    # exact trace only by off-diagonal terms, whose average over sources vanishes
    acc = np.zeros(L[0], dtype=complex)
    nsrc = 200
    rng = np.random.default_rng(5)
    for i in range(nsrc):
        z = (rng.choice([-1.0, 1.0], n) + 1j * rng.choice([-1.0, 1.0], n)) / np.sqrt(2)
        eta = synth.diluted_noise_columns(z)
        psi = np.einsum("xiyj,cyj->cxi", Sinv, eta.reshape(12, n, 12)).reshape(eta.shape)
        acc += oracle.noise_trace(L, o, e, eta, psi)
    est = acc / nsrc
    assert np.abs(est - exact).max() < 0.25 * np.abs(exact).max()


def test_free_field_correlators_match_golden_values():
    """Golden values written by tests/golden/make_golden.py from the momentum-space
    closed form; the C oracle's solve + contractions must reproduce them."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "free_field_8x4x4x4.json")))
    L = tuple(g["lattice"])
    U = synth.unit_gauge_field(L)
    S, *_ = oracle.propagator(U, L, AP, (0, 0, 0, 0), L, g["kappa"], (0, 0, 0, 0), tol=1e-13)
    assert _rel(oracle.pion(L, (0, 0, 0, 0), L, S), np.array(g["pion"])) < 1e-11
    want = np.array(g["nucleon_re"]) + 1j * np.array(g["nucleon_im"])
    assert _rel(oracle.nucleon(L, (0, 0, 0, 0), L, S), want) < 1e-10


# ------------------------------------------------------------ clover (O(a)-improvement) term
#
# The paper names the O(a)-improved operator (footnotes of Sec. 4 and Sec. 5)
# without writing it; the oracle uses the Sheikholeslami-Wohlert term
# c_sw (i/4) sum_{mu,nu} sigma_{mu nu} F_{mu nu}(x) with the clover-leaf F.
# These tests pin it with constant abelian fields, whose field strength and
# clover spectrum are known in closed form, and with the symmetries of D.

def _constant_flux(L, planes):
    """SU(3) links that are diagonal phases giving every plaquette of the (mu, nu)
    plane the phase exp(i n B q_c) per colour c (q = charges, sum q = 0) and every
    other plaquette 1: U_nu(x) = exp(i B x_mu q), U_mu(x) = exp(-i B L_mu x_nu q) on
    the last slice x_mu = L_mu - 1, with B = 2 pi n / (L_mu L_nu).
    planes: list of (mu, nu, n, q)."""
    V = int(np.prod(L))
    x = np.stack(np.unravel_index(np.arange(V), L), axis=1)
    ph = np.zeros((4, V, 3))
    for mu, nu, n, q in planes:
        B = 2 * np.pi * n / (L[mu] * L[nu])
        q = np.asarray(q, dtype=float)
        ph[nu] += np.outer(B * x[:, mu], q)
        last = x[:, mu] == L[mu] - 1
        ph[mu][last] -= np.outer(B * L[mu] * x[last, nu], q)
    U = np.zeros((4, V, 3, 3), dtype=np.complex128)
    for c in range(3):
        U[:, :, c, c] = np.exp(1j * ph[:, :, c])
    return U


@pytest.mark.parametrize("plane", [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)])
def test_clover_term_constant_field_spectrum(plane):
    """One constant field in the (mu, nu) plane: F_{mu nu} = i sin(B q_c) per colour, so
    the clover term -(c_sw/2) sigma_{mu nu} (x) diag sin(B q) has the eigenvalues
    +-(c_sw/2) sin(B q_c), each twice (sigma_{mu nu} has eigenvalues +-1, twice each),
    at every site."""
    L, csw = (4, 6, 4, 6), 1.7
    q = (1.0, 2.0, -3.0)
    mu, nu = plane
    U = _constant_flux(L, [(mu, nu, 1, q)])
    C = oracle.clover_field(U, L, csw)
    B = 2 * np.pi / (L[mu] * L[nu])
    want = np.sort(np.concatenate([[s * 0.5 * csw * np.sin(B * qc)] * 2 for qc in q for s in (1, -1)]))
    for site in (0, 17, 300, int(np.prod(L)) - 1):
        got = np.sort(np.linalg.eigvalsh(C[site]))
        assert np.allclose(got, want, atol=1e-13), (site, got, want)


def test_clover_term_two_planes_relative_orientation():
    """Fields in the (0,1) and (2,3) planes together: sigma_01 sigma_23 = -gamma_5 fixes
    how the two terms combine; per colour the spectrum is +-(c_sw/2)(a - b) and
    +-(c_sw/2)(a + b) with a, b the two sin(B q) (a dropped 1/2, a wrong sigma or a
    wrong plane orientation changes it)."""
    L, csw = (6, 4, 4, 6), 0.9
    qa, qb = (1.0, -2.0, 1.0), (2.0, 1.0, -3.0)
    U = _constant_flux(L, [(0, 1, 1, qa), (2, 3, 1, qb)])
    C = oracle.clover_field(U, L, csw)
    Ba, Bb = 2 * np.pi / (L[0] * L[1]), 2 * np.pi / (L[2] * L[3])
    want = []
    for c in range(3):
        a, b = np.sin(Ba * qa[c]), np.sin(Bb * qb[c])
        want += [0.5 * csw * v for v in (a - b, b - a, a + b, -a - b)]
    want = np.sort(want)
    for site in (0, 55, 250):
        assert np.allclose(np.sort(np.linalg.eigvalsh(C[site])), want, atol=1e-13)


def test_clover_term_vanishes_for_unit_links_and_is_hermitian(field44):
    L, U = field44
    assert np.abs(oracle.clover_field(synth.unit_gauge_field(L), L, 1.5)).max() < 1e-15
    C = oracle.clover_field(U, L, 1.5)
    assert np.abs(C - np.conj(np.swapaxes(C, 1, 2))).max() < 1e-14
    # commutes with gamma_5 (sigma_{mu nu} does): block diagonal in the chiral spin pairs
    g5 = np.kron(oracle.gamma()[4], np.eye(3))
    assert np.abs(C @ g5 - g5 @ C).max() < 1e-14


def test_clover_operator_adds_the_site_term(field44):
    """D(c_sw) - D(0) is site-local on a Dirichlet box and equals the clover term of the
    sites of the box (links outside the box included: D_Gamma = D[Gamma, Gamma])."""
    L, U = field44
    o, e = (3, 1, 0, 2), (2, 3, 4, 2)
    gi, _, _ = oracle.domain_maps(L, o, e)
    psi = synth.random_spinor(2, gi.size, 5)
    d = oracle.apply_dirac(U, L, AP, o, e, 0.13, psi, csw=1.3) - oracle.apply_dirac(U, L, AP, o, e, 0.13, psi)
    C = oracle.clover_field(U, L, 1.3)
    want = np.einsum("nij,cnj->cni", C[gi], psi.reshape(2, gi.size, 12)).reshape(psi.shape)
    assert _rel(d, want) < 1e-13


def test_clover_gamma5_hermiticity(field44):
    L, U = field44
    o, e = (3, 1, 0, 2), (2, 3, 4, 2)
    n = int(np.prod(e))
    g5 = oracle.gamma()[4]
    phi = synth.random_spinor(1, n, 1)
    psi = synth.random_spinor(1, n, 2)
    g5psi = np.einsum("ab,cnbk->cnak", g5, psi)
    lhs = np.vdot(phi, np.einsum("ab,cnbk->cnak", g5, oracle.apply_dirac(U, L, AP, o, e, 0.13, g5psi, csw=1.4)))
    rhs = np.vdot(oracle.apply_dirac(U, L, AP, o, e, 0.13, phi, csw=1.4), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_clover_gauge_covariance(field44):
    """With the clover term the propagator still transforms as S' = Lam(y) S Lam(x)^+:
    a leaf with its links in the wrong order would break it."""
    L, U = field44
    V = 256
    Lam = synth.random_gauge_transform(V, 78)
    Lr = Lam.reshape(L + (3, 3))
    Up = np.empty_like(U)
    for mu in range(4):
        Ur = U[mu].reshape(L + (3, 3))
        Lp = np.roll(Lr, -1, axis=mu)
        Up[mu] = (Lr @ Ur @ np.conj(np.swapaxes(Lp, -1, -2))).reshape(V, 3, 3)
    C, Cp = oracle.clover_field(U, L, 1.2), oracle.clover_field(Up, L, 1.2)
    Lam12 = np.einsum("st,nab->nsatb", np.eye(4), Lam).reshape(V, 12, 12)
    assert np.abs(Cp - Lam12 @ C @ np.conj(np.swapaxes(Lam12, 1, 2))).max() < 1e-13
    o, e, src = (3, 0, 1, 0), (3, 4, 2, 4), (3, 1, 1, 2)
    S, *_ = oracle.propagator(U, L, AP, o, e, 0.13, src, csw=1.2)
    Sp, *_ = oracle.propagator(Up, L, AP, o, e, 0.13, src, csw=1.2)
    assert _rel(oracle.pion(L, o, e, Sp), oracle.pion(L, o, e, S)) < 1e-10
    assert _rel(oracle.nucleon(L, o, e, Sp), oracle.nucleon(L, o, e, S)) < 1e-9


def test_clover_domain_propagator_is_inverse_of_sub_block(field44):
    """S^(i) with the clover term = inverse of the (Gamma, Gamma) block of the dense
    improved operator assembled column by column."""
    L, U = field44
    o, e = (1, 1, 0, 0), (2, 2, 4, 2)
    n = int(np.prod(e))
    csw, kappa = 1.1, 0.12
    Dm = np.zeros((12 * n, 12 * n), dtype=np.complex128)
    unit = np.zeros((1, n, 4, 3), dtype=np.complex128)
    for j in range(12 * n):
        unit.reshape(-1)[:] = 0
        unit.reshape(-1)[j] = 1.0
        Dm[:, j] = oracle.apply_dirac(U, L, AP, o, e, kappa, unit, csw=csw).reshape(-1)
    src = (2, 1, 3, 1)
    S, _, rr, st = oracle.propagator(U, L, AP, o, e, kappa, src, csw=csw)
    assert st == 0
    Sinv = np.linalg.inv(Dm)
    l = oracle.local_index(L, o, e, src)
    for c in range(12):
        assert _rel(S[c].reshape(-1), Sinv[:, 12 * l + c]) < 1e-10
