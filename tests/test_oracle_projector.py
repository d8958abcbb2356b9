"""Pins of the oracle's projector-cut factorization (Sec. 5, Eqs. proj,
approxlong2, fullfactpi, Bpions, W0tbary) against dense linear algebra.

The factorized propagator with the projector inserted,
    S~ = -D^-1_{G*} D[G*, Omega minus G*] P D^-1_{Gbar},  P = Phi Phi^+,
is built here from dense matrices of D (App. A, assembled from the covariant
derivatives by oracle.dense); the oracle's route through u_i, w_i, the
time-slice Gram blocks and the colourless spinors must reproduce its pion and
nucleon correlators, and a complete basis on the cut slice must give the exact
factorized propagator of Eq. approxlong.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import dense, projector

AP = oracle.BC_ANTIPERIODIC
L = (10, 2, 2, 4)
KAPPA = 0.12
GBAR = ((0, 0, 0, 0), (6, 2, 2, 4))    # slices 0..5   (x0cut = 4, Delta = 2)
GSTAR = ((4, 0, 0, 0), (5, 2, 2, 4))   # slices 4..8
OMEGA = ((2, 0, 0, 0), (4, 2, 2, 4))   # slices 2..5: the thick slice at the cut
VOL3 = L[1] * L[2] * L[3]


@pytest.fixture(scope="module")
def setup():
    U = synth.gauge_field(L, seed=31)
    D = dense.dirac_matrix(U, L, AP, KAPPA)
    return U, D


def _qr_positive(A):
    Q, R = np.linalg.qr(A)
    ph = np.diag(R) / np.abs(np.diag(R))
    return Q * ph[None, :]


def _random_orthonormal(m, n, seed):
    V = synth.random_spinor(m, n, seed)
    Q = _qr_positive(V.reshape(m, -1).T)
    return np.ascontiguousarray(Q.T.reshape(V.shape))


def test_orthonormalize_is_unique_qr():
    V = synth.random_spinor(5, 20, 3)
    Q = projector.orthonormalize(V).reshape(5, -1)
    want = _qr_positive(V.reshape(5, -1).T).T
    assert np.abs(Q - want).max() < 1e-13
    assert np.abs(Q.conj() @ Q.T - np.eye(5)).max() < 1e-13


def test_inverse_iteration_is_subspace_iteration(setup):
    """Orthonormalising after every step spans the same space as D^-k V0 and gives the
    same orthonormal basis: QR of D_Omega^-k V0 with a positive diagonal."""
    U, D = setup
    n = oracle.box_sites(OMEGA[1])
    V0 = synth.random_spinor(4, n, 5)
    got = projector.inverse_iteration(U, L, AP, *OMEGA, KAPPA, V0, 3).reshape(4, -1)
    Dinv = np.linalg.inv(dense.restricted(D, L, *OMEGA))
    X = V0.reshape(4, -1).T
    for _ in range(3):
        X = Dinv @ X
    want = _qr_positive(X).T
    assert np.abs(got - want).max() < 1e-9


def _dense_cut(D, Phi):
    """S~ as a matrix (components of G* x components of Gbar) for the columns Phi on Omega."""
    ib = dense.box_component_index(L, *GBAR)
    istar = dense.box_component_index(L, *GSTAR)
    io = dense.box_component_index(L, *OMEGA)
    Dbar_inv = np.linalg.inv(D[ib][:, ib].toarray())
    Dstar_inv = np.linalg.inv(D[istar][:, istar].toarray())
    star_sites = set((istar // 12).tolist())
    out = np.array([(c // 12) not in star_sites for c in io])
    P = Phi.reshape(Phi.shape[0], -1).T                      # (12 |Omega|, m)
    pos_b = {int(c): i for i, c in enumerate(ib)}
    rows_omega_in_bar = [pos_b[int(c)] for c in io]
    Dd = D[istar][:, io[out]].toarray()
    return -Dstar_inv @ Dd @ P[out] @ P.conj().T @ Dbar_inv[rows_omega_in_bar]


def _dense_pion(St):
    """(1/L^3) sum over the spatial sites of both slices of |S~(y, x)|^2."""
    tb = oracle.domain_maps(L, *GBAR)[0] // VOL3
    ts = oracle.domain_maps(L, *GSTAR)[0] // VOL3
    A = np.abs(St.reshape(ts.size, 12, tb.size, 12)) ** 2
    C = np.zeros((L[0], L[0]))
    for y0 in np.unique(ts):
        for x0 in np.unique(tb):
            C[y0, x0] = A[ts == y0][:, :, tb == x0].sum() / VOL3
    return C


def _oracle_pion(U, phi):
    u, w = projector.factorized_vectors(U, L, AP, KAPPA, GBAR, GSTAR, OMEGA, phi)
    M = projector.gram_slices(L, *GBAR, u)
    Mt = projector.gram_slices(L, *GSTAR, w)
    return projector.projected_pion(Mt, M, VOL3), u, w


def test_projected_pion_matches_dense_cut(setup):
    U, D = setup
    phi = _random_orthonormal(6, oracle.box_sites(OMEGA[1]), 9)
    C, _, _ = _oracle_pion(U, phi)
    want = _dense_pion(_dense_cut(D, phi))
    assert np.abs(C.imag).max() < 1e-12 * np.abs(want).max()
    assert np.linalg.norm(C.real - want) < 1e-10 * np.linalg.norm(want)


def test_complete_basis_on_the_cut_slice_is_exact(setup):
    """D[G*, Gbar minus G*] only reads the slice x0cut - 1: a complete basis there makes
    P act as the identity, and S~ becomes the factorized propagator of Eq. approxlong."""
    U, D = setup
    n_o = oracle.box_sites(OMEGA[1])
    t_o = oracle.domain_maps(L, *OMEGA)[0] // VOL3
    sites = np.flatnonzero(t_o == 3)
    phi = np.zeros((12 * sites.size, n_o, 4, 3), dtype=np.complex128)
    for i, (l, c) in enumerate((l, c) for l in sites for c in range(12)):
        phi[i, l, c // 3, c % 3] = 1.0
    C, _, _ = _oracle_pion(U, phi)
    # exact S^(f) = -D^-1_{G*} D[G*, Gbar minus G*] D^-1_{Gbar}
    ib = dense.box_component_index(L, *GBAR)
    istar = dense.box_component_index(L, *GSTAR)
    star_sites = set((istar // 12).tolist())
    out = np.array([(c // 12) not in star_sites for c in ib])
    Sf = -np.linalg.inv(D[istar][:, istar].toarray()) @ D[istar][:, ib[out]].toarray() @ \
        np.linalg.inv(D[ib][:, ib].toarray())[out]
    want = _dense_pion(Sf)
    assert np.linalg.norm(C.real - want) < 1e-10 * np.linalg.norm(want)
    # a basis that misses part of the slice is only an approximation
    C2, _, _ = _oracle_pion(U, phi[:12 * (sites.size - 1)])
    assert np.linalg.norm(C2.real - want) > 1e-3 * np.linalg.norm(want)


def test_projected_nucleon_matches_dense_cut(setup):
    """The colourless-spinor form of Eq. W0tbary equals the nucleon contraction (Sec. 4,
    W_N1 - W_N2, itself pinned by Wick enumeration) of the dense S~, summed over the
    spatial sites of the source slice."""
    U, D = setup
    phi = _random_orthonormal(4, oracle.box_sites(OMEGA[1]), 13)
    u, w = projector.factorized_vectors(U, L, AP, KAPPA, GBAR, GSTAR, OMEGA, phi)
    g5 = oracle.gamma()[4]
    xi = np.einsum("ab,mnbc->mnac", g5, np.conj(u))
    eta = -w
    X = projector.colourless_spinors(L, *GBAR, xi)
    Y = projector.colourless_spinors(L, *GSTAR, eta)
    C = projector.projected_nucleon(X, Y)
    St = _dense_cut(D, phi)
    gb = oracle.domain_maps(L, *GBAR)[0]
    n_star = oracle.box_sites(GSTAR[1])
    want = np.zeros((L[0], L[0]), dtype=np.complex128)
    for l, site in enumerate(gb):
        cols = St[:, 12 * l:12 * (l + 1)].T.reshape(12, n_star, 4, 3)   # S~(., x) column c = 3 beta + b
        want[:, site // VOL3] += oracle.nucleon(L, *GSTAR, np.ascontiguousarray(cols))
    assert np.linalg.norm(C - want) < 1e-10 * np.linalg.norm(want)
