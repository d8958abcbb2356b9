"""Projector-cut factorization of the pion and nucleon propagators (Sec. 5).

TEST INFRASTRUCTURE ONLY: a plain FP64 restatement, loaded by the tests, the
smoke check and the CPU-baseline leg of the benchmark; the CUDA library
never uses it.

The factorized propagator of Eq. approxlong, S^(f) = -D^-1_{G*} D_dG* D^-1_{Gbar},
is cut with the projector P = sum_i phi_i phi_i^+ on N_m orthonormal vectors
(Eq. proj; printed with its arguments in the other order, read as the
projector that acts on a field from the left), which gives Eq. approxlong2:
    S~(y, x) = - sum_i [D^-1_{G*} D_dG* phi_i](y) [phi_i^+ D^-1_{Gbar}](x).
With u_i = D^-1_{Gbar} g5 phi_i and w_i = D^-1_{G*} sigma_i, sigma_i = -D[G*, Omega \\ G*] phi_i
(so that w_i = -D^-1_{G*} D_dG* phi_i), gamma_5-hermiticity (Eq. g5h) gives
[phi_i^+ D^-1_{Gbar} g5](x) = u_i(x)^+, so that
  - the pion blocks of Eq. Bpions are B_ij(x) = u_i(x)^+ u_j(x) and
    B~_ij(y) = w_i(y)^+ w_j(y), and W~ = sum_ij B~_ij(y) B_ji(x) (Eq. fullfactpi);
  - xi_i(x) = g5 conj(u_i(x)) (the spinor of the row xi_i^T = phi_i^+ D^-1_{Gbar}) and
    eta_i(y) = -w_i(y) enter the colourless spinors
    B[s_i, s_j, s_k; x]_alpha = eps^{abc} (s_i^a)^T C g5 s_j^b (s_k^c)_alpha
    of the nucleon contractions (Eq. W0tbary; see projected_nucleon for the reading).

The vectors phi_i come from inverse iteration of the Dirichlet operator of the
thick time slice Omega (Sec. 5: 10 iterations on random vectors), read as
subspace iteration: V <- orthonormalize(D_Omega^-1 V) at every step, modified
Gram-Schmidt in column order.

Time-slice sums (x0 / y0 global) are returned for every global slice; slices
outside the box are zero.
"""
from __future__ import annotations

import numpy as np

from . import BC_OPEN, domain_maps, gamma, solve


def orthonormalize(V):
    """Modified Gram-Schmidt of the columns V[c] (shape (m, n, 4, 3)) in column
    order; returns the orthonormal columns (the Q of V = QR with R's diagonal
    real and positive)."""
    Q = np.array(V, dtype=np.complex128, copy=True).reshape(V.shape[0], -1)
    for i in range(Q.shape[0]):
        for j in range(i):
            Q[i] -= np.vdot(Q[j], Q[i]) * Q[j]
        Q[i] /= np.linalg.norm(Q[i])
    return Q.reshape(V.shape)


def inverse_iteration(U, L, bc, origin, extent, kappa, V0, iters, csw=0.0, tol=1e-12):
    """N_m orthonormal vectors on the box: `iters` times V <- orthonormalize(D_box^-1 V)
    starting from V0 (the random vectors, passed in)."""
    V = orthonormalize(V0)
    for _ in range(iters):
        X, _, _, st = solve(U, L, bc, origin, extent, kappa, V, tol=tol, csw=csw)
        if st:
            raise RuntimeError("inverse iteration: solve did not converge")
        V = orthonormalize(X)
    return V


def _slice_of_sites(L, origin, extent):
    gi, _, _ = domain_maps(L, origin, extent)
    return gi // (int(L[1]) * int(L[2]) * int(L[3]))


def gram_slices(L, origin, extent, A):
    """M[t][i][j] = sum_{x vec at time t} sum_{spin, colour} conj(A_i(x)) A_j(x)."""
    t = _slice_of_sites(L, origin, extent)
    m = A.shape[0]
    Af = A.reshape(m, -1, 12)
    M = np.zeros((int(L[0]), m, m), dtype=np.complex128)
    for s in np.unique(t):
        sel = Af[:, t == s, :].reshape(m, -1)
        M[s] = np.conj(sel) @ sel.T
    return M


def _cg5():
    g = gamma()
    C = 1j * g[0] @ g[2]
    return C @ g[4]


def colourless_spinors(L, origin, extent, S):
    """X[t][i][j][k][alpha] = sum_{x vec at time t} B[s_i, s_j, s_k; x]_alpha with
    B[s_i, s_j, s_k; x]_alpha = eps^{abc} sum_{beta gamma} s_i(x)_{beta a} (C g5)_{beta gamma}
    s_j(x)_{gamma b} s_k(x)_{alpha c}  (C = i g0 g2; S: (m, n, 4, 3))."""
    t = _slice_of_sites(L, origin, extent)
    m = S.shape[0]
    eps = np.zeros((3, 3, 3))
    for a, b, c in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        eps[a, b, c], eps[a, c, b] = 1.0, -1.0
    cg5 = _cg5()
    X = np.zeros((int(L[0]), m, m, m, 4), dtype=np.complex128)
    for s in np.unique(t):
        v = S[:, t == s]                                   # (m, ns, 4, 3)
        d = np.einsum("inba,bc,jncd->nijad", v, cg5, v)   # diquark (s_i^a)^T C g5 s_j^d per site
        X[s] = np.einsum("abc,nijab,knec->ijke", eps, d, v, optimize=True)
    return X


def projected_pion(Mt, M, vol3):
    """C(y0, x0) = (1/L^3) sum_{x vec, y vec} W~(y, x) = (1/L^3) sum_ij Mt_ij(y0) M_ji(x0)
    (Eq. fullfactpi summed over the two time slices)."""
    return np.einsum("yij,xji->yx", Mt, M) / float(vol3)


def projected_nucleon(X, Y):
    """C(y0, x0) = sum_{x vec, y vec} [W~_N1 - W~_N2](y, x): the nucleon contractions of
    Sec. 4 (W_N1 - W_N2) with S~ = -sum_i eta_i xi_i^T of Eq. approxlong2 substituted,
    X built from xi (x side), Y from eta (y side):
      W~_N1 = sum_ijk X_{jik}^T P- Y_{ijk},   W~_N2 = sum_ijk X_{kij}^T P- Y_{ijk}.
    (Eq. W0tbary prints -sum ... g5 P- between the spinors; the substitution, worked out
    term by term, has P- and a plus sign; the printed form corresponds to an x-side
    spinor carrying an extra -g5.)"""
    g = gamma()
    Pm = 0.5 * (np.eye(4) - g[0])
    n1 = np.einsum("xjika,ab,yijkb->yx", X, Pm, Y)
    n2 = np.einsum("xkija,ab,yijkb->yx", X, Pm, Y)
    return n1 - n2


def factorized_vectors(U, L, bc, kappa, gbar, gstar, omega, phi, csw=0.0, tol=1e-12):
    """u_i = D^-1_{Gbar} g5 phi_i on Gbar and w_i = D^-1_{G*} sigma_i on G* with
    sigma_i = -D[G*, Omega minus G*] phi_i (phi_i on Omega, inside Gbar)."""
    from . import dense
    g5 = gamma()[4]
    m = phi.shape[0]
    gi_b, _, _ = domain_maps(L, *gbar)
    gi_o, _, _ = domain_maps(L, *omega)
    pos = {int(s): i for i, s in enumerate(gi_b)}
    src = np.zeros((m, gi_b.size, 4, 3), dtype=np.complex128)
    src[:, [pos[int(s)] for s in gi_o]] = np.einsum("ab,mnbc->mnac", g5, phi)
    u, _, _, st = solve(U, L, bc, *gbar, kappa, src, tol=tol, csw=csw)
    if st:
        raise RuntimeError("solve on Gamma-bar did not converge")
    if bc == BC_OPEN:
        raise ValueError("the dense boundary coupling covers periodic and antiperiodic time")
    sigma = dense.boundary_source(U, L, bc, omega, phi, gstar)
    w, _, _, st = solve(U, L, bc, *gstar, kappa, sigma, tol=tol, csw=csw)
    if st:
        raise RuntimeError("solve on Gamma* did not converge")
    return u, w

