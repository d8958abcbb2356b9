"""Dense Wilson-Dirac matrix built directly from App. A (test infrastructure only).

The matrix is assembled as D = D_w + m0 with
    D_w = 1/2 sum_mu { gamma_mu (grad*_mu + grad_mu) - grad*_mu grad_mu },
    grad_mu psi(x)  = U_mu(x) psi(x+mu) - psi(x),
    grad*_mu psi(x) = psi(x) - U_mu(x-mu)^+ psi(x-mu),
i.e. from the covariant derivatives themselves rather than the expanded
hopping form used by oracle.c, so the two routes check each other.  The
Dirichlet operator of a box is the sub-block D[Gamma, Gamma] (Eq. blkdec,
Sec. 2).  Periodic and antiperiodic time boundaries only (the antiperiodic
sign is carried by the time links on the last time slice).  Index of a
component: site*12 + spin*3 + colour.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import gamma as _gamma


def _shift_operator(U, L, mu, bc):
    """T_mu with (T_mu psi)(x) = f(x) U_mu(x) psi(x+mu) as a sparse matrix."""
    L = tuple(int(l) for l in L)
    V = int(np.prod(L))
    x = np.indices(L).reshape(4, -1).T
    xp = x.copy()
    xp[:, mu] = (xp[:, mu] + 1) % L[mu]
    site = np.ravel_multi_index(x.T, L)
    nsite = np.ravel_multi_index(xp.T, L)
    f = np.ones(V)
    if mu == 0 and bc == 1:
        f[x[:, 0] == L[0] - 1] = -1.0
    rows, cols, vals = [], [], []
    for s in range(4):
        for a in range(3):
            for b in range(3):
                rows.append(site * 12 + s * 3 + a)
                cols.append(nsite * 12 + s * 3 + b)
                vals.append(f * U[mu, site, a, b])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(12 * V, 12 * V))


def dirac_matrix(U, L, bc, kappa):
    """Sparse D = D_w + m0 on the whole lattice, m0 = 1/(2 kappa) - 4 (Sec. 5)."""
    if bc not in (0, 1):
        raise ValueError("dense construction covers periodic/antiperiodic time only")
    L = tuple(int(l) for l in L)
    V = int(np.prod(L))
    N = 12 * V
    g = _gamma()
    Id = sp.identity(N, dtype=np.complex128, format="csr")
    m0 = 1.0 / (2.0 * kappa) - 4.0
    D = m0 * Id
    for mu in range(4):
        T = _shift_operator(U, L, mu, bc)
        grad = T - Id
        gradstar = Id - T.conj().T
        G = sp.kron(sp.identity(V), sp.kron(g[mu], sp.identity(3)), format="csr")
        D = D + 0.5 * (G @ (gradstar + grad) - gradstar @ grad)
    return D.tocsr()


def box_component_index(L, origin, extent):
    """Global component indices of the box's sites, in domain-local order."""
    L = tuple(int(l) for l in L)
    k = np.indices(tuple(int(e) for e in extent)).reshape(4, -1).T
    x = (k + np.asarray(origin)[None, :]) % np.asarray(L)[None, :]
    site = np.ravel_multi_index(x.T, L)
    return (site[:, None] * 12 + np.arange(12)[None, :]).reshape(-1)


def restricted(D, L, origin, extent):
    """D_Gamma = D[Gamma, Gamma] (Eq. blkdec) as a dense array."""
    idx = box_component_index(L, origin, extent)
    return D[idx][:, idx].toarray()


def boundary_source(U, L, bc, from_box, psi_from, to_box):
    """sigma = -D[Gamma_to, Gamma_from minus Gamma_to] psi_from: the couplings of D (App. A)
    from sites of the `from` box that lie outside the `to` box into the `to` box, i.e.
    the off-diagonal blocks D_dGamma of Eq. blkdec that the Dirichlet boundary of the
    `to` box drops.  With from = Gamma-bar_0, to = Gamma*_0 and psi = D^-1_{Gamma-bar_0} eta,
    D^-1_{Gamma*_0} sigma is the factorized propagator of Eq. approxlong.
    psi_from: (ncol, n_from, 4, 3); returns (ncol, n_to, 4, 3).  The hopping blocks
    do not depend on kappa (any value builds them)."""
    D = dirac_matrix(U, L, bc, 0.125)
    idx_to = box_component_index(L, *to_box)
    idx_from = box_component_index(L, *from_box)
    to_sites = set((idx_to // 12).tolist())
    keep = np.array([(i // 12) not in to_sites for i in idx_from])
    psi = np.asarray(psi_from).reshape(psi_from.shape[0], -1)
    B = D[idx_to][:, idx_from[keep]]
    sigma = -(B @ psi[:, keep].T).T
    n_to = len(idx_to) // 12
    return np.ascontiguousarray(sigma.reshape(psi_from.shape[0], n_to, 4, 3))
