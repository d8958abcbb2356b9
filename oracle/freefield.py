"""Free-field (unit-link) Wilson propagators in closed form (test infrastructure only).

With U = 1 the operator of App. A is diagonal in momentum space,
    D(p) = m0 + sum_mu (1 - cos p_mu) + i sum_mu gamma_mu sin p_mu,
with p_k = 2 pi n / L_k in space and p_0 = pi (2n+1) / T (antiperiodic) or
2 pi n / T (periodic) in time.  The propagator from the origin is
S(y, 0) = (1/V) sum_p e^{i p y} D(p)^{-1} (colour identity).

For a time slab with Dirichlet faces and periodic space, the spatial momenta
still diagonalise D; for each of them the operator is a 4*Delta x 4*Delta
block-tridiagonal matrix in time that is inverted densely.
"""
from __future__ import annotations

import numpy as np

from . import gamma as _gamma


def momentum_propagator(L, kappa, bc_time=1):
    """S_spin(y) for all y, shape L + (4, 4): S(y,0)_{alpha a, beta b} = delta_ab S_spin(y)_{alpha beta}."""
    L = tuple(int(l) for l in L)
    g = _gamma()
    m0 = 1.0 / (2.0 * kappa) - 4.0
    shift0 = np.pi / L[0] if bc_time == 1 else 0.0
    ps = [2 * np.pi * np.fft.fftfreq(L[m]) * 1.0 + (shift0 if m == 0 else 0.0) for m in range(4)]
    P = np.meshgrid(*ps, indexing="ij")
    scal = m0 + sum(1 - np.cos(P[m]) for m in range(4))
    Dp = scal[..., None, None] * np.eye(4) + 1j * sum(np.sin(P[m])[..., None, None] * g[m] for m in range(4))
    Dinv = np.linalg.inv(Dp)
    # the frequencies from fftfreq are 2 pi k / L with k in FFT order; numpy's
    # ifftn computes (1/N) sum_k X_k exp(+2 pi i k n / N), which is the sum over p.
    S = np.fft.ifftn(Dinv, axes=(0, 1, 2, 3))
    if shift0:
        y0 = np.arange(L[0])
        S = S * np.exp(1j * shift0 * y0)[:, None, None, None, None, None]
    return S


def slab_propagator(L, kappa, t_lo, thickness, src_t):
    """Free propagator on a Dirichlet time slab [t_lo, t_lo+thickness) (mod T),
    periodic space, source at (src_t, 0, 0, 0).  Returns S_spin with shape
    (thickness, L1, L2, L3, 4, 4) in slab-local time."""
    L = tuple(int(l) for l in L)
    g = _gamma()
    m0 = 1.0 / (2.0 * kappa) - 4.0
    D_ = thickness
    ks = [2 * np.pi * np.fft.fftfreq(L[m]) for m in (1, 2, 3)]
    K = np.meshgrid(*ks, indexing="ij")
    out = np.zeros((D_,) + L[1:] + (4, 4), dtype=np.complex128)
    src_local = (src_t - t_lo) % L[0]
    I4 = np.eye(4)
    for i1 in range(L[1]):
        for i2 in range(L[2]):
            for i3 in range(L[3]):
                p = [K[0][i1, i2, i3], K[1][i1, i2, i3], K[2][i1, i2, i3]]
                diag = (m0 + 1.0 + sum(1 - np.cos(p[j]) for j in range(3))) * I4 \
                    + 1j * sum(np.sin(p[j]) * g[1 + j] for j in range(3))
                M = np.zeros((4 * D_, 4 * D_), dtype=np.complex128)
                for t in range(D_):
                    M[4 * t:4 * t + 4, 4 * t:4 * t + 4] = diag
                    if t + 1 < D_:
                        M[4 * t:4 * t + 4, 4 * (t + 1):4 * (t + 1) + 4] = -0.5 * (I4 - g[0])
                        M[4 * (t + 1):4 * (t + 1) + 4, 4 * t:4 * t + 4] = -0.5 * (I4 + g[0])
                Minv = np.linalg.inv(M)
                out[:, i1, i2, i3] = Minv[:, 4 * src_local:4 * src_local + 4].reshape(D_, 4, 4)
    # back to position space: S(y) = (1/L^3) sum_p e^{i p y} S(p)
    out = np.fft.ifftn(out, axes=(1, 2, 3))
    return out
