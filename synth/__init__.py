"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds input generators only: random SU(3) gauge fields, the
tuning of their disorder, point/noise sources and the sizes of the standard
workloads.  It contains none of the arithmetic of the method itself (no
Dirac operator, solver, restriction or contraction), so that the FP64 oracle
and the CUDA path stay independent while consuming bit-identical inputs.

Gauge-field recipe (a synthetic stand-in for the quenched beta=6.0 ensembles
the paper measures on, Sec. 5): every link is drawn independently as
U = exp(i eps H), H = sum_a h_a lambda_a / 2 with h_a ~ N(0,1) and lambda_a the
Gell-Mann matrices.  eps is tuned so that the mean plaquette is 0.59.  Because
links are independent and the law of H is invariant under conjugation,
E[U] = c 1 with c = E[Re tr U / 3], hence E[plaquette] = c^4 exactly; the
tuning solves c(eps)^4 = 0.59 on a large single-link Monte Carlo sample.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Fixed seeds of the standard synthetic workloads.
SEED_GAUGE = 1601045871
SEED_VARIANT0 = 1601045872
SEED_NOISE0 = 1601045900
SEED_SERVING = 1601045999
SEED_TUNE = 1601045000

TARGET_PLAQUETTE = 0.59


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3) complex128."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / math.sqrt(3)
    lam[7][2, 2] = -2 / math.sqrt(3)
    return lam


_LAM = gell_mann()


def random_hermitian(n: int, rng: np.random.Generator) -> np.ndarray:
    """n traceless Hermitian matrices H = sum_a h_a lambda_a / 2, h_a ~ N(0,1)."""
    h = rng.standard_normal((n, 8))
    return np.einsum("na,aij->nij", h, _LAM) * 0.5


def exp_i_eps_h(H: np.ndarray, eps: float) -> np.ndarray:
    """U = exp(i eps H) through the Hermitian eigendecomposition (exactly SU(3))."""
    w, v = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    return np.einsum("nij,nj,nkj->nik", v, ph, np.conj(v))


def random_su3(n: int, eps: float, rng: np.random.Generator, chunk: int = 1 << 20) -> np.ndarray:
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        out[a:b] = exp_i_eps_h(random_hermitian(b - a, rng), eps)
    return out


def mean_link_trace(eps: float, n: int = 400_000, seed: int = SEED_TUNE) -> float:
    """Monte Carlo estimate of c(eps) = E[Re tr U / 3] with a fixed sample."""
    rng = np.random.default_rng(seed)
    H = random_hermitian(n, rng)
    U = exp_i_eps_h(H, eps)
    return float(np.mean(np.real(np.trace(U, axis1=1, axis2=2))) / 3.0)


_EPS_CACHE: dict = {}


def tune_eps(target: float = TARGET_PLAQUETTE, n: int = 400_000, seed: int = SEED_TUNE) -> float:
    """eps such that c(eps)^4 = target, by bisection on a fixed single-link sample."""
    key = (target, n, seed)
    if key in _EPS_CACHE:
        return _EPS_CACHE[key]
    rng = np.random.default_rng(seed)
    H = random_hermitian(n, rng)
    w, v = np.linalg.eigh(H)

    def c4(eps):
        # Re tr exp(i eps H) = sum_j cos(eps w_j)
        return (np.mean(np.sum(np.cos(eps * w), axis=1)) / 3.0) ** 4

    lo, hi = 0.0, 3.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if c4(mid) > target:
            lo = mid
        else:
            hi = mid
    eps = 0.5 * (lo + hi)
    _EPS_CACHE[key] = eps
    return eps


def volume(L) -> int:
    return int(L[0]) * int(L[1]) * int(L[2]) * int(L[3])


def gauge_field(L, seed: int = SEED_GAUGE, eps: float | None = None) -> np.ndarray:
    """Seeded gauge field, shape (4, V, 3, 3) complex128; site index
    ((x0*L1 + x1)*L2 + x2)*L3 + x3, direction 0 is time."""
    if eps is None:
        eps = tune_eps()
    V = volume(L)
    rng = np.random.default_rng(seed)
    U = random_su3(4 * V, eps, rng)
    return U.reshape(4, V, 3, 3)


def unit_gauge_field(L) -> np.ndarray:
    V = volume(L)
    U = np.zeros((4, V, 3, 3), dtype=np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1
    return U


def site_coords(L) -> np.ndarray:
    """(V, 4) int64 coordinates of every site in lexicographic order."""
    g = np.indices(tuple(int(l) for l in L)).reshape(4, -1).T
    return g.astype(np.int64)


def plaquette(U: np.ndarray, L) -> float:
    """Mean plaquette (1/(18 V)) sum_x sum_{mu<nu} Re tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+.
    Used only to tune and check the synthetic gauge recipe."""
    L = tuple(int(l) for l in L)
    V = volume(L)
    Ur = U.reshape((4,) + L + (3, 3))
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            a = Ur[mu]
            b = np.roll(Ur[nu], -1, axis=mu)
            c = np.conj(np.swapaxes(np.roll(Ur[mu], -1, axis=nu), -1, -2))
            d = np.conj(np.swapaxes(Ur[nu], -1, -2))
            p = a @ b @ c @ d
            tot += float(np.sum(np.real(np.trace(p, axis1=-2, axis2=-1))))
    return tot / (18.0 * V)


def random_gauge_transform(V: int, seed: int) -> np.ndarray:
    """V independent random SU(3) matrices (large eps: far from the identity)."""
    rng = np.random.default_rng(seed)
    return random_su3(V, 2.5, rng)


def variant_field(U_base: np.ndarray, L, t_lo: int, t_hi: int, seed: int,
                  eps: float | None = None) -> np.ndarray:
    """A level-1 variant of a time region [t_lo, t_hi): every link with both
    endpoints in the region is redrawn with the same eps, except the spatial
    links on the region's first time slice, which stay frozen (the paper keeps
    the spatial links at the cut fixed, Sec. 5).  Links leaving the region are
    unchanged."""
    if eps is None:
        eps = tune_eps()
    L = tuple(int(l) for l in L)
    V = volume(L)
    U = U_base.copy()
    x = site_coords(L)
    t = x[:, 0]
    in_region = (t >= t_lo) & (t < t_hi)
    rng = np.random.default_rng(seed)
    for mu in range(4):
        if mu == 0:
            sel = in_region & (t + 1 < t_hi)
        else:
            sel = in_region & (t != t_lo)
        idx = np.nonzero(sel)[0]
        U[mu, idx] = random_su3(idx.size, eps, rng)
    assert U.shape == (4, V, 3, 3)
    return U


def point_source_columns(n_sites: int, local_index: int) -> np.ndarray:
    """12 point-source columns on a domain, shape (12, n_sites, 4, 3): column
    c = 3*beta + b is 1 at (local_index, beta, b)."""
    eta = np.zeros((12, n_sites, 4, 3), dtype=np.complex128)
    for c in range(12):
        eta[c, local_index, c // 3, c % 3] = 1.0
    return eta


def noise_field(n_sites: int, seed: int) -> np.ndarray:
    """Complex Gaussian noise z(x) with E|z|^2 = 1, shape (n_sites,)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n_sites) + 1j * rng.standard_normal(n_sites)) / math.sqrt(2.0)


def diluted_noise_columns(z: np.ndarray) -> np.ndarray:
    """Spin-colour diluted volume sources eta_c(x) = z(x) e_c, shape (12, n, 4, 3)."""
    n = z.shape[0]
    eta = np.zeros((12, n, 4, 3), dtype=np.complex128)
    for c in range(12):
        eta[c, :, c // 3, c % 3] = z
    return eta


def random_spinor(ncol: int, n_sites: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((ncol, n_sites, 4, 3))
            + 1j * rng.standard_normal((ncol, n_sites, 4, 3)))


@dataclass(frozen=True)
class Box:
    origin: tuple
    extent: tuple

    @property
    def n_sites(self) -> int:
        return volume(self.extent)


def centered_time_slab(L, thickness: int, t_center: int = 0) -> Box:
    """Time slab [t_center - thickness/2, t_center + thickness/2 - 1] (mod T), full space."""
    o0 = (t_center - thickness // 2) % L[0]
    ext0 = thickness if thickness < L[0] else L[0]
    return Box((o0, 0, 0, 0), (ext0, L[1], L[2], L[3]))


# --- standard workload shapes (sizes only) -------------------------------------------

SMALL_LATTICE = (8, 4, 4, 4)        # plain FP64 case, kappa 0.120, full lattice
SMALL_KAPPA = 0.120
SLAB_LATTICE = (48, 24, 24, 24)     # nested slabs 8, 16, 24 and the full lattice
SLAB_KAPPA = 0.1550
SLAB_THICKNESS = (8, 16, 24)
BATCH_LATTICE = (32, 32, 32, 32)    # 256 blocks 8^4, 32 slabs 4x32^3, 16 slabs 8x32^3
BATCH_KAPPA = 0.1550
MULTILEVEL_LATTICE = (64, 32, 32, 32)
MULTILEVEL_KAPPA = 0.1550
MULTILEVEL_VARIANTS = 32


def batch_boxes(L=BATCH_LATTICE):
    """The uneven batch: 8^4 blocks tiling the lattice, 4xL^3 slabs at every t0,
    8xL^3 slabs at even t0."""
    boxes = []
    T, X, Y, Z = L
    for t in range(0, T, 8):
        for x in range(0, X, 8):
            for y in range(0, Y, 8):
                for z in range(0, Z, 8):
                    boxes.append(Box((t, x, y, z), (8, 8, 8, 8)))
    for t in range(T):
        boxes.append(Box((t, 0, 0, 0), (4, X, Y, Z)))
    for t in range(0, T, 2):
        boxes.append(Box((t, 0, 0, 0), (8, X, Y, Z)))
    return boxes


def box_center(box: Box):
    return tuple(box.origin[m] + box.extent[m] // 2 for m in range(4))


# --- the same recipe with torch (CUDA or CPU), for the large lattices ----------------

def _torch_gell_mann(torch, device):
    return torch.from_numpy(_LAM).to(device)


def _expm_i_eps_h_torch(H, eps):
    """exp(i eps H) for a batch of 3x3 Hermitian H by scaling and squaring of
    the Taylor series (order 14 after dividing by 2^5): the same matrix as the
    eigendecomposition route up to rounding, with batched matrix products only."""
    import torch
    A = (1j * eps / 32.0) * H
    n = H.shape[0]
    I = torch.eye(3, dtype=H.dtype, device=H.device).expand(n, 3, 3)
    P = I.clone()
    for k in range(14, 0, -1):
        P = I + (A @ P) / k
    for _ in range(5):
        P = P @ P
    return P


def random_su3_torch(n: int, eps: float, generator, device, chunk: int = 1 << 21):
    """n links exp(i eps H) drawn with a torch.Generator (same law as random_su3)."""
    import torch
    lam = _torch_gell_mann(torch, device)
    out = torch.empty((n, 3, 3), dtype=torch.complex128, device=device)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        h = torch.randn((b - a, 8), dtype=torch.float64, device=device, generator=generator)
        H = torch.einsum("na,aij->nij", h.to(torch.complex128), lam) * 0.5
        out[a:b] = _expm_i_eps_h_torch(H, eps)
    return out


def gauge_field_torch(L, seed: int = SEED_GAUGE, device="cuda", eps: float | None = None):
    """Seeded gauge field (4, V, 3, 3) complex128 on `device` (torch RNG stream)."""
    import torch
    if eps is None:
        eps = tune_eps()
    V = volume(L)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return random_su3_torch(4 * V, eps, g, device).reshape(4, V, 3, 3)


def variant_field_torch(U_base, L, t_lo: int, t_hi: int, seed: int, eps: float | None = None):
    """Torch version of variant_field: links with both ends in [t_lo, t_hi) redrawn,
    the spatial links of the region's first slice frozen."""
    import torch
    if eps is None:
        eps = tune_eps()
    L = tuple(int(l) for l in L)
    dev = U_base.device
    U = U_base.clone()
    slab = L[1] * L[2] * L[3]
    t = torch.arange(volume(L), device=dev) // slab
    in_region = (t >= t_lo) & (t < t_hi)
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed))
    for mu in range(4):
        sel = in_region & ((t + 1 < t_hi) if mu == 0 else (t != t_lo))
        idx = torch.nonzero(sel).flatten()
        U[mu, idx] = random_su3_torch(idx.numel(), eps, g, dev)
    return U
