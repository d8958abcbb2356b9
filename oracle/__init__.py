"""FP64 CPU oracle of the domain-restricted Wilson-Dirac propagators.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never imports it.

``oracle.c`` (compiled with gcc/OpenMP into ``liboracle.so`` by ``build()``)
holds the operator, the solver and the contractions; this module is a thin
ctypes wrapper.  ``dense.py`` builds the operator as a dense matrix directly
from the covariant derivatives of App. A, ``freefield.py`` holds the
momentum-space free propagator and ``wick.py`` a brute-force Wick
enumeration of the nucleon correlator; these three pin the C code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

BC_PERIODIC, BC_ANTIPERIODIC, BC_OPEN = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, -O2, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        i4 = ctypes.POINTER(ctypes.c_int)
        dp = ctypes.c_void_p
        L.orc_gamma.argtypes = [dp]
        L.orc_domain_maps.argtypes = [i4, i4, i4, dp, dp, dp]
        L.orc_apply_hop.argtypes = [i4, ctypes.c_int, dp, i4, i4, dp, dp, ctypes.c_int]
        L.orc_apply_dirac.argtypes = [i4, ctypes.c_int, dp, i4, i4, ctypes.c_double, ctypes.c_double, dp, dp,
                                      ctypes.c_int]
        L.orc_solve.argtypes = [i4, ctypes.c_int, dp, i4, i4, ctypes.c_double, ctypes.c_double, dp, dp,
                                ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, dp]
        L.orc_clover_field.argtypes = [i4, dp, ctypes.c_double, dp]
        L.orc_series_term.argtypes = [i4, i4, i4, dp, i4, i4, dp, dp, ctypes.c_int]
        L.orc_contract_local_trace.argtypes = [i4, i4, i4, dp, i4, dp]
        L.orc_contract_pion.argtypes = [i4, i4, i4, dp, dp]
        L.orc_contract_nucleon.argtypes = [i4, i4, i4, dp, dp]
        L.orc_contract_noise_trace.argtypes = [i4, i4, i4, dp, dp, ctypes.c_int, dp]
        L.orc_factorized_correlator.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                dp]
        _lib = L
    return _lib


def _i4(v):
    return (ctypes.c_int * 4)(*[int(x) for x in v])


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def gamma() -> np.ndarray:
    """gamma[0..3] = gamma_mu, gamma[4] = gamma_5 in the oracle's chiral basis."""
    g = np.zeros((5, 4, 4), dtype=np.complex128)
    lib().orc_gamma(_ptr(g))
    return g


def box_sites(extent) -> int:
    return int(extent[0]) * int(extent[1]) * int(extent[2]) * int(extent[3])


def domain_maps(L, origin, extent):
    """(global_index, eo_index, parity) for every site of the box in domain-local order."""
    n = box_sites(extent)
    gi = np.zeros(n, dtype=np.int64)
    eo = np.zeros(n, dtype=np.int64)
    par = np.zeros(n, dtype=np.int8)
    rc = lib().orc_domain_maps(_i4(L), _i4(origin), _i4(extent), _ptr(gi), _ptr(eo), _ptr(par))
    if rc:
        raise ValueError("bad box")
    return gi, eo, par


def apply_hop(U, L, bc, origin, extent, psi):
    U = _c(U)
    psi = _c(psi)
    out = np.zeros_like(psi)
    ncol = psi.shape[0] if psi.ndim == 4 else 1
    rc = lib().orc_apply_hop(_i4(L), bc, _ptr(U), _i4(origin), _i4(extent), _ptr(psi), _ptr(out), ncol)
    if rc:
        raise ValueError("bad arguments")
    return out


def hop_power(U, L, bc, origin, extent, kappa, p, psi):
    """(kappa D_hop)^p psi on the box: p applications of the Dirichlet-restricted
    hopping term (Sec. 2), each scaled by kappa, with 2 kappa D = 1 - kappa D_hop
    (Sec. 5).  With psi = D^-1 g5 eta and p = 8 it is the vector contracted with
    eta in the expanded stochastic trace of Eq. HPEtr."""
    if p < 0:
        raise ValueError("p must be >= 0")
    v = _c(psi)
    for _ in range(p):
        v = kappa * apply_hop(U, L, bc, origin, extent, v)
    return v


def clover_field(U, L, csw):
    """The clover term c_sw (i/4) sum_{mu,nu} sigma_{mu nu} F_{mu nu}(x) of every site,
    shape (V, 12, 12), rows and columns 3 spin + colour."""
    U = _c(U)
    V = int(np.prod(L))
    out = np.zeros((V, 12, 12), dtype=np.complex128)
    if lib().orc_clover_field(_i4(L), _ptr(U), float(csw), _ptr(out)):
        raise ValueError("bad lattice")
    return out


def apply_dirac(U, L, bc, origin, extent, kappa, psi, csw=0.0):
    """D_Gamma psi on the box; psi has shape (ncol, n, 4, 3) or (n, 4, 3).  csw != 0
    adds the clover term (clover_field) at every site of the box."""
    U = _c(U)
    psi = _c(psi)
    out = np.zeros_like(psi)
    ncol = psi.shape[0] if psi.ndim == 4 else 1
    rc = lib().orc_apply_dirac(_i4(L), bc, _ptr(U), _i4(origin), _i4(extent), float(kappa), float(csw),
                               _ptr(psi), _ptr(out), ncol)
    if rc:
        raise ValueError("bad arguments")
    return out


def solve(U, L, bc, origin, extent, kappa, eta, tol=1e-12, maxit=100000, csw=0.0):
    """psi = D_Gamma^-1 eta per column; returns (psi, iters, relres, status)."""
    U = _c(U)
    eta = _c(eta)
    psi = np.zeros_like(eta)
    ncol = eta.shape[0]
    it = np.zeros(ncol, dtype=np.int32)
    rr = np.zeros(ncol, dtype=np.float64)
    st = lib().orc_solve(_i4(L), bc, _ptr(U), _i4(origin), _i4(extent), float(kappa), float(csw), _ptr(eta),
                         _ptr(psi), ncol, float(tol), int(maxit), _ptr(it), _ptr(rr))
    if st == 1:
        raise ValueError("bad arguments")
    return psi, it, rr, st


def local_index(L, origin, extent, x):
    k = [((int(x[m]) - int(origin[m])) % int(L[m])) for m in range(4)]
    if any(k[m] >= int(extent[m]) for m in range(4)):
        raise ValueError("site outside the box")
    return ((k[0] * extent[1] + k[1]) * extent[2] + k[2]) * extent[3] + k[3]


def propagator(U, L, bc, origin, extent, kappa, src, tol=1e-12, maxit=100000, csw=0.0):
    """12-column point-source propagator S(., x) on the box (columns 3*spin+colour)."""
    n = box_sites(extent)
    eta = np.zeros((12, n, 4, 3), dtype=np.complex128)
    l = local_index(L, origin, extent, src)
    for c in range(12):
        eta[c, l, c // 3, c % 3] = 1.0
    return solve(U, L, bc, origin, extent, kappa, eta, tol, maxit, csw)


def series_term(L, small_o, small_e, S_small, big_o, big_e, S_big):
    S_small = _c(S_small)
    S_big = _c(S_big)
    T = np.zeros_like(S_big)
    rc = lib().orc_series_term(_i4(L), _i4(small_o), _i4(small_e), _ptr(S_small), _i4(big_o), _i4(big_e),
                               _ptr(S_big), _ptr(T), S_big.shape[0])
    if rc:
        raise ValueError("small box not inside big box")
    return T


def _twelve_columns(S, extent):
    """The point-source contractions read exactly 12 columns of the box."""
    if S.shape != (12, box_sites(extent), 4, 3):
        raise ValueError(f"expected a 12-column propagator of shape (12, {box_sites(extent)}, 4, 3), got {S.shape}")


def local_trace(L, origin, extent, S, src):
    S = _c(S)
    _twelve_columns(S, extent)
    out = np.zeros(2)
    if lib().orc_contract_local_trace(_i4(L), _i4(origin), _i4(extent), _ptr(S), _i4(src), _ptr(out)):
        raise ValueError("source outside the box")
    return complex(out[0], out[1])


def pion(L, origin, extent, S):
    S = _c(S)
    _twelve_columns(S, extent)
    out = np.zeros(int(L[0]))
    lib().orc_contract_pion(_i4(L), _i4(origin), _i4(extent), _ptr(S), _ptr(out))
    return out


def nucleon(L, origin, extent, S):
    S = _c(S)
    _twelve_columns(S, extent)
    out = np.zeros(2 * int(L[0]))
    lib().orc_contract_nucleon(_i4(L), _i4(origin), _i4(extent), _ptr(S), _ptr(out))
    return out[0::2] + 1j * out[1::2]


def noise_trace(L, origin, extent, eta, psi):
    eta = _c(eta)
    psi = _c(psi)
    out = np.zeros(2 * int(L[0]))
    lib().orc_contract_noise_trace(_i4(L), _i4(origin), _i4(extent), _ptr(eta), _ptr(psi), eta.shape[0],
                                   _ptr(out))
    return out[0::2] + 1j * out[1::2]


def factorized_correlator(TA, TB, L0, vol3):
    """C[y0][x0] = (1/L^3) mean_v TA[v][x0] * mean_w TB[w][y0] (Eq. factsing)."""
    TA = _c(TA)
    TB = _c(TB)
    C = np.zeros((L0, L0), dtype=np.complex128)
    if lib().orc_factorized_correlator(_ptr(TA), TA.shape[0], _ptr(TB), TB.shape[0], int(L0), float(vol3), _ptr(C)):
        raise ValueError("bad arguments")
    return C
