"""Domain-restricted Wilson-Dirac quark propagators on GB300 (sm_103a).

Thin Python binding of the C ABI in ``include/ddp.h`` (libddp.so, built by
``paper_1601_04587_gb300.build``).  Every function below marshals arguments
and calls the C entry point of the same name; all computation runs in the
library's CUDA kernels.  Arrays may be torch tensors (CUDA or CPU) or numpy
arrays; complex arrays are complex128.  There is no CPU fallback: importing
the binding without the compiled library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libddp.so")

DDP_OK, DDP_ERR_INVALID_ARG, DDP_ERR_UNSUPPORTED, DDP_ERR_OOM = 0, 1, 2, 3
DDP_ERR_NOT_CONVERGED, DDP_ERR_CUDA, DDP_ERR_BUSY, DDP_ERR_NOT_FOUND = 4, 5, 6, 7
DDP_BC_PERIODIC, DDP_BC_ANTIPERIODIC, DDP_BC_OPEN = 0, 1, 2
DDP_PREC_FP64, DDP_PREC_MIXED_FP32, DDP_PREC_MIXED_FP16, DDP_PREC_MIXED_BF16 = 0, 1, 2, 3
DDP_CONTRACT_PSEUDO_LOCAL, DDP_CONTRACT_PSEUDO_NOISE, DDP_CONTRACT_NUCLEON, DDP_CONTRACT_PION = 0, 1, 2, 3
DDP_HOP_PLAIN, DDP_HOP_SCHUR_RHAT, DDP_HOP_SCHUR_TS = 0, 1, 2
PRECISIONS = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}
DDP_INFO_COLS = 12


class ddp_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("ncol", ctypes.c_int), ("outer_cycles", ctypes.c_int),
                ("inner_iters", ctypes.c_int), ("max_rel_residual", ctypes.c_double),
                ("rel_residual", ctypes.c_double * DDP_INFO_COLS), ("seconds", ctypes.c_double),
                ("column_iters", ctypes.c_int64)]


class ddp_solve_req(ctypes.Structure):
    _fields_ = [("domain_id", ctypes.c_int), ("kappa", ctypes.c_double), ("csw", ctypes.c_double),
                ("src", ctypes.c_int * 4), ("eta", ctypes.c_void_p), ("ncol", ctypes.c_int),
                ("tol", ctypes.c_double), ("out", ctypes.c_void_p)]


class DDPError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        msg = f"{where}: {error_string(status)} ({status})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


_lib = None


def lib():
    """The loaded libddp.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libddp.so is missing ({LIB_PATH}); build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        i4 = ctypes.POINTER(ctypes.c_int)
        sig = {
            "ddp_error_string": ([i], ctypes.c_char_p),
            "ddp_last_error": ([vp], ctypes.c_char_p),
            "ddp_version": ([], i),
            "ddp_create": ([ctypes.POINTER(vp), i, vp], i),
            "ddp_destroy": ([vp], i),
            "ddp_set_stream": ([vp, vp], i),
            "ddp_load_gauge": ([vp, vp, i4, i, i4], i),
            "ddp_load_gauge_region": ([vp, i, i4, i4, vp, i4], i),
            "ddp_free_gauge": ([vp, i], i),
            "ddp_set_domain": ([vp, i, i4, i4, i4], i),
            "ddp_free_domain": ([vp, i], i),
            "ddp_domain_sites": ([vp, i, ctypes.POINTER(ctypes.c_int64), vp, vp], i),
            "ddp_apply_dirac": ([vp, i, d, d, vp, vp, i, i], i),
            "ddp_hop_power": ([vp, i, d, i, vp, vp, i], i),
            "ddp_boundary_source": ([vp, i, vp, i, vp, i], i),
            "ddp_solve_propagator": ([vp, i, d, d, i4, d, i, vp, ctypes.POINTER(ddp_solve_info)], i),
            "ddp_solve_sources": ([vp, i, d, d, vp, i, d, i, vp, ctypes.POINTER(ddp_solve_info)], i),
            "ddp_solve_batch": ([vp, ctypes.POINTER(ddp_solve_req), i, i, ctypes.POINTER(ddp_solve_info)], i),
            "ddp_series_terms": ([vp, i, vp, i, vp, vp, i], i),
            "ddp_contract": ([vp, i, i, vp, vp, i, i4, vp], i),
            "ddp_serve_config": ([vp, ctypes.c_uint64, i, i], i),
            "ddp_submit": ([vp, ctypes.POINTER(ddp_solve_req), ctypes.POINTER(ctypes.c_uint64)], i),
            "ddp_serve_step": ([vp, i4], i),
            "ddp_poll": ([vp, ctypes.c_uint64, i4, ctypes.POINTER(ddp_solve_info)], i),
            "ddp_serve_reset": ([vp], i),
            "ddp_set_param": ([vp, ctypes.c_char_p, d], i),
            "ddp_get_param": ([vp, ctypes.c_char_p, ctypes.POINTER(d)], i),
            "ddp_time_hop": ([vp, i, d, i, i, i, i, ctypes.POINTER(ctypes.c_float),
                              ctypes.POINTER(ctypes.c_double)], i),
            "ddp_kernel_launches": ([vp], ctypes.c_long),
            "ddp_contract_static": ([i, i4, i4, i4, vp, vp, i, i4, vp, vp], i),
            "ddp_factorized_correlator": ([vp, vp, i, vp, i, i, d, vp], i),
            "ddp_autotune": ([vp, i, d, i, i, i, i4, ctypes.POINTER(ctypes.c_float)], i),
            "ddp_propagator_series": ([vp, i, i4, d, d, i4, d, i, ctypes.POINTER(vp), ctypes.POINTER(vp), i, vp,
                                       ctypes.POINTER(ddp_solve_info)], i),
            "ddp_orthonormalize": ([vp, i, vp, i], i),
            "ddp_inverse_iteration": ([vp, i, d, d, vp, i, i, d, i, ctypes.POINTER(ddp_solve_info)], i),
            "ddp_embed": ([vp, i, vp, i, vp, i, i], i),
            "ddp_gram_slices": ([vp, i, vp, i, vp], i),
            "ddp_colourless_slices": ([vp, i, vp, i, i, vp], i),
            "ddp_projected_pion": ([vp, i, i, vp, vp, d, vp], i),
            "ddp_projected_nucleon": ([vp, i, i, vp, vp, vp], i),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols():
    """Names of the C entry points the binding expects in libddp.so."""
    lib()
    return [n for n in dir(_lib) if n.startswith("ddp_")]


def error_string(status: int) -> str:
    return lib().ddp_error_string(int(status)).decode()


def _i4(v):
    return (ctypes.c_int * 4)(*[int(x) for x in v])


def _ptr(a):
    """Raw pointer of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def _check(ctx, rc, where, allow=()):
    if rc != DDP_OK and rc not in allow:
        detail = lib().ddp_last_error(ctx).decode() if ctx else ""
        raise DDPError(rc, where, detail)
    return rc


# ------------------------------------------------------------- C ABI mirror

def ddp_create(device: int = 0, stream=None):
    h = ctypes.c_void_p()
    s = ctypes.c_void_p(int(stream)) if stream else None
    _check(None, lib().ddp_create(ctypes.byref(h), int(device), s), "ddp_create")
    return h


def ddp_destroy(ctx):
    return _check(ctx, lib().ddp_destroy(ctx), "ddp_destroy")


def ddp_set_stream(ctx, stream):
    return _check(ctx, lib().ddp_set_stream(ctx, ctypes.c_void_p(int(stream)) if stream else None), "ddp_set_stream")


def ddp_load_gauge(ctx, U, L, time_bc=DDP_BC_ANTIPERIODIC) -> int:
    gid = ctypes.c_int()
    _check(ctx, lib().ddp_load_gauge(ctx, _ptr(U), _i4(L), int(time_bc), ctypes.byref(gid)), "ddp_load_gauge")
    return gid.value


def ddp_load_gauge_region(ctx, base_gauge_id, origin, extent, U_box) -> int:
    gid = ctypes.c_int()
    _check(ctx, lib().ddp_load_gauge_region(ctx, int(base_gauge_id), _i4(origin), _i4(extent), _ptr(U_box),
                                            ctypes.byref(gid)), "ddp_load_gauge_region")
    return gid.value


def ddp_free_gauge(ctx, gauge_id):
    return _check(ctx, lib().ddp_free_gauge(ctx, int(gauge_id)), "ddp_free_gauge")


def ddp_set_domain(ctx, gauge_id, origin, extent) -> int:
    did = ctypes.c_int()
    _check(ctx, lib().ddp_set_domain(ctx, int(gauge_id), _i4(origin), _i4(extent), ctypes.byref(did)),
           "ddp_set_domain")
    return did.value


def ddp_free_domain(ctx, domain_id):
    return _check(ctx, lib().ddp_free_domain(ctx, int(domain_id)), "ddp_free_domain")


def ddp_domain_sites(ctx, domain_id, global_index_out=None, eo_index_out=None) -> int:
    n = ctypes.c_int64()
    _check(ctx, lib().ddp_domain_sites(ctx, int(domain_id), ctypes.byref(n), _ptr(global_index_out),
                                       _ptr(eo_index_out)), "ddp_domain_sites")
    return n.value


def ddp_apply_dirac(ctx, domain_id, kappa, psi, out, ncol, precision=DDP_PREC_FP64, csw=0.0):
    return _check(ctx, lib().ddp_apply_dirac(ctx, int(domain_id), float(kappa), float(csw), _ptr(psi), _ptr(out),
                                             int(ncol), int(precision)), "ddp_apply_dirac")


def ddp_hop_power(ctx, domain_id, kappa, p, psi, out, ncol=12):
    return _check(ctx, lib().ddp_hop_power(ctx, int(domain_id), float(kappa), int(p), _ptr(psi), _ptr(out), int(ncol)),
                  "ddp_hop_power")


def ddp_boundary_source(ctx, domain_from, psi, domain_to, sigma, ncol=12):
    return _check(ctx, lib().ddp_boundary_source(ctx, int(domain_from), _ptr(psi), int(domain_to), _ptr(sigma),
                                                 int(ncol)), "ddp_boundary_source")


def ddp_solve_propagator(ctx, domain_id, kappa, csw, src, tol, precision, S_out, raise_on_fail=False):
    info = ddp_solve_info()
    rc = lib().ddp_solve_propagator(ctx, int(domain_id), float(kappa), float(csw), _i4(src), float(tol),
                                    int(precision), _ptr(S_out), ctypes.byref(info))
    _check(ctx, rc, "ddp_solve_propagator", allow=() if raise_on_fail else (DDP_ERR_NOT_CONVERGED,))
    return rc, info


def ddp_solve_sources(ctx, domain_id, kappa, csw, eta, ncol, tol, precision, psi_out, raise_on_fail=False):
    info = ddp_solve_info()
    rc = lib().ddp_solve_sources(ctx, int(domain_id), float(kappa), float(csw), _ptr(eta), int(ncol), float(tol),
                                 int(precision), _ptr(psi_out), ctypes.byref(info))
    _check(ctx, rc, "ddp_solve_sources", allow=() if raise_on_fail else (DDP_ERR_NOT_CONVERGED,))
    return rc, info


def make_req(domain_id, kappa, src=(0, 0, 0, 0), tol=1e-10, out=None, eta=None, ncol=12, csw=0.0):
    r = ddp_solve_req()
    r.domain_id = int(domain_id)
    r.kappa = float(kappa)
    r.csw = float(csw)
    r.src = (ctypes.c_int * 4)(*[int(x) for x in src])
    r.eta = _ptr(eta).value if eta is not None else None
    r.ncol = int(ncol)
    r.tol = float(tol)
    r.out = _ptr(out).value
    return r


def ddp_solve_batch(ctx, reqs, precision):
    n = len(reqs)
    arr = (ddp_solve_req * n)(*reqs)
    infos = (ddp_solve_info * n)()
    rc = lib().ddp_solve_batch(ctx, arr, n, int(precision), infos)
    _check(ctx, rc, "ddp_solve_batch", allow=(DDP_ERR_NOT_CONVERGED,))
    return rc, list(infos)


def ddp_series_terms(ctx, domain_small, S_small, domain_big, S_big, T_out, ncol=12):
    return _check(ctx, lib().ddp_series_terms(ctx, int(domain_small), _ptr(S_small), int(domain_big), _ptr(S_big),
                                              _ptr(T_out), int(ncol)), "ddp_series_terms")


def ddp_contract(ctx, kind, domain_id, S, C_out, eta=None, ncol=12, src=(0, 0, 0, 0)):
    return _check(ctx, lib().ddp_contract(ctx, int(kind), int(domain_id), _ptr(S), _ptr(eta), int(ncol), _i4(src),
                                          _ptr(C_out)), "ddp_contract")


def ddp_propagator_series(ctx, domain_ids, kappa, src, tol, precision, S_out=None, T_out=None, contract_mask=0,
                          C_out=None, csw=0.0):
    """Nested-domain propagators, their series terms and contractions in one call
    (include/ddp.h).  S_out: list of n arrays or None entries; T_out: list of n-1;
    C_out: n x 4 x 2*L0 doubles.  Returns (status, infos)."""
    n = len(domain_ids)
    ids = (ctypes.c_int * n)(*[int(d) for d in domain_ids])
    sp = (ctypes.c_void_p * n)(*[(_ptr(x).value if x is not None else None) for x in (S_out or [None] * n)])
    tl = T_out or [None] * max(n - 1, 1)
    tp = (ctypes.c_void_p * len(tl))(*[(_ptr(x).value if x is not None else None) for x in tl])
    infos = (ddp_solve_info * n)()
    rc = lib().ddp_propagator_series(ctx, n, ids, float(kappa), float(csw), _i4(src), float(tol), int(precision),
                                     sp if S_out is not None else None, tp if T_out is not None else None,
                                     int(contract_mask), _ptr(C_out), infos)
    _check(ctx, rc, "ddp_propagator_series", allow=(DDP_ERR_NOT_CONVERGED,))
    return rc, list(infos)


def ddp_orthonormalize(ctx, domain_id, V, m):
    return _check(ctx, lib().ddp_orthonormalize(ctx, int(domain_id), _ptr(V), int(m)), "ddp_orthonormalize")


def ddp_inverse_iteration(ctx, domain_id, kappa, V, m, iters, tol, precision, csw=0.0):
    info = ddp_solve_info()
    rc = lib().ddp_inverse_iteration(ctx, int(domain_id), float(kappa), float(csw), _ptr(V), int(m), int(iters),
                                     float(tol), int(precision), ctypes.byref(info))
    _check(ctx, rc, "ddp_inverse_iteration", allow=(DDP_ERR_NOT_CONVERGED,))
    return rc, info


def ddp_embed(ctx, domain_from, psi, domain_to, out, ncol, gamma5=False):
    return _check(ctx, lib().ddp_embed(ctx, int(domain_from), _ptr(psi), int(domain_to), _ptr(out), int(ncol),
                                       1 if gamma5 else 0), "ddp_embed")


def ddp_gram_slices(ctx, domain_id, A, m, M_out):
    return _check(ctx, lib().ddp_gram_slices(ctx, int(domain_id), _ptr(A), int(m), _ptr(M_out)), "ddp_gram_slices")


def ddp_colourless_slices(ctx, domain_id, A, m, form, X_out):
    return _check(ctx, lib().ddp_colourless_slices(ctx, int(domain_id), _ptr(A), int(m), int(form), _ptr(X_out)),
                  "ddp_colourless_slices")


def ddp_projected_pion(ctx, L0, m, Mt, M, spatial_volume, C_out):
    return _check(ctx, lib().ddp_projected_pion(ctx, int(L0), int(m), _ptr(Mt), _ptr(M), float(spatial_volume),
                                                _ptr(C_out)), "ddp_projected_pion")


def ddp_projected_nucleon(ctx, L0, m, X, Y, C_out):
    return _check(ctx, lib().ddp_projected_nucleon(ctx, int(L0), int(m), _ptr(X), _ptr(Y), _ptr(C_out)),
                  "ddp_projected_nucleon")


def ddp_factorized_correlator(ctx, T_A, nvar_A, T_B, nvar_B, L0, spatial_volume, C_out):
    return _check(ctx, lib().ddp_factorized_correlator(ctx, _ptr(T_A), int(nvar_A), _ptr(T_B), int(nvar_B), int(L0),
                                                       float(spatial_volume), _ptr(C_out)),
                  "ddp_factorized_correlator")


def ddp_serve_config(ctx, mem_budget_bytes=0, max_active=64, precision=DDP_PREC_MIXED_FP32):
    return _check(ctx, lib().ddp_serve_config(ctx, int(mem_budget_bytes), int(max_active), int(precision)),
                  "ddp_serve_config")


def ddp_submit(ctx, req):
    t = ctypes.c_uint64()
    rc = lib().ddp_submit(ctx, ctypes.byref(req), ctypes.byref(t))
    _check(ctx, rc, "ddp_submit", allow=(DDP_ERR_BUSY,))
    return rc, t.value


def ddp_serve_step(ctx) -> int:
    n = ctypes.c_int()
    _check(ctx, lib().ddp_serve_step(ctx, ctypes.byref(n)), "ddp_serve_step")
    return n.value


def ddp_poll(ctx, ticket):
    done = ctypes.c_int()
    info = ddp_solve_info()
    _check(ctx, lib().ddp_poll(ctx, ctypes.c_uint64(ticket), ctypes.byref(done), ctypes.byref(info)), "ddp_poll")
    return bool(done.value), info


def ddp_serve_reset(ctx):
    return _check(ctx, lib().ddp_serve_reset(ctx), "ddp_serve_reset")


def ddp_set_param(ctx, name: str, value: float):
    return _check(ctx, lib().ddp_set_param(ctx, name.encode(), float(value)), "ddp_set_param")


def ddp_get_param(ctx, name: str) -> float:
    v = ctypes.c_double(0.0)
    _check(ctx, lib().ddp_get_param(ctx, name.encode(), ctypes.byref(v)), "ddp_get_param")
    return v.value


def ddp_time_hop(ctx, domain_id, kappa, ncol, precision, iters, kernel=DDP_HOP_PLAIN):
    """(ms per launch, algorithmic bytes per launch) of one inner-loop stencil variant."""
    ms = ctypes.c_float()
    by = ctypes.c_double()
    _check(ctx, lib().ddp_time_hop(ctx, int(domain_id), float(kappa), int(ncol), int(precision), int(kernel),
                                   int(iters), ctypes.byref(ms), ctypes.byref(by)), "ddp_time_hop")
    return ms.value, by.value


def ddp_autotune(ctx, domain_id, kappa, ncol, precision, iters=10):
    best = ctypes.c_int()
    ms = ctypes.c_float()
    _check(ctx, lib().ddp_autotune(ctx, int(domain_id), float(kappa), int(ncol), int(precision), int(iters),
                                   ctypes.byref(best), ctypes.byref(ms)), "ddp_autotune")
    return best.value, ms.value


_PREC_NAMES = {0: "fp64", 1: "fp32", 2: "fp16", 3: "bf16"}


def autotune_cached(ctx, domain_id, n_sites, kappa, ncol, precision, cache_path=None, iters=10):
    """ddp_autotune with a JSON cache keyed by storage format, columns and the
    domain's size class (powers of two of its site count); the cache path defaults
    to $DDP_TUNE_CACHE.  A cached choice is applied without timing."""
    import json
    path = cache_path or os.environ.get("DDP_TUNE_CACHE")
    key = f"{_PREC_NAMES[int(precision)]}/ncol{int(ncol)}/sites2^{max(0, int(n_sites).bit_length() - 1)}"
    cache = {}
    if path and os.path.exists(path):
        with open(path) as f:
            cache = json.load(f)
    name = _PREC_NAMES[int(precision)]
    if key in cache:
        ddp_set_param(ctx, f"tuned_cols_{name}", cache[key]["cols"])
        if "carveout" in cache[key]:
            ddp_set_param(ctx, f"tuned_carveout_{name}", cache[key]["carveout"])
        return cache[key]["cols"], cache[key]["ms"]
    cols, ms = ddp_autotune(ctx, domain_id, kappa, ncol, precision, iters)
    if path:
        cache[key] = {"cols": cols, "carveout": int(ddp_get_param(ctx, f"tuned_carveout_{name}")), "ms": ms}
        with open(path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return cols, ms


def ddp_kernel_launches(ctx) -> int:
    return int(lib().ddp_kernel_launches(ctx))


def _device_doubles(a, need, what):
    """Size in doubles of a CUDA complex128/float64 tensor, checked against `need`."""
    import torch
    if not isinstance(a, torch.Tensor) or not a.is_cuda:
        raise DDPError(DDP_ERR_INVALID_ARG, "ddp_contract_static", f"{what} must be a CUDA tensor")
    if a.dtype not in (torch.complex128, torch.float64):
        raise DDPError(DDP_ERR_INVALID_ARG, "ddp_contract_static", f"{what} must be complex128 or float64")
    nd = a.numel() * (2 if a.dtype == torch.complex128 else 1)
    if nd < need:
        raise DDPError(DDP_ERR_INVALID_ARG, "ddp_contract_static", f"{what} holds {nd} doubles, needs {need}")


def ddp_contract_static(kind, L, origin, extent, S, C_out, eta=None, ncol=12, src=(0, 0, 0, 0), stream=None):
    """Allocation-free contraction for callers that must not allocate device
    memory (see include/ddp.h); CUDA tensors only, enqueued on `stream`.  The
    tensors' device, dtype and size are checked here; the C entry point checks
    the pointer kinds again."""
    n = int(np.prod([int(e) for e in extent]))
    nc = int(ncol) if kind in (DDP_CONTRACT_PION, DDP_CONTRACT_PSEUDO_NOISE) else 12
    _device_doubles(S, 2 * 12 * nc * n, "S")
    if kind == DDP_CONTRACT_PSEUDO_NOISE:
        _device_doubles(eta, 2 * 12 * nc * n, "eta")
    _device_doubles(C_out, 2 if kind == DDP_CONTRACT_PSEUDO_LOCAL else 2 * int(L[0]), "C_out")
    s = ctypes.c_void_p(int(stream)) if stream else None
    return _check(None, lib().ddp_contract_static(int(kind), _i4(L), _i4(origin), _i4(extent), _ptr(S), _ptr(eta),
                                                  int(ncol), _i4(src), _ptr(C_out), s), "ddp_contract_static")


def info_dict(info: ddp_solve_info) -> dict:
    n = min(info.ncol, DDP_INFO_COLS)
    return {"status": info.status, "ncol": info.ncol, "outer_cycles": info.outer_cycles,
            "inner_iters": info.inner_iters, "column_iters": int(info.column_iters),
            "max_rel_residual": info.max_rel_residual,
            "rel_residual": [info.rel_residual[i] for i in range(n)], "seconds": info.seconds}
