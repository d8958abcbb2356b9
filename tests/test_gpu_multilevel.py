"""Two-level factorized disconnected correlator on the GPU against the oracle.

Two time regions of an 8 x 4^3 lattice are Dirichlet slabs; each gets level-1
variants of its own links (spatial links of its first slice frozen, Sec. 3 /
Sec. 5), the same diluted noise sources for every variant, a domain solve,
the noise estimate of its time-slice traces and finally the product of the
two level-1 means (Eq. factsing).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CORR_TOL = 1e-7
AP = oracle.BC_ANTIPERIODIC


@pytest.fixture(scope="module")
def ddp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_04587_gb300 import build
    build.build()
    import paper_1601_04587_gb300 as m
    return m


def test_two_level_factorized_correlator(ddp):
    L = (8, 4, 4, 4)
    kappa = 0.13
    nvar = 3
    U0 = synth.gauge_field(L, seed=71)
    ctx = ddp.ddp_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        gid0 = ddp.ddp_load_gauge(ctx, torch.from_numpy(U0).cuda(), L, ddp.DDP_BC_ANTIPERIODIC)
        regions = [(0, 4), (4, 8)]
        T_gpu, T_orc = [], []
        for r, (t_lo, t_hi) in enumerate(regions):
            o, e = (t_lo, 0, 0, 0), (t_hi - t_lo, 4, 4, 4)
            n = int(np.prod(e))
            gi, _, _ = oracle.domain_maps(L, o, e)
            eta = synth.diluted_noise_columns(synth.noise_field(n, synth.SEED_NOISE0 + r))
            tg = np.zeros((nvar, 2 * L[0]))
            to = np.zeros((nvar, L[0]), dtype=complex)
            for v in range(nvar):
                Uv = synth.variant_field(U0, L, t_lo, t_hi, seed=synth.SEED_VARIANT0 + 100 * r + v)
                vid = ddp.ddp_load_gauge_region(ctx, gid0, o, e, np.ascontiguousarray(Uv[:, gi]))
                did = ddp.ddp_set_domain(ctx, vid, o, e)
                psi = torch.zeros((12, n, 4, 3), dtype=torch.complex128, device="cuda")
                eta_d = torch.from_numpy(eta).cuda()
                rc, info = ddp.ddp_solve_sources(ctx, did, kappa, 0.0, eta_d, 12, 1e-10, ddp.DDP_PREC_MIXED_FP32, psi)
                assert rc == ddp.DDP_OK
                ddp.ddp_contract(ctx, ddp.DDP_CONTRACT_PSEUDO_NOISE, did, psi, tg[v], eta=eta_d, ncol=12)
                ddp.ddp_free_domain(ctx, did)
                ddp.ddp_free_gauge(ctx, vid)
                psi_o, *_ = oracle.solve(Uv, L, AP, o, e, kappa, eta)
                to[v] = oracle.noise_trace(L, o, e, eta, psi_o)
                assert np.linalg.norm(tg[v, 0::2] + 1j * tg[v, 1::2] - to[v]) <= CORR_TOL * np.linalg.norm(to[v])
            T_gpu.append(tg)
            T_orc.append(to)
        C = np.zeros(2 * L[0] * L[0])
        ddp.ddp_factorized_correlator(ctx, T_gpu[0], nvar, T_gpu[1], nvar, L[0], 64.0, C)
        Cg = (C[0::2] + 1j * C[1::2]).reshape(L[0], L[0])
        Co = oracle.factorized_correlator(T_orc[0], T_orc[1], L[0], 64.0)
        assert np.linalg.norm(Cg - Co) <= CORR_TOL * np.linalg.norm(Co)
        # region A's traces live on x0 < 4, region B's on y0 >= 4: C^(f) is supported there
        assert np.abs(Cg[:4, :]).max() == 0 and np.abs(Cg[:, 4:]).max() == 0
    finally:
        ddp.ddp_destroy(ctx)
