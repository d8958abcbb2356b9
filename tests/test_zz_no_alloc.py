"""The allocation-free contraction entry point (ddp_contract_static).

Some callers cannot allocate device memory at the moment they need a
correlator: a custom operator inside another framework whose allocator owns
the GPU, or a tight loop that cannot afford the device synchronisation
cudaMalloc/cudaFree can cause.  ddp_contract_static serves them: it takes device buffers only and
keeps its partial sums in one fixed array inside the library.  These tests call
it through the C ABI and check it against the allocating ddp_contract, twice
in a row, because the fixed array keeps the previous call's contents.

This file is collected last on purpose; it also passes on its own in a fresh
process (it sets up everything it uses).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CORR_TOL = 1e-7   # the correlator tolerance used by the other parity tests


@pytest.fixture(scope="module")
def ddp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_04587_gb300 import build
    build.build()
    import paper_1601_04587_gb300 as m
    return m


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def setup(ddp):
    L = (8, 4, 4, 6)
    U = synth.gauge_field(L, seed=4321)
    ctx = ddp.ddp_create(0, torch.cuda.current_stream().cuda_stream)
    gid = ddp.ddp_load_gauge(ctx, torch.from_numpy(U).cuda(), L, ddp.DDP_BC_ANTIPERIODIC)
    yield ctx, gid, L
    ddp.ddp_destroy(ctx)


@pytest.mark.parametrize("kind", ["nucleon", "pion", "noise", "local"])
def test_static_matches_allocating_entry_point_twice(ddp, setup, kind):
    ctx, gid, L = setup
    kinds = {"nucleon": ddp.DDP_CONTRACT_NUCLEON, "pion": ddp.DDP_CONTRACT_PION,
             "noise": ddp.DDP_CONTRACT_PSEUDO_NOISE, "local": ddp.DDP_CONTRACT_PSEUDO_LOCAL}
    k = kinds[kind]
    stream = torch.cuda.current_stream().cuda_stream
    # two different domains so that the second call cannot pass on the first call's leftovers
    for (o, e), seed in [(((6, 0, 0, 0), (4, 4, 4, 6)), 1), (((1, 1, 2, 0), (5, 3, 2, 6)), 2)]:
        did = ddp.ddp_set_domain(ctx, gid, o, e)
        n = int(np.prod(e))
        S = torch.from_numpy(synth.random_spinor(12, n, seed)).cuda()
        eta = torch.from_numpy(synth.random_spinor(12, n, seed + 10)).cuda()
        src = (o[0], o[1], o[2], o[3])
        nout = 2 if k == ddp.DDP_CONTRACT_PSEUDO_LOCAL else 2 * L[0]
        ref = torch.zeros(nout, dtype=torch.float64, device="cuda")
        ddp.ddp_contract(ctx, k, did, S, ref, eta=eta, ncol=12, src=src)
        want = ref.cpu().numpy()
        for _ in range(2):
            got = torch.full((nout,), np.nan, dtype=torch.float64, device="cuda")
            ddp.ddp_contract_static(k, L, o, e, S, got, eta=eta, ncol=12, src=src, stream=stream)
            torch.cuda.synchronize()
            g = got.cpu().numpy()
            assert np.all(np.isfinite(g))
            assert _rel(g, want) <= CORR_TOL
        ddp.ddp_free_domain(ctx, did)


def test_static_rejects_sizes_beyond_its_array(ddp):
    dummy = torch.zeros(1, dtype=torch.complex128, device="cuda")
    out = torch.zeros(2 * 132, dtype=torch.float64, device="cuda")
    L = (132, 32, 32, 32)   # 132 slices x 1024 nucleon chunks > the fixed array
    with pytest.raises(ddp.DDPError) as ei:
        ddp.ddp_contract_static(ddp.DDP_CONTRACT_NUCLEON, L, (0, 0, 0, 0), L, dummy, out)
    assert ei.value.status == ddp.DDP_ERR_INVALID_ARG
