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
            # same kernels and the same reduction order as ddp_contract: identical bits
            assert np.array_equal(g, want)
        ddp.ddp_free_domain(ctx, did)


def test_static_nucleon_matches_oracle(ddp, setup):
    """One case against the FP64 oracle directly, on an oracle propagator."""
    import oracle
    ctx, gid, L = setup
    o, e = (0, 0, 0, 0), L
    U = synth.gauge_field(L, seed=4321)
    ref, _, _, st = oracle.propagator(U, L, oracle.BC_ANTIPERIODIC, o, e, 0.12, (0, 0, 0, 0), tol=1e-12)
    assert st == 0
    S = torch.from_numpy(ref).cuda()
    got = torch.zeros(2 * L[0], dtype=torch.float64, device="cuda")
    ddp.ddp_contract_static(ddp.DDP_CONTRACT_NUCLEON, L, o, e, S, got,
                            stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    g = got.cpu().numpy()
    want = oracle.nucleon(L, o, e, ref)
    assert _rel(g[0::2] + 1j * g[1::2], want) <= CORR_TOL


def _raw_static(ddp, kind, L, o, e, S_ptr, out_ptr):
    """The C entry point itself, bypassing the binding's own checks."""
    import ctypes
    return ddp.lib().ddp_contract_static(int(kind), ddp._i4(L), ddp._i4(o), ddp._i4(e), S_ptr, None, 12,
                                         ddp._i4((0, 0, 0, 0)), out_ptr, None)


def test_static_rejects_sizes_beyond_its_array(ddp):
    dummy = torch.zeros(16, dtype=torch.complex128, device="cuda")
    out = torch.zeros(2 * 132, dtype=torch.float64, device="cuda")
    L = (132, 32, 32, 32)   # 132 slices x 1024 nucleon chunks > the fixed array
    rc = _raw_static(ddp, ddp.DDP_CONTRACT_NUCLEON, L, (0, 0, 0, 0), L, ddp._ptr(dummy), ddp._ptr(out))
    assert rc == ddp.DDP_ERR_INVALID_ARG
    torch.cuda.synchronize()


def test_static_rejects_host_and_short_buffers(ddp):
    L = (8, 4, 4, 6)
    n = int(np.prod(L))
    S_dev = torch.zeros((12, n, 4, 3), dtype=torch.complex128, device="cuda")
    out_dev = torch.zeros(2 * L[0], dtype=torch.float64, device="cuda")
    S_host = np.zeros((12, n, 4, 3), dtype=np.complex128)
    out_host = np.zeros(2 * L[0])
    # the C entry point refuses host memory before launching anything
    for s_ptr, o_ptr in [(ddp._ptr(S_host), ddp._ptr(out_dev)), (ddp._ptr(S_dev), ddp._ptr(out_host))]:
        assert _raw_static(ddp, ddp.DDP_CONTRACT_NUCLEON, L, (0, 0, 0, 0), L, s_ptr, o_ptr) == \
            ddp.DDP_ERR_INVALID_ARG
    # the binding refuses CPU tensors and tensors that are too short
    for S, out in [(S_dev.cpu(), out_dev), (S_dev[:6], out_dev), (S_dev, out_dev[:4])]:
        with pytest.raises(ddp.DDPError) as ei:
            ddp.ddp_contract_static(ddp.DDP_CONTRACT_NUCLEON, L, (0, 0, 0, 0), L, S, out)
        assert ei.value.status == ddp.DDP_ERR_INVALID_ARG
    # an odd extent in the x3 direction is the geometry the library does not support
    assert _raw_static(ddp, ddp.DDP_CONTRACT_NUCLEON, L, (0, 0, 0, 0), (8, 4, 4, 5), ddp._ptr(S_dev),
                       ddp._ptr(out_dev)) == ddp.DDP_ERR_UNSUPPORTED
    torch.cuda.synchronize()
