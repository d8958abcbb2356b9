"""Continuous batching: requests admitted while others run, each result identical
to the same request solved alone (GPU required)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
AP = oracle.BC_ANTIPERIODIC
LAT = (8, 4, 4, 6)


@pytest.fixture(scope="module")
def ddp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_04587_gb300 import build
    build.build()
    import paper_1601_04587_gb300 as m
    return m


@pytest.fixture(scope="module")
def env(ddp):
    U = synth.gauge_field(LAT, seed=2024)
    ctx = ddp.ddp_create(0, torch.cuda.current_stream().cuda_stream)
    gid = ddp.ddp_load_gauge(ctx, torch.from_numpy(U).cuda(), LAT, ddp.DDP_BC_ANTIPERIODIC)
    yield ctx, gid, U
    ddp.ddp_destroy(ctx)


SPECS = [(((6, 0, 0, 0), (4, 4, 4, 6)), (7, 1, 2, 3), 0.124),
         (((5, 1, 3, 2), (3, 2, 3, 4)), (6, 2, 0, 5), 0.120),
         (((0, 0, 0, 0), LAT), (3, 3, 3, 3), 0.122),
         (((2, 3, 0, 5), (5, 4, 2, 2)), (4, 3, 1, 0), 0.126)]


def _drain(ddp, ctx, tickets, results, max_steps=200):
    for _ in range(max_steps):
        left = ddp.ddp_serve_step(ctx)
        for t in list(tickets):
            done, info = ddp.ddp_poll(ctx, t)
            if done:
                results[t] = info
                tickets.remove(t)
        if left == 0 and not tickets:
            return
    raise AssertionError("serving did not finish")


@pytest.mark.parametrize("prec", [1, 2])
def test_mix_equals_alone(ddp, env, prec):
    ctx, gid, U = env
    ddp.ddp_serve_config(ctx, 256 << 20, 8, prec)
    outs, alone, reqs = [], [], []
    for (o, e), src, kappa in SPECS:
        did = ddp.ddp_set_domain(ctx, gid, o, e)
        n = int(np.prod(e))
        out = torch.zeros((12, n, 4, 3), dtype=torch.complex128, device="cuda")
        one = torch.zeros_like(out)
        rc, _ = ddp.ddp_solve_propagator(ctx, did, kappa, 0.0, src, 1e-10, prec, one)
        assert rc == ddp.DDP_OK
        outs.append(out)
        alone.append(one)
        reqs.append(ddp.make_req(did, kappa, src, 1e-10, out))
    results = {}
    tickets = []
    # two requests start, one more joins after the first cycle, the last after the second
    for r in reqs[:2]:
        rc, t = ddp.ddp_submit(ctx, r)
        assert rc == ddp.DDP_OK
        tickets.append(t)
    ddp.ddp_serve_step(ctx)
    rc, t = ddp.ddp_submit(ctx, reqs[2])
    assert rc == ddp.DDP_OK
    tickets.append(t)
    ddp.ddp_serve_step(ctx)
    rc, t = ddp.ddp_submit(ctx, reqs[3])
    assert rc == ddp.DDP_OK
    tickets.append(t)
    order = list(tickets)
    _drain(ddp, ctx, list(tickets), results)
    for t, out, one, ((o, e), src, kappa) in zip(order, outs, alone, SPECS):
        assert results[t].status == ddp.DDP_OK
        assert results[t].max_rel_residual <= 1e-10
        assert results[t].seconds > 0
        assert torch.equal(out, one)
        ref, *_ = oracle.propagator(U, LAT, AP, o, e, kappa, src, tol=1e-12)
        got = out.cpu().numpy()
        assert max(np.linalg.norm(got[c] - ref[c]) / np.linalg.norm(ref[c]) for c in range(12)) < 1e-8
    ddp.ddp_serve_reset(ctx)


def test_admission_by_slots_and_memory(ddp, env):
    ctx, gid, U = env
    (o, e), src, kappa = SPECS[2]
    did = ddp.ddp_set_domain(ctx, gid, o, e)
    n = int(np.prod(e))
    outs = [torch.zeros((12, n, 4, 3), dtype=torch.complex128, device="cuda") for _ in range(2)]
    # one active slot: the second request is refused until the first retires
    ddp.ddp_serve_config(ctx, 256 << 20, 1, ddp.DDP_PREC_MIXED_FP32)
    rc, t1 = ddp.ddp_submit(ctx, ddp.make_req(did, kappa, src, 1e-10, outs[0]))
    assert rc == ddp.DDP_OK
    rc, _ = ddp.ddp_submit(ctx, ddp.make_req(did, kappa, src, 1e-10, outs[1]))
    assert rc == ddp.DDP_ERR_BUSY
    res = {}
    _drain(ddp, ctx, [t1], res)
    rc, t2 = ddp.ddp_submit(ctx, ddp.make_req(did, kappa, src, 1e-10, outs[1]))
    assert rc == ddp.DDP_OK
    _drain(ddp, ctx, [t2], res)
    assert torch.equal(outs[0], outs[1])
    # a budget too small for the request: it can never be admitted
    ddp.ddp_serve_config(ctx, 4 << 20, 4, ddp.DDP_PREC_MIXED_FP32)
    with pytest.raises(ddp.DDPError) as ei:
        ddp.ddp_submit(ctx, ddp.make_req(did, kappa, src, 1e-10, outs[0]))
    assert ei.value.status == ddp.DDP_ERR_OOM
    # host output buffers are refused: serving works on resident device memory
    host = np.zeros((12, n, 4, 3), dtype=np.complex128)
    with pytest.raises(ddp.DDPError):
        ddp.ddp_submit(ctx, ddp.make_req(did, kappa, src, 1e-10, host))
    ddp.ddp_serve_reset(ctx)
