"""Multi-rank path on CPU: world-size-2 gloo ranks shard independent domain
solves (computed with the FP64 oracle) and the merged result equals the
unsharded run."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1601_04587_gb300 import shard  # noqa: E402

L = (4, 4, 2, 2)
KAPPA = 0.125


def _units():
    import synth
    boxes = [((0, 0, 0, 0), (2, 4, 2, 2)), ((2, 0, 0, 0), (2, 4, 2, 2)), ((1, 0, 0, 0), (2, 4, 2, 2)),
             ((3, 1, 1, 0), (3, 2, 1, 2)), ((0, 0, 0, 0), L)]
    return [(o, e, tuple((o[m] + e[m] // 2) % L[m] for m in range(4))) for o, e in boxes], synth


def _compute(unit):
    import oracle
    import synth
    U = synth.gauge_field(L, seed=77)
    o, e, src = unit
    S, *_ = oracle.propagator(U, L, oracle.BC_ANTIPERIODIC, o, e, KAPPA, src, tol=1e-12)
    return {"pion": oracle.pion(L, o, e, S), "trace": oracle.local_trace(L, o, e, S, src)}


def _worker(rank, world, port, outdir):
    # ranks share this host's cores: split the (already initialised) OpenMP pool between them
    torch.set_num_threads(max(1, (os.cpu_count() or 2) // world))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units, _ = _units()
    costs = [shard.solve_cost(int(np.prod(e))) for _, e, _ in units]
    res = shard.run_sharded(units, costs, _compute, dist)
    if rank == 0:
        np.save(os.path.join(outdir, "pion.npy"), np.array([r["pion"] for r in res]))
        np.save(os.path.join(outdir, "trace.npy"), np.array([r["trace"] for r in res]))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_partition_balanced_and_complete():
    costs = [5, 1, 9, 3, 3, 7, 2]
    for world in (1, 2, 3, 4):
        parts = shard.partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)
    assert shard.partition(costs, 2) == shard.partition(costs, 2)


def test_two_gloo_ranks_match_unsharded(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    units, _ = _units()
    ref = [_compute(u) for u in units]
    # the ranks' oracle runs use fewer OpenMP threads (another summation order): compare at the
    # oracle's solve tolerance
    np.testing.assert_allclose(np.load(tmp_path / "pion.npy"), np.array([r["pion"] for r in ref]), rtol=1e-10)
    np.testing.assert_allclose(np.load(tmp_path / "trace.npy"), np.array([r["trace"] for r in ref]), rtol=1e-10,
                               atol=1e-14)


def _batch_worker(rank, world, port, outdir):
    torch.set_num_threads(max(1, (os.cpu_count() or 2) // world))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units, _ = _units()
    costs = [shard.solve_cost(int(np.prod(e))) for _, e, _ in units]
    calls = []

    def batch(us):  # one batched call per rank, like one ddp_solve_batch of its share
        calls.append(len(us))
        return [_compute(u) for u in us]

    res = shard.run_sharded_batch(units, costs, batch, dist)
    np.save(os.path.join(outdir, f"calls{rank}.npy"), np.array(calls))
    if rank == 0:
        np.save(os.path.join(outdir, "bpion.npy"), np.array([r["pion"] for r in res]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_batched_shards(tmp_path):
    """run_sharded_batch: each rank makes exactly one batched call on its cost partition,
    and the merged results (unit order) equal the unsharded run."""
    port = _free_port()
    mp.start_processes(_batch_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    units, _ = _units()
    costs = [shard.solve_cost(int(np.prod(e))) for _, e, _ in units]
    parts = shard.partition(costs, 2)
    for r in range(2):
        assert list(np.load(tmp_path / f"calls{r}.npy")) == [len(parts[r])]
    ref = [_compute(u) for u in units]
    np.testing.assert_allclose(np.load(tmp_path / "bpion.npy"), np.array([r["pion"] for r in ref]), rtol=1e-10)


def test_batched_shards_single_process_is_one_call():
    calls = []
    out = shard.run_sharded_batch([3, 1, 2], [1, 1, 1], lambda us: calls.append(list(us)) or [u * 2 for u in us])
    assert out == [6, 2, 4] and calls == [[3, 1, 2]]
