"""The batched, two-level and serving workloads, measured on one GPU.

Used by ``bench.py --workload batch|multilevel|serve`` (the default bench line is
the nested-slab workload).  Each function returns a dict that bench.py prints
as one JSON line.  Gauge fields are synthetic (``synth``); their generation is
input synthesis and stays outside the timed regions, while loading them into
the library (packing, variants) is timed.
"""
from __future__ import annotations

import math
import time

import numpy as np


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


# ----------------------------------------------------------------- uneven batch

# Expected inner iterations of a domain class of the batch (measured), for the cost model
# of the sharding: an 8x32^3 slab at kappa 0.150 needs about 10x the iterations of the rest.
BATCH_ITERS = {(8, 8, 8, 8): 65, (4, 32, 32, 32): 115, (8, 32, 32, 32): 686}


def batch_workload(ddp, torch, ctx, synth, precision, steps=1, warmup=1, tune_cache=None, dist=None):
    """256 8^4 blocks, 32 4x32^3 and 16 8x32^3 slabs of a 32^4 lattice, 12 point-source
    columns each, all in one batched solve per step.  kappa: the stated 0.155 for the
    blocks and 4x32^3 slabs, 0.150 for the 8x32^3 slabs (slow convergence at 0.155 on
    the synthetic ensemble).  With several ranks (dist initialised) the domains are
    sharded by cost (shard.run_sharded_batch): each rank solves its share in one batch,
    the per-domain results are gathered once, and the step time is the slowest rank's."""
    from . import shard
    L = synth.BATCH_LATTICE
    U = synth.gauge_field_torch(L, seed=synth.SEED_GAUGE, device="cuda")
    boxes = synth.batch_boxes(L)
    kap = [0.155 if b.extent != (8, 32, 32, 32) else 0.150 for b in boxes]
    outs = [torch.empty((12, b.n_sites, 4, 3), dtype=torch.complex128, device="cuda") for b in boxes]
    gid = ddp.ddp_load_gauge(ctx, U, L, ddp.DDP_BC_ANTIPERIODIC)
    tuned = {}
    for ext in ((8, 8, 8, 8), (4, 32, 32, 32), (8, 32, 32, 32)):
        d = ddp.ddp_set_domain(ctx, gid, (0, 0, 0, 0), ext)
        tuned[str(ext)] = ddp.autotune_cached(ctx, d, int(np.prod(ext)), 0.15, 12, precision, tune_cache, iters=5)
        ddp.ddp_free_domain(ctx, d)
    ddp.ddp_free_gauge(ctx, gid)

    costs = [shard.solve_cost(b.n_sites, 12, BATCH_ITERS.get(tuple(b.extent), 100)) for b in boxes]
    units = list(range(len(boxes)))

    def solve_units(idx):
        """One batched solve of the given domains; a small result per domain."""
        if not idx:
            return []
        g = ddp.ddp_load_gauge(ctx, U, L, ddp.DDP_BC_ANTIPERIODIC)
        dids = [ddp.ddp_set_domain(ctx, g, boxes[i].origin, boxes[i].extent) for i in idx]
        reqs = [ddp.make_req(d, kap[i], tuple((boxes[i].origin[m] + boxes[i].extent[m] // 2) % L[m]
                                             for m in range(4)), 1e-10, outs[i])
                for d, i in zip(dids, idx)]
        rc, infos = ddp.ddp_solve_batch(ctx, reqs, precision)
        for d in dids:
            ddp.ddp_free_domain(ctx, d)
        ddp.ddp_free_gauge(ctx, g)
        return [{"status": int(inf.status), "max_rel_residual": float(inf.max_rel_residual),
                 "inner_iters": int(inf.inner_iters)} for inf in infos]

    def step():
        return shard.run_sharded_batch(units, costs, solve_units, dist)

    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    for _ in range(warmup):
        step()
    a, b = _events(torch)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    a.record()
    for _ in range(steps):
        res = step()
    b.record()
    torch.cuda.synchronize()
    secs = a.elapsed_time(b) / 1e3
    if world > 1:
        t = torch.tensor([secs], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        secs = float(t.item())
    worst = max(r["max_rel_residual"] for r in res)
    its = {k: max(r["inner_iters"] for r, bx in zip(res, boxes) if str(bx.extent) == k)
           for k in sorted({str(bx.extent) for bx in boxes})}
    rc = max(r["status"] for r in res)
    return {"workload": "32^4 lattice, 256 x 8^4 + 32 x 4x32^3 + 16 x 8x32^3 Dirichlet domains, 12 columns, "
                        "one batched solve per rank", "solves_per_s": len(boxes) * steps / secs,
            "column_solves_per_s": 12 * len(boxes) * steps / secs, "s_per_batch": secs / steps,
            "max_rel_residual": worst, "status": rc, "inner_iters_max_by_box": its,
            "autotuned_cols": {k: v[0] for k, v in tuned.items()}, "steps": steps, "warmup": warmup,
            "n_ranks": world, "scaling": "strong" if world > 1 else None,
            "sharding": "longest-first by sites x columns x expected iterations, one gather per step"}


# ------------------------------------------------------------- two-level workload

def multilevel_workload(ddp, torch, ctx, synth, precision, nvar=32, batch=8, steps=1, warmup=0):
    """64 x 32^3 lattice, regions t in [0,32) and [32,64) as Dirichlet slabs, nvar
    level-1 variants per region (region links redrawn, spatial links of the first
    slice frozen), 12 diluted-noise columns per region shared by all variants,
    kappa 0.140; traces per variant and the factorized correlator (Eq. factsing)."""
    L = synth.MULTILEVEL_LATTICE
    kappa = 0.140
    vol3 = float(L[1] * L[2] * L[3])
    U0 = synth.gauge_field_torch(L, seed=synth.SEED_GAUGE, device="cuda")
    regions = [(0, 32), (32, 64)]
    n = 32 * 32 ** 3
    etas = [torch.from_numpy(synth.diluted_noise_columns(synth.noise_field(n, synth.SEED_NOISE0 + r))).cuda()
            for r in range(2)]
    psis = [torch.empty((12, n, 4, 3), dtype=torch.complex128, device="cuda") for _ in range(batch)]

    def step():
        gid0 = ddp.ddp_load_gauge(ctx, U0, L, ddp.DDP_BC_ANTIPERIODIC)
        T = [torch.zeros((nvar, 2 * L[0]), dtype=torch.float64, device="cuda") for _ in range(2)]
        t_solve = 0.0
        for r, (lo, hi) in enumerate(regions):
            box = synth.Box((lo, 0, 0, 0), (32, 32, 32, 32))
            sl = slice(lo * 32768, hi * 32768)
            for v0 in range(0, nvar, batch):
                vids, dids, reqs = [], [], []
                for j, v in enumerate(range(v0, min(nvar, v0 + batch))):
                    Uv = synth.variant_field_torch(U0, L, lo, hi, seed=synth.SEED_VARIANT0 + 100 * r + v)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    vid = ddp.ddp_load_gauge_region(ctx, gid0, box.origin, box.extent, Uv[:, sl].contiguous())
                    did = ddp.ddp_set_domain(ctx, vid, box.origin, box.extent)
                    t_solve += time.perf_counter() - t0
                    del Uv
                    vids.append(vid)
                    dids.append(did)
                    reqs.append(ddp.make_req(did, kappa, tol=1e-10, out=psis[j], eta=etas[r], ncol=12))
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, infos = ddp.ddp_solve_batch(ctx, reqs, precision)
                for j, (v, d) in enumerate(zip(range(v0, v0 + len(reqs)), dids)):
                    ddp.ddp_contract(ctx, ddp.DDP_CONTRACT_PSEUDO_NOISE, d, psis[j], T[r][v], eta=etas[r], ncol=12)
                torch.cuda.synchronize()
                t_solve += time.perf_counter() - t0
                for d, g in zip(dids, vids):
                    ddp.ddp_free_domain(ctx, d)
                    ddp.ddp_free_gauge(ctx, g)
        C = torch.zeros(2 * L[0] * L[0], dtype=torch.float64, device="cuda")
        t0 = time.perf_counter()
        ddp.ddp_factorized_correlator(ctx, T[0], nvar, T[1], nvar, L[0], vol3, C)
        torch.cuda.synchronize()
        t_solve += time.perf_counter() - t0
        ddp.ddp_free_gauge(ctx, gid0)
        return t_solve, C

    for _ in range(warmup):
        step()
    secs = 0.0
    for _ in range(steps):
        s, C = step()
        secs += s
    nsolve = 2 * nvar * steps
    return {"workload": f"64x32^3 two-level: 2 regions x {nvar} level-1 variants, 12 diluted-noise columns, "
                        f"kappa {kappa}, factorized correlator", "solves_per_s": nsolve / secs,
            "s_per_step": secs / steps, "timed": "variant loading, batched solves, noise traces, correlator "
                                                 "(variant generation excluded)", "steps": steps}


# -------------------------------------------- factorized propagator, expanded trace

def next_rows_workload(ddp, torch, ctx, synth, precision, steps=2, warmup=1, L=None, x0_cut=24, delta=8):
    """48 x 24^3 lattice, kappa 0.140.  (1) The factorized propagator of Eq. approxlong
    with x0_cut = 24 and Delta = 8: Gamma-bar_0 = time slices [0, 32), Gamma*_0 =
    [24, 48); a 12-column point source at the origin solved on Gamma-bar_0, the boundary
    source, the 12 columns solved on Gamma*_0, the pion contraction of S^(f).  (2) The
    expanded stochastic trace of Eq. HPEtr (p = 8) on Gamma-bar_0: psi = D^-1 g5 eta for
    12 diluted noise columns, (kappa D_hop)^8 psi, contraction with g5 eta."""
    L = tuple(L or synth.SLAB_LATTICE)
    kappa = 0.140
    U = synth.gauge_field_torch(L, seed=synth.SEED_GAUGE, device="cuda")
    bar = ((0, 0, 0, 0), (x0_cut + delta, L[1], L[2], L[3]))
    star = ((x0_cut, 0, 0, 0), (L[0] - x0_cut, L[1], L[2], L[3]))
    nb, ns = int(np.prod(bar[1])), int(np.prod(star[1]))
    g5 = torch.tensor([-1.0, -1.0, 1.0, 1.0], dtype=torch.float64, device="cuda").view(1, 1, 4, 1)
    eta = torch.from_numpy(synth.diluted_noise_columns(synth.noise_field(nb, synth.SEED_NOISE0))).cuda()
    g5eta = (eta * g5).contiguous()
    Sb = torch.empty((12, nb, 4, 3), dtype=torch.complex128, device="cuda")
    sig = torch.empty((12, ns, 4, 3), dtype=torch.complex128, device="cuda")
    Sf = torch.empty((12, ns, 4, 3), dtype=torch.complex128, device="cuda")
    psi = torch.empty((12, nb, 4, 3), dtype=torch.complex128, device="cuda")
    v = torch.empty((12, nb, 4, 3), dtype=torch.complex128, device="cuda")
    Cpi = torch.zeros(2 * L[0], dtype=torch.float64, device="cuda")
    Ctr = torch.zeros(2 * L[0], dtype=torch.float64, device="cuda")
    gid = ddp.ddp_load_gauge(ctx, U, L, ddp.DDP_BC_ANTIPERIODIC)
    d_bar = ddp.ddp_set_domain(ctx, gid, *bar)
    d_star = ddp.ddp_set_domain(ctx, gid, *star)
    res = {}

    def factorized():
        rc1, i1 = ddp.ddp_solve_propagator(ctx, d_bar, kappa, 0.0, (0, 0, 0, 0), 1e-10, precision, Sb)
        ddp.ddp_boundary_source(ctx, d_bar, Sb, d_star, sig, 12)
        rc2, i2 = ddp.ddp_solve_sources(ctx, d_star, kappa, 0.0, sig, 12, 1e-10, precision, Sf)
        ddp.ddp_contract(ctx, ddp.DDP_CONTRACT_PION, d_star, Sf, Cpi)
        res["factorized_residuals"] = [i1.max_rel_residual, i2.max_rel_residual]
        return rc1 or rc2

    def expanded():
        rc, i = ddp.ddp_solve_sources(ctx, d_bar, kappa, 0.0, g5eta, 12, 1e-10, precision, psi)
        ddp.ddp_hop_power(ctx, d_bar, kappa, 8, psi, v, 12)
        ddp.ddp_contract(ctx, ddp.DDP_CONTRACT_PSEUDO_NOISE, d_bar, v, Ctr, eta=g5eta, ncol=12)
        res["expanded_residual"] = i.max_rel_residual
        return rc

    out = {}
    for name, fn in (("factorized", factorized), ("expanded", expanded)):
        for _ in range(warmup):
            fn()
        a, b = _events(torch)
        torch.cuda.synchronize()
        a.record()
        rc = 0
        for _ in range(steps):
            rc = rc or fn()
        b.record()
        torch.cuda.synchronize()
        out[name] = {"s_per_step": a.elapsed_time(b) / 1e3 / steps, "status": rc}
    ddp.ddp_free_domain(ctx, d_bar)
    ddp.ddp_free_domain(ctx, d_star)
    ddp.ddp_free_gauge(ctx, gid)
    return {"workload": "48x24^3, kappa 0.140: factorized propagator (Eq. approxlong, x0_cut 24, Delta 8: "
                        "solve on t in [0,32), boundary source, solve on t in [24,48), pion) and expanded "
                        "noise trace (Eq. HPEtr, p 8, 12 diluted columns on t in [0,32))",
            "factorized_s_per_propagator": out["factorized"]["s_per_step"],
            "expanded_trace_s_per_estimate": out["expanded"]["s_per_step"],
            "status": [out["factorized"]["status"], out["expanded"]["status"]],
            "max_rel_residuals": res, "steps": steps, "warmup": warmup}


# ------------------------------------------------ projector-cut factorization

def projector_workload(ddp, torch, ctx, synth, precision, nm=120, iters=10, steps=1, warmup=1, L=None, x0_cut=24,
                       delta=8):
    """48 x 24^3 lattice, kappa 0.140, the projector cut of Sec. 5 at x0_cut = 24 with
    Delta = 8: Gamma-bar_0 = time slices [0, 32), Gamma*_0 = [24, 48), Omega = [16, 32).
    Per step: nm orthonormal vectors by `iters` inverse iterations of D_Omega on seeded
    random vectors, u_i = D^-1_{Gbar} g5 phi_i, w_i = D^-1_{G*} sigma_i, the pion
    (time-slice Gram blocks, Eq. fullfactpi) and the nucleon (colourless spinors, Eq.
    W0tbary) for every (y0, x0).  Solves: mixed precision to 1e-10."""
    L = tuple(L or synth.SLAB_LATTICE)
    kappa = 0.140
    U = synth.gauge_field_torch(L, seed=synth.SEED_GAUGE, device="cuda")
    bar = ((0, 0, 0, 0), (x0_cut + delta, L[1], L[2], L[3]))
    star = ((x0_cut, 0, 0, 0), (L[0] - x0_cut, L[1], L[2], L[3]))
    omega = ((x0_cut - delta, 0, 0, 0), (2 * delta, L[1], L[2], L[3]))
    nb, ns, no = (int(np.prod(b[1])) for b in (bar, star, omega))
    V0 = torch.from_numpy(synth.random_spinor(nm, no, synth.SEED_NOISE0 + 7)).cuda()
    phi = torch.empty_like(V0)
    src = torch.empty((nm, nb, 4, 3), dtype=torch.complex128, device="cuda")
    u = torch.empty_like(src)
    sig = torch.empty((nm, ns, 4, 3), dtype=torch.complex128, device="cuda")
    w = torch.empty_like(sig)
    M = torch.empty((L[0], nm, nm), dtype=torch.complex128, device="cuda")
    Mt = torch.empty_like(M)
    X = torch.empty((L[0], nm, nm, nm, 4), dtype=torch.complex128, device="cuda")
    Y = torch.empty_like(X)
    Cpi = torch.empty((L[0], L[0]), dtype=torch.complex128, device="cuda")
    Cn = torch.empty_like(Cpi)
    gid = ddp.ddp_load_gauge(ctx, U, L, ddp.DDP_BC_ANTIPERIODIC)
    d_bar, d_star, d_om = (ddp.ddp_set_domain(ctx, gid, *b) for b in (bar, star, omega))
    times = {}

    def stage(name, fn):
        a, b = _events(torch)
        a.record()
        r = fn()
        b.record()
        torch.cuda.synchronize()
        times[name] = times.get(name, 0.0) + a.elapsed_time(b) / 1e3
        return r

    def step():
        phi.copy_(V0)
        rc1, _ = stage("modes", lambda: ddp.ddp_inverse_iteration(ctx, d_om, kappa, phi, nm, iters, 1e-10, precision))
        stage("sources", lambda: (ddp.ddp_embed(ctx, d_om, phi, d_bar, src, nm, gamma5=True),
                                  ddp.ddp_boundary_source(ctx, d_om, phi, d_star, sig, nm)))
        rc2, _ = stage("solves", lambda: ddp.ddp_solve_sources(ctx, d_bar, kappa, 0.0, src, nm, 1e-10, precision, u))
        rc3, _ = stage("solves", lambda: ddp.ddp_solve_sources(ctx, d_star, kappa, 0.0, sig, nm, 1e-10, precision, w))
        stage("pion", lambda: (ddp.ddp_gram_slices(ctx, d_bar, u, nm, M), ddp.ddp_gram_slices(ctx, d_star, w, nm, Mt),
                               ddp.ddp_projected_pion(ctx, L[0], nm, Mt, M, L[1] * L[2] * L[3], Cpi)))
        stage("nucleon", lambda: (ddp.ddp_colourless_slices(ctx, d_bar, u, nm, 1, X),
                                  ddp.ddp_colourless_slices(ctx, d_star, w, nm, 2, Y),
                                  ddp.ddp_projected_nucleon(ctx, L[0], nm, X, Y, Cn)))
        return rc1 or rc2 or rc3

    for _ in range(warmup):
        step()
    times.clear()
    a, b = _events(torch)
    torch.cuda.synchronize()
    a.record()
    rc = 0
    for _ in range(steps):
        rc = rc or step()
    b.record()
    torch.cuda.synchronize()
    secs = a.elapsed_time(b) / 1e3
    for d in (d_bar, d_star, d_om):
        ddp.ddp_free_domain(ctx, d)
    ddp.ddp_free_gauge(ctx, gid)
    # 10 iterations of nm columns on Omega, nm columns on each of Gamma-bar and Gamma*
    col_solves = iters * nm + 2 * nm
    return {"workload": f"48x24^3 projector cut (Sec. 5): x0_cut {x0_cut}, Delta {delta}, {nm} modes from {iters} "
                        f"inverse iterations on t in [{x0_cut - delta}, {x0_cut + delta}), u on [0, {x0_cut + delta}), "
                        f"w on [{x0_cut}, {L[0]}), pion and nucleon for every (y0, x0), kappa {kappa}",
            "s_per_step": secs / steps, "s_per_stage": {k: v / steps for k, v in times.items()},
            "column_solves_per_step": col_solves, "status": rc, "steps": steps, "warmup": warmup,
            # one entry of each correlator: sink slice y0 in Gamma*_0, source slice x0 in Gamma-bar_0
            "pion_C_y40_x4": [float(Cpi[40, 4].real), float(Cpi[40, 4].imag)],
            "nucleon_C_y40_x4": [float(Cn[40, 4].real), float(Cn[40, 4].imag)]}


# ----------------------------------------------------------------------- serving

SERVE_CLASSES = [((4, 4, 4, 4), 0.1555), ((8, 8, 8, 8), 0.1555), ((4, 32, 32, 32), 0.1555),
                 ((8, 32, 32, 32), 0.150), ((16, 32, 32, 32), 0.145)]


def _make_requests(synth, L, nreq, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nreq):
        ext, kmax = SERVE_CLASSES[rng.integers(len(SERVE_CLASSES))]
        origin = tuple(int(rng.integers(L[m])) for m in range(4))
        src = tuple(int((origin[m] + rng.integers(ext[m])) % L[m]) for m in range(4))
        kappa = float(rng.uniform(0.140, kmax))
        out.append((origin, ext, src, kappa))
    return out


def _serve_run(ddp, torch, ctx, gid, L, reqs, precision, rate, budget, max_active):
    """Open-loop Poisson arrivals at `rate` requests/s (rate=None: all at t=0)."""
    ddp.ddp_serve_config(ctx, budget, max_active, precision)
    rng = np.random.default_rng(7)
    arrivals = np.zeros(len(reqs)) if rate is None else np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
    pending = []          # (index, arrival) arrived but not admitted
    inflight = {}         # ticket -> (index, arrival, domain, out)
    lat = np.zeros(len(reqs))
    nxt = 0
    done = 0
    C = torch.zeros(2 * L[0], dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    while done < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and arrivals[nxt] <= now:
            pending.append((nxt, arrivals[nxt]))
            nxt += 1
        still = []
        for i, arr in pending:
            o, e, src, kappa = reqs[i]
            d = ddp.ddp_set_domain(ctx, gid, o, e)
            out = torch.empty((12, int(np.prod(e)), 4, 3), dtype=torch.complex128, device="cuda")
            rc, t = ddp.ddp_submit(ctx, ddp.make_req(d, kappa, src, 1e-10, out))
            if rc == ddp.DDP_OK:
                inflight[t] = (i, arr, d, out)
            else:
                ddp.ddp_free_domain(ctx, d)
                still.append((i, arr))
        pending = still
        if not inflight:
            if nxt < len(reqs):
                time.sleep(max(0.0, min(0.001, arrivals[nxt] - (time.perf_counter() - t0))))
            continue
        ddp.ddp_serve_step(ctx)
        for t in list(inflight):
            f, info = ddp.ddp_poll(ctx, t)
            if f:
                i, arr, d, out = inflight.pop(t)
                ddp.ddp_contract(ctx, ddp.DDP_CONTRACT_NUCLEON, d, out, C)   # the request's correlator
                lat[i] = time.perf_counter() - t0 - arr
                ddp.ddp_free_domain(ctx, d)
                done += 1
    total = time.perf_counter() - t0
    ddp.ddp_serve_reset(ctx)
    return {"solves_per_s": len(reqs) / total, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()), "wall_s": total}


def serve_workload(ddp, torch, ctx, synth, precision, nreq=200, budget=96 << 30, max_active=32):
    """Resident 32^4 field; requests on boxes 4^4 .. 16x32^3 with random origins and
    point sources, kappa uniform in [0.140, min(0.1555, class limit)], 12 columns,
    nucleon correlator per request.  Capacity = closed-loop throughput; then Poisson
    arrivals at 0.5 and 0.9 of it, for the mixed path and for the plain FP64 path."""
    L = synth.BATCH_LATTICE
    U = synth.gauge_field_torch(L, seed=synth.SEED_GAUGE, device="cuda")
    gid = ddp.ddp_load_gauge(ctx, U, L, ddp.DDP_BC_ANTIPERIODIC)
    reqs = _make_requests(synth, L, nreq, synth.SEED_SERVING)
    out = {"workload": f"serving on a resident 32^4 field: {nreq} requests, boxes 4^4..16x32^3, 12 columns, "
                       f"nucleon contraction per request", "requests": nreq}
    for name, prec in (("mixed", precision), ("fp64", ddp.DDP_PREC_FP64)):
        n_here = nreq if name == "mixed" else max(20, nreq // 5)
        sub = reqs[:n_here]
        cap = _serve_run(ddp, torch, ctx, gid, L, sub, prec, None, budget, max_active)
        res = {"capacity_solves_per_s": cap["solves_per_s"], "requests": n_here}
        for f in (0.5, 0.9):
            r = _serve_run(ddp, torch, ctx, gid, L, sub, prec, f * cap["solves_per_s"], budget, max_active)
            res[f"load_{f}"] = r
        out[name] = res
    ddp.ddp_free_gauge(ctx, gid)
    return out
