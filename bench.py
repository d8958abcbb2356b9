"""Benchmark of the domain-propagator hot path on GB300.

Workload (default): a 48 x 24^3 lattice (antiperiodic in time, periodic in
space) with the seeded synthetic SU(3) field of plaquette 0.59, nested time
slabs of thickness 8, 16, 24 around a point source at the origin plus the
full lattice; per step:
  a1 load + pack the gauge field (from a device copy),
  a3-a5 the four 12-column domain propagators S^(0), S^(1), S^(2), S to a
        true FP64 residual of 1e-10 in one batched solve,
  a6 the three series terms S^(i) - S^(i-1) and S - S^(2),
  a7 nucleon and pion correlators of each propagator and tr{g5 S(x,x)}.
`value` counts domain-propagator solves (12 columns each) per second with
inputs resident in HBM; `e2e` runs the same step through the C ABI with host
buffers (pinned), every transfer inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp16|bf16|fp64]
  python bench.py --impl reference ...   (the FP64 CPU oracle on a bounded sample)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

L = synth.SLAB_LATTICE
THICK = synth.SLAB_THICKNESS
# kappa of the benchmark: the stated 0.1550 lies beyond the critical point of
# the i.i.d. synthetic ensemble (BiCGStab diverges on the 16, 24 and full
# domains), 0.1400 is the largest value on a 0.005 grid at which every domain
# of the workload converges.
KAPPA = 0.1400
CSW = 0.0        # clover coefficient of the operator (0: plain Wilson); --csw
TOL = 1e-10
SRC = (0, 0, 0, 0)
METRIC = "domain-propagator solves/s (12 columns, true FP64 residual 1e-10)"
UNIT = "solves/s"


def boxes():
    out = [synth.centered_time_slab(L, t, 0) for t in THICK]
    out.append(synth.Box((0, 0, 0, 0), L))
    return out


NOMINAL_HBM_GBPS = 7900.0  # GB300 HBM3e, nominal


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _stencil_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in ("ddp_device.cuh", "ddp_kernels.cuh", "clover.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1601_04587_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def hop_traffic_record():
    """ncu DRAM bytes per launch of the stencil kernel, if the committed record
    matches the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "hop_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        rec = json.load(open(p))
        if rec.get("sources_sha256") != _stencil_sources_sha256():
            return None
        return rec
    except Exception:
        return None


HOP_TRAFFIC_LATTICE = (32, 24, 24, 24)
HOP_TRAFFIC_METRICS = ("gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum,"
                       "l1tex__m_xbar2l1tex_read_bytes.sum,launch__registers_per_thread")


def write_hop_traffic(csv_path, out_path=None):
    """profiles/hop_traffic.json (or out_path) from the ncu CSV of the three FP32 stencils
    on the 32x24^3 lattice (the --workload hop run with --iters 1 under
    `ncu --metrics HOP_TRAFFIC_METRICS --clock-control none -k regex:k_hop --csv`):
    DRAM bytes per launch, scaled by site-columns to the 48x24^3 bench launch."""
    import csv
    rows = [r for r in csv.reader(open(csv_path)) if r]
    hdr = next(r for r in rows if "Kernel Name" in r and "Metric Name" in r)
    ix = {k: hdr.index(k) for k in ("Kernel Name", "Metric Name", "Metric Value", "ID")}
    per = {}
    for r in rows[rows.index(hdr) + 1:]:
        if len(r) != len(hdr) or "k_hop" not in r[ix["Kernel Name"]]:
            continue
        d = per.setdefault(r[ix["ID"]], {"name": r[ix["Kernel Name"]]})
        d[r[ix["Metric Name"]]] = float(r[ix["Metric Value"]].replace(",", ""))
    names = {"k_hop<PF32, 0, 0,": "fp32/plain", "k_hop<PF32, 1, 1,": "fp32/schur_rhat", "k_hop<PF32, 1, 2,": "fp32/schur_ts"}
    captured = {}
    for d in per.values():
        key = next((v for k, v in names.items() if k in d["name"].replace("ddp::", "")), None)
        if key is not None and "dram__bytes_read.sum" in d:
            b = d["dram__bytes_read.sum"] + d["dram__bytes_write.sum"]
            captured[key] = min(captured.get(key, b), b)  # launches after the first: warm L2
    sites = HOP_TRAFFIC_LATTICE[0] * HOP_TRAFFIC_LATTICE[1] * HOP_TRAFFIC_LATTICE[2] * HOP_TRAFFIC_LATTICE[3] // 2
    per_site_col = {"fp32/plain": 224, "fp32/schur_rhat": 368, "fp32/schur_ts": 320}
    scale = 48 / HOP_TRAFFIC_LATTICE[0]
    rec = {"what": "ncu DRAM bytes (read + write) per launch of the three inner-loop stencils, FP32 storage, 12 columns",
           "captured_lattice": list(HOP_TRAFFIC_LATTICE), "ncol": 12,
           "captured_bytes": captured,
           "captured_algorithmic_bytes": {k: per_site_col[k] * sites * 12 for k in captured},
           "scale_to_bench": scale,
           "note": "the 48x24^3 launch has 1.5x the captured site-columns; DRAM traffic of these kernels scales with "
                   "site-columns (their re-reads are neighbour gathers missing L2), so the bench's per-launch traffic "
                   "is the captured bytes x 1.5",
           "kernels": {k: v * scale for k, v in captured.items()},
           "command": "python bench.py --workload hop --lattice 32 24 24 24 --precision fp32 --kernel "
                      "plain,schur_rhat,schur_ts --iters 1 (under ncu --metrics " + HOP_TRAFFIC_METRICS +
                      " --clock-control none -k regex:k_hop --csv), then python bench.py --write-hop-traffic CSV",
           "sources_sha256": _stencil_sources_sha256()}
    with open(out_path or os.path.join(ROOT, "profiles", "hop_traffic.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))
    return rec


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = str(device_index)
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.dev, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- GPU arm

CONTRACT_MASK = 0b1101   # local trace (kind 0), nucleon (kind 2), pion (kind 3)


class Workload:
    def __init__(self, ddp, torch, ctx, precision, U):
        self.ddp, self.torch, self.ctx, self.prec = ddp, torch, ctx, precision
        self.U_dev = torch.from_numpy(U).cuda()
        self.bx = boxes()
        self.outs = [torch.zeros((12, b.n_sites, 4, 3), dtype=torch.complex128, device="cuda") for b in self.bx]
        self.terms = [torch.zeros_like(o) for o in self.outs[1:]]
        # [domain][contraction kind][2 L0]: kind 0 local trace (first 2 entries), 2 nucleon, 3 pion
        self.C = torch.zeros((len(self.bx), 4, 2 * L[0]), dtype=torch.float64, device="cuda")
        self.infos = None

    def step(self, host=None):
        """One pass of the hot path: gauge field in, the four nested propagators, their
        series terms and contractions out, in one library call.  host: pinned host
        buffers for the end-to-end variant (the gauge field is uploaded, every result
        downloaded, nothing uploaded twice)."""
        ddp, ctx = self.ddp, self.ctx
        U = self.U_dev if host is None else host["U"]
        outs = self.outs if host is None else host["S"]
        terms = self.terms if host is None else host["T"]
        C = self.C if host is None else host["C"]
        gid = ddp.ddp_load_gauge(ctx, U, L, ddp.DDP_BC_ANTIPERIODIC)
        dids = [ddp.ddp_set_domain(ctx, gid, b.origin, b.extent) for b in self.bx]
        rc, self.infos = ddp.ddp_propagator_series(ctx, dids, KAPPA, SRC, TOL, self.prec, S_out=outs, T_out=terms,
                                                   contract_mask=CONTRACT_MASK, C_out=C, csw=CSW)
        for d in dids:
            ddp.ddp_free_domain(ctx, d)
        ddp.ddp_free_gauge(ctx, gid)
        return rc

    def host_buffers(self):
        t = self.torch
        h = {"U": t.from_numpy(np.ascontiguousarray(self.U_dev.cpu().numpy())).pin_memory(),
             "S": [t.zeros(o.shape, dtype=o.dtype).pin_memory() for o in self.outs],
             "T": [t.zeros(o.shape, dtype=o.dtype).pin_memory() for o in self.terms],
             "C": t.zeros(self.C.shape, dtype=t.float64).pin_memory()}
        nb = lambda x: x.numel() * x.element_size()  # noqa: E731
        # H2D: the gauge field only; D2H: the propagators, the series terms and the correlators
        h2d = nb(h["U"])
        d2h = sum(nb(x) for x in h["S"]) + sum(nb(x) for x in h["T"]) + nb(h["C"])
        return h, h2d, d2h


def pinned_link_rate(torch, bufs):
    """Host<->device copy rates (GB/s) over the step's pinned host buffers, taken
    just before the end-to-end timing: the host->device rate of this shared
    link varies from run to run (the device->host rate much less), and the
    end-to-end figure moves with it."""
    nbytes = sum(b.numel() * b.element_size() for b in bufs)
    devs = [torch.empty_like(b, device="cuda") for b in bufs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for d, b in zip(devs, bufs):
        d.copy_(b, non_blocking=True)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for d, b in zip(devs, bufs):
        b.copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    del devs
    return {"h2d": round(nbytes / (t1 - t0) / 1e9, 1), "d2h": round(nbytes / (t2 - t1) / 1e9, 1)}


def timed(torch, fn, steps, dist=None):
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    start.record()
    for _ in range(steps):
        fn()
    end.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    return start.elapsed_time(end) / 1e3


CPU_SAMPLE = "1 of the 12 columns of the 8-thick and of the 16-thick slab propagators (2 of the step's 48 " \
             "column-solves, the two cheapest domains of the step)"


def oracle_columns(U, kappa, boxes_, tol):
    """Column 0 (spin 0, colour 0) of the point-source propagator of each box, solved
    by the FP64 oracle as it stands; returns (seconds, columns)."""
    import oracle
    cols = []
    t0 = time.perf_counter()
    for b in boxes_:
        n = b.n_sites
        eta = np.zeros((1, n, 4, 3), dtype=np.complex128)
        eta[0, oracle.local_index(L, b.origin, b.extent, SRC), 0, 0] = 1.0
        psi, _, _, _ = oracle.solve(U, L, oracle.BC_ANTIPERIODIC, b.origin, b.extent, kappa, eta, tol=tol, csw=CSW)
        cols.append(psi[0])
    return time.perf_counter() - t0, cols


def cpu_oracle_sample(U, kappa):
    """The timed CPU baseline: the oracle on column 0 of the 8- and the 16-thick slab
    propagators at the metric's tolerance, 2 of the step's 48 column-solves."""
    return oracle_columns(U, kappa, boxes()[:2], TOL)


def cpu_baseline_line(dt, cores):
    """The timed oracle sample as it was run: 2 column-solves in dt seconds; `value`
    expresses those 2 column-solves in the metric's unit (12 column-solves make one
    propagator solve), with no other extrapolation."""
    return {"value": (2.0 / 12.0) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "column_solves_per_s": 2.0 / dt, "timed": "2 of 48 column-solves of one step",
            "seconds": dt, "sample": CPU_SAMPLE + f", {dt:.1f} s of FP64 CPU work at the metric's tolerance "
                                                 f"{TOL}; value = (2/12) propagator solves / time"}


def _rel(a, b):
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def parity_block(ddp, torch, ctx, wl, U, cpu_cols):
    """Error of the measured run against the FP64 oracle.
    columns: the GPU columns the CPU leg solved, relative L2 error per column and of
      the pion correlator of that column;
    propagators: every column of every propagator, the oracle's own true residual
      |eta - D_Gamma psi_gpu| / |eta| (oracle operator, FP64);
    correlators: every correlator of the step, relative L2 error of the GPU value
      against the oracle's contraction of the same propagator."""
    import oracle
    out = {"columns": [], "propagators": [], "correlators": []}
    S_host = [o.cpu().numpy() for o in wl.outs]
    for i, (b, ref) in enumerate(zip(wl.bx[:2], cpu_cols)):
        got = S_host[i][0]
        # the pion contraction of one column: the oracle's contraction with the other 11
        # columns zero (sum over the column's own |psi|^2 per time slice)
        one = np.zeros((12,) + got.shape, dtype=np.complex128)
        one[0] = ref
        pi_ref = oracle.pion(L, b.origin, b.extent, one)
        one[0] = got
        pi_gpu = oracle.pion(L, b.origin, b.extent, one)
        del one
        out["columns"].append({"domain": list(b.extent), "column": 0, "rel_l2_error": _rel(got, ref),
                               "pion_rel_l2_error": _rel(pi_gpu, pi_ref)})
    for i, b in enumerate(wl.bx):
        S = S_host[i]
        eta = np.zeros_like(S)
        l = oracle.local_index(L, b.origin, b.extent, SRC)
        for c in range(12):
            eta[c, l, c // 3, c % 3] = 1.0
        r = eta - oracle.apply_dirac(U, L, oracle.BC_ANTIPERIODIC, b.origin, b.extent, KAPPA, S, csw=CSW)
        rr = [float(np.linalg.norm(r[c]) / np.linalg.norm(eta[c])) for c in range(12)]
        out["propagators"].append({"domain": list(b.extent), "oracle_max_rel_residual": max(rr)})
        C = wl.C[i].cpu().numpy()
        nuc = oracle.nucleon(L, b.origin, b.extent, S)
        pio = oracle.pion(L, b.origin, b.extent, S)
        ltr = oracle.local_trace(L, b.origin, b.extent, S, SRC)
        tr = C[0]
        out["correlators"].append({"domain": list(b.extent),
                                   "nucleon_rel_l2_error": _rel(C[2, 0::2] + 1j * C[2, 1::2], nuc),
                                   "pion_rel_l2_error": _rel(C[3, 0::2], pio),
                                   "local_trace_rel_error": abs(complex(tr[0], tr[1]) - ltr) / abs(ltr)})
    out["max_column_rel_l2_error"] = max(c["rel_l2_error"] for c in out["columns"])
    out["max_oracle_rel_residual"] = max(p["oracle_max_rel_residual"] for p in out["propagators"])
    out["max_correlator_rel_l2_error"] = max(max(c["nucleon_rel_l2_error"], c["pion_rel_l2_error"],
                                                 c["local_trace_rel_error"]) for c in out["correlators"])
    out["tolerances"] = {"column": 1e-8, "correlator": 1e-7}
    return out


HOP_KERNELS = (("plain", "DDP_HOP_PLAIN", 2, "tmp = H_oe p"),
               ("schur_rhat", "DDP_HOP_SCHUR_RHAT", 1, "v = p - k^2 H_eo tmp; (rh, v)"),
               ("schur_ts", "DDP_HOP_SCHUR_TS", 1, "t = s - k^2 H_eo tmp; (t, s), (t, t)"))


def stencil_roofline(ddp, ctx, U_dev, prec, precision_name, iters=50):
    """CUDA-event time of every inner-loop stencil variant on the full 48x24^3 domain
    with 12 columns; the dominant one (largest share of a BiCGStab iteration:
    launches per iteration x time per launch) is the roofline kernel."""
    gid = ddp.ddp_load_gauge(ctx, U_dev, L, ddp.DDP_BC_ANTIPERIODIC)
    did = ddp.ddp_set_domain(ctx, gid, (0, 0, 0, 0), L)
    peak, peak_kind = measured_peaks()
    rec = hop_traffic_record()
    per = {}
    for name, const, per_iter, what in HOP_KERNELS:
        ms, nbytes = ddp.ddp_time_hop(ctx, did, KAPPA, 12, prec, iters, getattr(ddp, const))
        achieved = nbytes / (ms * 1e-3) / 1e9
        traffic = None
        if rec:
            traffic = rec.get("kernels", {}).get(f"{precision_name}/{name}")
        per[name] = {"computes": what, "launches_per_iteration": per_iter, "ms_per_launch": ms,
                     "algorithmic_bytes_per_launch": nbytes, "achieved": achieved, "frac": achieved / peak,
                     "traffic": traffic,
                     # the ncu DRAM bytes of a launch over its CUDA-event time
                     "dram_gbps": (traffic / (ms * 1e-3) / 1e9) if traffic else None}
    ddp.ddp_free_domain(ctx, did)
    ddp.ddp_free_gauge(ctx, gid)
    tot = sum(v["launches_per_iteration"] * v["ms_per_launch"] for v in per.values())
    for v in per.values():
        v["share_of_stencil_time"] = v["launches_per_iteration"] * v["ms_per_launch"] / tot
    dom = max(per, key=lambda k: per[k]["share_of_stencil_time"])
    d = per[dom]
    return {"bound": "hbm", "achieved": d["achieved"], "peak": peak, "unit": "GB/s", "frac": d["frac"],
            "traffic": d["traffic"], "kernel": f"k_hop<{precision_name}> {dom}: {d['computes']}",
            "ms_per_launch": d["ms_per_launch"], "algorithmic_bytes_per_launch": d["algorithmic_bytes_per_launch"],
            "launch": "48x24^3 full lattice, 12 columns, 3,981,312 output site-columns",
            "peak_kind": f"{peak_kind} HBM copy bandwidth", "dram_gbps": d["dram_gbps"],
            "frac_of_nominal": d["achieved"] / NOMINAL_HBM_GBPS, "nominal_peak": NOMINAL_HBM_GBPS, "per_kernel": per}


def run_gpu(args):
    import torch

    import paper_1601_04587_gb300 as ddp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    prec = ddp.PRECISIONS[args.precision]
    U = synth.gauge_field(L, seed=synth.SEED_GAUGE + rank)
    ctx = ddp.ddp_create(torch.cuda.current_device(), torch.cuda.current_stream().cuda_stream)
    if args.no_conditional:
        ddp.ddp_set_param(ctx, "conditional", 0)
    for kv in args.param:
        k, v = kv.split("=")
        ddp.ddp_set_param(ctx, k, float(v))
    wl = Workload(ddp, torch, ctx, prec, U)
    for _ in range(args.warmup):
        wl.step()
    launches0 = ddp.ddp_kernel_launches(ctx)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    secs = timed(torch, wl.step, args.steps, dist)
    clk = clocks.stop()
    launches = ddp.ddp_kernel_launches(ctx) - launches0
    infos = [ddp.info_dict(i) for i in wl.infos]
    # slowest rank decides
    if dist:
        t = torch.tensor([secs], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        secs = float(t.item())
    nsolve = len(wl.bx) * args.steps * world
    value = nsolve / secs

    # end to end: host buffers through the C ABI, transfers inside the timed region
    host, h2d, d2h = wl.host_buffers()
    wl.step(host)
    link = pinned_link_rate(torch, [host["U"]] + host["S"] + host["T"])
    e2e_secs = timed(torch, lambda: wl.step(host), max(1, args.steps // 2), dist)
    if dist:
        t = torch.tensor([e2e_secs], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_secs = float(t.item())
    e2e_value = len(wl.bx) * max(1, args.steps // 2) * world / e2e_secs

    # plain FP64 GPU path on the same workload
    fp64 = None
    if not args.skip_fp64 and prec != ddp.DDP_PREC_FP64:
        wl64 = Workload(ddp, torch, ctx, ddp.DDP_PREC_FP64, U)
        wl64.step()
        s64 = timed(torch, wl64.step, 1, dist)
        fp64 = {"solves_per_s": len(wl.bx) / s64, "ms_per_step": 1e3 * s64,
                "max_rel_residual": max(i.max_rel_residual for i in wl64.infos)}
        del wl64

    roof = stencil_roofline(ddp, ctx, wl.U_dev, prec, args.precision)
    col_iters = sum(i["column_iters"] for i in infos)
    site_col_iters = sum(i["column_iters"] * b.n_sites // 2 for i, b in zip(infos, wl.bx))

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "fp16": "f16",
                                                           "bf16": "bf16"}[args.precision],
        "data": "synthetic (seeded SU(3) field, plaquette 0.59)",
        "config": {"workload": f"48x24^3 nested time slabs 8/16/24 + full lattice, 12-column point-source "
                               f"propagators, kappa {KAPPA}, tol {TOL}" + (f", clover c_sw {CSW}" if CSW else ""),
                   "lattice": list(L), "kappa": KAPPA, "kappa_stated": 0.155, "tol": TOL, "csw": CSW,
                   "precision": f"mixed: FP32 inner on {args.precision} storage, FP64 defect correction"
                   if prec else "fp64",
                   "l2": "inputs larger than L2 (links 0.38 GB FP64, propagators 3.1 GB)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "pinned_GBps": link},
        "gpu_launches": int(launches),
        "clocks": clk,
        "roofline": roof,
        # kappa-independent throughput of the inner solver: BiCGStab iterations of single
        # columns (and of even site-columns) per second, summed over the step's 48 columns
        "column_iterations_per_s": col_iters * args.steps * world / secs,
        "site_column_iterations_per_s": site_col_iters * args.steps * world / secs,
        "inner_iterations_per_step": col_iters,
        "fp64_path": fp64,
        "speedup_vs_fp64": (value / fp64["solves_per_s"]) if fp64 else None,
        "solves": infos,
    }
    if rank == 0 and world == 1 and not args.skip_cpu:
        import oracle
        dt, _ = cpu_oracle_sample(U, KAPPA)
        line["cpu_baseline"] = cpu_baseline_line(dt, oracle.num_threads())
        # parity columns at the oracle's own tolerance (1e-12), so that its error is negligible
        _, cols = oracle_columns(U, KAPPA, boxes()[:2], 1e-12)
        line["parity"] = parity_block(ddp, torch, ctx, wl, U, cols)
    ddp.ddp_destroy(ctx)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def run_other(args):
    """Extra measurement lines: the uneven batch, the two-level workload, serving."""
    import torch

    import paper_1601_04587_gb300 as ddp
    from paper_1601_04587_gb300 import workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        # the uneven batch shards its domains across the ranks; the other workloads
        # are single-GPU measurements that rank 0 makes alone
        if args.workload != "batch":
            if rank != 0:
                return
            world = 1
        else:
            import torch.distributed as dist
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            dist.init_process_group("nccl")
    if dist is None:
        torch.cuda.set_device(0)
    prec = ddp.PRECISIONS[args.precision]
    ctx = ddp.ddp_create(torch.cuda.current_device(), torch.cuda.current_stream().cuda_stream)
    for kv in args.param:
        k, v = kv.split("=")
        ddp.ddp_set_param(ctx, k, float(v))
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if args.workload == "batch":
        res = workloads.batch_workload(ddp, torch, ctx, synth, prec, steps=args.steps, warmup=args.warmup, dist=dist)
    elif args.workload == "multilevel":
        res = workloads.multilevel_workload(ddp, torch, ctx, synth, prec, steps=args.steps, warmup=args.warmup)
    elif args.workload == "next":
        res = workloads.next_rows_workload(ddp, torch, ctx, synth, prec, steps=args.steps, warmup=args.warmup)
    elif args.workload == "projector":
        res = workloads.projector_workload(ddp, torch, ctx, synth, prec, nm=args.modes, steps=args.steps,
                                           warmup=args.warmup)
    else:
        res = workloads.serve_workload(ddp, torch, ctx, synth, prec)
    res["clocks"] = clocks.stop()
    res["precision"] = args.precision
    res["gpu_launches"] = ddp.ddp_kernel_launches(ctx)
    ddp.ddp_destroy(ctx)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res))


# ---------------------------------------------------------- reference arm

REF_SAMPLE = "column 0 of the 8-thick slab propagator (1 of the step's 48 column-solves, the step's cheapest domain)"


def run_reference(args):
    """The oracle as it stands on the host cores: per step, one column-solve of the
    workload (bounded so that the whole run takes a few minutes); value = that
    column-solve in the metric's unit (1/12 of a propagator solve) per second."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    U = synth.gauge_field(L, seed=synth.SEED_GAUGE)
    for _ in range(args.warmup):
        oracle_columns(U, KAPPA, boxes()[:1], TOL)
    dt = 0.0
    for _ in range(args.steps):
        d, _ = oracle_columns(U, KAPPA, boxes()[:1], TOL)
        dt += d
    value = args.steps * (1.0 / 12.0) / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded SU(3) field, plaquette 0.59)",
            "config": {"workload": f"48x24^3 nested time slabs 8/16/24 + full lattice, 12-column point-source "
                                   f"propagators, kappa {KAPPA}, tol {TOL}", "kappa": KAPPA},
            "cpu_baseline": {"kind": "oracle", "cores": oracle.num_threads(), "value": value, "unit": UNIT,
                             "column_solves_per_s": args.steps / dt, "timed": "1 of 48 column-solves per step",
                             "sample": "per step: " + REF_SAMPLE + f", at tolerance {TOL}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_colourless(args):
    """The colourless-spinor sums of the projector cut (Eq. W0tbary) on one 24^3 time slice
    with --modes spinor columns (random, seeded, device-resident), the size of every slice
    of the 48x24^3 projector workload: CUDA-event time per call (diquarks, splitting,
    the emulated-FP64 tensor-core product, exponents and symmetric fill) and the rate of
    the slice-pair MMA work that the product issues."""
    import torch

    import paper_1601_04587_gb300 as ddp

    m = args.modes
    Ls = (2, 24, 24, 24)
    box = ((0, 0, 0, 0), (1, 24, 24, 24))
    ns = 24 ** 3
    ctx = ddp.ddp_create(0, torch.cuda.current_stream().cuda_stream)
    U = synth.gauge_field_torch(Ls, seed=synth.SEED_GAUGE, device="cuda")
    gid = ddp.ddp_load_gauge(ctx, U, Ls, ddp.DDP_BC_ANTIPERIODIC)
    did = ddp.ddp_set_domain(ctx, gid, *box)
    A = torch.from_numpy(synth.random_spinor(m, ns, synth.SEED_NOISE0 + 11)).cuda()
    X = torch.zeros((Ls[0], m, m, m, 4), dtype=torch.complex128, device="cuda")
    ddp.ddp_colourless_slices(ctx, did, A, m, 1, X)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(args.iters):
        ddp.ddp_colourless_slices(ctx, did, A, m, 1, X)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.iters
    ddp.ddp_destroy(ctx)
    rows, q = m * (m + 1) // 2, 4 * m
    mt, nt = -(-rows // 128), -(-(2 * q) // 64)
    kp = -(-(2 * 3 * ns) // 16) * 16  # [Re | Im] halves of the 3 x sites reduction, 16-deep steps
    mma_flop = 28 * 2.0 * (mt * 128) * (nt * 64) * kp  # 28 slice-pair products per padded tile
    fp64_flop = 8.0 * rows * q * 3 * ns  # the complex product itself, one multiply-add = 8 flops
    print(json.dumps({"workload": "colourless", "slice": [24, 24, 24], "modes": m, "diquark_rows": rows,
                      "tiles": [mt, nt], "ms_per_slice": ms, "mma_tflops": mma_flop / ms / 1e9,
                      "fp64_equivalent_tflops": fp64_flop / ms / 1e9}))


def run_hop(args):
    """One stencil variant alone on a whole lattice (the ncu target for the stencil
    profiles): average CUDA-event time of `--iters` launches and the bandwidth its
    algorithmic bytes imply."""
    import torch

    import paper_1601_04587_gb300 as ddp

    Lh = tuple(args.lattice)
    U = synth.gauge_field_torch(Lh, seed=synth.SEED_GAUGE, device="cuda")
    ctx = ddp.ddp_create(0, torch.cuda.current_stream().cuda_stream)
    for kv in args.param:
        k, v = kv.split("=")
        ddp.ddp_set_param(ctx, k, float(v))
    gid = ddp.ddp_load_gauge(ctx, U, Lh, ddp.DDP_BC_ANTIPERIODIC)
    did = ddp.ddp_set_domain(ctx, gid, (0, 0, 0, 0), Lh)
    kern = {"plain": ddp.DDP_HOP_PLAIN, "schur_rhat": ddp.DDP_HOP_SCHUR_RHAT, "schur_ts": ddp.DDP_HOP_SCHUR_TS}
    res = {}
    for name in (args.kernel.split(",") if args.kernel != "all" else list(kern)):
        ms, nbytes = ddp.ddp_time_hop(ctx, did, KAPPA, args.ncol, ddp.PRECISIONS[args.precision], args.iters,
                                      kern[name])
        res[name] = {"ms_per_launch": ms, "algorithmic_bytes": nbytes, "GBps": nbytes / ms / 1e6}
    ddp.ddp_destroy(ctx)
    print(json.dumps({"workload": "hop", "lattice": Lh, "ncol": args.ncol, "precision": args.precision,
                      "kernels": res}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 5; 1 for the two-level workload, whose steps take minutes)")
    ap.add_argument("--warmup", type=int, default=None,
                    help="untimed warm-up steps (default 3; 0 for the two-level workload)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp16", "bf16"])
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--workload", default="slabs", choices=["slabs", "batch", "multilevel", "serve", "next", "hop",
                                                         "projector", "colourless"],
                    help="slabs: the benchmark line; the others print their own measurement line")
    ap.add_argument("--lattice", type=int, nargs=4, default=[32, 24, 24, 24], help="--workload hop: lattice")
    ap.add_argument("--kernel", default="all", help="--workload hop: plain, schur_rhat, schur_ts or all")
    ap.add_argument("--ncol", type=int, default=12, help="--workload hop: columns")
    ap.add_argument("--iters", type=int, default=20,
                    help="--workload hop: timed launches per kernel; colourless: timed calls")
    ap.add_argument("--param", action="append", default=[],
                    help="solver parameter name=value passed to ddp_set_param (repeatable)")
    ap.add_argument("--modes", type=int, default=120,
                    help="--workload projector / colourless: number of modes N_m (default 120, the paper's)")
    ap.add_argument("--kappa", type=float, default=None, help="slabs: kappa (default 0.14)")
    ap.add_argument("--csw", type=float, default=0.0, help="slabs: clover coefficient c_sw (default 0)")
    ap.add_argument("--no-conditional", action="store_true",
                    help="run the inner loop as host-polled graph chunks (profilers see its kernels)")
    ap.add_argument("--write-hop-traffic", metavar="CSV", default=None,
                    help="write profiles/hop_traffic.json from an ncu CSV of the stencil bytes and exit")
    args = ap.parse_args()
    if args.write_hop_traffic:
        write_hop_traffic(args.write_hop_traffic)
        return
    global KAPPA, CSW
    if args.kappa is not None:
        KAPPA = args.kappa
    CSW = args.csw
    long_steps = args.workload == "multilevel"
    short = args.workload in ("next", "projector")
    if args.steps is None:
        args.steps = 1 if long_steps else (2 if short else 5)
    if args.warmup is None:
        args.warmup = 0 if long_steps else (1 if short else 3)
    if args.warmup < 3 and args.workload == "slabs" and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "hop":
        run_hop(args)
    elif args.workload == "colourless":
        run_colourless(args)
    elif args.workload != "slabs":
        run_other(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
