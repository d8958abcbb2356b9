"""The measurement script's own arithmetic and output contract (CPU only): the DRAM
traffic record built from an ncu CSV, and the JSON line of the reference arm (the FP64
oracle on the host cores)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

HDR = ['"ID"', '"Kernel Name"', '"Metric Name"', '"Metric Unit"', '"Metric Value"']


def _csv(tmp_path, rows):
    p = tmp_path / "bytes.csv"
    lines = ["==PROF== a line ncu writes before the table", ",".join(HDR)]
    for i, name, metric, value in rows:
        lines.append(",".join(f'"{x}"' for x in (i, name, metric, "byte", value)))
    p.write_text("\n".join(lines) + "\n")
    return str(p)


def test_hop_traffic_record_from_ncu_csv(tmp_path):
    """Per variant the smallest read + write of its launches, scaled by the 48/32 ratio of
    site-columns, beside the algorithmic bytes of 224, 368 (BF16 shadow residual) and 320
    bytes per site-column of the 32x24^3 lattice with 12 columns."""
    names = {"plain": "void ddp::k_hop<ddp::PF32, 0, 0, 0>(ddp::HopArgs)",
             "schur_rhat": "void ddp::k_hop<ddp::PF32, 1, 1, 0>(ddp::HopArgs)",
             "schur_ts": "void ddp::k_hop<ddp::PF32, 1, 2, 0>(ddp::HopArgs)"}
    rows, i = [], 0
    for key, (r1, w1, r2, w2) in {"plain": (400, 230, 384, 226), "schur_rhat": (800, 240, 797, 241),
                                  "schur_ts": (660, 240, 654, 237)}.items():
        for r, w in ((r1, w1), (r2, w2)):
            rows += [(i, names[key], "dram__bytes_read.sum", f"{r}000000"),
                     (i, names[key], "dram__bytes_write.sum", f"{w}000000")]
            i += 1
    rows.append((i, "void other(int)", "dram__bytes_read.sum", "5"))
    out = tmp_path / "rec.json"
    rec = bench.write_hop_traffic(_csv(tmp_path, rows), str(out))
    assert json.loads(out.read_text()) == rec
    assert rec["captured_bytes"] == {"fp32/plain": 610e6, "fp32/schur_rhat": 1038e6, "fp32/schur_ts": 891e6}
    sites = 32 * 24 ** 3 // 2
    assert rec["captured_algorithmic_bytes"] == {"fp32/plain": 224 * sites * 12,
                                                 "fp32/schur_rhat": 368 * sites * 12,
                                                 "fp32/schur_ts": 320 * sites * 12}
    assert rec["scale_to_bench"] == 1.5
    assert rec["kernels"]["fp32/plain"] == 610e6 * 1.5
    assert rec["sources_sha256"] == bench._stencil_sources_sha256()


def test_reference_arm_line():
    """One step of the reference arm: the oracle's column-solve on the host cores, in the
    metric and unit of the GPU line, with its CPU-baseline description and a zero-copy e2e."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("48x24^3 nested time slabs")
