"""Summaries of Nsight Compute output for the kernels of the field-advance
library (measurement tooling beside bench.py, not part of the library).

    python ncu_report.py launches launches.csv
        per-kernel launches, total device time and share from a launch list
        (ncu --metrics gpu__time_duration.sum --csv --log-file launches.csv ...)
    python ncu_report.py full raw.csv
        key counters per captured launch from `ncu -i rep --page raw --csv`
    python ncu_report.py traffic raw.csv out.json
        dram bytes (read + write) per launch of each TE / TM kernel, stored
        with the hash of the kernel sources they were taken on (bench.py
        reports them as `traffic` only while the hash still matches)

Times under ncu are cold-cache and serialised: compare shares, not absolutes.
"""
from __future__ import annotations

import collections
import csv
import hashlib
import json
import os
import sys

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "paper_1907_13088_gb300", "csrc")
KERNEL_SOURCES = ("fused2d_pol.cu", "pol_tile.cuh", "pair2.cuh", "fused2d.h", "fmx_internal.h")


def kernel_hash() -> str:
    """First 16 hex digits of the sha256 of the TE / TM kernel sources."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(_CSRC, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def short_name(name: str) -> str:
    """Kernel label used by bench.py's per-kernel timings where one exists."""
    if "k_pol2d<0" in name:
        return "k_pol2d TE (Ex, Ey, Bz)"
    if "k_pol2d<1" in name:
        return "k_pol2d TM (Ez, Bx, By)"
    if name.startswith("void at::") or " at::" in name:
        return "PyTorch buffer fill (allocation zeroing, outside the timed region)"
    return name.split("(")[0].replace("void ", "").split("::")[-1]


def launches(path: str) -> str:
    with open(path) as f:
        lines = [l for l in f if l.startswith('"')]
    agg = collections.OrderedDict()
    for r in csv.DictReader(lines):
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        scale = {"ns": 1e-3, "nsecond": 1e-3, "usecond": 1.0, "us": 1.0, "msecond": 1e3, "ms": 1e3}.get(
            r["Metric Unit"], 1.0)
        n = short_name(r["Kernel Name"])
        c, s = agg.get(n, (0, 0.0))
        agg[n] = (c + 1, s + float(r["Metric Value"].replace(",", "")) * scale)
    total = sum(s for _, s in agg.values()) or 1.0
    out = ["| kernel | launches | total us | mean us | share |", "|---|---|---|---|---|"]
    for n, (c, s) in sorted(agg.items(), key=lambda x: -x[1][1]):
        out.append(f"| `{n}` | {c} | {s:.1f} | {s / c:.1f} | {100 * s / total:.1f}% |")
    return "\n".join(out)


FULL_METRICS = (
    ("gpu__time_duration.sum", "duration"),
    ("dram__bytes_read.sum", "DRAM read"),
    ("dram__bytes_write.sum", "DRAM write"),
    ("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "DRAM throughput % of peak"),
    ("launch__grid_size", "CTAs"),
    ("launch__registers_per_thread", "registers / thread"),
    ("launch__shared_mem_per_block_dynamic", "dynamic smem / CTA"),
    ("launch__occupancy_limit_registers", "CTAs / SM (register limit)"),
    ("launch__occupancy_limit_shared_mem", "CTAs / SM (smem limit)"),
    ("sm__warps_active.avg.pct_of_peak_sustained_active", "warps active % of peak"),
    ("smsp__issue_active.avg.pct_of_peak_sustained_active", "issue active %"),
    ("smsp__inst_executed.sum", "warp instructions"),
    ("sass__inst_executed_shared_loads", "shared loads (warp instr.)"),
    ("sass__inst_executed_shared_stores", "shared stores (warp instr.)"),
    ("l1tex__data_pipe_lsu_wavefronts_mem_shared.sum", "shared wavefronts"),
    ("l1tex__data_bank_conflicts_pipe_lsu_mem_shared.sum", "shared bank conflicts"),
    ("l1tex__throughput.avg.pct_of_peak_sustained_active", "L1 throughput %"),
    ("lts__t_sector_hit_rate.pct", "L2 hit rate %"),
    ("sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active", "FMA pipe %"),
    ("sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active", "ALU pipe %"),
    ("sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active", "LSU pipe %"),
    ("sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active", "tensor pipe %"),
)


def _raw_rows(path):
    with open(path) as f:
        rows = list(csv.reader(l for l in f if l.startswith('"')))
    return rows[0], rows[1], rows[2:]


def full(path: str) -> str:
    hdr, units, rows = _raw_rows(path)
    col = {h: i for i, h in enumerate(hdr)}
    out = []
    for v in rows:
        name = short_name(v[col["Kernel Name"]]) if "Kernel Name" in col else "?"
        out.append(f"### {name}\n\n| counter | value |\n|---|---|")
        for m, label in FULL_METRICS:
            if m in col and v[col[m]] != "":
                out.append(f"| {label} (`{m}`) | {v[col[m]]} {units[col[m]]} |")
        stalls = [(h[len("smsp__average_warps_issue_stalled_"):-len("_per_issue_active.ratio")], v[i])
                  for h, i in col.items()
                  if h.startswith("smsp__average_warps_issue_stalled") and h.endswith("_per_issue_active.ratio")]
        stalls = sorted(((n, float(x)) for n, x in stalls if x), key=lambda t: -t[1])[:6]
        out.append("| top stall reasons (warps per issue) | " + ", ".join(f"{n} {x:.2f}" for n, x in stalls) + " |")
        out.append("")
    return "\n".join(out)


def _bytes(val: str, unit: str) -> float:
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}.get(unit, 1.0)
    return float(val.replace(",", "")) * scale


def traffic(path: str, out_json: str) -> dict:
    hdr, units, rows = _raw_rows(path)
    col = {h: i for i, h in enumerate(hdr)}
    per = collections.defaultdict(list)
    for v in rows:
        name = short_name(v[col["Kernel Name"]])
        rd = _bytes(v[col["dram__bytes_read.sum"]], units[col["dram__bytes_read.sum"]])
        wr = _bytes(v[col["dram__bytes_write.sum"]], units[col["dram__bytes_write.sum"]])
        per[name].append(rd + wr)
    d = {"kernel_sha256_16": kernel_hash(),
         "dram_bytes_per_launch": {n: sum(x) / len(x) for n, x in per.items()},
         "source": os.path.basename(path)}
    with open(out_json, "w") as f:
        json.dump(d, f, indent=1)
    return d


if __name__ == "__main__":
    mode = sys.argv[1]
    if mode == "launches":
        print(launches(sys.argv[2]))
    elif mode == "full":
        print(full(sys.argv[2]))
    elif mode == "traffic":
        print(json.dumps(traffic(sys.argv[2], sys.argv[3]), indent=1))
    else:
        raise SystemExit(__doc__)
