"""Summarise an ncu launch list (--metrics gpu__time_duration.sum --csv) per
kernel: launches, total device time, share.  Usage:
    python profiles/summarize_launches.py launches.csv
"""
import collections
import csv
import sys


def main(path):
    rows = []
    with open(path) as f:
        lines = [l for l in f if l.startswith('"')]
    for r in csv.DictReader(lines):
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        unit = r["Metric Unit"]
        v = float(r["Metric Value"].replace(",", ""))
        scale = {"ns": 1e-3, "usecond": 1.0, "us": 1.0, "msecond": 1e3, "ms": 1e3}.get(unit, 1.0)
        name = r["Kernel Name"]
        short = name.split("(")[0].replace("void ", "").split("::")[-1]
        if name.startswith("void at::") or " at::" in name:
            short = "PyTorch buffer fill (allocation zeroing, outside the timed region)"
        if "k_pol2d<0" in name:
            short = "k_pol2d TE " + name[name.index("k_pol2d<"):].split(">")[0] + ">"
        elif "k_pol2d<1" in name:
            short = "k_pol2d TM " + name[name.index("k_pol2d<"):].split(">")[0] + ">"
        rows.append((short, v * scale))
    agg = collections.OrderedDict()
    for n, t in rows:
        c, s = agg.get(n, (0, 0.0))
        agg[n] = (c + 1, s + t)
    total = sum(s for _, s in agg.values())
    print(f"| kernel | launches | total us | mean us | share |")
    print(f"|---|---|---|---|---|")
    for n, (c, s) in sorted(agg.items(), key=lambda x: -x[1][1]):
        print(f"| `{n}` | {c} | {s:.1f} | {s / c:.1f} | {100 * s / total:.1f}% |")


if __name__ == "__main__":
    main(sys.argv[1])
