"""The Nsight Compute summaries in profiles/ are made by ncu_report.py; its
parsing of ncu's CSV (units, thousands separators, tool chatter lines,
aggregation and shares) is checked here on small hand-made files in ncu's
column layout (no GPU, no ncu)."""
import json

import ncu_report

LAUNCH_HDR = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
              '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')


def _launch_row(i, kernel, unit, value):
    return (f'"{i}","1","python3","h","{kernel}","1","7","(128, 1, 1)","(450, 1, 1)","0","10.3",'
            f'"Command line profiler metrics","gpu__time_duration.sum","{unit}","{value}"')


def test_launch_list_aggregates_with_units_and_shares(tmp_path):
    # kernel names as ncu prints them
    te = "void fmx::<unnamed>::k_pol2d<0, 4, 3, 1, 128>(fmx::Fused2dArgs<float>, fmx::Geo, pair2::Coef2, int, int, int)"
    tm = "void fmx::<unnamed>::k_pol2d<1, 4, 3, 1, 128>(fmx::Fused2dArgs<float>, fmx::Geo, pair2::Coef2, int, int, int)"
    fill = "void at::vectorized_elementwise_kernel<4, at::FillFunctor<float>>(int)"
    lines = ["==PROF== Connected to process 1", LAUNCH_HDR,
             _launch_row(0, fill, "ns", "4,000"),
             _launch_row(1, te, "usecond", "150"),
             _launch_row(2, tm, "ns", "110,000"),
             _launch_row(3, te, "msecond", "0.15"),
             "==PROF== Disconnected from process 1"]
    p = tmp_path / "launches.csv"
    p.write_text("\n".join(lines) + "\n")
    table = ncu_report.launches(str(p)).splitlines()
    assert table[0].startswith("| kernel | launches | total us")
    rows = {r.split("|")[1].strip(" `"): [c.strip() for c in r.split("|")[2:6]] for r in table[2:]}
    te_row = rows["k_pol2d TE (Ex, Ey, Bz)"]
    assert te_row[0] == "2" and te_row[1] == "300.0" and te_row[2] == "150.0"
    tm_row = rows["k_pol2d TM (Ez, Bx, By)"]
    assert tm_row[1] == "110.0"
    assert rows["PyTorch buffer fill (allocation zeroing, outside the timed region)"][1] == "4.0"
    # shares of the total device time, largest first
    assert table[2].split("|")[1].strip(" `") == "k_pol2d TE (Ex, Ey, Bz)"
    assert te_row[3] == f"{100 * 300 / 414:.1f}%"


def test_raw_page_counters_and_traffic(tmp_path):
    hdr = ["ID", "Kernel Name", "dram__bytes_read.sum", "dram__bytes_write.sum", "gpu__time_duration.sum",
           "smsp__average_warps_issue_stalled_barrier_per_issue_active.ratio",
           "smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio"]
    units = ["", "", "Mbyte", "Kbyte", "usecond", "", ""]
    te = "void fmx::<unnamed>::k_pol2d<0, 4, 3, 1, 128>(fmx::Fused2dArgs<float>, fmx::Geo, pair2::Coef2, int, int, int)"
    tm = "void fmx::<unnamed>::k_pol2d<1, 4, 3, 1, 128>(fmx::Fused2dArgs<float>, fmx::Geo, pair2::Coef2, int, int, int)"
    rows = [["0", te, "400.5", "170,000", "144.1", "0.39", "1.35"],
            ["1", tm, "325", "168,000", "115.2", "0.2", "1.03"],
            ["2", te, "399.5", "170,000", "144.0", "0.4", "1.3"]]
    q = lambda r: ",".join(f'"{c}"' for c in r)
    p = tmp_path / "raw.csv"
    p.write_text("==PROF== chatter\n" + "\n".join(q(r) for r in [hdr, units] + rows) + "\n")
    text = ncu_report.full(str(p))
    assert text.count("### k_pol2d TE (Ex, Ey, Bz)") == 2 and "### k_pol2d TM (Ez, Bx, By)" in text
    assert "| DRAM read (`dram__bytes_read.sum`) | 400.5 Mbyte |" in text
    assert "long_scoreboard 1.35, barrier 0.39" in text  # stalls sorted, largest first
    out = tmp_path / "traffic.json"
    d = ncu_report.traffic(str(p), str(out))
    assert json.loads(out.read_text()) == d
    assert d["kernel_sha256_16"] == ncu_report.kernel_hash()
    per = d["dram_bytes_per_launch"]
    assert abs(per["k_pol2d TE (Ex, Ey, Bz)"] - (400e6 + 170e6)) < 1.0  # mean of two launches
    assert abs(per["k_pol2d TM (Ez, Bx, By)"] - (325e6 + 168e6)) < 1.0
