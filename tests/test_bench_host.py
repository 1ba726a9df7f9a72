"""Host-side arithmetic of bench.py's roofline objects (no GPU needed)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_alu_roofline_of_the_3d_step():
    b = _bench()
    # as the factored z-march kernels evaluate it: filter 63, source 53, four
    # sweeps of 112, update 3, Faraday 24
    assert b.FLOPS_PER_CELL_STEP_3D == 591
    assert abs(b.FP32_PEAK_TFLOPS - 80.548) < 1e-3
    r = b.alu_roofline(512 ** 3, 5.5e-3)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 591 * 512 ** 3 / 5.5e-3 / 1e12) < 0.01
    assert abs(r["frac"] - r["achieved"] / b.FP32_PEAK_TFLOPS) < 1e-3
    # below the ridge: flops per algorithmic byte under peak flops per HBM byte,
    # so the step's roof is HBM
    assert b.FLOPS_PER_CELL_STEP_3D / b.BYTES_PER_CELL < b.FP32_PEAK_TFLOPS * 1e12 / (6761.6e9)


def _commands():
    """Command lines quoted in the profile summaries (continuations joined)."""
    out = []
    pdir = os.path.join(ROOT, "profiles")
    for name in sorted(os.listdir(pdir)):
        if not name.endswith(".md"):
            continue
        with open(os.path.join(pdir, name)) as f:
            lines = f.read().splitlines()
        buf = ""
        for line in lines:
            t = line.strip()
            if buf:
                buf += " " + t.rstrip("\\").strip()
                if not t.endswith("\\"):
                    out.append((name, buf))
                    buf = ""
            elif t.startswith(("python ", "ncu ")):
                if t.endswith("\\"):
                    buf = t.rstrip("\\").strip()
                else:
                    out.append((name, t))
    return out


def test_profile_commands_run_committed_files():
    """Every command a profile summary quotes names a bench.py option set the
    parser accepts, an existing ncu_report mode, or the build module's
    resource report: the summaries stay reproducible from committed files."""
    import shlex
    b = _bench()
    import ncu_report
    from paper_1907_13088_gb300 import build
    cmds = _commands()
    assert len(cmds) >= 8
    seen_bench = 0
    for name, cmd in cmds:
        words = shlex.split(cmd)
        if "bench.py" in words:
            args = words[words.index("bench.py") + 1:]
            b._parser().parse_args(args)  # raises SystemExit on an unknown option
            seen_bench += 1
        if "ncu_report.py" in words:
            mode = words[words.index("ncu_report.py") + 1]
            assert hasattr(ncu_report, mode), (name, mode)
        if "paper_1907_13088_gb300.build" in words:
            assert "--resources" in words and hasattr(build, "resources"), (name, cmd)
        if words[0] == "ncu" and "-i" not in words:
            assert "--clock-control" in words and words[words.index("--clock-control") + 1] == "none", (name, cmd)
    assert seen_bench >= 5


def test_resource_summary_matches_the_sources():
    """The ptxas table in profiles/ptxas_resources_sm103a.md is what its quoted
    command prints for the sources as committed (registers, spills, stack and
    shared memory of every listed kernel): a kernel change that moves them, or
    a template change that drops a kernel from the pattern, shows here."""
    import shlex
    from paper_1907_13088_gb300 import build

    cmd = [c for n, c in _commands() if n == "ptxas_resources_sm103a.md" and "--resources" in c]
    assert len(cmd) == 1, cmd
    args = shlex.split(cmd[0])
    pattern = args[args.index("--resources") + 1]
    with open(os.path.join(ROOT, "profiles", "ptxas_resources_sm103a.md")) as f:
        committed = [line for line in f.read().splitlines() if line.startswith("| `")]
    now = [line for line in build.resources(pattern).splitlines() if line.startswith("| `")]
    assert any("k_pol2d<0, 4, 3, true, 128, true>" in line for line in now)  # the 4096^2 TE kernel is listed
    assert now == committed
