"""Builds the in-tree CUDA library ``_build/libfmx.so`` for sm_103a.

Every translation unit under ``csrc/`` is compiled by nvcc in parallel and
linked into one shared library with the C ABI of ``include/fmx.h``.  Host
code is compiled without floating-point contraction so that the scheme's
coefficients are the binary64 values of the expressions documented in
``fmx.h`` on any host architecture.
"""
from __future__ import annotations

import concurrent.futures
import os
import re
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfmx.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the fmx CUDA library cannot be built")


def sources():
    out = []
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cpp")):
            out.append(os.path.join(CSRC, name))
    return out


def _deps():
    return [os.path.join(CSRC, n) for n in os.listdir(CSRC)] + [os.path.join(INCLUDE, n) for n in os.listdir(INCLUDE)]


def _up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _flags(nvcc: str, src: str, obj: str, extra=()) -> list:
    return [nvcc, "-std=c++17", ARCH, "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
            *extra, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]


def _compile(src: str, nvcc: str) -> str:
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    r = subprocess.run(_flags(nvcc, src, obj), capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link the library if any source changed; returns its path."""
    if not force and _up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    srcs = sources()
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, nvcc), srcs))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, ARCH, "-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}", file=sys.stderr)
    return LIB


def _demangle(names):
    tool = shutil.which("c++filt")
    if not tool or not names:
        return list(names)
    r = subprocess.run([tool], input="\n".join(names), capture_output=True, text=True)
    out = r.stdout.splitlines()
    return out if r.returncode == 0 and len(out) == len(names) else list(names)


def _short(name: str) -> str:
    """Kernel name with its template arguments, without return type, namespaces
    or parameter list."""
    name = re.sub(r"^void ", "", name).replace("(anonymous namespace)::", "")
    depth, cut = 0, len(name)
    for i, ch in enumerate(name):  # drop the parameter list: the first '(' outside <...>
        if ch == "<":
            depth += 1
        elif ch == ">":
            depth -= 1
        elif ch == "(" and depth == 0:
            cut = i
            break
    name = name[:cut]
    base, _, targs = name.partition("<")
    base = base.split("::")[-1]
    targs = re.sub(r"\([A-Za-z0-9_:]+\)", "", targs)  # enum casts such as (fmx::pol2d::Pol)0
    return base + ("<" + targs if targs else "")


def resources(pattern: str = "") -> str:
    """Per-kernel resources that ptxas reports with -Xptxas -v (registers,
    spill stores and loads, stack frame, static shared memory) for every
    kernel of the library whose short name matches ``pattern``, as a
    markdown table.  Only the compiler's summary lines are read."""
    nvcc = _nvcc()
    srcs = [s for s in sources() if s.endswith(".cu")]
    with tempfile.TemporaryDirectory() as tmp:
        def one(src):
            obj = os.path.join(tmp, os.path.basename(src) + ".o")
            r = subprocess.run(_flags(nvcc, src, obj, ("-Xptxas", "-v")), capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
            return os.path.basename(src), r.stderr

        with concurrent.futures.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
            logs = list(ex.map(one, srcs))
    rows = []
    for tu, log in logs:
        cur = None
        for line in log.splitlines():
            m = re.search(r"Compiling entry function '([^']+)'", line)
            if m:
                cur = {"tu": tu, "name": m.group(1), "stack": 0, "spill_st": 0, "spill_ld": 0, "smem": 0}
                continue
            if cur is None:
                continue
            m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", line)
            if m:
                cur["stack"], cur["spill_st"], cur["spill_ld"] = (int(v) for v in m.groups())
                continue
            m = re.search(r"Used (\d+) registers", line)
            if m:
                cur["regs"] = int(m.group(1))
                sm = re.search(r"(\d+) bytes smem", line)
                cur["smem"] = int(sm.group(1)) if sm else 0
                rows.append(cur)
                cur = None
    for r, d in zip(rows, _demangle([r["name"] for r in rows])):
        r["short"] = _short(d)
    keep = [r for r in rows if re.search(pattern, r["short"])]
    keep.sort(key=lambda r: (r["tu"], r["short"]))
    out = ["| file | kernel | registers | spill stores / loads (B) | stack (B) | static smem (B) |",
           "|---|---|---|---|---|---|"]
    for r in keep:
        out.append(f"| `{r['tu']}` | `{r['short']}` | {r['regs']} | {r['spill_st']} / {r['spill_ld']} | "
                   f"{r['stack']} | {r['smem']} |")
    return "\n".join(out)


if __name__ == "__main__":
    if "--resources" in sys.argv:
        i = sys.argv.index("--resources")
        print(resources(sys.argv[i + 1] if len(sys.argv) > i + 1 else ""))
    else:
        print(build(force="--force" in sys.argv, verbose=True))
