"""The boundary is a C ABI: include/fmx.h compiles as plain C11 without
warnings, and a C program links libfmx.so and drives its host-side entry
points (create, coefficients, time step, sizes, status strings) with no GPU."""
import math
import os
import shutil
import subprocess

import pytest

from paper_1907_13088_gb300 import build as fbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "fmx.h"

int main(void) {
    fmx_params p;
    memset(&p, 0, sizeof(p));
    p.dims = 2; p.n[0] = 64; p.n[1] = 48; p.n[2] = 1;
    p.d[0] = p.d[1] = p.d[2] = 1.0; p.c = 1.0; p.courant = 0.5;
    p.precision = FMX_F64; p.iter_mode = FMX_ITER_FIXED; p.m = 4;
    fmx_grid *g = NULL;
    int warn = 0;
    fmx_status s = fmx_create(&p, &g, &warn);
    if (s != FMX_OK) { printf("create failed %d %s\n", (int)s, fmx_last_error()); return 1; }
    double co[FMX_NCOEF];
    if (fmx_coefficients(g, co, FMX_NCOEF) != FMX_OK) return 2;
    printf("dt %.17g\nc6 %.17g\nfield_bytes %zu\nworkspace %zu\n", fmx_time_step(g), co[4],
           fmx_field_bytes(&p), fmx_workspace_bytes(&p));
    fmx_destroy(g);
    p.courant = 1.5;
    s = fmx_create(&p, &g, NULL);
    printf("cfl %d %s\n", (int)s, fmx_strerror(s));
    return g == NULL ? 0 : 3;
}
"""


def test_header_compiles_as_c_and_the_library_links(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lib = fbuild.build()
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib)
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-L", libdir, "-lfmx", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    out = dict(line.split(" ", 1) for line in r.stdout.strip().splitlines())
    assert math.isclose(float(out["dt"]), 0.5 / math.sqrt(2.0), rel_tol=1e-15)  # courant x dt_CFL, 1/sqrt(2) in 2D
    assert float(out["c6"]) == 1.0 / 6.0
    assert int(out["field_bytes"]) == 64 * 48 * 8
    assert int(out["workspace"]) >= int(out["field_bytes"])
    assert out["cfl"].startswith("2 ")  # FMX_ECFL
