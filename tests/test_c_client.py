"""The boundary from plain C (CPU): a C99 program that includes only
include/mbt.h compiles with warnings as errors, links against libmbt.so and
drives the host-side calls (version and status strings, context creation
with a resonator and the mesh, argument errors, the planning queries)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "mbt.h"

int main(void)
{
    if (mbt_version() != 100) return 10;
    if (strcmp(mbt_status_string(MBT_OK), "ok") != 0) return 11;
    mbt_ring ring;
    memset(&ring, 0, sizeof ring);
    ring.E0_eV = 2.4e9;
    ring.T0_s = 288.0 / 299792458.0;
    ring.h = 480;
    ring.V_rf_V = 2.1e6;
    ring.alpha_c = 6e-4;
    ring.U0_eV = 0.5e6;
    ring.sigma_delta = 9e-4;
    ring.tau_z_s = 4.5e-3;
    mbt_ctx *ctx = NULL;
    if (mbt_create(&ring, MBT_PREC_MIXED, 0, 7, &ctx) != MBT_OK || !ctx) return 12;
    if (mbt_add_resonator(ctx, 1e6, 1.5e9, 2e4, MBT_RANGE_BOTH) != MBT_OK) return 13;
    if (mbt_set_grid(ctx, 200, 5.0) != MBT_ERR_UNSUPPORTED) return 14;   /* mixed: 128 or 256 cells */
    if (mbt_last_error(ctx) == NULL || mbt_last_error(ctx)[0] == 0) return 15;
    if (mbt_set_grid(ctx, 256, 5.0) != MBT_OK) return 16;
    mbt_destroy(ctx);

    int64_t run_n[1] = {39000000};
    int32_t run_nb[1] = {390};
    int streams = -1;
    if (mbt_plan_streams(1, run_n, run_nb, 0, 152, &streams) != MBT_OK || streams != 1) return 17;
    int32_t run[3] = {0, 0, 0};
    int64_t n[3] = {10, 37, 5};
    int64_t ntiles = 0, out[4 * 16];
    if (mbt_plan_stream_split(3, run, n, 4, NULL, 0, &ntiles) != MBT_OK || ntiles < 3 || ntiles > 16) return 18;
    if (mbt_plan_stream_split(3, run, n, 4, out, 16, &ntiles) != MBT_OK) return 19;
    int64_t total = 0;
    for (int64_t k = 0; k < ntiles; ++k) total += out[4 * k + 2];
    if (total != 52) return 20;
    if (mbt_plan_stream_split(3, run, n, 0, out, 16, &ntiles) != MBT_ERR_ARG) return 21;
    printf("c client ok: %lld tiles\n", (long long)ntiles);
    return 0;
}
"""


def test_c_program_uses_the_boundary(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    import paper_1809_00391_gb300 as pkg
    pkg.build()
    lib = os.path.dirname(str(pkg._LIB_PATH))
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
           "-L", lib, "-lmbt", "-Wl,-rpath," + lib, "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, f"exit {r.returncode}: {r.stdout}{r.stderr}"
    assert r.stdout.startswith("c client ok")
