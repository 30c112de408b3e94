"""The boundary is a C ABI: include/lbm.h must compile as plain C99 and a C
program must link against liblbm.so and call it. Only calls that need no GPU
are made here (parameter validation, error paths)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "lbm.h"

int main(void) {
    lbm_params p;
    lbm_sp_params sp;
    lbm_ctx* ctx = 0;
    lbm_sp_ctx* sctx = 0;
    memset(&p, 0, sizeof p);
    p.nx = 0;                                        /* invalid: no CUDA call is made */
    if (lbm_validate_params(&p) != LBM_EINVAL) return 1;
    if (lbm_create(&p, 1, LBM_F64, 0, &ctx) != LBM_EINVAL || ctx != 0) return 2;
    memset(&sp, 0, sizeof sp);
    sp.nx = 2; sp.ny = 16; sp.nu = 0.1;              /* nx < 3 */
    if (lbm_sp_create(&sp, LBM_F64, 0, &sctx) != LBM_EINVAL || sctx != 0) return 3;
    if (lbm_step(0, 1) != LBM_EINVAL || lbm_sp_step(0, 1) != LBM_EINVAL) return 4;
    if (lbm_autotune_shape(0, 0, 0) != LBM_EINVAL) return 5;
    if (lbm_measure_fp64_fma(0, 0) != LBM_EINVAL) return 6;
    lbm_destroy(0);
    lbm_sp_destroy(0);
    printf("ok %d %d %d %d\n", (int)sizeof(lbm_params), (int)sizeof(lbm_sp_params),
           (int)sizeof(lbm_monitor), (int)sizeof(lbm_launch_shape));
    return 0;
}
"""


def test_header_compiles_as_c99_and_links(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1902_08933_gb300 import build
    lib = build.build()
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                        str(src), lib, "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), (r.returncode, r.stdout, r.stderr)
    # the Python binding's structures have the C layout
    from paper_1902_08933_gb300 import lbm
    import ctypes
    _, n_params, n_sp, n_mon, n_shape = r.stdout.split()
    assert ctypes.sizeof(lbm.lbm_params) == int(n_params)
    assert ctypes.sizeof(lbm.lbm_sp_params) == int(n_sp)
    assert ctypes.sizeof(lbm.lbm_monitor) == int(n_mon)
    assert ctypes.sizeof(lbm.lbm_launch_shape) == int(n_shape)
