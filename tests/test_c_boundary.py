"""The boundary from plain C: include/lpbatch.h compiles as strict C99, and a
C program links against the library and gets argument errors as codes before
any device work (CPU only; no GPU call is made)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "lpbatch.h"

int main(void) {
    lp_batch_opts o;
    lpb_default_opts(&o);
    if (o.precision != LP_PREC_FP64) return 1;
    if (strlen(lpb_strerror(LPB_EINVAL)) == 0) return 2;
    int32_t m[1] = {2}, n[1] = {2}, st[1], it[1];
    double A[4] = {1, 0, 0, 1}, b[2] = {1, 1}, c[2] = {1, 1}, obj[1], x[2];
    lpb_err e = lp_solve_host(0, m, n, NULL, A, 4, NULL, b, 2, NULL, c, 2, NULL, 0, st, it, obj, x, NULL);
    if (e != LPB_EINVAL) return 3;
    e = lp_solve_host(1, m, n, NULL, A, 3, NULL, b, 2, NULL, c, 2, NULL, 0, st, it, obj, x, NULL);
    if (e != LPB_EINVAL || strstr(lpb_last_error(), "offset out of range") == NULL) return 4;
    lp_batch *h = NULL;
    e = lp_batch_create(&h, 1, m, n, NULL, A, 4, NULL, b, 2, NULL, c, 2, 7, NULL, NULL);
    if (e != LPB_EINVAL || h != NULL) return 5;
    if (lp_batch_destroy(NULL) != LPB_OK) return 6;
    puts("c boundary ok");
    return 0;
}
"""


def test_header_is_strict_c99():
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no C compiler")
    r = subprocess.run([gcc, "-fsyntax-only", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-x", "c",
                        os.path.join(INCLUDE, "lpbatch.h")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_links_and_gets_error_codes(tmp_path):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no C compiler")
    from paper_1802_08557_gb300 import build
    lib = build.build()
    src = tmp_path / "use_lpbatch.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "use_lpbatch"
    libdir = os.path.dirname(lib)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", INCLUDE, str(src), "-o", str(exe),
                        "-L", libdir, "-l:" + os.path.basename(lib), "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "c boundary ok" in r.stdout, (r.returncode, r.stdout, r.stderr)
