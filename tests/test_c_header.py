"""The C ABI seen from C: include/sapmg.h compiles on its own as C99 with
warnings as errors, and a C program linked against libsapmg.so calls a
host-only entry point (no GPU needed)."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include "sapmg.h"
#include <stdio.h>

int main(void) {
  mg_params p;
  if (mg_default_params(&p) != MG_OK) return 1;
  if (mg_sizeof_params() != sizeof(mg_params)) return 2;
  if (p.n_mr != 4 || p.fgmres_m != 20 || p.setup2_iters != 0) return 3;
  if (mg_cgn_solve(NULL, NULL, NULL, 1, MG_FP64, 1e-10, 10, NULL) != MG_ERR_ARG) return 4;
  printf("ok\n");
  return 0;
}
"""


def test_header_is_self_contained_c(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib_dir = os.path.join(ROOT, "paper_1202_2462_gb300")
    if not os.path.exists(os.path.join(lib_dir, "libsapmg.so")):
        pytest.skip("libsapmg.so not built")
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           str(src), "-L", lib_dir, "-lsapmg", "-Wl,-rpath," + lib_dir, "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
