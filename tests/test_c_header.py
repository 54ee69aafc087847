"""The C ABI from plain C: `include/mgard_gb.h` compiles as C99 with all
warnings as errors, a C program links against `libmgardgb.so`, and the
host-only entry points answer as documented (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

from paper_2010_05872_gb300 import build as build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_PROGRAM = r"""
#include <stdint.h>
#include <stdio.h>
#include <stddef.h>
#include "mgard_gb.h"

int main(void) {
  int64_t dims[3] = {65, 65, 65};
  int L = -1;
  if (mgard_num_levels(3, dims, &L) != MGARD_OK || L != 5) return 1;
  size_t ws = 0;
  if (mgard_workspace_size(3, dims, MGARD_F32, &ws) != MGARD_OK || ws == 0 || ws % 256) return 2;
  double tau[6];
  if (mgard_level_tolerances(3, dims, NULL, 0, 1e-3, tau) != MGARD_OK) return 3;
  double sum = 0.0;
  for (int l = 0; l <= L; ++l) sum += tau[l];
  if (!(sum < 1e-3)) return 4; /* sum of tau_l = tau / C_Linf, C_Linf > 1 */
  int64_t d4[4] = {9, 9, 9, 9};
  if (mgard_num_levels_4d(d4, &L) != MGARD_OK || L != 2) return 5;
  uint64_t counts[6] = {45, 13, 12, 16, 9, 5};
  uint8_t len[6];
  const uint8_t expect[6] = {1, 3, 3, 3, 4, 4};
  if (mgard_huffman_lengths(6, counts, len) != MGARD_OK) return 6;
  for (int i = 0; i < 6; ++i)
    if (len[i] != expect[i]) return 7;
  int64_t bad[3] = {2, 5, 5};
  if (mgard_num_levels(3, bad, &L) != MGARD_ERR_SHAPE) return 8;
  if (mgard_decompose(3, bad, NULL, MGARD_F32, 0, NULL, NULL, 0, NULL) != MGARD_ERR_SHAPE) return 9;
  printf("%s\n", mgard_error_string(MGARD_ERR_SHAPE));
  return 0;
}
"""


def test_header_is_c99_and_links(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lib = build_mod.build()
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
           "-L", libdir, "-lmgardgb", "-Wl,-rpath," + libdir]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True,
                         env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert run.returncode == 0, (run.returncode, run.stderr)
    assert run.stdout.startswith("invalid shape")
