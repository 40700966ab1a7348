"""The boundary from C: a C99 program that includes include/lbm.h compiles
with warnings as errors, links against liblbm.so and calls the entry points
that need no GPU (lbm_plan, lbm_jet_fit, lbm_create_error)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIBDIR = os.path.join(ROOT, "paper_1206_0389_gb300")

PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include <string.h>
#include "lbm.h"

int main(void) {
  lbm_grid g;
  memset(&g, 0, sizeof g);
  g.nbx = 4; g.nby = 3; g.nbz = 3; g.periodic_x = 0; g.levels = 1; g.refine = NULL;
  g.walls = 15; g.slip = 8; g.outlet = 1;
  g.nozzle_y0 = 12.0; g.nozzle_z0 = 12.0; g.nozzle_r = 0.0;
  lbm_plan_info info;
  memset(&info, 0, sizeof info);
  if (lbm_plan(&g, LBM_D3Q27_FCLB, LBM_F32, &info) != LBM_OK) return 1;
  if (info.levels != 1 || info.active_cells[0] != 32 * 24 * 24 || info.nozzle_level != -1) return 2;
  g.walls = 1;                                   /* an unpaired wall is rejected */
  if (lbm_plan(&g, LBM_D3Q27_FCLB, LBM_F32, &info) != LBM_ERR_ARG) return 3;
  double mean[4] = {1.0, 0.8, 0.3, 0.1}, var[4] = {0.01, 0.0, 0.0, 0.0}, out[5];
  int64_t counts[4] = {3, 8, 12, 16};
  if (lbm_jet_fit(4, 1.0, mean, var, counts, out) != LBM_OK) return 4;
  if (!(out[0] == 1.0 && fabs(out[2] - 0.1) < 1e-15 && out[1] > 1.0 && out[1] < 2.5)) return 5;
  if (lbm_jet_fit(0, 1.0, mean, var, counts, out) != LBM_ERR_ARG) return 6;
  printf("ok %s\n", lbm_create_error());
  return 0;
}
"""


def test_c_program_uses_the_header_and_library(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    if not os.path.exists(os.path.join(LIBDIR, "liblbm.so")):
        pytest.skip("liblbm.so not built")
    src = tmp_path / "use_lbm.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "use_lbm"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", LIBDIR, "-llbm", "-Wl,-rpath," + LIBDIR, "-lm"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.startswith("ok")
