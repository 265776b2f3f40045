"""libstmg.so used from a C program (gcc -std=c99, linked against the library, no Python
in between): the header's defaults, the host-side set-up calls, the status strings, and
stmg_create returning an error status, not crashing, on a machine without a GPU (CPU only)."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2502_09159_gb300")

PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include "stmg.h"

int main(void) {
  stmg_config cfg;
  if (stmg_default_config(&cfg) != STMG_OK) return 1;
  if (cfg.omega != 0.7 || cfg.nu1 != 1 || cfg.nu2 != 1 || cfg.gmres_max_iter != 200 || cfg.rel_tol != 1e-8)
    return 2;
  int levels[3 * STMG_MAX_LEVELS], count = 0;
  if (stmg_host_default_hierarchy(64, 2, 2, 8, 2, levels, &count) != STMG_OK || count != 5) return 3;
  if (levels[3] != 64 || levels[4] != 1 || levels[5] != 2 || levels[12] != 8) return 4;
  double A[9] = {0, 2, 0, 1, 0, 0, 0, 0, 4};          /* needs a row interchange */
  if (stmg_host_invert(A, 3, 0) != STMG_OK) return 5;
  const double want[9] = {0, 1, 0, 0.5, 0, 0, 0, 0, 0.25};
  for (int i = 0; i < 9; ++i)
    if (fabs(A[i] - want[i]) > 1e-15) return 6;
  double S[4] = {1, 2, 2, 4};
  if (stmg_host_invert(S, 2, 0) != STMG_ERR_SINGULAR) return 7;
  if (stmg_host_invert(NULL, 2, 0) != STMG_ERR_ARG) return 8;
  cfg.dim = 2; cfg.n_cells = 4; cfg.r = 1; cfg.k = 1; cfg.n_slabs = 2;
  stmg_handle* h = (stmg_handle*)0x1;
  const int st = stmg_create(&cfg, &h);
  printf("create: %d %s\n", st, stmg_status_string(st));
  if (st == STMG_OK) { stmg_destroy(h); return 9; }   /* no GPU here: must fail */
  if (h != NULL) return 10;                           /* no handle on failure */
  cfg.dim = 4;
  if (stmg_create(&cfg, &h) != STMG_ERR_ARG) return 11;
  printf("ok\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def lib_built():
    import paper_2502_09159_gb300 as p
    p.build()
    return os.path.join(PKG, "libstmg.so")


def test_c_program_links_and_runs(lib_built, tmp_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present: stmg_create would succeed")
    src, exe = tmp_path / "client.c", tmp_path / "client"
    src.write_text(PROGRAM)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", PKG, "-l:libstmg.so", f"-Wl,-rpath,{PKG}", "-lm"], check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    assert out.stdout.strip().endswith("ok")
