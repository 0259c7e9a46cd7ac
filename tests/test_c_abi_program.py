"""The boundary is a C ABI: a C99 program compiled against include/fftb.h
with gcc and linked to libfftb.so calls the host-only entry points and the
error paths (no GPU needed) and gets the oracle's sphere sizes."""
import os
import shutil
import subprocess

import pytest

from oracle import sphere_gvectors

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "fftb.h"

int main(void) {
  const int32_t n[3] = {24, 24, 24};
  int64_t ngw = 0;
  if (fftb_sphere_enumerate(n, 6.0, NULL, NULL, 0, &ngw) != FFTB_OK) return 2;
  int32_t* g = (int32_t*)malloc((size_t)ngw * 3 * sizeof(int32_t));
  if (fftb_sphere_enumerate(n, 6.0, NULL, g, ngw, &ngw) != FFTB_OK) return 3;
  int32_t sticks = 0, slabs = 0;
  if (fftb_sphere_sticks(n, g, ngw, &sticks, &slabs) != FFTB_OK) return 4;
  const int32_t m[3] = {4, 6, 5};
  int32_t box[4 * 6 * 5 * 3];
  if (fftb_box_enumerate(m, box, 4 * 6 * 5) != FFTB_OK) return 5;
  /* an invalid description: the status and the message, no exception, *out NULL */
  fftb_desc d;
  memset(&d, 0, sizeof d);
  d.n[0] = d.n[1] = d.n[2] = 24;
  d.n_kpoints = 1;
  d.radius = 6.0;
  d.layout = 7;
  fftb_plan p = (fftb_plan)&d;
  const fftb_status st = fftb_plan_create(&p, &d, FFTB_ROUNDTRIP, FFTB_FP32);
  printf("%lld %d %d %d %d %d %s|%s|%s\n", (long long)ngw, sticks, slabs, box[0], box[1], box[2],
         fftb_error_string(st), p == NULL ? "null" : "set", fftb_version());
  free(g);
  return st == FFTB_ERR_INVALID_ARG ? 0 : 6;
}
"""


@pytest.fixture(scope="module")
def lib_dir():
    from paper_2406_05577_gb300 import build
    build.build()
    return os.path.join(ROOT, "paper_2406_05577_gb300")


def test_c_program_against_the_header(lib_dir, tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe), "-L", lib_dir, "-lfftb", f"-Wl,-rpath,{lib_dir}"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    fields = out.stdout.split()
    assert int(fields[0]) == len(sphere_gvectors((24, 24, 24), 6.0)) == 925
    assert int(fields[1]) == 113 and int(fields[2]) == 13
    assert [int(v) for v in fields[3:6]] == [-2, -3, -2]   # first box G: (gx, gy, gz) lowest
    status_msg, plan_ptr, version = out.stdout.strip().split(" ", 6)[6].split("|")
    assert "invalid" in status_msg and plan_ptr == "null" and version
