"""A C99 program drives the transform through the C ABI alone: compiled with
gcc against include/fftb.h and linked to libfftb.so, it creates FP64 plans
on a 24^3 grid (|G| <= 6, 3 bands), runs G -> r and r -> G with host buffers
(fftb_execute_host), reads the plan's sphere back, and writes everything to
files; the test compares them with the FP64 oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import fftb_inputs as fi
import oracle

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "fftb.h"

static int fail(const char* what, fftb_status st) {
  fprintf(stderr, "%s: %s (%s)\n", what, fftb_error_string(st), fftb_last_error());
  return 10 + (int)st;
}

static int read_all(const char* path, void* buf, size_t bytes) {
  FILE* f = fopen(path, "rb");
  if (!f) return 0;
  const size_t got = fread(buf, 1, bytes, f);
  fclose(f);
  return got == bytes;
}

static int write_all(const char* path, const void* buf, size_t bytes) {
  FILE* f = fopen(path, "wb");
  if (!f) return 0;
  const size_t put = fwrite(buf, 1, bytes, f);
  fclose(f);
  return put == bytes;
}

int main(int argc, char** argv) {
  if (argc != 2) return 2;
  char path[4096];
  const int32_t bands = 3;
  fftb_desc d;
  memset(&d, 0, sizeof d);
  d.n[0] = d.n[1] = d.n[2] = 24;
  d.n_kpoints = 1;
  d.bands = &bands;
  d.radius = 6.0;
  fftb_plan g2r = NULL, r2g = NULL;
  fftb_status st = fftb_plan_create(&g2r, &d, FFTB_G_TO_R, FFTB_FP64);
  if (st != FFTB_OK) return fail("create g2r", st);
  st = fftb_plan_create(&r2g, &d, FFTB_R_TO_G, FFTB_FP64);
  if (st != FFTB_OK) return fail("create r2g", st);
  int64_t ngw = 0;
  if ((st = fftb_plan_ngw(g2r, 0, &ngw)) != FFTB_OK) return fail("ngw", st);
  const size_t vol = 24 * 24 * 24;
  const size_t sph_b = (size_t)bands * (size_t)ngw * 16, cube_b = (size_t)bands * vol * 16;
  int32_t* g = (int32_t*)malloc((size_t)ngw * 3 * sizeof(int32_t));
  double* c = (double*)malloc(sph_b);
  double* cube = (double*)malloc(cube_b);
  double* rin = (double*)malloc(cube_b);
  double* sph = (double*)malloc(sph_b);
  if (!g || !c || !cube || !rin || !sph) return 3;
  if ((st = fftb_plan_sphere(g2r, 0, g)) != FFTB_OK) return fail("sphere", st);
  snprintf(path, sizeof path, "%s/c.bin", argv[1]);
  if (!read_all(path, c, sph_b)) return 4;
  snprintf(path, sizeof path, "%s/rin.bin", argv[1]);
  if (!read_all(path, rin, cube_b)) return 5;
  /* host buffers, legacy default stream; the call synchronises */
  if ((st = fftb_execute_host(g2r, c, cube, NULL, NULL)) != FFTB_OK) return fail("g2r", st);
  if ((st = fftb_execute_host(r2g, rin, sph, NULL, NULL)) != FFTB_OK) return fail("r2g", st);
  if ((st = fftb_plan_check(g2r)) != FFTB_OK) return fail("check", st);
  snprintf(path, sizeof path, "%s/g.bin", argv[1]);
  if (!write_all(path, g, (size_t)ngw * 3 * sizeof(int32_t))) return 6;
  snprintf(path, sizeof path, "%s/cube.bin", argv[1]);
  if (!write_all(path, cube, cube_b)) return 7;
  snprintf(path, sizeof path, "%s/sph.bin", argv[1]);
  if (!write_all(path, sph, sph_b)) return 8;
  printf("%lld\n", (long long)ngw);
  fftb_destroy(g2r);
  fftb_destroy(r2g);
  free(g); free(c); free(cube); free(rin); free(sph);
  return 0;
}
"""


def test_c_program_runs_the_transform(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    from paper_2406_05577_gb300 import build
    build.build()
    lib_dir = os.path.join(ROOT, "paper_2406_05577_gb300")
    n, bands = (24, 24, 24), 3
    g = oracle.sphere_gvectors(n, 6.0)
    c = fi.complex_gaussian((bands, len(g)), 801)
    rin = fi.complex_gaussian((bands, 24, 24, 24), 802)
    c.astype(np.complex128).tofile(tmp_path / "c.bin")
    rin.astype(np.complex128).tofile(tmp_path / "rin.bin")
    src = tmp_path / "run.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "run"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe), "-L", lib_dir, "-lfftb", f"-Wl,-rpath,{lib_dir}"], check=True)
    out = subprocess.run([str(exe), str(tmp_path)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    assert int(out.stdout.split()[0]) == len(g) == 925
    gp = np.fromfile(tmp_path / "g.bin", dtype=np.int32).reshape(-1, 3)
    assert np.array_equal(gp, g)  # the plan's canonical order is the oracle's
    cube = np.fromfile(tmp_path / "cube.bin", dtype=np.complex128).reshape(bands, 24, 24, 24)
    want = oracle.g2r(g, c, n)
    assert np.linalg.norm(cube - want) <= 1e-12 * np.linalg.norm(want)
    sph = np.fromfile(tmp_path / "sph.bin", dtype=np.complex128).reshape(bands, -1)
    want = oracle.r2g(g, rin, n)
    assert np.linalg.norm(sph - want) <= 1e-12 * np.linalg.norm(want)
