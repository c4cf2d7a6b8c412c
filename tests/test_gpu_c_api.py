"""The C ABI from a plain C program: no Python binding, no PyTorch allocator.

A small C caller includes include/dsdna.h, links libdsdna.so, creates a
context with the default allocator (cudaMalloc) on the default stream, loads
and steps two tethered molecules, reads energies, observables and the state,
and checks the error path.  The same system stepped through the binding must
give the same state bit for bit (the library owns every computation).
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1608_03722_gb300 import _build
from paper_1608_03722_gb300 import dsdna as D

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SRC = r"""
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include "dsdna.h"

int main(void) {
  dsdna_params p;
  dsdna_default_params(&p);
  p.seed = 11;
  int n_bp[2] = {300, 120};
  int tether[2] = {1, 1};
  dsdna_system s = {0};
  s.n_mol = 2; s.n_bp = n_bp; s.tether = tether;
  dsdna_ctx* ctx = NULL;
  int rc = dsdna_create(&p, &s, NULL, NULL, &ctx);
  if (rc != DSDNA_OK) { printf("create %d %s\n", rc, dsdna_last_error(NULL)); return 1; }
  double f[3] = {0, 0, 2.0}, t[3] = {0, 0, 1.0};
  if (dsdna_set_external_force_torque(ctx, 0, f, t) != DSDNA_OK) return 2;
  if (dsdna_step(ctx, 500) != DSDNA_OK) { printf("step %s\n", dsdna_last_error(ctx)); return 3; }
  double E[DSDNA_NTERMS], W[6];
  if (dsdna_energy_virial(ctx, -1, E, W) != DSDNA_OK) return 4;
  dsdna_obs o;
  if (dsdna_observables(ctx, 0, DSDNA_OBS_EXT | DSDNA_OBS_TW | DSDNA_OBS_LK, &o) != DSDNA_OK) return 5;
  const int n = 2 * (300 + 120);
  double* X = malloc(sizeof(double) * 3 * n);
  if (dsdna_get_state(ctx, -1, X, NULL, NULL, NULL) != DSDNA_OK) return 6;
  double e = 0.0;
  for (int k = 0; k < DSDNA_NTERMS; ++k) e += E[k];
  printf("E %.17g rz %.17g tw %.17g lk %.17g steps %lld\n", e, o.rz, o.tw, o.lk, (long long)dsdna_step_counter(ctx));
  FILE* out = fopen(getenv("DSDNA_C_OUT"), "wb");
  fwrite(X, sizeof(double), 3 * n, out);
  fclose(out);
  /* the error path: a molecule index out of range is refused with a message */
  if (dsdna_observables(ctx, 7, DSDNA_OBS_EXT, &o) != DSDNA_EINVAL) return 7;
  printf("error: %s\n", dsdna_last_error(ctx));
  dsdna_destroy(ctx);
  free(X);
  return isfinite(e) ? 0 : 8;
}
"""


def test_c_caller_steps_with_the_default_allocator():
    D.load()                                    # builds libdsdna.so if needed
    libdir = os.path.dirname(_build.LIB)
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "caller.c")
        exe = os.path.join(d, "caller")
        with open(src, "w") as f:
            f.write(C_SRC)
        subprocess.check_call(["gcc", "-std=c11", "-O1", "-I", os.path.join(ROOT, "include"), src, "-o", exe,
                               "-L", libdir, "-ldsdna", "-lm", "-Wl,-rpath," + libdir])
        out_path = os.path.join(d, "X.bin")
        r = subprocess.run([exe], capture_output=True, text=True, env=dict(os.environ, DSDNA_C_OUT=out_path),
                           timeout=300)
        assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
        assert "steps 500" in r.stdout and "error: " in r.stdout
        Xc = np.fromfile(out_path, dtype=np.float64).reshape(-1, 3)
    # the same system through the binding (PyTorch allocator): the same state
    p = D.dsdna_default_params(seed=11)
    ctx = D.Context(p, [300, 120], tether=[1, 1])
    ctx.set_external_force_torque(0, [0, 0, 2.0], [0, 0, 1.0])
    ctx.step(500)
    Xp, _, _, _ = ctx.get_state()
    ctx.close()
    assert np.array_equal(Xc, Xp)
