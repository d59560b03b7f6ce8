"""The C ABI header is plain C: a C99 translation unit that includes it and
calls every entry point (arguments type-checked, never run) compiles with
-std=c99 -pedantic -Werror, and the same source compiles as C++."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")

SRC = r"""
#include <stddef.h>
#include "wdweno.h"

int main(void) {
  weno_params p = weno_params_default();
  weno_image im = {0, 1, 1, 1, 1, 1, 1};
  unsigned int timeouts = 0;
  int rc = 0;
  size_t n = 0;
  if (p.beta < 0.f) {  /* never taken: the calls are only type-checked */
    rc += weno_zoom2x_fwd(&im, WENO_U8, &im, WENO_U8, &p, NULL);
    rc += weno_zoom2x_fwd_tiled(&im, WENO_F16, &im, WENO_F16, &p, 0, 0, NULL);
    rc += weno_zoom2x_bwd(&im, &im, &im, &p, NULL, 0, NULL);
    n += weno_zoom2x_bwd_workspace_bytes(&im);
    n += weno_zoom2x_batched_workspace_bytes(1);
    rc += weno_zoom2x_batched(1, &im, WENO_BF16, &im, WENO_F32, &p, NULL, 0, 0, 0, NULL);
    rc += weno_zoom2x_batched_noalloc(1, &im, WENO_U8, &im, WENO_U8, &p, 0, 0, NULL);
    rc += weno_zoom2x_cascade(&im, WENO_U8, &im, WENO_U8, 3, &p, NULL, 0, NULL);
    n += weno_zoom2x_cascade_workspace_bytes(&im, 3, &p);
    rc += weno_resample(&im, WENO_U8, &im, WENO_U8, &p, NULL);
    rc += weno_wait_timeouts(&timeouts, 0);
    rc += (int)(weno_status_string(rc)[0] == 0);
  }
  return rc + (int)n + (int)(p.data_bound != 0.f) + WENO_CASCADE_MAX_LEVELS * 0 +
         WENO_NOALLOC_MAX_IMAGES * 0;
}
"""


@pytest.mark.parametrize("compiler,args", [("gcc", ["-std=c99", "-pedantic", "-x", "c"]),
                                           ("g++", ["-std=c++11", "-x", "c++"])])
def test_header_compiles(tmp_path, compiler, args):
    cc = shutil.which(compiler)
    if cc is None:
        pytest.skip(f"{compiler} not found")
    src = tmp_path / "use_header.c"
    src.write_text(SRC)
    r = subprocess.run([cc, "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I", INCLUDE] +
                       args + [str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
