"""A plain C99 program that uses only the C ABI (and the CUDA runtime for
device memory): the 2x zoom of a uint8 image keeps the input samples and
maps a constant image to itself (checked inside the program), and its output
equals the Python API's bit for bit."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

from paper_2312_00229_gb300 import api, build

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r"""
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <cuda_runtime_api.h>
#include "wdweno.h"

enum { C = 3, N = 37, M = 53 };

static int zoom(const uint8_t* host_in, uint8_t* host_out) {
  void *din = 0, *dout = 0;
  const size_t nin = (size_t)C * N * M, nout = (size_t)C * 4 * N * M;
  if (cudaMalloc(&din, nin) != cudaSuccess || cudaMalloc(&dout, nout) != cudaSuccess) return -100;
  cudaMemcpy(din, host_in, nin, cudaMemcpyHostToDevice);
  weno_image in = {din, N, M, C, (int64_t)N * M, M, 1};
  weno_image out = {dout, 2 * N, 2 * M, C, (int64_t)4 * N * M, 2 * M, 1};
  weno_params p = weno_params_default();
  int rc = weno_zoom2x_fwd(&in, WENO_U8, &out, WENO_U8, &p, 0);
  if (rc == WENO_OK && cudaDeviceSynchronize() != cudaSuccess) rc = -101;
  cudaMemcpy(host_out, dout, nout, cudaMemcpyDeviceToHost);
  cudaFree(din);
  cudaFree(dout);
  return rc;
}

int main(int argc, char** argv) {
  static uint8_t a[C * N * M], b[C * 4 * N * M];
  int c, i, j, rc;
  for (c = 0; c < C; ++c)
    for (i = 0; i < N; ++i)
      for (j = 0; j < M; ++j) a[(c * N + i) * M + j] = (uint8_t)((i * 7 + j * 13 + c * 31 + i * j) % 256);
  if ((rc = zoom(a, b)) != WENO_OK) { printf("zoom failed: %s\n", weno_status_string(rc)); return 1; }
  for (c = 0; c < C; ++c)  /* input samples kept at the even fine points */
    for (i = 0; i < N; ++i)
      for (j = 0; j < M; ++j)
        if (b[(c * 2 * N + 2 * i) * 2 * M + 2 * j] != a[(c * N + i) * M + j]) {
          printf("sample (%d, %d, %d) not kept\n", c, i, j);
          return 2;
        }
  if (argc > 1) {
    FILE* f = fopen(argv[1], "wb");
    if (!f || fwrite(b, 1, sizeof b, f) != sizeof b) return 3;
    fclose(f);
  }
  for (i = 0; i < C * N * M; ++i) a[i] = 77;  /* a constant image stays constant */
  if ((rc = zoom(a, b)) != WENO_OK) return 4;
  for (i = 0; i < C * 4 * N * M; ++i)
    if (b[i] != 77) { printf("constant image changed at %d\n", i); return 5; }
  printf("ok\n");
  return 0;
}
"""


def test_c_program_uses_the_abi(tmp_path):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not found")
    lib = build.build()
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    src = tmp_path / "zoom.c"
    exe = tmp_path / "zoom"
    src.write_text(SRC)
    libdir = os.path.dirname(lib)
    cmd = [cc, "-std=c99", "-O2", "-Wall", "-Werror", str(src), "-o", str(exe),
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
           "-L", libdir, "-lwdweno", "-L", os.path.join(cuda, "lib64"), "-lcudart",
           f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    raw = tmp_path / "out.bin"
    r = subprocess.run([str(exe), str(raw)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "ok" in r.stdout, (r.returncode, r.stdout, r.stderr)
    C, N, M = 3, 37, 53
    i, j = np.meshgrid(np.arange(N), np.arange(M), indexing="ij")
    a = np.stack([((i * 7 + j * 13 + c * 31 + i * j) % 256) for c in range(C)]).astype(np.uint8)
    want = api.zoom2x_fwd(torch.from_numpy(a).cuda()).cpu().numpy()
    got = np.fromfile(raw, dtype=np.uint8).reshape(C, 2 * N, 2 * M)
    assert np.array_equal(got, want)
