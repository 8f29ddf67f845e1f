"""The FP64 reciprocal square root and quotient of the push's Boris step (csrc/fastmath.cuh:
Newton-Raphson refinement of an FP32 estimate, with a residual step for the quotient) against the
GPU's IEEE FP64 results, 1 / sqrt(x) and a / b, on the argument ranges the step produces: 1 + u^2
and 1 + t^2 for momenta up to 1e6, gamma + 1, and numerators of either sign. A small kernel that
includes the header is built here with nvcc and run through ctypes."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_1401_0838_gb300 import build as B

pytestmark = pytest.mark.gpu

SRC = r"""
#include <cuda_runtime.h>
#include "fastmath.cuh"

__global__ void k_fastmath(const double* x, const double* a, const double* b, double* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[4 * i + 0] = picgb::fast_rsqrt(x[i]);
  out[4 * i + 1] = 1.0 / sqrt(x[i]);
  out[4 * i + 2] = picgb::fast_div(a[i], b[i]);
  out[4 * i + 3] = a[i] / b[i];
}

extern "C" int run_fastmath(const double* x, const double* a, const double* b, double* out, int n) {
  double *dx = nullptr, *da = nullptr, *db = nullptr, *dout = nullptr;
  const size_t bytes = sizeof(double) * (size_t)n;
  int rc = 0;
  if (cudaMalloc(&dx, bytes) || cudaMalloc(&da, bytes) || cudaMalloc(&db, bytes) || cudaMalloc(&dout, 4 * bytes))
    rc = 1;
  if (!rc && (cudaMemcpy(dx, x, bytes, cudaMemcpyHostToDevice) || cudaMemcpy(da, a, bytes, cudaMemcpyHostToDevice) ||
              cudaMemcpy(db, b, bytes, cudaMemcpyHostToDevice)))
    rc = 2;
  if (!rc) {
    k_fastmath<<<(n + 255) / 256, 256>>>(dx, da, db, dout, n);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) rc = 3;
  }
  if (!rc && cudaMemcpy(out, dout, 4 * bytes, cudaMemcpyDeviceToHost)) rc = 4;
  cudaFree(dx);
  cudaFree(da);
  cudaFree(db);
  cudaFree(dout);
  return rc;
}
"""


@pytest.fixture(scope="module")
def fastmath_lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("fastmath")
    src = d / "fastmath_test.cu"
    src.write_text(SRC)
    so = d / "libfastmath_test.so"
    cmd = [B.nvcc(), "-shared", "-Xcompiler", "-fPIC", "-O3", "-std=c++17", *B.ARCH, "-I", B.CSRC, "-o", str(so),
           str(src), "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(str(so))
    P = ctypes.POINTER(ctypes.c_double)
    lib.run_fastmath.argtypes = [P, P, P, P, ctypes.c_int]
    lib.run_fastmath.restype = ctypes.c_int
    return lib


def _run(lib, x, a, b):
    n = len(x)
    out = np.empty(4 * n)
    P = ctypes.POINTER(ctypes.c_double)
    args = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, a, b)]
    rc = lib.run_fastmath(*(v.ctypes.data_as(P) for v in args), out.ctypes.data_as(P), n)
    assert rc == 0
    return out.reshape(n, 4)


def test_fp64_rsqrt_and_quotient_within_three_ulp(fastmath_lib):
    rng = np.random.default_rng(7)
    n = 1 << 20
    u = 10.0 ** rng.uniform(-8, 6, n)                    # momenta (grid units) from thermal to extreme
    x = 1.0 + u * u                                      # 1 + u^2 of the Boris step
    x[:4] = [1.0, 1.0 + 2.0 ** -52, 16901.0, 1e12]       # the edges and gamma = 130
    b = np.where(rng.random(n) < 0.5, 1.0 + 10.0 ** rng.uniform(-8, 4, n), 2.0 + u)  # 1 + t^2 or gamma + 1
    a = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-12, 12, n)
    a[:2] = [2.0, 0.0]
    r = _run(fastmath_lib, x, a, b)
    ulp_rs = np.abs(r[:, 0] - r[:, 1]) / np.spacing(np.abs(r[:, 1]))
    ulp_q = np.abs(r[:, 2] - r[:, 3]) / np.where(r[:, 3] == 0, 1.0, np.spacing(np.abs(r[:, 3])))
    assert np.isfinite(r).all()
    assert ulp_rs.max() <= 3.0, ulp_rs.max()
    assert ulp_q.max() <= 3.0, ulp_q.max()
    assert r[1, 2] == 0.0  # 0 / b stays an exact zero
