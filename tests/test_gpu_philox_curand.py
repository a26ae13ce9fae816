"""Cross-check of the oracle's Philox4x32-10 against CUDA's own public
implementation (curand_Philox4x32_10 from curand_philox4x32_x.h), called from
a tiny kernel on the GPU on 4,096 seeded (counter, key) pairs. The oracle is
also pinned to the published Random123 known-answer vectors on the CPU; this
extends the pin to many more inputs with an independent implementation."""
import os
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SRC = r"""
#include <cstdio>
#include <cstdlib>
#include <curand_philox4x32_x.h>
__global__ void run(const uint4 *c, const uint2 *k, uint4 *out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = curand_Philox4x32_10(c[i], k[i]);
}
int main(int argc, char **argv) {
  const int n = atoi(argv[1]);
  uint4 *hc = (uint4 *)malloc(n * sizeof(uint4)); uint2 *hk = (uint2 *)malloc(n * sizeof(uint2));
  uint4 *ho = (uint4 *)malloc(n * sizeof(uint4));
  FILE *f = fopen(argv[2], "rb");
  if (!f || fread(hc, sizeof(uint4), n, f) != (size_t)n || fread(hk, sizeof(uint2), n, f) != (size_t)n) return 2;
  fclose(f);
  uint4 *dc, *dout; uint2 *dk;
  if (cudaMalloc(&dc, n * sizeof(uint4)) || cudaMalloc(&dk, n * sizeof(uint2)) || cudaMalloc(&dout, n * sizeof(uint4))) return 3;
  cudaMemcpy(dc, hc, n * sizeof(uint4), cudaMemcpyHostToDevice);
  cudaMemcpy(dk, hk, n * sizeof(uint2), cudaMemcpyHostToDevice);
  run<<<(n + 127) / 128, 128>>>(dc, dk, dout, n);
  if (cudaMemcpy(ho, dout, n * sizeof(uint4), cudaMemcpyDeviceToHost) != cudaSuccess) return 4;
  f = fopen(argv[3], "wb");
  fwrite(ho, sizeof(uint4), n, f);
  fclose(f);
  return 0;
}
"""


def test_oracle_philox_matches_curand(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
    src = tmp_path / "philox_curand.cu"
    src.write_text(SRC)
    exe = tmp_path / "philox_curand"
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", str(src), "-o", str(exe)])
    n = 4096
    rng = np.random.default_rng(2510)
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:16] = 0                                   # structured corners: zero and all-ones words
    ctr[16:32] = 0xFFFFFFFF
    key[:8] = 0
    key[24:32] = 0xFFFFFFFF
    inp = tmp_path / "in.bin"
    inp.write_bytes(ctr.astype("<u4").tobytes() + key.astype("<u4").tobytes())
    out = tmp_path / "out.bin"
    subprocess.check_call([str(exe), str(n), str(inp), str(out)])
    got = np.frombuffer(out.read_bytes(), dtype="<u4").reshape(n, 4)
    for i in range(n):
        want = oracle.philox4x32_10([int(v) for v in ctr[i]], [int(v) for v in key[i]])
        assert tuple(int(v) for v in got[i]) == want, i
