"""FMA throughput probe: the FP64 (and FP32) rate that the "alu" rooflines of bench.py divide by.

``python -m paper_2109_08547_gb300.fp64_peak`` compiles a small kernel for sm_103a with nvcc,
runs it on device 0 and prints {"fp64_fma_tflops": ..., "fp32_fma_tflops": ...}.  Each thread
runs 8 independent FMA chains with no memory traffic in the loop; the grid is 8 blocks of 256
threads per SM; the best of 5 CUDA-event timings counts.  The figures measured on this GPU
type are recorded beside the constant in bench.py.
"""
import json
import os
import subprocess
import tempfile

_SRC = r"""
#include <cstdio>
#include <cuda_runtime.h>
template <typename T> __global__ void chains(T *out, int iters, T a, T b) {
  T x[8];
  for (int j = 0; j < 8; ++j) x[j] = T(threadIdx.x) * T(1e-3) + T(j);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = x[j] * a + b;
  T s = 0;
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == T(12345.678)) out[0] = s;   // keeps the chains alive
}
template <typename T> double tflops(int iters) {
  T *d = nullptr;
  cudaMalloc(&d, sizeof(T));
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int grid = sms * 8, block = 256;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  chains<T><<<grid, block>>>(d, iters, T(0.999999), T(1e-7));
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    chains<T><<<grid, block>>>(d, iters, T(0.999999), T(1e-7));
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = ms < best ? ms : best;
  }
  cudaFree(d);
  return 2.0 * 8 * iters * double(grid) * block / (best * 1e-3) / 1e12;
}
int main() {
  printf("fp64_fma_tflops %.4f\nfp32_fma_tflops %.4f\n", tflops<double>(4096), tflops<float>(16384));
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
"""


def measure() -> dict:
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "fma.cu"), os.path.join(d, "fma")
        with open(src, "w") as f:
            f.write(_SRC)
        subprocess.run(["nvcc", "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe, src], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}


if __name__ == "__main__":
    print(json.dumps(measure()))
