// FP64 throughput probe: DFMA chains vs mma.sync.m8n8k4.f64 (the legacy FP64
// tensor path), the best of a few launch shapes per form, CUDA events.
// Prints one JSON line.
#include <cstdio>
#include <cuda_runtime.h>

__global__ void dfma_kernel(double *out, int iters, double b, double c) {
  double a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
    a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
  }
  const double s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == 1.2345) out[0] = s;  // keeps the chains live
}

__global__ void dmma_kernel(double *out, int iters, double av, double bv) {
  double d[4][2];
#pragma unroll
  for (int c = 0; c < 4; ++c) { d[c][0] = threadIdx.x + c; d[c][1] = 1.0 + c; }
  const double a = av + threadIdx.x, b = bv;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(d[c][0]), "+d"(d[c][1])
                   : "d"(a), "d"(b));
  double s = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += d[c][0] + d[c][1];
  if (s == 1.2345) out[0] = s;
}

template <typename K>
static double time_ms(K k, int grid, int block, int iters, double *out) {
  k<<<grid, block>>>(out, 16, 1.0000001, 1e-12);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0);
  k<<<grid, block>>>(out, iters, 1.0000001, 1e-12);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms;
}

int main() {
  int nsm = 0, clk = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  double *out;
  cudaMalloc(&out, 8);
  const int iters = 8192;
  double f_dfma = 0, f_dmma = 0;
  for (int per_sm : {1, 2, 4})
    for (int block : {128, 256, 512}) {
      const int grid = nsm * per_sm;
      const double threads = (double)grid * block;
      const double t1 = time_ms(dfma_kernel, grid, block, iters, out);
      f_dfma = fmax(f_dfma, threads * iters * 8 * 2 / (t1 * 1e-3) / 1e12);
      const double t2 = time_ms(dmma_kernel, grid, block, iters, out);
      // m8n8k4: 8 x 8 x 4 FMAs per warp instruction
      f_dmma = fmax(f_dmma, (threads / 32) * iters * 4 * (8 * 8 * 4 * 2) / (t2 * 1e-3) / 1e12);
    }
  const cudaError_t e = cudaDeviceSynchronize();
  printf("{\"sms\": %d, \"max_clock_mhz\": %.0f, \"dfma_tflops\": %.4f, \"dmma_m8n8k4_tflops\": %.4f, \"status\": \"%s\"}\n",
         nsm, clk / 1e3, f_dfma, f_dmma, cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
