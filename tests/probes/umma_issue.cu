// tcgen05.mma issue probe (M 128, N 128, K 16, BF16 -> FP32 in tensor
// memory, operands resident in shared memory): cycles per MMA when
//   plain   - one thread issues groups of 4 MMAs back to back;
//   poll    - the same thread also commits each group to a ring of mbarriers
//             and polls (bounded) the barrier of 4 groups earlier, long
//             complete, before the next group;
//   handoff - a second warp does that polling and hands each group to the
//             issuing warp at a named barrier.
// Prints one JSON line.  Every wait is bounded; the kernel frees its tensor
// memory on every path.
#include <cstdio>
#include <cuda.h>
#include <cuda_runtime.h>

#include "ftgemm_common.cuh"
#include "ftgemm_tc.cuh"

using namespace ftg;

constexpr int GROUPS = 5000, PER = 4;

template <int MODE>
__global__ void __launch_bounds__(128, 1) issue_kernel(unsigned long long *cycles, int *err) {
  extern __shared__ unsigned char raw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tslot;
  __shared__ __align__(8) uint64_t ring[8];
  __shared__ __align__(8) uint64_t done;
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < 2 * 128 * 128 / 4; i += 128) ((uint32_t *)sm)[i] = 0x3f803f80u;  // bf16 1.0
  if (threadIdx.x == 0) {
    for (int q = 0; q < 8; ++q) mbar_init(smem_u32(&ring[q]), 1);
    mbar_init(smem_u32(&done), 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(&tslot), 128);
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot, a0 = smem_u32(sm), b0 = a0 + 128 * 128;
  const uint32_t idesc = tc_idesc_bf16_f32(128, 128);
  const unsigned long long lim = 1000000000ull;
  if (MODE == 2 && warp == 2) {  // waiter
    for (int g = 0; g < GROUPS; ++g) {
      if (g >= 4 && threadIdx.x == 64) mbar_wait_bounded(smem_u32(&ring[(g - 4) & 7]), ((g - 4) >> 3) & 1, lim, err);
      __syncwarp();
      asm volatile("bar.sync 2, 64;" ::: "memory");
    }
  }
  if (warp == 1) {
    const unsigned long long t0 = clock64();
    for (int g = 0; g < GROUPS; ++g) {
      if (MODE == 1 && g >= 4 && threadIdx.x == 32)
        mbar_wait_bounded(smem_u32(&ring[(g - 4) & 7]), ((g - 4) >> 3) & 1, lim, err);
      if (MODE == 2) asm volatile("bar.sync 2, 64;" ::: "memory");
      if (elect_one()) {
#pragma unroll
        for (int kk = 0; kk < PER; ++kk)
          tc_mma_bf16(tbase, tc_desc_k128(a0 + 32 * kk), tc_desc_k128(b0 + 32 * kk), idesc, (g | kk) ? 1u : 0u);
        if (MODE != 0) tc_commit(smem_u32(&ring[g & 7]));
      }
      __syncwarp();
    }
    if (elect_one()) tc_commit(smem_u32(&done));
    __syncwarp();
    if (threadIdx.x == 32) {
      mbar_wait_bounded(smem_u32(&done), 0, lim, err);
      cycles[blockIdx.x] = clock64() - t0;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, 128);
  }
}

template <int MODE>
static double run(int nsm, unsigned long long *cyc, int *err, double *tflops) {
  const int smem = 2 * 128 * 128 + 1024;
  cudaFuncSetAttribute(issue_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  issue_kernel<MODE><<<nsm, 128, smem>>>(cyc, err);  // warm-up
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0);
  issue_kernel<MODE><<<nsm, 128, smem>>>(cyc, err);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  unsigned long long h = 0;
  cudaMemcpy(&h, cyc, 8, cudaMemcpyDeviceToHost);
  *tflops = 2.0 * 128 * 128 * 16 * (double)GROUPS * PER * nsm / (ms * 1e-3) / 1e12;
  return (double)h / (GROUPS * PER);
}

int main() {
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  unsigned long long *cyc;
  int *err;
  cudaMalloc(&cyc, 8 * nsm);
  cudaMalloc(&err, 4);
  cudaMemset(err, 0, 4);
  double t0, t1, t2;
  const double c0 = run<0>(nsm, cyc, err, &t0);
  const double c1 = run<1>(nsm, cyc, err, &t1);
  const double c2 = run<2>(nsm, cyc, err, &t2);
  int herr = 0;
  cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaDeviceSynchronize();
  printf("{\"cycles_per_mma\": {\"plain\": %.1f, \"poll\": %.1f, \"handoff\": %.1f}, "
         "\"tflops\": {\"plain\": %.1f, \"poll\": %.1f, \"handoff\": %.1f}, \"wait_error\": %d, \"status\": \"%s\"}\n",
         c0, c1, c2, t0, t1, t2, herr, cudaGetErrorString(e));
  return (e == cudaSuccess && herr == 0) ? 0 : 1;
}
