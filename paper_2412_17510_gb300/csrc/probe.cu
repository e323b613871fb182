// probe.cu -- binary64 pipe throughput probe (roofline denominator).
//
// The multiple-precision kernels are bound by the binary64 instruction rate,
// which GB300 does not publish per instruction kind.  This probe measures it
// at the clocks of the moment: every thread runs 8 independent dependency
// chains of one instruction kind (DFMA, DADD or DMUL) over a grid of 8 CTAs
// of 256 threads per SM, timed with CUDA events.
#include <algorithm>

#include "internal.h"

namespace {

constexpr int kChains = 8;

template <int OP>
__global__ void fp64_chain_kernel(double* out, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; i++) a[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < kChains; i++) {
      if (OP == 0) a[i] = __fma_rn(a[i], b, c);
      else if (OP == 1) a[i] = __dadd_rn(a[i], c);
      else a[i] = __dmul_rn(a[i], b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; i++) s = __dadd_rn(s, a[i]);
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int mpspmv_probe_fp64(int op, int iters, double* instr_per_s, void* stream) {
  if (op < 0 || op > 2 || iters < 1 || !instr_per_s) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  int dev = 0, sms = 0;
  MPS_CUDA(cudaGetDevice(&dev));
  MPS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = sms * 8;
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * (size_t)blocks * threads) != cudaSuccess) return MPSPMV_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int st = MPSPMV_OK;
  for (int rep = 0; rep < 3 && st == MPSPMV_OK; rep++) {
    cudaEventRecord(e0, s);
    switch (op) {
      case 0: fp64_chain_kernel<0><<<blocks, threads, 0, s>>>(buf, iters, 0.999999, 1e-7); break;
      case 1: fp64_chain_kernel<1><<<blocks, threads, 0, s>>>(buf, iters, 0.999999, 1e-7); break;
      default: fp64_chain_kernel<2><<<blocks, threads, 0, s>>>(buf, iters, 0.999999, 1e-7); break;
    }
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) st = MPSPMV_ECUDA;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (st != MPSPMV_OK) return st;
  *instr_per_s = (double)blocks * threads * (double)iters * kChains / (best * 1e-3);
  return MPSPMV_OK;
}
