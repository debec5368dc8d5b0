// rate.cu -- the floating-point rate of the GPU, measured: the bound of the
// FP64 path of the step, whose stencil arithmetic runs on the FP64 units
// (a small fraction of the FP32 rate on GB300), and the FP32 rate beside it.
//
// Every thread runs NCHAIN independent chains x <- x a + b of fused
// multiply-adds (two floating-point operations each), enough chains that the
// dependent latency of one is hidden behind the others, over a grid of
// several resident blocks per SM.  a = 1 - 2^-20 and b = 2^-20 keep every x
// at a fixed point 1 + O(2^-20) (no overflow, no denormals), and the chains'
// sum is compared with a value it cannot take, so the compiler keeps every
// multiply-add.  The rate is the operations over the kernel's CUDA-event
// time on the caller's stream, the best of three launches after a warm-up.
#include <cuda_runtime.h>

#include "../../include/gpe2p.h"

namespace {

constexpr int RT_THREADS = 256;
constexpr int RT_NCHAIN = 8;

// never written in practice: the kernels store there only if the chains'
// sum takes an impossible value
__device__ double g_rate_sink[2];

template <typename real>
__global__ void __launch_bounds__(RT_THREADS) fma_chain_kernel(int iters, real a, real b) {
  real x[RT_NCHAIN];
#pragma unroll
  for (int c = 0; c < RT_NCHAIN; ++c) x[c] = real(1) + real(c) * real(1e-3) + real(threadIdx.x) * real(1e-6);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < RT_NCHAIN; ++c) x[c] = fma(x[c], a, b);
  }
  real s = real(0);
#pragma unroll
  for (int c = 0; c < RT_NCHAIN; ++c) s += x[c];
  if (s == real(-1)) g_rate_sink[sizeof(real) == 8] = (double)s;
}

template <typename real>
cudaError_t time_chains(int blocks, int iters, cudaStream_t s, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  const real a = real(1) - real(1.0 / 1048576.0), b = real(1.0 / 1048576.0);
  cudaEventRecord(e0, s);
  fma_chain_kernel<real><<<blocks, RT_THREADS, 0, s>>>(iters, a, b);
  e = cudaGetLastError();
  cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

template <typename real>
int measure(double* flops_per_s, double* out_ms, cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GPE2P_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GPE2P_ECUDA;
  const int blocks = sms * 8;  // 64 warps per SM
  const double ops_per_iter = 2.0 * RT_NCHAIN * (double)blocks * RT_THREADS;
  // calibrate on a short launch, then size the timed ones to about 50 ms
  float ms = 0.f;
  int iters = 256;
  if (time_chains<real>(blocks, iters, s, &ms) != cudaSuccess) return GPE2P_ECUDA;
  const double per_iter = ms > 0.f ? ms / iters : 1e-3;
  iters = (int)(50.0 / per_iter);
  if (iters < 256) iters = 256;
  if (iters > (1 << 26)) iters = 1 << 26;
  float best = 0.f;
  for (int r = 0; r < 4; ++r) {
    if (time_chains<real>(blocks, iters, s, &ms) != cudaSuccess) return GPE2P_ECUDA;
    if (r > 0 && (best == 0.f || ms < best)) best = ms;
  }
  *flops_per_s = ops_per_iter * iters / (best * 1e-3);
  if (out_ms) *out_ms = best;
  return GPE2P_OK;
}

}  // namespace

extern "C" int gpe2p_fma_rate(int precision, double* flops_per_s, double* ms, void* stream) {
  if (!flops_per_s || (precision != 32 && precision != 64)) return GPE2P_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  return precision == 64 ? measure<double>(flops_per_s, ms, s) : measure<float>(flops_per_s, ms, s);
}
