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
#include <stdint.h>

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

// ---------------------------------------------------------------------------
// tcgen05.mma issue rate
// ---------------------------------------------------------------------------
// One CTA (one SM).  Lane 0 of warps 0 .. issuers-1 each issues MR_ITERS
// back-to-back tcgen05.mma (kind::f16, BF16 operands, M = 128, N = n,
// K = 16) into its own accumulator of n tensor-memory columns, from a zeroed
// shared-memory operand in the no-swizzle K-major layout, commits them to its
// own mbarrier and waits for their completion (bounded).  The elapsed SM
// clock of the slowest issuer, over the MMAs of all issuers, is the SM's
// cycles per MMA at that N with that many issuing threads.
constexpr int MR_ITERS = 1 + 8 * 128;  // MMAs per issuer
constexpr int MR_SMEM = 65536 + 1024;

__device__ long long g_mma_cycles;
__device__ int g_mma_status;

__device__ __forceinline__ uint32_t mr_su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t mr_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the tcgen05 family; no swizzle
  return d;
}

__device__ __forceinline__ void mr_mma(uint32_t t, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(t),
               "l"(a), "l"(b), "r"(id), "r"(acc)
               : "memory");
}

__global__ void __launch_bounds__(128) mma_rate_kernel(int n, int issuers) {
  extern __shared__ unsigned char mr_raw[];
  unsigned char* sm = mr_raw + ((1024 - (mr_su32(mr_raw) & 1023)) & 1023);  // 1024-byte aligned
  __shared__ uint64_t bar[4];
  __shared__ uint32_t slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 65536 / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(sm)[i] = 0u;
  if (tid == 0) {
    for (int w = 0; w < 4; ++w) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mr_su32(&bar[w])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(mr_su32(&slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tm = slot;
  bool done = true;
  if (warp < issuers && lane == 0) {
    const uint32_t A = mr_su32(sm), B = mr_su32(sm + 16384);
    const uint64_t ad = mr_desc(A, 2048, 128), bd = mr_desc(B, (uint32_t)(n / 8) * 128, 128);
    const uint32_t id = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint32_t t = tm + (uint32_t)(warp * n);
    const long long t0 = clock64();
    mr_mma(t, ad, bd, id, 0u);
    for (int i = 0; i < (MR_ITERS - 1) / 8; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) mr_mma(t, ad, bd, id, 1u);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     mr_su32(&bar[warp]))
                 : "memory");
    uint32_t ok = 0;
    while (!ok && clock64() - t0 < 2000000000LL) {
      asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                   "selp.u32 %0, 1, 0, p;\n\t}"
                   : "=r"(ok)
                   : "r"(mr_su32(&bar[warp]))
                   : "memory");
    }
    atomicMax(&g_mma_cycles, clock64() - t0);
    done = ok != 0;
    if (!done) atomicExch(&g_mma_status, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  if (__syncthreads_or(!done)) {
    // a wait that ran out: give the MMAs a bounded time to finish before the memory is freed
    const long long t1 = clock64();
    while (clock64() - t1 < 100000000LL) {}
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tm) : "memory");
}

}  // namespace

extern "C" int gpe2p_mma_rate(int n, int issuers, double* cycles_per_mma, void* stream) {
  if (!cycles_per_mma || (n != 32 && n != 64 && n != 128 && n != 256) ||
      (issuers != 1 && issuers != 2 && issuers != 4) || n * issuers > 512)
    return GPE2P_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaFuncSetAttribute(mma_rate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MR_SMEM) != cudaSuccess)
    return GPE2P_ECUDA;
  long long best = 0;
  for (int r = 0; r < 4; ++r) {
    const long long zero = 0;
    const int zs = 0;
    if (cudaMemcpyToSymbolAsync(g_mma_cycles, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(g_mma_status, &zs, sizeof(zs), 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return GPE2P_ECUDA;
    mma_rate_kernel<<<1, 128, MR_SMEM, s>>>(n, issuers);
    if (cudaGetLastError() != cudaSuccess) return GPE2P_ECUDA;
    long long c = 0;
    int st = 0;
    if (cudaMemcpyFromSymbolAsync(&c, g_mma_cycles, sizeof(c), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyFromSymbolAsync(&st, g_mma_status, sizeof(st), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return GPE2P_ECUDA;
    if (st != 0) return GPE2P_ETIMEOUT;
    if (r > 0 && (best == 0 || c < best)) best = c;  // the first launch warms up
  }
  *cycles_per_mma = (double)best / ((double)MR_ITERS * issuers);
  return GPE2P_OK;
}

extern "C" int gpe2p_fma_rate(int precision, double* flops_per_s, double* ms, void* stream) {
  if (!flops_per_s || (precision != 32 && precision != 64)) return GPE2P_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  return precision == 64 ? measure<double>(flops_per_s, ms, s) : measure<float>(flops_per_s, ms, s);
}
