// noalloc.cu -- diagnostics of a state the caller holds, without allocating.
//
// Some callers cannot allocate device memory when they need the diagnostics:
// code running inside a CUDA-graph capture or a custom memory pool, a host
// that has handed the whole device to another allocator, or a real-time
// loop that must not block in cudaMalloc.  This entry point computes the
// same four scalars as gpe2p_diagnostics from device pointers the caller
// passes in; its only scratch (one slot of partial sums per thread block) is a
// fixed array in this file's device memory, which every GPU that loads the
// library holds until the process exits.
//
// Set-up: the first call on a device, with that device current, looks up the
// device address of the array (cudaGetSymbolAddress) and keeps it; that first
// call should therefore come before any stream capture.  Later calls that are
// not made while their stream is capturing look the address up again, so
// that a device reset (which reloads the library's device code, possibly at
// another address) does not leave a stale one behind.  All calls share the
// array: each call overwrites the slots it uses before reading them, and two
// calls whose kernels overlap on the GPU race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/gpe2p.h"
#include "gpe2p_dev.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_CELLS_PER_THREAD = 16;
constexpr long long NA_CELLS_PER_BLOCK = (long long)NA_THREADS * NA_CELLS_PER_THREAD;  // 4096
constexpr int NA_MAX_BLOCKS = 16384;
static_assert(NA_CELLS_PER_BLOCK * NA_MAX_BLOCKS == GPE2P_NOALLOC_MAX_CELLS, "limit mismatch");

// 4 doubles of partial results per block: 512 KiB
static __device__ __align__(256) double g_noalloc_scratch[4 * NA_MAX_BLOCKS];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_mu;
double* g_scratch_ptr[NA_MAX_DEVICES] = {};

using gpe2p::KParams;

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double na_warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// block b reduces the cells [b*4096, (b+1)*4096) into scratch slot b
template <typename real, int DIM>
__global__ void __launch_bounds__(NA_THREADS) na_partial_kernel(const KParams<real> P, const real* p, const real* u0,
                                                                const real* u1, const real* u2, const real* phi,
                                                                const real* phi_lo, double* slots,
                                                                long long ncell) {
  const real* U[3] = {u0, u1, u2};
  double sphi = 0.0, ke = 0.0, umax = 0.0, bad = 0.0;
  const long long base = (long long)blockIdx.x * NA_CELLS_PER_BLOCK;
  for (int r = 0; r < NA_CELLS_PER_THREAD; ++r) {
    const long long id = base + (long long)r * NA_THREADS + threadIdx.x;
    if (id >= ncell) break;
    const int i = (int)(id % P.n[0]);
    const int j = (int)((id / P.n[0]) % P.n[1]);
    const int k = (int)(id / ((long long)P.n[0] * P.n[1]));
    const long long q = gpe2p::lin(P, i, j, k);
    // phi of the cell: the stored value plus, under the compensated
    // accumulation, its low part; the lower neighbour's phi in the face
    // density is the stored value alone, as in gpe2p_diagnostics
    const double f = (double)phi[q] + (phi_lo ? (double)phi_lo[q] : 0.0);
    sphi += f;
    if (!isfinite(f) || !isfinite((double)p[q])) bad = 1.0;
    const double rho0 = 0.5 * ((double)P.rhoL * (1.0 + f) + (double)P.rhoG * (1.0 - f));
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const double fm = (double)gpe2p::ld_cen(phi, P, i - (c == 0), j - (c == 1), k - (c == 2));
      const double rhom = 0.5 * ((double)P.rhoL * (1.0 + fm) + (double)P.rhoG * (1.0 - fm));
      const double uc = (double)U[c][q];
      ke += 0.5 * (0.5 * (rhom + rho0)) * uc * uc;
      umax = fmax(umax, fabs(uc));
      if (!isfinite(uc)) bad = 1.0;
    }
  }
  __shared__ double red[4][NA_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  sphi = na_warp_sum(sphi);
  ke = na_warp_sum(ke);
  umax = na_warp_max(umax);
  bad = na_warp_max(bad);
  if (lane == 0) {
    red[0][wid] = sphi;
    red[1][wid] = ke;
    red[2][wid] = umax;
    red[3][wid] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
    for (int w = 0; w < NA_THREADS / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
      c = fmax(c, red[2][w]);
      d = fmax(d, red[3][w]);
    }
    slots[4 * blockIdx.x + 0] = a;
    slots[4 * blockIdx.x + 1] = b;
    slots[4 * blockIdx.x + 2] = c;
    slots[4 * blockIdx.x + 3] = d;
  }
}

// one block sums the nblocks slots in a fixed order and writes out[0..3]
__global__ void __launch_bounds__(NA_THREADS) na_final_kernel(const double* slots, int nblocks, double vol,
                                                              double* out) {
  __shared__ double red[4][NA_THREADS];
  double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
  for (int q = threadIdx.x; q < nblocks; q += NA_THREADS) {
    a += slots[4 * q + 0];
    b += slots[4 * q + 1];
    c = fmax(c, slots[4 * q + 2]);
    d = fmax(d, slots[4 * q + 3]);
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  red[2][threadIdx.x] = c;
  red[3][threadIdx.x] = d;
  __syncthreads();
  for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
      red[2][threadIdx.x] = fmax(red[2][threadIdx.x], red[2][threadIdx.x + s]);
      red[3][threadIdx.x] = fmax(red[3][threadIdx.x], red[3][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = red[0][0] * vol;
    out[1] = red[1][0] * vol;
    out[2] = red[2][0];
    out[3] = red[3][0];
  }
}

// the device address of the scratch array on the current device: looked up on
// the first call on a device, and again on every call whose stream is not
// capturing (a capture keeps the address found before it)
cudaError_t scratch_on_current_device(cudaStream_t s, double** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capturing = cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
  if (capturing) cudaGetLastError();  // a query refused during a capture leaves no sticky error
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev] || !capturing) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *ptr = g_scratch_ptr[dev];
  return cudaSuccess;
}

template <typename real, int DIM>
cudaError_t launch(const KParams<real>& P, const void* p, const void* u, const void* v, const void* w,
                   const void* phi, const void* phi_lo, double* slots, long long ncell, int nblocks, double vol,
                   double* out, cudaStream_t s) {
  na_partial_kernel<real, DIM><<<nblocks, NA_THREADS, 0, s>>>(P, (const real*)p, (const real*)u, (const real*)v,
                                                              (const real*)w, (const real*)phi,
                                                              (const real*)phi_lo, slots, ncell);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  na_final_kernel<<<1, NA_THREADS, 0, s>>>(slots, nblocks, vol, out);
  return cudaGetLastError();
}

template <typename real>
KParams<real> na_params(const gpe2p_params& q, long long row_pitch) {
  KParams<real> P{};
  P.n[0] = q.nx;
  P.n[1] = q.ny;
  P.n[2] = q.dim == 3 ? q.nz : 1;
  for (int a = 0; a < 3; ++a) P.bc[a] = (a < q.dim) ? q.bc[a] : gpe2p::BC_PERIODIC;
  P.sy = row_pitch;
  P.sz = row_pitch * q.ny;
  P.rhoL = (real)q.rhoL;
  P.rhoG = (real)q.rhoG;
  P.inv_dx = (real)(1.0 / q.dx);
  return P;
}

}  // namespace

extern "C" int gpe2p_diagnostics_noalloc(const gpe2p_params* q, const void* p, const void* u, const void* v,
                                         const void* w, const void* phi, const void* phi_lo,
                                         long long row_pitch, double* out, void* stream) {
  if (!q || !p || !u || !v || !phi || !out) return GPE2P_EINVAL;
  if (q->dim != 2 && q->dim != 3) return GPE2P_EINVAL;
  if (q->dim == 3 && !w) return GPE2P_EINVAL;
  if (q->precision != 32 && q->precision != 64) return GPE2P_EINVAL;
  const long long nz = q->dim == 3 ? q->nz : 1;
  if (q->nx < 1 || q->ny < 1 || nz < 1 || row_pitch < q->nx) return GPE2P_EINVAL;
  if (!(q->dx > 0.0) || !std::isfinite(q->dx)) return GPE2P_EINVAL;
  for (int a = 0; a < q->dim; ++a)
    if (q->bc[a] < 0 || q->bc[a] > 2) return GPE2P_EINVAL;
  const long long ncell = (long long)q->nx * q->ny * nz;
  if (ncell > GPE2P_NOALLOC_MAX_CELLS) return GPE2P_EINVAL;  // more cells than the scratch slots cover
  cudaStream_t s = (cudaStream_t)stream;
  double* slots = nullptr;
  if (scratch_on_current_device(s, &slots) != cudaSuccess) return GPE2P_ECUDA;
  const int nblocks = (int)((ncell + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
  const double vol = q->dim == 3 ? q->dx * q->dx * q->dx : q->dx * q->dx;
  cudaError_t e;
  if (q->precision == 32) {
    const KParams<float> P = na_params<float>(*q, row_pitch);
    e = q->dim == 2 ? launch<float, 2>(P, p, u, v, w, phi, phi_lo, slots, ncell, nblocks, vol, out, s)
                    : launch<float, 3>(P, p, u, v, w, phi, phi_lo, slots, ncell, nblocks, vol, out, s);
  } else {
    const KParams<double> P = na_params<double>(*q, row_pitch);
    e = q->dim == 2 ? launch<double, 2>(P, p, u, v, w, phi, phi_lo, slots, ncell, nblocks, vol, out, s)
                    : launch<double, 3>(P, p, u, v, w, phi, phi_lo, slots, ncell, nblocks, vol, out, s);
  }
  return e == cudaSuccess ? GPE2P_OK : GPE2P_ECUDA;
}
