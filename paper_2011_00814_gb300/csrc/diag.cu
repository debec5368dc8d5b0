// diag.cu -- FP64 diagnostics of the state (sum of phi, kinetic energy with
// the face density, max |u|, NaN/Inf flag) and the FP64 <-> working-precision
// copies used at the host boundary.
//
// The sum of phi is the integral the Cahn-Hilliard equation (Eq. che)
// conserves. The advective form conserves it only up to the flow's
// compressibility, so its drift measures the method. The kinetic energy takes
// each face velocity with the density of its face, the mean of the two cells'
// densities (Eq. density-viscosity-op-two-phase, linear in phi). max |u| gives
// the spurious currents of a drop at rest.
//
// The reduction is deterministic: a fixed grid of blocks walks the cells with
// a grid-stride loop, each block reduces its partial sums with warp shuffles
// into a slot of a scratch array, and a single block then sums the slots in
// a fixed order.
#include "gpe2p_dev.cuh"
#include "gpe2p_launch.h"

namespace gpe2p {

constexpr int DIAG_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <typename real, int DIM>
__global__ void __launch_bounds__(DIAG_THREADS) diag_partial_kernel(const KParams<real> P, const real* p,
                                                                    const real* u0, const real* u1,
                                                                    const real* u2, const real* phi,
                                                                    const real* phi_lo, double* partial) {
  // blocks stride over the rows (j, k), threads along x; per cell, in FP64:
  // phi, and for each face the face density (the mean of the two cells'
  // rho(phi) = (rhoL + rhoG)/2 + phi (rhoL - rhoG)/2) times u^2; the factor
  // 1/2 of the kinetic energy is applied once per thread
  const int nx = P.n[0], ny = P.n[1];
  const long long rows = (long long)ny * P.n[2];
  const double rm = 0.5 * ((double)P.rhoL + (double)P.rhoG), rd = 0.25 * ((double)P.rhoL - (double)P.rhoG);
  double sphi = 0.0, ke = 0.0;
  real umax = real(0);
  bool bad = false;
  const real* U[3] = {u0, u1, u2};
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const int j = (int)(r % ny), k = (int)(r / ny);
    const long long q0 = lin(P, 0, j, k);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const long long q = q0 + i;
      const real fr = phi[q];
      const double f = (double)fr + (phi_lo ? (double)phi_lo[q] : 0.0);
      sphi += f;
      bad = bad || !isfinite(fr) || !isfinite(p[q]);
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const double fm = (double)ld_cen(phi, P, i - (c == 0), j - (c == 1), k - (c == 2));
        const real uc = U[c][q];
        const double ud = (double)uc;
        ke = fma(fma(rd, fm + f, rm), ud * ud, ke);
        umax = fmax(umax, fabs(uc));
        bad = bad || !isfinite(uc);
      }
    }
  }
  ke *= 0.5;
  double umaxd = (double)umax, badd = bad ? 1.0 : 0.0;
  __shared__ double red[4][DIAG_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  sphi = warp_sum(sphi);
  ke = warp_sum(ke);
  umaxd = warp_max(umaxd);
  badd = warp_max(badd);
  if (lane == 0) {
    red[0][wid] = sphi;
    red[1][wid] = ke;
    red[2][wid] = umaxd;
    red[3][wid] = badd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
    for (int w = 0; w < DIAG_THREADS / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
      c = fmax(c, red[2][w]);
      d = fmax(d, red[3][w]);
    }
    partial[4 * blockIdx.x + 0] = a;
    partial[4 * blockIdx.x + 1] = b;
    partial[4 * blockIdx.x + 2] = c;
    partial[4 * blockIdx.x + 3] = d;
  }
}

__global__ void diag_final_kernel(const double* partial, int nblocks, double vol, double* out) {
  __shared__ double red[4][DIAG_THREADS];
  double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
  for (int q = threadIdx.x; q < nblocks; q += blockDim.x) {
    a += partial[4 * q + 0];
    b += partial[4 * q + 1];
    c = fmax(c, partial[4 * q + 2]);
    d = fmax(d, partial[4 * q + 3]);
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  red[2][threadIdx.x] = c;
  red[3][threadIdx.x] = d;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
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

template <typename real, int DIM>
cudaError_t launch_diag(const KParams<real>& P, const real* p, const real* const U[3], const real* phi,
                        const real* phi_lo, double* partial, int nblocks, double* out, cudaStream_t s) {
  const double dx = 1.0 / (double)P.inv_dx;
  const double vol = DIM == 3 ? dx * dx * dx : dx * dx;
  diag_partial_kernel<real, DIM><<<nblocks, DIAG_THREADS, 0, s>>>(P, p, U[0], U[1], U[2], phi, phi_lo, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final_kernel<<<1, DIAG_THREADS, 0, s>>>(partial, nblocks, vol, out);
  return cudaGetLastError();
}

// dense FP64 (host layout) -> padded rows in the working precision.  Blocks
// stride over the rows (j, k) and threads along x, so that both sides are
// read and written in order; src may be a pinned host array read in place,
// in 16-byte pairs where the rows allow.  With ABS, the block also sums
// |src| and the stored value (in FP64, fixed order) into partial[4 b] and
// partial[4 b + 1], in the layout diag_final_kernel reduces: the integral of
// |phi_0| and that of phi_0 as stored (the reference of the conservation
// drift) need no second read.
template <typename real, bool ABS>
__global__ void __launch_bounds__(DIAG_THREADS) from_double_kernel(const KParams<real> P, const double* src,
                                                                   real* dst, int c, double* partial) {
  const int nx = P.n[0], ny = P.n[1];
  const long long rows = (long long)ny * P.n[2];
  const bool pairs = (nx & 1) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0;
  double a = 0.0, b = 0.0;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const int j = (int)(r % ny), k = (int)(r / ny);
    const bool wall_row = c >= 0 && P.bc[c] != BC_PERIODIC && ((c == 1 && j == 0) || (c == 2 && k == 0));
    const bool wall_x = c == 0 && P.bc[0] != BC_PERIODIC;
    const double* s = src + r * nx;
    real* d = dst + lin(P, 0, j, k);
    if (pairs) {
      const double2* s2 = reinterpret_cast<const double2*>(s);
      for (int i2 = threadIdx.x; i2 < (nx >> 1); i2 += blockDim.x) {
        const double2 x = s2[i2];
        if (ABS) a += fabs(x.x) + fabs(x.y);
        real v0 = (real)x.x, v1 = (real)x.y;
        if (wall_row || (wall_x && i2 == 0)) v0 = real(0);
        if (wall_row) v1 = real(0);
        if (ABS) b += (double)v0 + (double)v1;
        d[2 * i2] = v0;
        d[2 * i2 + 1] = v1;
      }
    } else {
      for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const double x = s[i];
        if (ABS) a += fabs(x);
        real v = (real)x;
        if (wall_row || (wall_x && i == 0)) v = real(0);
        if (ABS) b += (double)v;
        d[i] = v;
      }
    }
  }
  if (ABS) {
    __shared__ double red[2][DIAG_THREADS / 32];
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = a;
      red[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0, u = 0.0;
      for (int w = 0; w < DIAG_THREADS / 32; ++w) {
        t += red[0][w];
        u += red[1][w];
      }
      partial[4 * blockIdx.x + 0] = t;
      partial[4 * blockIdx.x + 1] = u;
      partial[4 * blockIdx.x + 2] = 0.0;
      partial[4 * blockIdx.x + 3] = 0.0;
    }
  }
}

// padded rows -> dense FP64 (plus a low part, when given); dst may be a
// pinned host array written in place
template <typename real>
__global__ void to_double_kernel(const KParams<real> P, const real* src, double* dst, const real* lo) {
  const int nx = P.n[0], ny = P.n[1];
  const long long rows = (long long)ny * P.n[2];
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const int j = (int)(r % ny), k = (int)(r / ny);
    const long long q0 = lin(P, 0, j, k);
    double* d = dst + r * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x)
      d[i] = (double)src[q0 + i] + (lo ? (double)lo[q0 + i] : 0.0);
  }
}

// blocks for a row-strided conversion: every row gets a block up to 32 per SM
template <typename real>
static unsigned grid_rows(const KParams<real>& P) {
  long long rows = (long long)P.n[1] * P.n[2];
  if (rows > 152 * 32) rows = 152 * 32;
  return (unsigned)(rows < 1 ? 1 : rows);
}

template <typename real>
cudaError_t launch_from_double(const KParams<real>& P, const double* src, real* dst, int c, long long n,
                               cudaStream_t s) {
  (void)n;
  from_double_kernel<real, false><<<grid_rows(P), DIAG_THREADS, 0, s>>>(P, src, dst, c, nullptr);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_from_double_abs(const KParams<real>& P, const double* src, real* dst, double* partial,
                                   int nblocks, double vol, double* out, cudaStream_t s) {
  unsigned nb = grid_rows(P);
  if (nb > (unsigned)nblocks) nb = (unsigned)nblocks;
  from_double_kernel<real, true><<<nb, DIAG_THREADS, 0, s>>>(P, src, dst, -1, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final_kernel<<<1, DIAG_THREADS, 0, s>>>(partial, (int)nb, vol, out);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_to_double(const KParams<real>& P, const real* src, double* dst, long long n, cudaStream_t s,
                             const real* lo) {
  (void)n;
  to_double_kernel<real><<<grid_rows(P), 256, 0, s>>>(P, src, dst, lo);
  return cudaGetLastError();
}

template cudaError_t launch_diag<float, 2>(const KParams<float>&, const float*, const float* const[3],
                                           const float*, const float*, double*, int, double*, cudaStream_t);
template cudaError_t launch_diag<float, 3>(const KParams<float>&, const float*, const float* const[3],
                                           const float*, const float*, double*, int, double*, cudaStream_t);
template cudaError_t launch_diag<double, 2>(const KParams<double>&, const double*, const double* const[3],
                                            const double*, const double*, double*, int, double*, cudaStream_t);
template cudaError_t launch_diag<double, 3>(const KParams<double>&, const double*, const double* const[3],
                                            const double*, const double*, double*, int, double*, cudaStream_t);
template cudaError_t launch_from_double<float>(const KParams<float>&, const double*, float*, int, long long,
                                               cudaStream_t);
template cudaError_t launch_from_double<double>(const KParams<double>&, const double*, double*, int,
                                                long long, cudaStream_t);
template cudaError_t launch_from_double_abs<float>(const KParams<float>&, const double*, float*, double*, int,
                                                   double, double*, cudaStream_t);
template cudaError_t launch_from_double_abs<double>(const KParams<double>&, const double*, double*, double*, int,
                                                    double, double*, cudaStream_t);
template cudaError_t launch_to_double<float>(const KParams<float>&, const float*, double*, long long,
                                             cudaStream_t, const float*);
template cudaError_t launch_to_double<double>(const KParams<double>&, const double*, double*, long long,
                                              cudaStream_t, const double*);

}  // namespace gpe2p
