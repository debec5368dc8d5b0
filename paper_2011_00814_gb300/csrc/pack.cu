// pack.cu -- the state of a 2D problem as a network tensor and back, and the
// distance between a state and such a tensor.
//
// tensor[j][i][c] for the cell (i, j), c < nch, with the channels
//   0 phi, 1 u, 2 v, 3 p (velocity components on the cell's low faces),
//   4 rho(phi) / rho_L (Eq. of the material laws; nch = 5 only),
// normalised as (field - mean[c]) / scale[c] on packing and mapped back as
// mean[c] + scale[c] * tensor on unpacking and in the distance (mean and
// scale have nch entries).
#include "gpe2p_dev.cuh"
#include "gpe2p_launch.h"

namespace gpe2p {

struct Affine {
  float mean[5], scale[5];
};

template <typename real>
__global__ void pack_kernel(const KParams<real> P, const real* __restrict__ phi, const real* __restrict__ u,
                            const real* __restrict__ v, const real* __restrict__ p, float* __restrict__ out, int nch,
                            const Affine A) {
  const long long n = (long long)P.n[0] * P.n[1];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id % P.n[0]), j = (int)(id / P.n[0]);
    const long long q = lin(P, i, j, 0);
    const real f[4] = {phi[q], u[q], v[q], p[q]};
    float* o = out + id * nch;
#pragma unroll
    for (int c = 0; c < 4; ++c) o[c] = ((float)f[c] - A.mean[c]) / A.scale[c];
    if (nch > 4) o[4] = ((float)(rho_of(P, f[0]) / P.rhoL) - A.mean[4]) / A.scale[4];
  }
}

template <typename real>
__global__ void unpack_kernel(const KParams<real> P, real* __restrict__ phi, real* __restrict__ u, real* __restrict__ v,
                              real* __restrict__ p, const float* __restrict__ in, int nch, const Affine A) {
  const long long n = (long long)P.n[0] * P.n[1];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id % P.n[0]), j = (int)(id / P.n[0]);
    const long long q = lin(P, i, j, 0);
    const float* t = in + id * nch;
    phi[q] = (real)(A.mean[0] + A.scale[0] * t[0]);
    u[q] = (P.bc[0] != BC_PERIODIC && i == 0) ? real(0) : (real)(A.mean[1] + A.scale[1] * t[1]);
    v[q] = (P.bc[1] != BC_PERIODIC && j == 0) ? real(0) : (real)(A.mean[2] + A.scale[2] * t[2]);
    p[q] = (real)(A.mean[3] + A.scale[3] * t[3]);
  }
}

// per block: for each channel c < 4, sum (field - value)^2 and sum field^2 in FP64
template <typename real>
__global__ void distance_kernel(const KParams<real> P, const real* __restrict__ phi, const real* __restrict__ u,
                                const real* __restrict__ v, const real* __restrict__ p, const float* __restrict__ in,
                                int nch, const Affine A, double* __restrict__ part) {
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const long long n = (long long)P.n[0] * P.n[1];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id % P.n[0]), j = (int)(id / P.n[0]);
    const long long q = lin(P, i, j, 0);
    const real f[4] = {phi[q], u[q], v[q], p[q]};
    const float* t = in + id * nch;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double fv = (double)f[c];
      const double d = fv - ((double)A.mean[c] + (double)A.scale[c] * (double)t[c]);
      s[2 * c] += d * d;
      s[2 * c + 1] += fv * fv;
    }
  }
  __shared__ double red[8][8];  // [value][warp]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    double x = s[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[k][w] = x;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    double x = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) x += red[threadIdx.x][k];
    part[blockIdx.x * 8 + threadIdx.x] = x;
  }
}

// fixed-order sum of the block partials
__global__ void distance_final_kernel(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  if (threadIdx.x < 8) {
    double x = 0.0;
    for (int b = 0; b < nblk; ++b) x += part[b * 8 + threadIdx.x];
    out[threadIdx.x] = x;
  }
}

// per block: the displacement of the phi = 0 interface between the state's
// phi (the reference phi_b) and the tensor's phi channel (phi_a), in cells:
// sum |phi_a - phi_b|, sum |grad phi_b| (central differences with the
// boundaries' ghost rules), and over the cells with |phi_b| < 1/2 the max of
// |phi_a - phi_b| / |grad phi_b| and their count (FP64)
template <typename real>
__global__ void iface_kernel(const KParams<real> P, const real* __restrict__ phi, const float* __restrict__ in,
                             int nch, const Affine A, double* __restrict__ part) {
  double sd = 0.0, sg = 0.0, mx = 0.0, cnt = 0.0;
  const long long n = (long long)P.n[0] * P.n[1];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id % P.n[0]), j = (int)(id / P.n[0]);
    const double fb = (double)phi[lin(P, i, j, 0)];
    const double fa = (double)A.mean[0] + (double)A.scale[0] * (double)in[id * nch];
    const double gx = 0.5 * ((double)ld_cen(phi, P, i + 1, j, 0) - (double)ld_cen(phi, P, i - 1, j, 0));
    const double gy = 0.5 * ((double)ld_cen(phi, P, i, j + 1, 0) - (double)ld_cen(phi, P, i, j - 1, 0));
    const double g = sqrt(gx * gx + gy * gy);
    const double d = fabs(fa - fb);
    sd += d;
    sg += g;
    if (fabs(fb) < 0.5) {
      mx = fmax(mx, d / fmax(g, 1e-12));
      cnt += 1.0;
    }
  }
  __shared__ double red[4][8];  // [value][warp]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double v[4] = {sd, sg, mx, cnt};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      x = k == 2 ? fmax(x, y) : x + y;
    }
    if (lane == 0) red[k][w] = x;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double x = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k)
      x = threadIdx.x == 2 ? fmax(x, red[threadIdx.x][k]) : x + red[threadIdx.x][k];
    part[blockIdx.x * 4 + threadIdx.x] = x;
  }
}

// fixed-order combination of the block partials: out[0] max displacement,
// out[1] mean displacement, out[2] band cells
__global__ void iface_final_kernel(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double sd = 0.0, sg = 0.0, mx = 0.0, cnt = 0.0;
    for (int b = 0; b < nblk; ++b) {
      sd += part[b * 4 + 0];
      sg += part[b * 4 + 1];
      mx = fmax(mx, part[b * 4 + 2]);
      cnt += part[b * 4 + 3];
    }
    out[0] = mx;
    out[1] = sd / fmax(sg, 1e-300);
    out[2] = cnt;
  }
}

static Affine affine(const float* mean, const float* scale, int nch) {
  Affine A;
  for (int c = 0; c < 5; ++c) {
    if (c >= nch) { A.mean[c] = 0.f; A.scale[c] = 1.f; continue; }
    A.mean[c] = mean ? mean[c] : 0.f;
    A.scale[c] = scale ? scale[c] : 1.f;
  }
  return A;
}

static unsigned grid_for(long long n) {
  long long nb = (n + 255) / 256;
  return (unsigned)(nb < 152 * 8 ? nb : 152 * 8);
}

template <typename real>
cudaError_t launch_pack(const KParams<real>& P, const real* const f[4], float* out, int nch, const float* mean,
                        const float* scale, cudaStream_t s) {
  const long long n = (long long)P.n[0] * P.n[1];
  pack_kernel<real><<<grid_for(n), 256, 0, s>>>(P, f[0], f[1], f[2], f[3], out, nch, affine(mean, scale, nch));
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_unpack(const KParams<real>& P, real* const f[4], const float* in, int nch, const float* mean,
                          const float* scale, cudaStream_t s) {
  const long long n = (long long)P.n[0] * P.n[1];
  unpack_kernel<real><<<grid_for(n), 256, 0, s>>>(P, f[0], f[1], f[2], f[3], in, nch, affine(mean, scale, nch));
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_distance(const KParams<real>& P, const real* const f[4], const float* in, int nch, const float* mean,
                            const float* scale, double* part, double* out, cudaStream_t s) {
  distance_kernel<real><<<kDistanceBlocks, 256, 0, s>>>(P, f[0], f[1], f[2], f[3], in, nch, affine(mean, scale, nch), part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  distance_final_kernel<<<1, 32, 0, s>>>(part, kDistanceBlocks, out);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_interface_distance(const KParams<real>& P, const real* phi, const float* in, int nch,
                                      const float* mean, const float* scale, double* part, double* out,
                                      cudaStream_t s) {
  iface_kernel<real><<<kDistanceBlocks, 256, 0, s>>>(P, phi, in, nch, affine(mean, scale, nch), part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  iface_final_kernel<<<1, 32, 0, s>>>(part, kDistanceBlocks, out);
  return cudaGetLastError();
}

#define GPE2P_PACK_INST(real)                                                                                       \
  template cudaError_t launch_pack<real>(const KParams<real>&, const real* const[4], float*, int, const float*,     \
                                         const float*, cudaStream_t);                                               \
  template cudaError_t launch_unpack<real>(const KParams<real>&, real* const[4], const float*, int, const float*,   \
                                           const float*, cudaStream_t);                                             \
  template cudaError_t launch_distance<real>(const KParams<real>&, const real* const[4], const float*, int,         \
                                             const float*, const float*, double*, double*, cudaStream_t);   \
  template cudaError_t launch_interface_distance<real>(const KParams<real>&, const real*, const float*, int,       \
                                                       const float*, const float*, double*, double*, cudaStream_t);
GPE2P_PACK_INST(float)
GPE2P_PACK_INST(double)

}  // namespace gpe2p
