// ch.cu -- the Cahn-Hilliard part of a step (Sec. 3): chemical potential
// (Eq. chem-pot), one RK stage of Eq. che with the isotropic stencils of
// Eqs. 1st-der-iso and laplacian-iso, and the time-centred cell velocity of
// Eq. u-center-2d.  Same tiling as the flow stage: a block stages phi_s and
// mu_s (and, for the conservative form, the cell velocity) with a one-cell
// halo in shared memory and marches along z in 3D.
#include "gpe2p_dev.cuh"
#include "gpe2p_launch.h"

namespace gpe2p {

// which lattice shells a model uses: D2Q9 {1,2}, D3Q15 {1,3}, D3Q19 {1,2}, D3Q27 {1,2,3}
template <int ISO>
struct Shells {
  static constexpr bool s2 = ISO == 9 || ISO == 19 || ISO == 27;
  static constexpr bool s3 = ISO == 15 || ISO == 27;
};

template <typename real, int DIM, int ISO, int NPL>
__device__ __forceinline__ real lap_iso(const Tile<real, NPL>& S, const KParams<real>& P, int f) {
  real s = real(0);
#pragma unroll
  for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int sh = dx * dx + dy * dy + dz * dz;
        if (sh == 0) continue;
        if (sh == 2 && !Shells<ISO>::s2) continue;
        if (sh == 3 && !Shells<ISO>::s3) continue;
        s += shell_w(P, sh) * S(f, dx, dy, dz);
      }
  return P.lap_c * (s - P.one_m_w0 * S(f, 0, 0, 0));
}

// the DIM components of the isotropic gradient of staged field f
template <typename real, int DIM, int ISO, int NPL>
__device__ __forceinline__ void grad_iso(const Tile<real, NPL>& S, const KParams<real>& P, int f, real g[3]) {
  real s[3] = {real(0), real(0), real(0)};
#pragma unroll
  for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int sh = dx * dx + dy * dy + dz * dz;
        if (sh == 0) continue;
        if (sh == 2 && !Shells<ISO>::s2) continue;
        if (sh == 3 && !Shells<ISO>::s3) continue;
        const real w = shell_w(P, sh);
        const real v = S(f, dx, dy, dz);
        if (dx != 0) s[0] += (dx > 0 ? w : -w) * v;
        if (dy != 0) s[1] += (dy > 0 ? w : -w) * v;
        if (DIM == 3 && dz != 0) s[2] += (dz > 0 ? w : -w) * v;
      }
#pragma unroll
  for (int a = 0; a < DIM; ++a) g[a] = P.grad_c * s[a];
}

enum { C_PHI = 0, C_MU = 1, C_UH = 2, C_N = 5 };

template <typename real, int DIM, int ISO>
__global__ void __launch_bounds__(NTHR) ch_stage_kernel(const KParams<real> P, const CHArgs<real> A,
                                                        const int kchunk) {
  constexpr int NPL = DIM == 3 ? 3 : 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  real* sm = reinterpret_cast<real*>(smraw);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int kbeg = DIM == 3 ? blockIdx.z * kchunk : 0;
  const int kend = DIM == 3 ? min(kbeg + kchunk, P.n[2]) : 1;
  const int nx = P.n[0], ny = P.n[1];
  const bool cons = A.conservative != 0;

  auto load_plane = [&](int kk, int slot) {
    for (int idx = tid; idx < PL; idx += NTHR) {
      const int ly = idx / SX, lx = idx - ly * SX;
      const int gi = clampi(i0 - 1 + lx, -1, nx), gj = clampi(j0 - 1 + ly, -1, ny);
      real* b = sm + slot * PL + idx;
      b[(C_PHI * NPL) * PL] = ld_cen(A.phis, P, gi, gj, kk);
      b[(C_MU * NPL) * PL] = ld_cen(A.mus, P, gi, gj, kk);
      if (cons) {
        b[((C_UH + 0) * NPL) * PL] = ld_cvec<0>(A.uh[0], P, gi, gj, kk);
        b[((C_UH + 1) * NPL) * PL] = ld_cvec<1>(A.uh[1], P, gi, gj, kk);
        if (DIM == 3) b[((C_UH + 2) * NPL) * PL] = ld_cvec<2>(A.uh[2], P, gi, gj, kk);
      }
    }
  };

  if (DIM == 3) {
    load_plane(kbeg - 1, (kbeg + 2) % 3);
    load_plane(kbeg, kbeg % 3);
  } else {
    load_plane(0, 0);
  }
  const int i = i0 + tx, j = j0 + ty;
  const bool active = i < nx && j < ny;
  for (int k = kbeg; k < kend; ++k) {
    if (DIM == 3) load_plane(k + 1, (k + 1) % 3);
    __syncthreads();
    if (active) {
      Tile<real, NPL> S;
      S.sm = sm;
      S.c = (ty + 1) * SX + (tx + 1);
      S.s0 = DIM == 3 ? k % 3 : 0;
      S.sm1 = DIM == 3 ? (k + 2) % 3 : 0;
      S.sp1 = DIM == 3 ? (k + 1) % 3 : 0;
      const long long id = lin(P, i, j, k);
      const real lapmu = lap_iso<real, DIM, ISO, NPL>(S, P, C_MU);
      real adv = real(0);
      if (!cons) {
        real uh[3];
        if (A.compute_uh) {
          uh[0] = real(0.25) * ((ld_face<0>(A.u0[0], P, i, j, k) + ld_face<0>(A.u0[0], P, i + 1, j, k)) +
                                (ld_face<0>(A.u1[0], P, i, j, k) + ld_face<0>(A.u1[0], P, i + 1, j, k)));
          uh[1] = real(0.25) * ((ld_face<1>(A.u0[1], P, i, j, k) + ld_face<1>(A.u0[1], P, i, j + 1, k)) +
                                (ld_face<1>(A.u1[1], P, i, j, k) + ld_face<1>(A.u1[1], P, i, j + 1, k)));
          if (DIM == 3)
            uh[2] = real(0.25) * ((ld_face<2>(A.u0[2], P, i, j, k) + ld_face<2>(A.u0[2], P, i, j, k + 1)) +
                                  (ld_face<2>(A.u1[2], P, i, j, k) + ld_face<2>(A.u1[2], P, i, j, k + 1)));
          if (A.stage != 0)
            for (int a = 0; a < DIM; ++a) A.uh[a][id] = uh[a];
        } else {
          for (int a = 0; a < DIM; ++a) uh[a] = A.uh[a][id];
        }
        real g[3];
        grad_iso<real, DIM, ISO, NPL>(S, P, C_PHI, g);
#pragma unroll
        for (int a = 0; a < DIM; ++a) adv += uh[a] * g[a];
      } else {
        // -div_iso(uhat phi): the isotropic first derivative of the product
        real s[3] = {real(0), real(0), real(0)};
#pragma unroll
        for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz)
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
              const int sh = dx * dx + dy * dy + dz * dz;
              if (sh == 0) continue;
              if (sh == 2 && !Shells<ISO>::s2) continue;
              if (sh == 3 && !Shells<ISO>::s3) continue;
              const real w = shell_w(P, sh);
              const real ph = S(C_PHI, dx, dy, dz);
              if (dx != 0) s[0] += (dx > 0 ? w : -w) * S(C_UH + 0, dx, dy, dz) * ph;
              if (dy != 0) s[1] += (dy > 0 ? w : -w) * S(C_UH + 1, dx, dy, dz) * ph;
              if (DIM == 3 && dz != 0) s[2] += (dz > 0 ? w : -w) * S(C_UH + 2, dx, dy, dz) * ph;
            }
#pragma unroll
        for (int a = 0; a < DIM; ++a) adv += P.grad_c * s[a];
      }
      const real L = -adv + P.M * lapmu;
      real o;
      if (A.stage == 0) {
        o = L;
      } else if (A.scheme == 2) {
        if (A.stage == 1) o = A.phin[id] + P.dt * L;
        else o = real(0.5) * A.phin[id] + real(0.5) * (S(C_PHI, 0, 0, 0) + P.dt * L);
      } else {
        const real d = P.dt * L;
        const real pn = A.phin[id];
        if (A.stage == 1) { A.acc[id] = d; o = pn + real(0.5) * d; }
        else if (A.stage == 2) { A.acc[id] = A.acc[id] + real(2) * d; o = pn + real(0.5) * d; }
        else if (A.stage == 3) { A.acc[id] = A.acc[id] + real(2) * d; o = pn + d; }
        else { o = pn + (A.acc[id] + d) / real(6); }
      }
      A.out[id] = o;
    }
    __syncthreads();
  }
}

template <typename real, int DIM, int ISO>
__global__ void __launch_bounds__(NTHR) mu_kernel(const KParams<real> P, const real* __restrict__ phi,
                                                  real* __restrict__ mu, const int kchunk) {
  constexpr int NPL = DIM == 3 ? 3 : 1;
  __shared__ real sm[NPL * PL];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int kbeg = DIM == 3 ? blockIdx.z * kchunk : 0;
  const int kend = DIM == 3 ? min(kbeg + kchunk, P.n[2]) : 1;
  const int nx = P.n[0], ny = P.n[1];
  auto load_plane = [&](int kk, int slot) {
    for (int idx = tid; idx < PL; idx += NTHR) {
      const int ly = idx / SX, lx = idx - ly * SX;
      const int gi = clampi(i0 - 1 + lx, -1, nx), gj = clampi(j0 - 1 + ly, -1, ny);
      sm[slot * PL + idx] = ld_cen(phi, P, gi, gj, kk);
    }
  };
  if (DIM == 3) {
    load_plane(kbeg - 1, (kbeg + 2) % 3);
    load_plane(kbeg, kbeg % 3);
  } else {
    load_plane(0, 0);
  }
  const int i = i0 + tx, j = j0 + ty;
  const bool active = i < nx && j < ny;
  for (int k = kbeg; k < kend; ++k) {
    if (DIM == 3) load_plane(k + 1, (k + 1) % 3);
    __syncthreads();
    if (active) {
      Tile<real, NPL> S;
      S.sm = sm;
      S.c = (ty + 1) * SX + (tx + 1);
      S.s0 = DIM == 3 ? k % 3 : 0;
      S.sm1 = DIM == 3 ? (k + 2) % 3 : 0;
      S.sp1 = DIM == 3 ? (k + 1) % 3 : 0;
      const real f = S(0, 0, 0, 0);
      mu[lin(P, i, j, k)] = P.a4 * f * (f * f - real(1)) - P.kappa * lap_iso<real, DIM, ISO, NPL>(S, P, 0);
    }
    __syncthreads();
  }
}

template <typename real, int DIM>
__global__ void center_velocity_kernel(const KParams<real> P, const real* u00, const real* u01,
                                       const real* u02, const real* u10, const real* u11, const real* u12,
                                       real* uh0, real* uh1, real* uh2) {
  const long long n = (long long)P.n[0] * P.n[1] * P.n[2];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
       id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id % P.n[0]);
    const int j = (int)((id / P.n[0]) % P.n[1]);
    const int k = (int)(id / ((long long)P.n[0] * P.n[1]));
    uh0[id] = real(0.25) * ((ld_face<0>(u00, P, i, j, k) + ld_face<0>(u00, P, i + 1, j, k)) +
                            (ld_face<0>(u10, P, i, j, k) + ld_face<0>(u10, P, i + 1, j, k)));
    uh1[id] = real(0.25) * ((ld_face<1>(u01, P, i, j, k) + ld_face<1>(u01, P, i, j + 1, k)) +
                            (ld_face<1>(u11, P, i, j, k) + ld_face<1>(u11, P, i, j + 1, k)));
    if (DIM == 3)
      uh2[id] = real(0.25) * ((ld_face<2>(u02, P, i, j, k) + ld_face<2>(u02, P, i, j, k + 1)) +
                              (ld_face<2>(u12, P, i, j, k) + ld_face<2>(u12, P, i, j, k + 1)));
  }
}

template <typename real, int DIM>
static size_t ch_smem() {
  return sizeof(real) * (size_t)C_N * (DIM == 3 ? 3 : 1) * PL;
}

template <typename real, int DIM, int ISO>
static cudaError_t ch_go(const KParams<real>& P, const CHArgs<real>& A, int kchunk, cudaStream_t s) {
  const size_t sm = ch_smem<real, DIM>();
  cudaError_t e = cudaFuncSetAttribute(ch_stage_kernel<real, DIM, ISO>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 blk(TX, TY, 1);
  dim3 grd((P.n[0] + TX - 1) / TX, (P.n[1] + TY - 1) / TY, DIM == 3 ? (P.n[2] + kchunk - 1) / kchunk : 1);
  ch_stage_kernel<real, DIM, ISO><<<grd, blk, sm, s>>>(P, A, kchunk);
  return cudaGetLastError();
}

template <typename real, int DIM>
cudaError_t launch_ch_stage(const KParams<real>& P, const CHArgs<real>& A, int iso, int kchunk,
                            cudaStream_t s) {
  if constexpr (DIM == 2) {
    return ch_go<real, DIM, 9>(P, A, kchunk, s);
  } else {
    switch (iso) {
      case 15: return ch_go<real, DIM, 15>(P, A, kchunk, s);
      case 19: return ch_go<real, DIM, 19>(P, A, kchunk, s);
      default: return ch_go<real, DIM, 27>(P, A, kchunk, s);
    }
  }
}

template <typename real, int DIM, int ISO>
static cudaError_t mu_go(const KParams<real>& P, const real* phi, real* mu, int kchunk, cudaStream_t s) {
  dim3 blk(TX, TY, 1);
  dim3 grd((P.n[0] + TX - 1) / TX, (P.n[1] + TY - 1) / TY, DIM == 3 ? (P.n[2] + kchunk - 1) / kchunk : 1);
  mu_kernel<real, DIM, ISO><<<grd, blk, 0, s>>>(P, phi, mu, kchunk);
  return cudaGetLastError();
}

template <typename real, int DIM>
cudaError_t launch_mu(const KParams<real>& P, const real* phi, real* mu, int iso, int kchunk, cudaStream_t s) {
  if constexpr (DIM == 2) {
    return mu_go<real, DIM, 9>(P, phi, mu, kchunk, s);
  } else {
    switch (iso) {
      case 15: return mu_go<real, DIM, 15>(P, phi, mu, kchunk, s);
      case 19: return mu_go<real, DIM, 19>(P, phi, mu, kchunk, s);
      default: return mu_go<real, DIM, 27>(P, phi, mu, kchunk, s);
    }
  }
}

template <typename real, int DIM>
cudaError_t launch_center_velocity(const KParams<real>& P, const real* const u0[3], const real* const u1[3],
                                   real* const uh[3], cudaStream_t s) {
  const long long n = (long long)P.n[0] * P.n[1] * P.n[2];
  long long nb = (n + 255) / 256;
  if (nb > 152 * 16) nb = 152 * 16;
  center_velocity_kernel<real, DIM><<<(unsigned)nb, 256, 0, s>>>(P, u0[0], u0[1], u0[2], u1[0], u1[1], u1[2],
                                                                 uh[0], uh[1], uh[2]);
  return cudaGetLastError();
}

#define GPE2P_CH_INST(R, D)                                                                                 \
  template cudaError_t launch_ch_stage<R, D>(const KParams<R>&, const CHArgs<R>&, int, int, cudaStream_t); \
  template cudaError_t launch_mu<R, D>(const KParams<R>&, const R*, R*, int, int, cudaStream_t);           \
  template cudaError_t launch_center_velocity<R, D>(const KParams<R>&, const R* const[3], const R* const[3], \
                                                    R* const[3], cudaStream_t);
GPE2P_CH_INST(float, 2)
GPE2P_CH_INST(float, 3)
GPE2P_CH_INST(double, 2)
GPE2P_CH_INST(double, 3)
#undef GPE2P_CH_INST

}  // namespace gpe2p
