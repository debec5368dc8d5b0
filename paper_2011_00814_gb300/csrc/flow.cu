// flow.cu -- one TVD-RK3 stage of the GPE flow update (Sec. 3):
//   out = a q^n + b (q + dt L(q)),  q = (p, u, v[, w]),
// with L the semi-discrete operators of Eq. p-u-v-semidiscrete-2d built from
// Eqs. div-v-discretization, diff-p-discretization, conv-u-discretization,
// u-stress-discretization (a)-(d), st-u-discretization, gradp-u-discretization
// and gradp-u-p-ave-3d, with phi and mu frozen (Sec. 3, after Eq. tvd-rk3).
//
// One thread per cell computes the pressure rate at the cell centre and the
// rate of each velocity component on the cell's low faces.  A block stages the
// fields of its tile plus a one-cell halo in shared memory (ghosts already
// mapped by the boundary rules), together with rho, eta and nu = eta/rho
// computed once per staged cell; 3D blocks march along z through a rolling
// window of three planes, so every input value is read from global memory
// once per tile.
#include "gpe2p_dev.cuh"
#include "gpe2p_launch.h"

namespace gpe2p {

enum { F_P = 0, F_U = 1, F_V = 2, F_W = 3, F_PHI = 4, F_RHO = 5, F_ETA = 6, F_NU = 7, F_MU = 8, F_N = 9 };

template <typename real, int DIM>
struct FlowOps {
  static constexpr int NPL = DIM == 3 ? 3 : 1;
  using T = Tile<real, NPL>;

  // velocity divergence of the cell at offset (ox,oy,oz), Eq. div-v-discretization
  __device__ __forceinline__ static real div(const T& S, const KParams<real>& P, int ox, int oy, int oz) {
    real d = (S(F_U, ox + 1, oy, oz) - S(F_U, ox, oy, oz)) + (S(F_V, ox, oy + 1, oz) - S(F_V, ox, oy, oz));
    if (DIM == 3) d += S(F_W, ox, oy, oz + 1) - S(F_W, ox, oy, oz);
    return d * P.inv_dx;
  }

  // averaged pressure of the cell at offset o for the gradient along C
  // (Eq. gradp-u-discretization in 2D, Eq. gradp-u-p-ave-3d in 3D)
  template <int C>
  __device__ __forceinline__ static real pbar(const T& S, const KParams<real>& P, int ox, int oy, int oz) {
    if (!P.pavg) return S(F_P, ox, oy, oz);
    if (DIM == 2) {
      constexpr int tx = C == 1, ty = C == 0;
      return (real(4) * S(F_P, ox, oy, oz) + S(F_P, ox + tx, oy + ty, oz) + S(F_P, ox - tx, oy - ty, oz)) *
             real(1.0 / 6.0);
    } else {
      constexpr int T1 = (C + 1) % 3, T2 = (C + 2) % 3;
      constexpr int ax = T1 == 0, ay = T1 == 1, az = T1 == 2;  // unit vector t1
      constexpr int bx = T2 == 0, by = T2 == 1, bz = T2 == 2;  // unit vector t2
      const real s4 = S(F_P, ox + ax, oy + ay, oz + az) + S(F_P, ox - ax, oy - ay, oz - az) +
                      S(F_P, ox + bx, oy + by, oz + bz) + S(F_P, ox - bx, oy - by, oz - bz);
      const real s1 = S(F_P, ox + ax + bx, oy + ay + by, oz + az + bz) +
                      S(F_P, ox - ax - bx, oy - ay - by, oz - az - bz) +
                      S(F_P, ox - ax + bx, oy - ay + by, oz - az + bz) +
                      S(F_P, ox + ax - bx, oy + ay - by, oz + az - bz);
      return (real(16) * S(F_P, ox, oy, oz) + real(4) * s4 + s1) * real(1.0 / 36.0);
    }
  }

  // pressure rate at the cell centre: -rho c_s^2 div u + div(nu grad p)
  __device__ __forceinline__ static real rate_p(const T& S, const KParams<real>& P, real D0) {
    real diff = real(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int ex = a == 0, ey = a == 1, ez = a == 2;
      const real nup = real(0.5) * (S(F_NU, 0, 0, 0) + S(F_NU, ex, ey, ez));
      const real num = real(0.5) * (S(F_NU, 0, 0, 0) + S(F_NU, -ex, -ey, -ez));
      diff += (nup * (S(F_P, ex, ey, ez) - S(F_P, 0, 0, 0)) - num * (S(F_P, 0, 0, 0) - S(F_P, -ex, -ey, -ez))) *
              P.inv_dx2;
    }
    return -S(F_RHO, 0, 0, 0) * P.cs2 * D0 + diff;
  }

  // rate of velocity component C on the cell's low face along C
  template <int C>
  __device__ __forceinline__ static real rate_vel(const T& S, const KParams<real>& P, real D0) {
    constexpr int cx = C == 0, cy = C == 1, cz = C == 2;
    const int FC = F_U + C;
    const real rb = real(0.5) * (S(F_RHO, -cx, -cy, -cz) + S(F_RHO, 0, 0, 0));
    const real gradp = (pbar<C>(S, P, 0, 0, 0) - pbar<C>(S, P, -cx, -cy, -cz)) * P.inv_dx;
    const real uc0 = S(FC, 0, 0, 0);
    const real t_cc = (S(F_ETA, 0, 0, 0) * (S(FC, cx, cy, cz) - uc0) -
                       S(F_ETA, -cx, -cy, -cz) * (uc0 - S(FC, -cx, -cy, -cz))) *
                      P.inv_dx2;
    real t_tr = real(0), conv_tr = real(0);
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
      if (t == C) continue;
      const int tx = t == 0, ty = t == 1, tz = t == 2;
      const int FT = F_U + t;
      const real etp = (S(F_ETA, 0, 0, 0) + S(F_ETA, tx, ty, tz) + S(F_ETA, -cx, -cy, -cz) +
                        S(F_ETA, tx - cx, ty - cy, tz - cz)) *
                       real(0.25);
      const real etm = (S(F_ETA, 0, 0, 0) + S(F_ETA, -tx, -ty, -tz) + S(F_ETA, -cx, -cy, -cz) +
                        S(F_ETA, -tx - cx, -ty - cy, -tz - cz)) *
                       real(0.25);
      const real t_tt = (etp * (S(FC, tx, ty, tz) - uc0) - etm * (uc0 - S(FC, -tx, -ty, -tz))) * P.inv_dx2;
      const real t_tc = (etp * (S(FT, tx, ty, tz) - S(FT, tx - cx, ty - cy, tz - cz)) -
                         etm * (S(FT, 0, 0, 0) - S(FT, -cx, -cy, -cz))) *
                        P.inv_dx2;
      t_tr += t_tt + t_tc;
      const real ubar = (S(FT, 0, 0, 0) + S(FT, -cx, -cy, -cz) + S(FT, tx, ty, tz) +
                         S(FT, tx - cx, ty - cy, tz - cz)) *
                        real(0.25);
      conv_tr += ubar * (S(FC, tx, ty, tz) - S(FC, -tx, -ty, -tz)) * P.inv_2dx;
    }
    real t_b = real(0);
    if (P.bulk) t_b = (S(F_ETA, 0, 0, 0) * D0 - S(F_ETA, -cx, -cy, -cz) * div(S, P, -cx, -cy, -cz)) * P.inv_dx;
    const real st = -P.sigma * (S(F_PHI, 0, 0, 0) + S(F_PHI, -cx, -cy, -cz)) *
                    (S(F_MU, 0, 0, 0) - S(F_MU, -cx, -cy, -cz)) * P.inv_2dx;
    const real grav = (rb - P.rho_ref) * P.g[C];
    const real force = -gradp + real(2) * t_cc + t_tr + t_b + st + grav;
    const real conv = uc0 * (S(FC, cx, cy, cz) - S(FC, -cx, -cy, -cz)) * P.inv_2dx + conv_tr;
    return force / rb - conv;
  }
};

// MODE 0: out = L(q);  MODE 1: out = q + dt L(q);  MODE 2: out = a q0 + b (q + dt L(q))
template <typename real, int DIM, int MODE>
__global__ void __launch_bounds__(NTHR) flow_stage_kernel(const KParams<real> P, const FlowArgs<real> A,
                                                          const int kchunk) {
  constexpr int NPL = DIM == 3 ? 3 : 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  real* sm = reinterpret_cast<real*>(smraw);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int kbeg = DIM == 3 ? blockIdx.z * kchunk : 0;
  const int kend = DIM == 3 ? min(kbeg + kchunk, P.n[2]) : 1;
  const int nx = P.n[0], ny = P.n[1];

  auto load_plane = [&](int kk, int slot) {
    for (int idx = tid; idx < PL; idx += NTHR) {
      const int ly = idx / SX, lx = idx - ly * SX;
      const int gi = clampi(i0 - 1 + lx, -1, nx), gj = clampi(j0 - 1 + ly, -1, ny);
      const real phi = ld_cen(A.phi, P, gi, gj, kk);
      const real rho = rho_of(P, phi), eta = eta_of(P, phi);
      real* b = sm + slot * PL + idx;
      b[(F_P * NPL) * PL] = ld_cen(A.q[0], P, gi, gj, kk);
      b[(F_U * NPL) * PL] = ld_face<0>(A.q[1], P, gi, gj, kk);
      b[(F_V * NPL) * PL] = ld_face<1>(A.q[2], P, gi, gj, kk);
      if (DIM == 3) b[(F_W * NPL) * PL] = ld_face<2>(A.q[3], P, gi, gj, kk);
      b[(F_PHI * NPL) * PL] = phi;
      b[(F_RHO * NPL) * PL] = rho;
      b[(F_ETA * NPL) * PL] = eta;
      b[(F_NU * NPL) * PL] = eta / rho;
      b[(F_MU * NPL) * PL] = ld_cen(A.mu, P, gi, gj, kk);
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
      using Ops = FlowOps<real, DIM>;
      const real D0 = Ops::div(S, P, 0, 0, 0);
      real L[4];
      L[0] = Ops::rate_p(S, P, D0);
      L[1] = (P.bc[0] != BC_PERIODIC && i == 0) ? real(0) : Ops::template rate_vel<0>(S, P, D0);
      L[2] = (P.bc[1] != BC_PERIODIC && j == 0) ? real(0) : Ops::template rate_vel<1>(S, P, D0);
      if (DIM == 3) L[3] = (P.bc[2] != BC_PERIODIC && k == 0) ? real(0) : Ops::template rate_vel<2>(S, P, D0);
      const long long id = lin(P, i, j, k);
      const int F[4] = {F_P, F_U, F_V, F_W};
#pragma unroll
      for (int f = 0; f < DIM + 1; ++f) {
        real o;
        if (MODE == 0) {
          o = L[f];
        } else {
          const real q = S(F[f], 0, 0, 0);
          if (MODE == 1) o = q + P.dt * L[f];
          else o = A.a * A.q0[f][id] + A.b * (q + P.dt * L[f]);
        }
        A.out[f][id] = o;
      }
    }
    __syncthreads();
  }
}

template <typename real, int DIM>
static size_t flow_smem() {
  return sizeof(real) * (size_t)F_N * (DIM == 3 ? 3 : 1) * PL;
}

template <typename real, int DIM>
cudaError_t launch_flow_stage(const KParams<real>& P, const FlowArgs<real>& A, int mode, int kchunk,
                              cudaStream_t s) {
  const size_t sm = flow_smem<real, DIM>();
  dim3 blk(TX, TY, 1);
  dim3 grd((P.n[0] + TX - 1) / TX, (P.n[1] + TY - 1) / TY, DIM == 3 ? (P.n[2] + kchunk - 1) / kchunk : 1);
  cudaError_t e;
#define GPE2P_FLOW_CASE(M)                                                                                \
  e = cudaFuncSetAttribute(flow_stage_kernel<real, DIM, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                           (int)sm);                                                                      \
  if (e != cudaSuccess) return e;                                                                         \
  flow_stage_kernel<real, DIM, M><<<grd, blk, sm, s>>>(P, A, kchunk);
  if (mode == 0) { GPE2P_FLOW_CASE(0) }
  else if (mode == 1) { GPE2P_FLOW_CASE(1) }
  else { GPE2P_FLOW_CASE(2) }
#undef GPE2P_FLOW_CASE
  return cudaGetLastError();
}

template cudaError_t launch_flow_stage<float, 2>(const KParams<float>&, const FlowArgs<float>&, int, int,
                                                 cudaStream_t);
template cudaError_t launch_flow_stage<float, 3>(const KParams<float>&, const FlowArgs<float>&, int, int,
                                                 cudaStream_t);
template cudaError_t launch_flow_stage<double, 2>(const KParams<double>&, const FlowArgs<double>&, int, int,
                                                  cudaStream_t);
template cudaError_t launch_flow_stage<double, 3>(const KParams<double>&, const FlowArgs<double>&, int, int,
                                                  cudaStream_t);

}  // namespace gpe2p
