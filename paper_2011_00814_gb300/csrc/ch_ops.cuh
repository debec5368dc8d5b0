// ch_ops.cuh -- the Cahn-Hilliard step of one cell (Sec. 3): chemical
// potential (Eq. chem-pot), one RK stage of Eq. che with the isotropic
// stencils of Eqs. 1st-der-iso and laplacian-iso, the time-centred cell
// velocity of Eq. u-center-2d; and the 2D CH stage and mu on one tile, shared
// by the single-instance and the batched 2D kernels.
#pragma once

#include "flow_ops.cuh"
#include "gpe2p_dev.cuh"
#include "gpe2p_launch.h"

namespace gpe2p {

// which lattice shells a model uses: D2Q9 {1,2}, D3Q15 {1,3}, D3Q19 {1,2}, D3Q27 {1,2,3}
template <int ISO>
struct Shells {
  static constexpr bool s2 = ISO == 9 || ISO == 19 || ISO == 27;
  static constexpr bool s3 = ISO == 15 || ISO == 27;
};

// Eq. laplacian-iso written as sum_i w_i (f(x + e_i) - f(x)) (the same
// operator, since the non-rest weights sum to 1 - w0): every difference
// enters the two cells it joins with opposite signs and the same weight, so
// the Laplacian sums to zero over a periodic grid in any precision, which
// keeps the Cahn-Hilliard update conservative in FP32 as well
template <typename real, int DIM, int ISO, typename T>
__device__ __forceinline__ real lap_iso(const T& S, const KParams<real>& P, int f) {
  real s = real(0);
  const real f0 = S(f, 0, 0, 0);
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
        s += shell_w(P, sh) * (S(f, dx, dy, dz) - f0);
      }
  return P.lap_c * s;
}

// the same operator as a weighted sum per shell, sum_s w_s (sum_{|e|^2 = s}
// f(x + e) - n_s f(x)): fewer operations, but rounding that depends on the
// cell, so the Laplacians it sums need not cancel over the grid.  For mu,
// which nothing conserves.
template <typename real, int DIM, int ISO, typename T>
__device__ __forceinline__ real lap_iso_shells(const T& S, const KParams<real>& P, int f) {
  real s1 = real(0), s2 = real(0), s3 = real(0);
  const real f0 = S(f, 0, 0, 0);
#pragma unroll
  for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int sh = dx * dx + dy * dy + dz * dz;
        if (sh == 1) s1 += S(f, dx, dy, dz);
        if (sh == 2 && Shells<ISO>::s2) s2 += S(f, dx, dy, dz);
        if (sh == 3 && Shells<ISO>::s3) s3 += S(f, dx, dy, dz);
      }
  real s = P.w1 * fma(real(-2 * DIM), f0, s1);
  if (Shells<ISO>::s2) s = fma(P.w2, fma(real(DIM == 3 ? -12 : -4), f0, s2), s);
  if (Shells<ISO>::s3) s = fma(P.w3, fma(real(-8), f0, s3), s);
  return P.lap_c * s;
}

// the DIM components of the isotropic gradient of staged field f
template <typename real, int DIM, int ISO, typename T>
__device__ __forceinline__ void grad_iso(const T& S, const KParams<real>& P, int f, real g[3]) {
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

// (1/r) df/dr of the axisymmetric form (Eqs. che-axisym, chem-pot-axisym) at
// the cell of a 2D tile, column i at r = (i + 1/2) dx: the x component of the
// D2Q9 isotropic gradient over r
template <typename real, typename T>
__device__ __forceinline__ real axis_grad_over_r(const T& S, const KParams<real>& P, int f) {
  const real sx = fma(P.w1, S(f, 1, 0, 0) - S(f, -1, 0, 0),
                      mul_rn(P.w2, (S(f, 1, 1, 0) - S(f, -1, 1, 0)) + (S(f, 1, -1, 0) - S(f, -1, -1, 0))));
  return mul_rn(mul_rn(P.grad_c, sx), fdiv(real(2) * P.inv_dx, real(2 * S.gi + 1)));
}

enum { C_PHI = 0, C_MU = 1, C_UH = 2, C_N = 5 };

// face value of component C on the high face of cell (i,j,k) (the low face of
// the next cell along C): zero on a wall, wrapped when periodic
template <int C, typename real>
__device__ __forceinline__ real face_next(const real* __restrict__ f, const KParams<real>& P, int i, int j, int k,
                                          long long id) {
  const int x = C == 0 ? i : (C == 1 ? j : k);
  const long long st = C == 0 ? 1 : (C == 1 ? P.sy : P.sz);
  if (x + 1 < P.n[C]) return f[id + st];
  if (P.bc[C] == BC_PERIODIC) return f[id + st - (long long)P.n[C] * st];
  return real(0);
}

// the values a CH stage reads at the cell itself (no halo): the stage-1
// time-centred velocity from the two face velocities (Eq. u-center-2d) or the
// stored one, phi^{n+1/2} and the RK4 accumulator; loaded before the stencil
// so that their latency overlaps the wait for the staged planes
template <typename real>
struct CHPoint {
  real uh[3];
  real pn, acc;
  real pnl;  // low part of phi^{n+1/2} (compensated accumulation)
};

// USUM: the stage-1 uhat from the face sums u^n + u^{n+1} the last flow stage
// left in A.usum: uhat_a = (s_a + s_a(+e_a)) / 4
template <typename real, int DIM, bool USUM = false>
__device__ __forceinline__ void ch_point_load(const KParams<real>& P, const CHArgs<real>& A, int i, int j, int k,
                                              CHPoint<real>& c) {
  const long long id = lin(P, i, j, k);
  if (!A.conservative) {
    if (USUM) {
      c.uh[0] = real(0.25) * (A.usum[0][id] + face_next<0>(A.usum[0], P, i, j, k, id));
      c.uh[1] = real(0.25) * (A.usum[1][id] + face_next<1>(A.usum[1], P, i, j, k, id));
      if (DIM == 3) c.uh[2] = real(0.25) * (A.usum[2][id] + face_next<2>(A.usum[2], P, i, j, k, id));
    } else if (A.compute_uh) {
      c.uh[0] = real(0.25) * ((A.u0[0][id] + face_next<0>(A.u0[0], P, i, j, k, id)) +
                              (A.u1[0][id] + face_next<0>(A.u1[0], P, i, j, k, id)));
      c.uh[1] = real(0.25) * ((A.u0[1][id] + face_next<1>(A.u0[1], P, i, j, k, id)) +
                              (A.u1[1][id] + face_next<1>(A.u1[1], P, i, j, k, id)));
      if (DIM == 3)
        c.uh[2] = real(0.25) * ((A.u0[2][id] + face_next<2>(A.u0[2], P, i, j, k, id)) +
                                (A.u1[2][id] + face_next<2>(A.u1[2], P, i, j, k, id)));
    } else {
      for (int a = 0; a < DIM; ++a) c.uh[a] = A.uh[a][id];
    }
  }
  // (USUM: phi^{n+1/2} is phi_s itself, which the caller takes from its tile)
  if (A.stage != 0 && !USUM) c.pn = A.phin[id];
  c.pnl = (A.phi_lo && A.stage != 0) ? A.phi_lo[id] : real(0);
  // RK4 stages 2-4 read the accumulated increments; with the compensated
  // accumulation the RK2 stage 2 reads the increment of stage 1
  if ((A.scheme == 4 && A.stage >= 2) || (A.phi_lo && A.scheme == 2 && A.stage == 2)) c.acc = A.acc[id];
}

// the CH rate of one cell: -uhat.grad(phi_s) + M lap(mu_s), or its conservative form
template <typename real, int DIM, int ISO, typename T>
__device__ __forceinline__ real ch_rate(const T& S, const KParams<real>& P, const CHArgs<real>& A,
                                       const CHPoint<real>& c) {
  real lapmu = lap_iso<real, DIM, ISO>(S, P, C_MU);
  if constexpr (DIM == 2) {
    if (P.axisym) lapmu = add_rn(lapmu, axis_grad_over_r(S, P, C_MU));
  }
  real adv = real(0);
  if (!A.conservative) {
    real g[3];
    grad_iso<real, DIM, ISO>(S, P, C_PHI, g);
#pragma unroll
    for (int a = 0; a < DIM; ++a) adv += c.uh[a] * g[a];
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
  return -adv + P.M * lapmu;
}

// the RK combination of a CH stage for one cell with rate L (phis0 = phi_s
// at the cell) and its stores; also stores the stage-1 cell velocity
template <typename real, int DIM>
__device__ __forceinline__ void ch_finish(const KParams<real>& P, const CHArgs<real>& A, long long id,
                                          const CHPoint<real>& c, real L, real phis0) {
  if (!A.conservative && A.compute_uh && A.stage != 0)
    for (int a = 0; a < DIM; ++a) A.uh[a][id] = c.uh[a];
  real o;
  const bool last = A.stage == A.scheme;
  if (A.phi_lo && last) {
    // phi^{n+3/2} in FP64 from the high/low pair of phi^{n+1/2} and the stage
    // increments (never from a rounded stage state), stored back as a pair:
    // RK2 phi^n + (d1 + d2)/2, RK4 phi^n + (d1 + 2 d2 + 2 d3 + d4)/6
    const double pn = (double)c.pn + (double)c.pnl;
    const real d = P.dt * L;
    double od;
    if (A.scheme == 2) od = pn + 0.5 * ((double)c.acc + (double)d);
    else od = fma((double)c.acc + (double)d, 1.0 / 6.0, pn);
    const real hi = (real)od;
    A.phi_lo[id] = (real)(od - (double)hi);
    A.out[id] = hi;
    return;
  }
  if (A.stage == 0) {
    o = L;
  } else if (A.scheme == 2) {
    // explicit fused multiply-adds: the kernels that share this code round alike
    if (A.stage == 1) {
      o = fma(P.dt, L, c.pn);
      if (A.phi_lo) A.acc[id] = P.dt * L;
    } else {
      o = fma(real(0.5), c.pn, real(0.5) * fma(P.dt, L, phis0));
    }
  } else {
    const real d = P.dt * L;
    const real pn = c.pn;
    if (A.stage == 1) { A.acc[id] = d; o = pn + real(0.5) * d; }
    else if (A.stage == 2) { A.acc[id] = c.acc + real(2) * d; o = pn + real(0.5) * d; }
    else if (A.stage == 3) { A.acc[id] = c.acc + real(2) * d; o = pn + d; }
    else { o = fma(c.acc + d, real(1.0 / 6.0), pn); }  // a multiply, not an IEEE divide
  }
  A.out[id] = o;
}

// one cell of a CH stage: rate and RK combination
template <typename real, int DIM, int ISO, typename T>
__device__ __forceinline__ void ch_cell(const T& S, const KParams<real>& P, const CHArgs<real>& A, int i, int j,
                                        int k, const CHPoint<real>& c) {
  ch_finish<real, DIM>(P, A, lin(P, i, j, k), c, ch_rate<real, DIM, ISO>(S, P, A, c), S(C_PHI, 0, 0, 0));
}

// One 2D CH stage on the tile of TXv x TYv cells at (i0, j0), by a block of
// TXv*TYv/2 threads (thread t computes the cells (t % TXv, 2 (t / TXv) + r),
// r = 0, 1).  sm holds C_N * (TXv+2)*(TYv+2) reals, staged straight from the
// fields on an interior tile and through the boundary maps at the edges.
// Stage 1 of the advective form with A.usum set forms the time-centred
// velocity from the face sums u^n + u^{n+1} the last flow stage left.
template <typename real, int TXv, int TYv>
__device__ __forceinline__ void ch2d_tile(const KParams<real>& P, const CHArgs<real>& A, int i0, int j0,
                                          real* sm) {
  constexpr int SXv = TXv + 2, SYv = TYv + 2, PLv = SXv * SYv;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int tx = tid % TXv, ty = tid / TXv;
  const int nx = P.n[0], ny = P.n[1];
  const bool cons = A.conservative != 0;
  const bool usum = !cons && A.usum[0] && A.stage == 1;
  const int i = i0 + tx;
  // the per-cell values, loaded first so that their latency overlaps the staging
  CHPoint<real> c[2] = {};
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int j = j0 + 2 * ty + r;
    if (i < nx && j < ny) {
      if (usum) ch_point_load<real, 2, true>(P, A, i, j, 0, c[r]);
      else ch_point_load<real, 2>(P, A, i, j, 0, c[r]);
    }
  }
  stage2d<real, TXv, TYv>(P, i0, j0, tile_interior<real, TXv, TYv>(P, i0, j0),
                          [&](int e, int lx, int ly, long long q) {
    real* b = sm + e;
    if (q >= 0) {
      b[C_PHI * PLv] = A.phis[q];
      b[C_MU * PLv] = A.mus[q];
      if (cons) {
        b[(C_UH + 0) * PLv] = A.uh[0][q];
        b[(C_UH + 1) * PLv] = A.uh[1][q];
      }
    } else {
      const int gi = clampi(i0 - 1 + lx, -1, nx), gj = clampi(j0 - 1 + ly, -1, ny);
      b[C_PHI * PLv] = ld_cen(A.phis, P, gi, gj, 0);
      b[C_MU * PLv] = ld_cen(A.mus, P, gi, gj, 0);
      if (cons) {
        b[(C_UH + 0) * PLv] = ld_cvec<0>(A.uh[0], P, gi, gj, 0);
        b[(C_UH + 1) * PLv] = ld_cvec<1>(A.uh[1], P, gi, gj, 0);
      }
    }
  });
  __syncthreads();
  real L[2], ph0[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    Tile2<real, SXv, PLv> S;
    S.sm = sm;
    S.c = (2 * ty + r + 1) * SXv + (tx + 1);
    S.gi = i;
    L[r] = ch_rate<real, 2, 9>(S, P, A, c[r]);
    ph0[r] = S(C_PHI, 0, 0, 0);
    if (usum) c[r].pn = ph0[r];  // stage 1: phi^{n+1/2} = phi_s
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int j = j0 + 2 * ty + r;
    if (i < nx && j < ny) ch_finish<real, 2>(P, A, lin(P, i, j, 0), c[r], L[r], ph0[r]);
  }
  __syncthreads();
}

// mu of a 2D tile (Eq. chem-pot with the D2Q9 Laplacian) by TXv*TYv/2 threads,
// two cells each; sm holds (TXv+2)*(TYv+2) reals
template <typename real, int TXv, int TYv>
__device__ __forceinline__ void mu2d_tile(const KParams<real>& P, const real* __restrict__ phi,
                                          real* __restrict__ mu, int i0, int j0, real* sm) {
  constexpr int SXv = TXv + 2, PLv = SXv * (TYv + 2);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int tx = tid % TXv, ty = tid / TXv;
  const int nx = P.n[0], ny = P.n[1];
  stage2d<real, TXv, TYv>(P, i0, j0, tile_interior<real, TXv, TYv>(P, i0, j0),
                          [&](int e, int lx, int ly, long long q) {
    if (q >= 0) {
      sm[e] = phi[q];
    } else {
      const int gi = clampi(i0 - 1 + lx, -1, nx), gj = clampi(j0 - 1 + ly, -1, ny);
      sm[e] = ld_cen(phi, P, gi, gj, 0);
    }
  });
  __syncthreads();
  const int i = i0 + tx;
  real out[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    Tile2<real, SXv, PLv> S;
    S.sm = sm;
    S.c = (2 * ty + r + 1) * SXv + (tx + 1);
    S.gi = i;
    const real f = S(0, 0, 0, 0);
    real lap = lap_iso<real, 2, 9>(S, P, 0);
    if (P.axisym) lap = add_rn(lap, axis_grad_over_r(S, P, 0));  // Eq. chem-pot-axisym
    out[r] = fma(P.a4 * f, fma(f, f, real(-1)), -(P.kappa * lap));
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int j = j0 + 2 * ty + r;
    if (i < nx && j < ny) mu[lin(P, i, j, 0)] = out[r];
  }
  __syncthreads();
}

}  // namespace gpe2p
