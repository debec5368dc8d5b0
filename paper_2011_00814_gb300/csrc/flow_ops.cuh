// flow_ops.cuh -- the semi-discrete flow operators of one cell (Sec. 3) and
// the 2D flow stage on one tile, shared by the single-instance and the
// batched 2D kernels so that both compute bit-identical results.
//
//   out = a q^n + b (q + dt L(q)),  q = (p, u, v[, w]),
// with L of Eq. p-u-v-semidiscrete-2d built from Eqs. div-v-discretization,
// diff-p-discretization, conv-u-discretization, u-stress-discretization
// (a)-(d), st-u-discretization, gradp-u-discretization and gradp-u-p-ave-3d,
// phi and mu frozen (Sec. 3, after Eq. tvd-rk3).
//
// The axisymmetric form (2D, KParams::axisym; x = r, y = z, cell column i
// centred at r = (i + 1/2) dx, u face i at r = i dx) adds, as printed in
// Eqs. div-v-axisym, gpe-pressure-two-phase-axisym and
// gpe-momentum-two-phase-axisym-r/-z: u_r / r to the divergence (u_r at the
// centre = mean of its faces), (nu / r) dp/dr to the pressure rate,
// (eta / r)(du_r/dr - u_r / r) to the radial and (eta / r) du_z/dr to the
// axial momentum, with central differences and the face viscosity the mean
// of the two cells the face separates.
#pragma once

#include "gpe2p_dev.cuh"
#include "gpe2p_launch.h"

namespace gpe2p {

enum { F_P = 0, F_U = 1, F_V = 2, F_W = 3, F_PHI = 4, F_RHO = 5, F_ETA = 6, F_NU = 7, F_MU = 8, F_N = 9 };

// The rates below gather every term with its grid factor applied once:
// sums of the four edge viscosities, face velocities and transverse
// pressures are formed unnormalised and scaled together at the end.  Every
// sum of two products is written as the fused multiply-add it is meant to be
// (the compiler could otherwise fuse either product, and two kernels that
// inline this code could round differently).
template <typename real, int DIM, typename T>
struct FlowOps {
  // dx / (2 r) at the centre of the cell column at x offset ox (axisymmetric form, 2D tiles)
  __device__ __forceinline__ static real dx_2r(const T& S, int ox) {
    return fdiv(real(1), real(2 * (S.gi + ox) + 1));
  }

  // velocity divergence of the cell at offset (ox,oy,oz) times dx, Eq. div-v-discretization
  // (plus dx u_r / r, Eq. div-v-axisym, in the axisymmetric form)
  __device__ __forceinline__ static real divsum(const T& S, const KParams<real>& P, int ox, int oy, int oz) {
    real d = (S(F_U, ox + 1, oy, oz) - S(F_U, ox, oy, oz)) + (S(F_V, ox, oy + 1, oz) - S(F_V, ox, oy, oz));
    if constexpr (DIM == 3) {
      d += S(F_W, ox, oy, oz + 1) - S(F_W, ox, oy, oz);
    } else {
      if (P.axisym) d += (S(F_U, ox, oy, oz) + S(F_U, ox + 1, oy, oz)) * dx_2r(S, ox);
    }
    return d;
  }

  // 4 x (eta averaged over the four cells around the edge shared by the faces
  // of components C and t), Eq. u-stress-discretization (eta bar at i, j+-1/2):
  // the edge on the +t side (e4p) and on the -t side (e4m) of the C face
  template <int C>
  __device__ __forceinline__ static void edge_eta4(const T& S, int t, real& e4p, real& e4m) {
    const int cx = C == 0, cy = C == 1, cz = C == 2;
    const int tx = t == 0, ty = t == 1, tz = t == 2;
    if constexpr (DIM == 3) {
      // summed in one order per edge whichever face asks (pairs along the
      // lower axis first), so that the rates of the two components and the
      // two cells that share an edge share its sum
      const int a = C < t ? C : t, b = C < t ? t : C;
      auto e4 = [&](int ox, int oy, int oz) {
        const int ax = a == 0, ay = a == 1, az = a == 2, bx = b == 0, by = b == 1, bz = b == 2;
        return (S(F_ETA, ox, oy, oz) + S(F_ETA, ox + ax, oy + ay, oz + az)) +
               (S(F_ETA, ox + bx, oy + by, oz + bz) + S(F_ETA, ox + ax + bx, oy + ay + by, oz + az + bz));
      };
      e4p = e4(-cx, -cy, -cz);
      e4m = e4(-cx - tx, -cy - ty, -cz - tz);
    } else {
      e4p = (S(F_ETA, 0, 0, 0) + S(F_ETA, tx, ty, tz)) + (S(F_ETA, -cx, -cy, -cz) + S(F_ETA, tx - cx, ty - cy, tz - cz));
      e4m = (S(F_ETA, 0, 0, 0) + S(F_ETA, -tx, -ty, -tz)) +
            (S(F_ETA, -cx, -cy, -cz) + S(F_ETA, -tx - cx, -ty - cy, -tz - cz));
    }
  }

  // whether the pressure gradient averages transversally (Eq. gradp-u-p-ave-3d)
  __device__ __forceinline__ static bool averaged(const KParams<real>& P) {
    if constexpr (T::PAVG == 0) return false;
    else if constexpr (T::PAVG > 0) return true;
    else return P.pavg != 0;
  }

  // the averaged pressure of the cell at offset o for the gradient along C,
  // unnormalised: 6 pbar in 2D (Eq. gradp-u-discretization), 36 pbar in 3D
  template <int C>
  __device__ __forceinline__ static real psum(const T& S, int ox, int oy, int oz) {
    if (DIM == 2) {
      constexpr int tx = C == 1, ty = C == 0;
      return real(4) * S(F_P, ox, oy, oz) + (S(F_P, ox + tx, oy + ty, oz) + S(F_P, ox - tx, oy - ty, oz));
    } else {
      constexpr int T1 = (C + 1) % 3, T2 = (C + 2) % 3;
      constexpr int ax = T1 == 0, ay = T1 == 1, az = T1 == 2;  // unit vector t1
      constexpr int bx = T2 == 0, by = T2 == 1, bz = T2 == 2;  // unit vector t2
      const real s4 = (S(F_P, ox + ax, oy + ay, oz + az) + S(F_P, ox - ax, oy - ay, oz - az)) +
                      (S(F_P, ox + bx, oy + by, oz + bz) + S(F_P, ox - bx, oy - by, oz - bz));
      const real s1 = (S(F_P, ox + ax + bx, oy + ay + by, oz + az + bz) +
                       S(F_P, ox - ax - bx, oy - ay - by, oz - az - bz)) +
                      (S(F_P, ox - ax + bx, oy - ay + by, oz - az + bz) +
                       S(F_P, ox + ax - bx, oy + ay - by, oz + az - bz));
      return real(16) * S(F_P, ox, oy, oz) + (real(4) * s4 + s1);
    }
  }

  // pressure rate at the cell centre: -rho c_s^2 div u + div(nu grad p); d0 = dx div u
  __device__ __forceinline__ static real rate_p(const T& S, const KParams<real>& P, real d0) {
    real diff = real(0);
    const real nu0 = S(F_NU, 0, 0, 0), p0 = S(F_P, 0, 0, 0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int ex = a == 0, ey = a == 1, ez = a == 2;
      diff = fma(nu0 + S(F_NU, ex, ey, ez), S(F_P, ex, ey, ez) - p0, diff);
      diff = fma(nu0 + S(F_NU, -ex, -ey, -ez), S(F_P, -ex, -ey, -ez) - p0, diff);
    }
    if constexpr (DIM == 2) {
      // (nu / r) dp/dr, Eq. gpe-pressure-two-phase-axisym
      if (P.axisym) diff = fma(real(2) * nu0 * (S(F_P, 1, 0, 0) - S(F_P, -1, 0, 0)), dx_2r(S, 0), diff);
    }
    return fma(diff, real(0.5) * P.inv_dx2, -(S(F_RHO, 0, 0, 0) * P.cs2 * mul_rn(d0, P.inv_dx)));
  }

  // rate of velocity component C on the cell's low face along C; d0 = dx div u of the cell
  template <int C>
  __device__ __forceinline__ static real rate_vel(const T& S, const KParams<real>& P, real d0) {
    constexpr int cx = C == 0, cy = C == 1, cz = C == 2;
    const int FC = F_U + C;
    const real rb2 = S(F_RHO, -cx, -cy, -cz) + S(F_RHO, 0, 0, 0);   // 2 rho on the face
    real gradp;
    if (averaged(P))
      gradp = (psum<C>(S, 0, 0, 0) - psum<C>(S, -cx, -cy, -cz)) *
              (P.inv_dx * real(DIM == 2 ? 1.0 / 6.0 : 1.0 / 36.0));
    else
      gradp = (S(F_P, 0, 0, 0) - S(F_P, -cx, -cy, -cz)) * P.inv_dx;
    const real uc0 = S(FC, 0, 0, 0);
    const real tcc = fma(S(F_ETA, -cx, -cy, -cz), S(FC, -cx, -cy, -cz) - uc0,
                         mul_rn(S(F_ETA, 0, 0, 0), S(FC, cx, cy, cz) - uc0));
    real edge = real(0), conv4 = real(0);
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
      if (t == C) continue;
      const int tx = t == 0, ty = t == 1, tz = t == 2;
      const int FT = F_U + t;
      real e4p, e4m;
      edge_eta4<C>(S, t, e4p, e4m);
      const real ucp = S(FC, tx, ty, tz), ucm = S(FC, -tx, -ty, -tz);
      const real ut0 = S(FT, 0, 0, 0), utc = S(FT, -cx, -cy, -cz);
      const real utp = S(FT, tx, ty, tz), utpc = S(FT, tx - cx, ty - cy, tz - cz);
      edge = fma(e4p, (ucp - uc0) + (utp - utpc), edge);
      edge = fma(e4m, (ucm - uc0) + (utc - ut0), edge);
      conv4 = fma((ut0 + utc) + (utp + utpc), ucp - ucm, conv4);
    }
    real visc = fma(real(2), tcc, mul_rn(real(0.25), edge));
    if (P.bulk) {
      visc = fma(S(F_ETA, 0, 0, 0), d0, visc);
      visc = fma(-S(F_ETA, -cx, -cy, -cz), divsum(S, P, -cx, -cy, -cz), visc);
    }
    if constexpr (DIM == 2) {
      if (P.axisym) {
        const real eta_f = real(0.5) * (S(F_ETA, -cx, -cy, 0) + S(F_ETA, 0, 0, 0));
        const real dudr2 = S(FC, 1, 0, 0) - S(FC, -1, 0, 0);  // 2 dx du_c/dr
        if (C == 0) {
          // (eta / r)(du_r/dr - u_r / r) on the u face i, r = i dx (i >= 1)
          const real ir = fdiv(real(1), real(S.gi));
          visc = fma(mul_rn(eta_f, ir), fma(real(0.5), dudr2, -mul_rn(uc0, ir)), visc);
        } else {
          // (eta / r) du_z/dr on the v face of column i, r = (i + 1/2) dx
          visc = fma(mul_rn(eta_f, dudr2), dx_2r(S, 0), visc);
        }
      }
    }
    const real st = -P.sigma * (S(F_PHI, 0, 0, 0) + S(F_PHI, -cx, -cy, -cz)) *
                    (S(F_MU, 0, 0, 0) - S(F_MU, -cx, -cy, -cz));
    const real grav = fma(real(0.5), rb2, -P.rho_ref);
    real force = fma(visc, P.inv_dx2, -gradp);
    force = fma(st, P.inv_2dx, force);
    force = fma(grav, P.g[C], force);
    const real conv = fma(uc0, S(FC, cx, cy, cz) - S(FC, -cx, -cy, -cz), mul_rn(real(0.25), conv4));
    return fma(-conv, P.inv_2dx, fdiv(real(2) * force, rb2));
  }
};

// 2D tile accessor: NF staged fields of (TXv+2) x (TYv+2) elements
template <typename real, int SXv, int PLv>
struct Tile2 {
  static constexpr int PAVG = -1;  // pressure averaging decided at run time
  const real* sm;
  int c;   // the thread's cell within a staged field
  int gi;  // its global column index (the radius of the axisymmetric form)
  __device__ __forceinline__ real operator()(int f, int dx, int dy, int) const {
    return sm[f * PLv + c + dy * SXv + dx];
  }
};

// Whether the one-cell halo of the TXv x TYv tile at (i0, j0) lies inside
// the domain, so that its staged values need no boundary map: every staged
// cell (gi, gj) then has 0 <= gi < nx and 0 <= gj < ny, and a face value on
// it is the stored one (the wall faces 0 of a walled axis lie outside such a
// halo, since i0, j0 >= 1).
template <typename real, int TXv, int TYv>
__device__ __forceinline__ bool tile_interior(const KParams<real>& P, int i0, int j0) {
  return i0 >= 1 && i0 + TXv + 1 <= P.n[0] && j0 >= 1 && j0 + TYv + 1 <= P.n[1];
}

// The staged region of a 2D tile, (TXv + 2) x (TYv + 2) cells, spread over
// the block's threads.  fn(e, lx, ly, off) is called for every staged cell
// e = ly (TXv + 2) + lx, i.e. the cell (i0 - 1 + lx, j0 - 1 + ly); off is its
// element offset when the tile is interior (every staged cell inside the
// domain; formed from one per-tile base in 32-bit arithmetic), else -1.
template <typename real, int TXv, int TYv, typename Fn>
__device__ __forceinline__ void stage2d(const KParams<real>& P, int i0, int j0, bool interior, Fn fn) {
  constexpr int SXv = TXv + 2, PLv = SXv * (TYv + 2), NT = TXv * TYv / 2;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const long long base = interior ? lin(P, i0 - 1, j0 - 1, 0) : -1LL;
  const int sy = (int)P.sy;
  for (int e = tid; e < PLv; e += NT) {
    const int ly = e / SXv, lx = e - ly * SXv;
    fn(e, lx, ly, interior ? base + (ly * sy + lx) : -1LL);
  }
}

// MODE 0: out = L(q);  MODE 1: out = q + dt L(q);  MODE 2: out = a q0 + b (q + dt L(q)).
// One 2D flow stage on the tile of TXv x TYv cells at (i0, j0), by a block of
// TXv*TYv/2 threads: thread t computes the cells (t % TXv, 2 (t / TXv) + r),
// r = 0, 1, whose stencils share most of their staged values.  The block
// stages p, u, v, phi, rho, eta, nu = eta/rho and mu with a one-cell halo in
// sm, F_N * (TXv+2)*(TYv+2) reals: straight from the fields on an interior
// tile, through the boundary maps (ghosts) on a tile at the domain's edge.
// With A.usum set (MODE 2, the last stage), it also stores u^n + u^{n+1} on
// the cells' faces, from which the CH step forms the time-centred velocity.
template <typename real, int MODE, int TXv, int TYv>
__device__ __forceinline__ void flow2d_tile(const KParams<real>& P, const FlowArgs<real>& A, int i0, int j0,
                                            real* sm) {
  constexpr int SXv = TXv + 2, SYv = TYv + 2, PLv = SXv * SYv;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int tx = tid % TXv, ty = tid / TXv;
  const int nx = P.n[0], ny = P.n[1];
  const int i = i0 + tx;
  // q^n at the thread's cells, loaded first so that its latency overlaps the staging
  real q0v[2][3];
  if (MODE == 2) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int j = j0 + 2 * ty + r;
      const bool act = i < nx && j < ny;
#pragma unroll
      for (int f = 0; f < 3; ++f) q0v[r][f] = act ? A.q0[f][lin(P, i, j, 0)] : real(0);
    }
  }
  stage2d<real, TXv, TYv>(P, i0, j0, tile_interior<real, TXv, TYv>(P, i0, j0),
                          [&](int e, int lx, int ly, long long q) {
    real pv, uv, vv, phi, muv;
    if (q >= 0) {
      pv = A.q[0][q];
      uv = A.q[1][q];
      vv = A.q[2][q];
      phi = A.phi[q];
      muv = A.mu[q];
    } else {
      const int gi = clampi(i0 - 1 + lx, -1, nx), gj = clampi(j0 - 1 + ly, -1, ny);
      pv = ld_cen(A.q[0], P, gi, gj, 0);
      uv = ld_face<0>(A.q[1], P, gi, gj, 0);
      vv = ld_face<1>(A.q[2], P, gi, gj, 0);
      phi = ld_cen(A.phi, P, gi, gj, 0);
      muv = ld_cen(A.mu, P, gi, gj, 0);
    }
    const real rho = rho_of(P, phi), eta = eta_of(P, phi);
    real* b = sm + e;
    b[F_P * PLv] = pv;
    b[F_U * PLv] = uv;
    b[F_V * PLv] = vv;
    b[F_PHI * PLv] = phi;
    b[F_RHO * PLv] = rho;
    b[F_ETA * PLv] = eta;
    b[F_NU * PLv] = fdiv(eta, rho);
    b[F_MU * PLv] = muv;
  });
  __syncthreads();
  real out[2][3];
  using Ops = FlowOps<real, 2, Tile2<real, SXv, PLv>>;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int j = j0 + 2 * ty + r;
    Tile2<real, SXv, PLv> S;
    S.sm = sm;
    S.c = (2 * ty + r + 1) * SXv + (tx + 1);
    S.gi = i;
    const real D0 = Ops::divsum(S, P, 0, 0, 0);
    real L[3];
    L[0] = Ops::rate_p(S, P, D0);
    L[1] = (P.bc[0] != BC_PERIODIC && i == 0) ? real(0) : Ops::template rate_vel<0>(S, P, D0);
    L[2] = (P.bc[1] != BC_PERIODIC && j == 0) ? real(0) : Ops::template rate_vel<1>(S, P, D0);
    const int F[3] = {F_P, F_U, F_V};
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      if (MODE == 0) {
        out[r][f] = L[f];
      } else {
        const real q = S(F[f], 0, 0, 0);
        const real s1 = fma(P.dt, L[f], q);
        if (MODE == 1) out[r][f] = s1;
        else out[r][f] = fma(A.a, q0v[r][f], mul_rn(A.b, s1));
      }
    }
  }
  // stores after both cells, so that nothing separates their shared loads
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int j = j0 + 2 * ty + r;
    if (i < nx && j < ny) {
      const long long id = lin(P, i, j, 0);
#pragma unroll
      for (int f = 0; f < 3; ++f) A.out[f][id] = out[r][f];
      if (MODE == 2 && A.usum[0]) {
        A.usum[0][id] = q0v[r][1] + out[r][1];
        A.usum[1][id] = q0v[r][2] + out[r][2];
      }
    }
  }
  __syncthreads();
}

}  // namespace gpe2p
