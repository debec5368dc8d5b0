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
#include "ring3d.cuh"

// Whether the 3D flow stage precomputes the divergence and the edge
// viscosities per staged cell (fewer instructions per cell, but four more
// shared-memory planes per derived slot, which costs occupancy).
#ifndef GPE2P_FLOW_PRECOMPUTE
#define GPE2P_FLOW_PRECOMPUTE 0
#endif

namespace gpe2p {

enum { F_P = 0, F_U = 1, F_V = 2, F_W = 3, F_PHI = 4, F_RHO = 5, F_ETA = 6, F_NU = 7, F_MU = 8, F_N = 9 };
// precomputed per-cell quantities offered by the 3D ring accessor: the
// divergence of the cell and the viscosity of the cell's low edge in each
// coordinate plane (mean of eta over the four cells around the edge)
enum { F_DIV = 9, F_EXY = 10, F_EXZ = 11, F_EYZ = 12 };

// accessors that stage only the raw fields (the 2D plane kernel)
template <typename T>
struct HasPre {
  static constexpr bool value = false;
};

template <typename real, int DIM, typename T>
struct FlowOps {
  static constexpr bool PRE = HasPre<T>::value;

  // velocity divergence of the cell at offset (ox,oy,oz), Eq. div-v-discretization
  __device__ __forceinline__ static real div(const T& S, const KParams<real>& P, int ox, int oy, int oz) {
    if constexpr (PRE) {
      return S(F_DIV, ox, oy, oz);
    } else {
      real d = (S(F_U, ox + 1, oy, oz) - S(F_U, ox, oy, oz)) + (S(F_V, ox, oy + 1, oz) - S(F_V, ox, oy, oz));
      if (DIM == 3) d += S(F_W, ox, oy, oz + 1) - S(F_W, ox, oy, oz);
      return d * P.inv_dx;
    }
  }

  // eta averaged over the four cells around the edge shared by the faces of
  // components C and t (Eq. u-stress-discretization, eta bar at i, j+-1/2):
  // the edge on the +t side (etp) or on the -t side (etm) of the C face
  template <int C>
  __device__ __forceinline__ static void edge_eta(const T& S, int t, real& etp, real& etm) {
    const int cx = C == 0, cy = C == 1, cz = C == 2;
    const int tx = t == 0, ty = t == 1, tz = t == 2;
    if constexpr (PRE) {
      const int a = C < t ? C : t, b = C < t ? t : C;
      const int FE = (a == 0 && b == 1) ? F_EXY : ((a == 0 && b == 2) ? F_EXZ : F_EYZ);
      etp = S(FE, tx, ty, tz);
      etm = S(FE, 0, 0, 0);
    } else {
      etp = (S(F_ETA, 0, 0, 0) + S(F_ETA, tx, ty, tz) + S(F_ETA, -cx, -cy, -cz) +
             S(F_ETA, tx - cx, ty - cy, tz - cz)) *
            real(0.25);
      etm = (S(F_ETA, 0, 0, 0) + S(F_ETA, -tx, -ty, -tz) + S(F_ETA, -cx, -cy, -cz) +
             S(F_ETA, -tx - cx, -ty - cy, -tz - cz)) *
            real(0.25);
    }
  }

  // averaged pressure of the cell at offset o for the gradient along C
  // (Eq. gradp-u-discretization in 2D, Eq. gradp-u-p-ave-3d in 3D)
  template <int C>
  __device__ __forceinline__ static real pbar(const T& S, const KParams<real>& P, int ox, int oy, int oz) {
    if constexpr (T::PAVG == 0) {
      return S(F_P, ox, oy, oz);
    } else if constexpr (T::PAVG < 0) {
      if (!P.pavg) return S(F_P, ox, oy, oz);
    }
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
      real etp, etm;
      edge_eta<C>(S, t, etp, etm);
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
    return fdiv(force, rb) - conv;
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
      b[(F_NU * NPL) * PL] = fdiv(eta, rho);
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
      using Ops = FlowOps<real, DIM, Tile<real, NPL>>;
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

// ---------------------------------------------------------------------------
// 3D: the same stage fed by the TMA plane ring of ring3d.cuh
// ---------------------------------------------------------------------------

// raw (copied) fields of the ring and the derived planes rho, eta, nu, the
// divergence and the three edge viscosities
enum { R_P = 0, R_U = 1, R_V = 2, R_W = 3, R_PHI = 4, R_MU = 5, NRAW_FLOW = 6 };
enum { D_RHO = 0, D_ETA = 1, D_NU = 2, D_DIV = 3, D_EXY = 4, D_EXZ = 5, D_EYZ = 6 };
constexpr int NDER_FLOW = GPE2P_FLOW_PRECOMPUTE ? 7 : 3;

template <typename real, int PAVG_>
struct RingTile {
  static constexpr int PAVG = PAVG_;
  using G = RingGeom<real>;
  const real* sm;  // the block's shared memory
  int r[3];        // index of the thread's cell in raw field 0 of planes k-1, k, k+1
  int d[3];        // index of the thread's cell in derived field 0 of planes k-1, k, k+1
  __device__ __forceinline__ real operator()(int f, int dx, int dy, int dz) const {
    const int o = dy * G::BX + dx;
    switch (f) {
      case F_P: return sm[r[dz + 1] + R_P * G::PE + o];
      case F_U: return sm[r[dz + 1] + R_U * G::PE + o];
      case F_V: return sm[r[dz + 1] + R_V * G::PE + o];
      case F_W: return sm[r[dz + 1] + R_W * G::PE + o];
      case F_PHI: return sm[r[dz + 1] + R_PHI * G::PE + o];
      case F_MU: return sm[r[dz + 1] + R_MU * G::PE + o];
      case F_RHO: return sm[d[dz + 1] + D_RHO * G::PE + o];
      case F_ETA: return sm[d[dz + 1] + D_ETA * G::PE + o];
      case F_NU: return sm[d[dz + 1] + D_NU * G::PE + o];
      case F_DIV: return sm[d[dz + 1] + D_DIV * G::PE + o];
      case F_EXY: return sm[d[dz + 1] + D_EXY * G::PE + o];
      case F_EXZ: return sm[d[dz + 1] + D_EXZ * G::PE + o];
      default: return sm[d[dz + 1] + D_EYZ * G::PE + o];
    }
  }
};
template <typename real, int PAVG_>
struct HasPre<RingTile<real, PAVG_>> {
  static constexpr bool value = GPE2P_FLOW_PRECOMPUTE != 0;
};

template <typename real, int MODE, int RING, int PAVG>
__global__ void __launch_bounds__(NTHR, 2) flow3d_kernel(const __grid_constant__ Maps<NRAW_FLOW> maps,
                                                      const KParams<real> P, const FlowArgs<real> A,
                                                      const int kchunk, int* err) {
  using G = RingGeom<real>;
  extern __shared__ __align__(128) unsigned char smraw[];
  Ring<real, NRAW_FLOW, RING> R;
  unsigned char* sbase = smem_base128(smraw);
  R.bar = reinterpret_cast<uint64_t*>(sbase);
  R.raw = reinterpret_cast<real*>(sbase + 128);
  real* der = R.raw + (size_t)RING * NRAW_FLOW * G::PE;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(kbeg + kchunk, P.n[2]);
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
  const bool edge_tile = i0 == 0 || i0 + TX + 1 > nx || j0 == 0 || j0 + TY + 1 > ny;
  const int i = i0 + tx, j = j0 + ty;
  const bool active = i < nx && j < ny;
  auto dplane = [&](int kk) { return der + (size_t)((unsigned)(kk + 4) & 3u) * NDER_FLOW * G::PE; };

  R.start(P, maps.m, kbeg, kend, i0, j0);

  // wait for plane kk; overwrite its out-of-domain cells; derive rho, eta, nu
  // of plane kk, then the divergence of plane kk - 1 and the edge viscosities
  // of plane kk
  auto acquire = [&](int kk, bool refill) -> bool {
    if (!R.wait(kk)) return false;
    if (refill && tid == 0) R.refill(P, maps.m, kk);
    const bool ghost_plane = kk < 0 || kk >= nz;
    real* pl[NRAW_FLOW];
#pragma unroll
    for (int f = 0; f < NRAW_FLOW; ++f) pl[f] = R.plane(kk, f);
    real* dk = dplane(kk);
    for (int idx = tid; idx < SX * SY; idx += NTHR) {
      const int ly = idx / SX, lx = idx - ly * SX;
      const int e = G::at(lx, ly);
      if (ghost_plane || edge_tile) {
        const int gi = i0 - 1 + lx, gj = j0 - 1 + ly;
        if (ghost_plane || gi < 0 || gi >= nx || gj < 0 || gj >= ny) {
          const int ci = clampi(gi, -1, nx), cj = clampi(gj, -1, ny);
          pl[R_P][e] = ld_cen(A.q[0], P, ci, cj, kk);
          pl[R_U][e] = ld_face<0>(A.q[1], P, ci, cj, kk);
          pl[R_V][e] = ld_face<1>(A.q[2], P, ci, cj, kk);
          pl[R_W][e] = ld_face<2>(A.q[3], P, ci, cj, kk);
          pl[R_PHI][e] = ld_cen(A.phi, P, ci, cj, kk);
          pl[R_MU][e] = ld_cen(A.mu, P, ci, cj, kk);
        }
      }
      const real phi = pl[R_PHI][e];
      const real rho = rho_of(P, phi), eta = eta_of(P, phi);
      dk[D_RHO * G::PE + e] = rho;
      dk[D_ETA * G::PE + e] = eta;
      dk[D_NU * G::PE + e] = fdiv(eta, rho);
    }
    if (ghost_plane || edge_tile) fence_proxy_async_smem();
    if (!GPE2P_FLOW_PRECOMPUTE) return true;
    __syncthreads();
    const bool have_prev = kk > R.first;
    const real* um = R.plane(kk - 1, R_U);
    const real* vm = R.plane(kk - 1, R_V);
    const real* wm = R.plane(kk - 1, R_W);
    const real* wk = pl[R_W];
    real* dm = dplane(kk - 1);
    const real* em = dplane(kk - 1) + D_ETA * G::PE;
    const real* ek = dk + D_ETA * G::PE;
    for (int idx = tid; idx < SX * SY; idx += NTHR) {
      const int ly = idx / SX, lx = idx - ly * SX;
      const int e = G::at(lx, ly);
      if (have_prev && lx < SX - 1 && ly < SY - 1)
        dm[D_DIV * G::PE + e] =
            ((um[e + 1] - um[e]) + (vm[e + G::BX] - vm[e]) + (wk[e] - wm[e])) * P.inv_dx;
      if (lx > 0 && ly > 0) {
        dk[D_EXY * G::PE + e] = ((ek[e] + ek[e - 1]) + (ek[e - G::BX] + ek[e - 1 - G::BX])) * real(0.25);
        if (have_prev) {
          dk[D_EXZ * G::PE + e] = ((ek[e] + ek[e - 1]) + (em[e] + em[e - 1])) * real(0.25);
          dk[D_EYZ * G::PE + e] = ((ek[e] + ek[e - G::BX]) + (em[e] + em[e - G::BX])) * real(0.25);
        }
      }
    }
    return true;
  };

  if (!acquire(kbeg - 1, false)) { R.fail(err, kbeg - 1); return; }
  if (!acquire(kbeg, false)) { R.fail(err, kbeg); return; }
  const real* smr = reinterpret_cast<const real*>(smraw);
  const int raw0 = (int)(R.raw - smr), der0 = (int)(der - smr);
  const int cell = G::at(tx + 1, ty + 1);
  long long id = lin(P, i, j, kbeg);
  for (int k = kbeg; k < kend; ++k, id += P.sz) {
    real q0v[4];
    if (MODE == 2 && active) {
#pragma unroll
      for (int f = 0; f < 4; ++f) q0v[f] = A.q0[f][id];
    }
    if (!acquire(k + 1, true)) { R.fail(err, k + 1); return; }
    __syncthreads();
    if (active) {
      RingTile<real, PAVG> S;
      S.sm = smr;
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz) {
        S.r[dz + 1] = raw0 + R.slot(k + dz) * NRAW_FLOW * G::PE + cell;
        S.d[dz + 1] = der0 + (int)((unsigned)(k + dz + 4) & 3u) * NDER_FLOW * G::PE + cell;
      }
      using Ops = FlowOps<real, 3, RingTile<real, PAVG>>;
      const real D0 = Ops::div(S, P, 0, 0, 0);
      real L[4];
      L[0] = Ops::rate_p(S, P, D0);
      L[1] = Ops::template rate_vel<0>(S, P, D0);
      L[2] = Ops::template rate_vel<1>(S, P, D0);
      L[3] = Ops::template rate_vel<2>(S, P, D0);
      // faces on a wall are never updated
      if (P.bc[0] != BC_PERIODIC && i == 0) L[1] = real(0);
      if (P.bc[1] != BC_PERIODIC && j == 0) L[2] = real(0);
      if (P.bc[2] != BC_PERIODIC && k == 0) L[3] = real(0);
      const int F[4] = {F_P, F_U, F_V, F_W};
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        real o;
        if (MODE == 0) {
          o = L[f];
        } else {
          const real q = S(F[f], 0, 0, 0);
          if (MODE == 1) o = q + P.dt * L[f];
          else o = A.a * q0v[f] + A.b * (q + P.dt * L[f]);
        }
        A.out[f][id] = o;
      }
    }
  }
}

#ifndef GPE2P_FLOW_RING
#define GPE2P_FLOW_RING 4
#endif
template <typename real>
constexpr int flow_ring() { return GPE2P_FLOW_RING; }

template <typename real, int DIM>
static size_t flow_smem() {
  return sizeof(real) * (size_t)F_N * (DIM == 3 ? 3 : 1) * PL;
}

template <typename real, int DIM>
cudaError_t launch_flow_stage(const KParams<real>& P, const FlowArgs<real>& A, int mode, int kchunk,
                              cudaStream_t s, const Maps<6>* maps, int* err) {
  dim3 blk(TX, TY, 1);
  dim3 grd((P.n[0] + TX - 1) / TX, (P.n[1] + TY - 1) / TY, DIM == 3 ? (P.n[2] + kchunk - 1) / kchunk : 1);
  cudaError_t e;
  if constexpr (DIM == 3) {
    constexpr int RING = flow_ring<real>();
    const size_t sm = ring_smem_bytes<real, NRAW_FLOW, NDER_FLOW, RING>();
#define GPE2P_FLOW3_CASE(M)                                                                                 \
  if (P.pavg) {                                                                                             \
    e = cudaFuncSetAttribute(flow3d_kernel<real, M, RING, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                             (int)sm);                                                                      \
    if (e != cudaSuccess) return e;                                                                         \
    flow3d_kernel<real, M, RING, 1><<<grd, blk, sm, s>>>(*maps, P, A, kchunk, err);                         \
  } else {                                                                                                  \
    e = cudaFuncSetAttribute(flow3d_kernel<real, M, RING, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                             (int)sm);                                                                      \
    if (e != cudaSuccess) return e;                                                                         \
    flow3d_kernel<real, M, RING, 0><<<grd, blk, sm, s>>>(*maps, P, A, kchunk, err);                         \
  }
    if (mode == 0) { GPE2P_FLOW3_CASE(0) }
    else if (mode == 1) { GPE2P_FLOW3_CASE(1) }
    else { GPE2P_FLOW3_CASE(2) }
#undef GPE2P_FLOW3_CASE
  } else {
    const size_t sm = flow_smem<real, DIM>();
#define GPE2P_FLOW_CASE(M)                                                                                \
  e = cudaFuncSetAttribute(flow_stage_kernel<real, DIM, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                           (int)sm);                                                                      \
  if (e != cudaSuccess) return e;                                                                         \
  flow_stage_kernel<real, DIM, M><<<grd, blk, sm, s>>>(P, A, kchunk);
    if (mode == 0) { GPE2P_FLOW_CASE(0) }
    else if (mode == 1) { GPE2P_FLOW_CASE(1) }
    else { GPE2P_FLOW_CASE(2) }
#undef GPE2P_FLOW_CASE
  }
  return cudaGetLastError();
}

#define GPE2P_FLOW_INST(R, D)                                                                      \
  template cudaError_t launch_flow_stage<R, D>(const KParams<R>&, const FlowArgs<R>&, int, int, cudaStream_t, \
                                               const Maps<6>*, int*);
GPE2P_FLOW_INST(float, 2)
GPE2P_FLOW_INST(float, 3)
GPE2P_FLOW_INST(double, 2)
GPE2P_FLOW_INST(double, 3)
#undef GPE2P_FLOW_INST

}  // namespace gpe2p
