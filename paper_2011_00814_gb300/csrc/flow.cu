// flow.cu -- one TVD-RK3 stage of the GPE flow update (Sec. 3):
//   out = a q^n + b (q + dt L(q)),  q = (p, u, v[, w]),
// with L the semi-discrete operators of Eq. p-u-v-semidiscrete-2d built from
// Eqs. div-v-discretization, diff-p-discretization, conv-u-discretization,
// u-stress-discretization (a)-(d), st-u-discretization, gradp-u-discretization
// and gradp-u-p-ave-3d, with phi and mu frozen (Sec. 3, after Eq. tvd-rk3).
//
// One thread per cell computes the pressure rate at the cell centre and the
// rate of each velocity component on the cell's low faces (the operators are
// in flow_ops.cuh).  2D blocks stage one tile with its halo; 3D blocks march
// along z fed by the TMA plane ring of ring3d.cuh, two cells per thread.
#include "flow_ops.cuh"
#include "gpe2p_dev.cuh"
#include "gpe2p_launch.h"
#include "ring3d.cuh"

namespace gpe2p {

// The single-instance 2D flow stage: one tile per block, two cells per thread.
template <typename real, int MODE>
__global__ void __launch_bounds__(NTHR / 2) flow2d_kernel(const KParams<real> P, const FlowArgs<real> A) {
  extern __shared__ __align__(16) unsigned char smraw[];
  flow2d_tile<real, MODE, TX, TY>(P, A, blockIdx.x * TX, blockIdx.y * TY, reinterpret_cast<real*>(smraw));
}

// ---------------------------------------------------------------------------
// 3D: the same stage fed by the TMA plane ring of ring3d.cuh
// ---------------------------------------------------------------------------

// fields staged per plane; rho, eta and nu are formed from phi where they are read
enum { R_P = 0, R_U = 1, R_V = 2, R_W = 3, R_PHI = 4, R_MU = 5, NRAW_FLOW = 6 };

template <typename real, int PAVG_>
struct RingTile {
  static constexpr int PAVG = PAVG_;
  using G = RingGeom<real, FLOW_K3_SY>;
  const real* sm;           // the block's shared memory
  const KParams<real>* P;
  int r[3];                 // index of the thread's cell in raw field 0 of planes k-1, k, k+1
  __device__ __forceinline__ real raw(int f, int o, int dz) const { return sm[r[dz + 1] + f * G::PE + o]; }
  __device__ __forceinline__ real operator()(int f, int dx, int dy, int dz) const {
    const int o = dy * G::BX + dx;
    switch (f) {
      case F_P: return raw(R_P, o, dz);
      case F_U: return raw(R_U, o, dz);
      case F_V: return raw(R_V, o, dz);
      case F_W: return raw(R_W, o, dz);
      case F_PHI: return raw(R_PHI, o, dz);
      case F_MU: return raw(R_MU, o, dz);
      case F_RHO: return rho_of(*P, raw(R_PHI, o, dz));
      case F_ETA: return eta_of(*P, raw(R_PHI, o, dz));
      default: {  // F_NU
        const real phi = raw(R_PHI, o, dz);
        return fdiv(eta_of(*P, phi), rho_of(*P, phi));
      }
    }
  }
};

// The -z side terms of a cell's 3D rates are what the same thread formed on
// the +z side of the cell below, one plane earlier: the stresses on the x-z
// and y-z edges between the two planes (the u and v faces' -z edge terms, and
// the w face's -x and -y edge terms, are their negatives), the averaged
// pressure and the divergence of the cell below (the w face's gradient and
// bulk terms), and the flux nu (p_k - p_{k-1}) of the pressure diffusion.
// The block marches along z, so these are carried in registers.
template <typename real>
struct ZCarry {
  real tau_xz, tau_yz;  // 4 eta_edge x (du/dz + dw/dx) and (dv/dz + dw/dy), times dx, on the +z edges
  real psum2;           // 36 x the pressure averaged over the x-y plane (Eq. gradp-u-p-ave-3d)
  real div;             // dx div u
  real pflux;           // (nu + nu(+z)) (p(+z) - p)
};

// FlowOps with the -z side terms taken from the carry of the plane below and
// the +z side terms returned for the plane above (3D ring tiles only)
template <typename real, typename T>
struct FlowOpsZ : FlowOps<real, 3, T> {
  using B = FlowOps<real, 3, T>;

  // the +z side terms of the cell (planes 0 and +1 only); d0 = dx div u of the cell
  __device__ __forceinline__ static void plus_z(const T& S, const KParams<real>& P, real d0, ZCarry<real>& o) {
    real e4p, e4m;
    B::template edge_eta4<0>(S, 2, e4p, e4m);
    o.tau_xz = e4p * ((S(F_U, 0, 0, 1) - S(F_U, 0, 0, 0)) + (S(F_W, 0, 0, 1) - S(F_W, -1, 0, 1)));
    B::template edge_eta4<1>(S, 2, e4p, e4m);
    o.tau_yz = e4p * ((S(F_V, 0, 0, 1) - S(F_V, 0, 0, 0)) + (S(F_W, 0, 0, 1) - S(F_W, 0, -1, 1)));
    o.psum2 = B::averaged(P) ? B::template psum<2>(S, 0, 0, 0) : real(0);
    o.div = d0;
    o.pflux = (S(F_NU, 0, 0, 0) + S(F_NU, 0, 0, 1)) * (S(F_P, 0, 0, 1) - S(F_P, 0, 0, 0));
  }

  // the pressure rate with the -z flux from the carry
  __device__ __forceinline__ static real rate_p(const T& S, const KParams<real>& P, real d0, const ZCarry<real>& in,
                                                const ZCarry<real>& out) {
    real diff = out.pflux - in.pflux;
    const real nu0 = S(F_NU, 0, 0, 0), p0 = S(F_P, 0, 0, 0);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int ex = a == 0, ey = a == 1;
      diff = fma(nu0 + S(F_NU, ex, ey, 0), S(F_P, ex, ey, 0) - p0, diff);
      diff = fma(nu0 + S(F_NU, -ex, -ey, 0), S(F_P, -ex, -ey, 0) - p0, diff);
    }
    return fma(diff, real(0.5) * P.inv_dx2, -(S(F_RHO, 0, 0, 0) * P.cs2 * mul_rn(d0, P.inv_dx)));
  }

  // the velocity rate of component C with its z-side (C = 0, 1) or x- and
  // y-side (C = 2) edge terms below the cell, and the w face's averaged
  // pressure and divergence below, from the carry
  template <int C>
  __device__ __forceinline__ static real rate_vel(const T& S, const KParams<real>& P, real d0,
                                                  const ZCarry<real>& in, const ZCarry<real>& out) {
    constexpr int cx = C == 0, cy = C == 1, cz = C == 2;
    const int FC = F_U + C;
    const real rb2 = S(F_RHO, -cx, -cy, -cz) + S(F_RHO, 0, 0, 0);
    real gradp;
    if (B::averaged(P)) {
      const real pm = C == 2 ? in.psum2 : B::template psum<C>(S, -cx, -cy, -cz);
      const real p0 = C == 2 ? out.psum2 : B::template psum<C>(S, 0, 0, 0);
      gradp = (p0 - pm) * (P.inv_dx * real(1.0 / 36.0));
    } else {
      gradp = (S(F_P, 0, 0, 0) - S(F_P, -cx, -cy, -cz)) * P.inv_dx;
    }
    const real uc0 = S(FC, 0, 0, 0);
    const real tcc = fma(S(F_ETA, -cx, -cy, -cz), S(FC, -cx, -cy, -cz) - uc0,
                         mul_rn(S(F_ETA, 0, 0, 0), S(FC, cx, cy, cz) - uc0));
    real edge = real(0), conv4 = real(0);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      if (t == C) continue;
      const int tx = t == 0, ty = t == 1, tz = t == 2;
      const int FT = F_U + t;
      const real ucp = S(FC, tx, ty, tz), ucm = S(FC, -tx, -ty, -tz);
      const real ut0 = S(FT, 0, 0, 0), utc = S(FT, -cx, -cy, -cz);
      const real utp = S(FT, tx, ty, tz), utpc = S(FT, tx - cx, ty - cy, tz - cz);
      if (t == 2) {
        // the x-z or y-z edges above and below the u or v face
        edge += (C == 0 ? out.tau_xz : out.tau_yz) - (C == 0 ? in.tau_xz : in.tau_yz);
      } else if (C == 2) {
        // the w face: the edge on its -t side lies between the planes, below the cell
        real e4p, e4m;
        B::template edge_eta4<C>(S, t, e4p, e4m);
        edge = fma(e4p, (ucp - uc0) + (utp - utpc), edge);
        edge -= t == 0 ? in.tau_xz : in.tau_yz;
      } else {
        real e4p, e4m;
        B::template edge_eta4<C>(S, t, e4p, e4m);
        edge = fma(e4p, (ucp - uc0) + (utp - utpc), edge);
        edge = fma(e4m, (ucm - uc0) + (utc - ut0), edge);
      }
      conv4 = fma((ut0 + utc) + (utp + utpc), ucp - ucm, conv4);
    }
    real visc = fma(real(2), tcc, mul_rn(real(0.25), edge));
    if (P.bulk) {
      const real dm = C == 2 ? in.div : B::divsum(S, P, -cx, -cy, -cz);
      visc = fma(S(F_ETA, 0, 0, 0), d0, visc);
      visc = fma(-S(F_ETA, -cx, -cy, -cz), dm, visc);
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

// One block: a TX x FLOW_K3_TY column of cells over the planes [kbeg, kend);
// thread (tx, ty) computes the cells (i0 + tx, j0 + 2 ty + r), r = 0, 1.  The
// two cells share most of their stencil, so the loads and sub-expressions
// they have in common are formed once.
// resident blocks per SM the 3D flow stage is compiled for (FLOW_MINB: up to
// 128 registers, no spills; three blocks of 256 threads cap them at 80 with
// spills and measured slower, 5.61 against 4.88 ms per step of the
// 256x256x512 bubble)

template <typename real, int MODE, int RING, int PAVG>
__global__ void __launch_bounds__(FLOW_NTHR, FLOW_MINB) flow3d_kernel(const __grid_constant__ Maps<NRAW_FLOW> maps,
                                                      const __grid_constant__ KParams<real> P,
                                                      const FlowArgs<real> A, const int kchunk, int* err) {
  constexpr int SYv = FLOW_K3_SY;
  using G = RingGeom<real, SYv>;
  extern __shared__ __align__(128) unsigned char smraw[];
  Ring<real, NRAW_FLOW, RING, SYv> R;
  unsigned char* sbase = smem_base128(smraw);
  R.bar = reinterpret_cast<uint64_t*>(sbase);
  R.raw = reinterpret_cast<real*>(sbase + 128);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * FLOW_K3_TY;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(kbeg + kchunk, P.n[2]);
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
  const bool edge_tile = i0 == 0 || i0 + TX + 1 > nx || j0 == 0 || j0 + FLOW_K3_TY + 1 > ny;
  const bool ragged = i0 + TX > nx || j0 + FLOW_K3_TY > ny;
  const int i = i0 + tx, ja = j0 + 2 * ty;
  const bool act[2] = {i < nx && ja < ny, i < nx && ja + 1 < ny};

  R.start(P, maps.m, kbeg, kend, i0, j0, (P.wait_fault & WF_FLOW_RING) != 0);

  // wait for plane kk and overwrite its out-of-domain cells (all cells of a
  // ghost plane or of a tile overhanging the domain end, else the perimeter
  // of a tile on the boundary)
  auto acquire = [&](int kk, bool refill) -> bool {
    if (!R.wait(kk)) return false;
    if (refill && tid == 0) R.refill(P, maps.m, kk);
    const bool ghost_plane = kk < 0 || kk >= nz;
    if (!ghost_plane && !edge_tile) return true;
    real* pl[NRAW_FLOW];
#pragma unroll
    for (int f = 0; f < NRAW_FLOW; ++f) pl[f] = R.plane(kk, f);
    const bool full = ghost_plane || ragged;
    const int ncell = full ? SX * SYv : perim<SYv>();
    for (int q = tid; q < ncell; q += FLOW_NTHR) {
      int lx, ly;
      if (full) { ly = q / SX; lx = q - ly * SX; }
      else perim_cell<SYv>(q, lx, ly);
      const int gi = i0 - 1 + lx, gj = j0 - 1 + ly;
      if (ghost_plane || gi < 0 || gi >= nx || gj < 0 || gj >= ny) {
        const int e = G::at(lx, ly);
        const int ci = clampi(gi, -1, nx), cj = clampi(gj, -1, ny);
        pl[R_P][e] = ld_cen(A.q[0], P, ci, cj, kk);
        pl[R_U][e] = ld_face<0>(A.q[1], P, ci, cj, kk);
        pl[R_V][e] = ld_face<1>(A.q[2], P, ci, cj, kk);
        pl[R_W][e] = ld_face<2>(A.q[3], P, ci, cj, kk);
        pl[R_PHI][e] = ld_cen(A.phi, P, ci, cj, kk);
        pl[R_MU][e] = ld_cen(A.mu, P, ci, cj, kk);
      }
    }
    fence_proxy_async_smem();
    return true;
  };

  if (!acquire(kbeg - 1, false)) { R.fail(err, kbeg - 1); return; }
  if (!acquire(kbeg, false)) { R.fail(err, kbeg); return; }
  const real* smr = reinterpret_cast<const real*>(smraw);
  const int raw0 = (int)(R.raw - smr);
  const int cell0 = G::at(tx + 1, 2 * ty + 1);
  using Ops = FlowOpsZ<real, RingTile<real, PAVG>>;
  // the +z side terms of the cells of plane kbeg - 1 (planes kbeg - 1 and kbeg
  // only), after every thread's writes of the two planes' out-of-domain cells
  if (edge_tile || kbeg == 0 || kbeg + 1 >= nz) __syncthreads();
  ZCarry<real> zc[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    RingTile<real, PAVG> S;
    S.sm = smr;
    S.P = &P;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) S.r[dz + 1] = raw0 + R.slot(kbeg - 1 + dz) * NRAW_FLOW * G::PE + cell0 + r * G::BX;
    Ops::plus_z(S, P, Ops::divsum(S, P, 0, 0, 0), zc[r]);
  }
  long long id = lin(P, i, ja, kbeg);
  for (int k = kbeg; k < kend; ++k, id += P.sz) {
    real q0v[2][4];
    if (MODE == 2) {
#pragma unroll
      for (int r = 0; r < 2; ++r)
        if (act[r]) {
#pragma unroll
          for (int f = 0; f < 4; ++f) q0v[r][f] = A.q0[f][id + r * P.sy];
        }
    }
    if (!acquire(k + 1, true)) { R.fail(err, k + 1); return; }
    // the threads' writes of out-of-domain cells must be seen by all before the
    // stencil reads them; a plane that needed none is visible to every thread
    // after its own wait on the plane's barrier
    if (edge_tile || k + 1 >= nz) __syncthreads();
    real out[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      RingTile<real, PAVG> S;
      S.sm = smr;
      S.P = &P;
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz) S.r[dz + 1] = raw0 + R.slot(k + dz) * NRAW_FLOW * G::PE + cell0 + r * G::BX;
      const real D0 = Ops::divsum(S, P, 0, 0, 0);
      ZCarry<real> zo;
      Ops::plus_z(S, P, D0, zo);
      real L[4];
      L[0] = Ops::rate_p(S, P, D0, zc[r], zo);
      L[1] = Ops::template rate_vel<0>(S, P, D0, zc[r], zo);
      L[2] = Ops::template rate_vel<1>(S, P, D0, zc[r], zo);
      L[3] = Ops::template rate_vel<2>(S, P, D0, zc[r], zo);
      zc[r] = zo;
      // faces on a wall are never updated
      if (P.bc[0] != BC_PERIODIC && i == 0) L[1] = real(0);
      if (P.bc[1] != BC_PERIODIC && ja + r == 0) L[2] = real(0);
      if (P.bc[2] != BC_PERIODIC && k == 0) L[3] = real(0);
      const int F[4] = {F_P, F_U, F_V, F_W};
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        if (MODE == 0) {
          out[r][f] = L[f];
        } else {
          const real q = S(F[f], 0, 0, 0);
          if (MODE == 1) out[r][f] = q + P.dt * L[f];
          else out[r][f] = A.a * q0v[r][f] + A.b * (q + P.dt * L[f]);
        }
      }
    }
    // stores after both cells, so that nothing separates their shared loads
#pragma unroll
    for (int r = 0; r < 2; ++r)
      if (act[r]) {
#pragma unroll
        for (int f = 0; f < 4; ++f) A.out[f][id + r * P.sy] = out[r][f];
      }
    // the last stage also leaves u^n + u^{n+1} on every face, from which the
    // CH step forms the time-centred cell velocity with half the loads
    if (MODE == 2 && A.usum[0]) {
#pragma unroll
      for (int r = 0; r < 2; ++r)
        if (act[r]) {
#pragma unroll
          for (int a = 0; a < 3; ++a) A.usum[a][id + r * P.sy] = q0v[r][1 + a] + out[r][1 + a];
        }
    }
  }
}

#ifndef GPE2P_FLOW_RING
#define GPE2P_FLOW_RING 4
#endif
template <typename real>
constexpr int flow_ring() { return GPE2P_FLOW_RING; }

template <typename real>
static size_t flow2d_smem() {
  return sizeof(real) * (size_t)F_N * PL;
}

template <typename real, int DIM>
cudaError_t launch_flow_stage(const KParams<real>& P, const FlowArgs<real>& A, int mode, int kchunk,
                              cudaStream_t s, const Maps<6>* maps, int* err) {
  dim3 blk(TX, TY, 1);
  dim3 grd((P.n[0] + TX - 1) / TX, (P.n[1] + TY - 1) / TY, DIM == 3 ? (P.n[2] + kchunk - 1) / kchunk : 1);
  cudaError_t e;
  if constexpr (DIM == 3) {
    constexpr int RING = flow_ring<real>();
    const size_t sm = ring_smem_bytes<real, NRAW_FLOW, 0, RING, FLOW_K3_SY>();
    blk.y = FLOW_TY;
    grd.y = (P.n[1] + FLOW_K3_TY - 1) / FLOW_K3_TY;
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
    const size_t sm = flow2d_smem<real>();
    blk.y = TY / 2;  // two cells per thread
#define GPE2P_FLOW_CASE(M)                                                                                \
  e = cudaFuncSetAttribute(flow2d_kernel<real, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
  if (e != cudaSuccess) return e;                                                                         \
  flow2d_kernel<real, M><<<grd, blk, sm, s>>>(P, A);
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
