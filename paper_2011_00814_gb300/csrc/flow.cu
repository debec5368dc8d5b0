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
// along z fed by the TMA plane ring of ring3d.cuh.
#include "flow_ops.cuh"
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

// The single-instance 2D flow stage: one tile per block.
template <typename real, int MODE>
__global__ void __launch_bounds__(NTHR) flow2d_kernel(const KParams<real> P, const FlowArgs<real> A) {
  extern __shared__ __align__(16) unsigned char smraw[];
  flow2d_tile<real, MODE, TX, TY>(P, A, blockIdx.x * TX, blockIdx.y * TY, reinterpret_cast<real*>(smraw));
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
    const size_t sm = flow2d_smem<real>();
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
