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
    using Ops = FlowOps<real, 3, RingTile<real, PAVG>>;
    real out[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      RingTile<real, PAVG> S;
      S.sm = smr;
      S.P = &P;
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz) S.r[dz + 1] = raw0 + R.slot(k + dz) * NRAW_FLOW * G::PE + cell0 + r * G::BX;
      const real D0 = Ops::divsum(S, P, 0, 0, 0);
      real L[4];
      L[0] = Ops::rate_p(S, P, D0);
      L[1] = Ops::template rate_vel<0>(S, P, D0);
      L[2] = Ops::template rate_vel<1>(S, P, D0);
      L[3] = Ops::template rate_vel<2>(S, P, D0);
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
