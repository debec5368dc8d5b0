// ch.cu -- the Cahn-Hilliard part of a step (Sec. 3): chemical potential
// (Eq. chem-pot), one RK stage of Eq. che with the isotropic stencils of
// Eqs. 1st-der-iso and laplacian-iso, and the time-centred cell velocity of
// Eq. u-center-2d.  Same tiling as the flow stage: a block stages phi_s and
// mu_s (and, for the conservative form, the cell velocity) with a one-cell
// halo in shared memory and marches along z in 3D.
#include "ch_ops.cuh"
#include "gpe2p_dev.cuh"
#include "gpe2p_launch.h"
#include "ring3d.cuh"

namespace gpe2p {

// The single-instance 2D CH stage and mu: one tile per block.
template <typename real>
__global__ void __launch_bounds__(NTHR / 2) ch2d_kernel(const KParams<real> P, const CHArgs<real> A) {
  extern __shared__ __align__(16) unsigned char smraw2d[];
  ch2d_tile<real, TX, TY>(P, A, blockIdx.x * TX, blockIdx.y * TY, reinterpret_cast<real*>(smraw2d));
}

template <typename real>
__global__ void __launch_bounds__(NTHR / 2) mu2d_kernel(const KParams<real> P, const real* __restrict__ phi,
                                                    real* __restrict__ mu) {
  __shared__ real sm[PL];
  mu2d_tile<real, TX, TY>(P, phi, mu, blockIdx.x * TX, blockIdx.y * TY, sm);
}

// ---------------------------------------------------------------------------
// 3D: the CH stage and mu fed by the TMA plane ring of ring3d.cuh
// ---------------------------------------------------------------------------

template <typename real, int NRAW, int SYv>
struct RawTile {
  using G = RingGeom<real, SYv>;
  const real* sm;  // the block's shared memory
  int r[3];        // index of the thread's cell in field 0 of planes k-1, k, k+1
  __device__ __forceinline__ real operator()(int f, int dx, int dy, int dz) const {
    return sm[r[dz + 1] + f * G::PE + dy * G::BX + dx];
  }
};

// wait for plane kk, refill the slot of plane kk - 3 + RING, overwrite the
// out-of-domain cells of the staged fields with the boundary rules (a block
// of NT threads staging SYv rows)
template <typename real, int NRAW, int RING, int SYv, int NT, typename Fix>
__device__ __forceinline__ bool ring_acquire(Ring<real, NRAW, RING, SYv>& R, const KParams<real>& P,
                                             const CUtensorMap* maps, int kk, bool refill, bool edge_tile,
                                             Fix fix) {
  using G = RingGeom<real, SYv>;
  if (!R.wait(kk)) return false;
  const int tid = threadIdx.y * TX + threadIdx.x;
  if (refill && tid == 0) R.refill(P, maps, kk);
  const bool ghost_plane = kk < 0 || kk >= P.n[2];
  if (ghost_plane || edge_tile) {
    // a full tile can reach outside the domain only on the staged region's
    // perimeter; a tile that overhangs the domain end has its ghost column or
    // row inside the region, so it and a ghost plane are scanned in full
    const bool full = ghost_plane || R.i0 + TX > P.n[0] || R.j0 + (SYv - 2) > P.n[1];
    const int ncell = full ? SX * SYv : perim<SYv>();
    for (int q = tid; q < ncell; q += NT) {
      int lx, ly;
      if (full) { ly = q / SX; lx = q - ly * SX; }
      else perim_cell<SYv>(q, lx, ly);
      const int gi = R.i0 - 1 + lx, gj = R.j0 - 1 + ly;
      if (ghost_plane || gi < 0 || gi >= P.n[0] || gj < 0 || gj >= P.n[1]) {
        const int ci = clampi(gi, -1, P.n[0]), cj = clampi(gj, -1, P.n[1]);
        const int e = G::at(lx, ly);
#pragma unroll
        for (int f = 0; f < NRAW; ++f) R.plane(kk, f)[e] = fix(f, ci, cj, kk);
      }
    }
    fence_proxy_async_smem();
  }
  return true;
}

// One block: a TX x CH_K3_TY column of cells over the planes [kbeg, kend);
// thread (tx, ty) takes the cells (i0 + tx, j0 + 2 ty + r), r = 0, 1, whose
// stencils share most of their loads.
// PTS: an advective stage after the first takes its per-cell values (uhat,
// phi^{n+1/2}, the accumulator) from point planes that TMA brings in one
// plane ahead (boxes of the block's own TX x CH_K3_TY cells, no halo, two
// slots after the ring) instead of loading them per thread; pmaps: uhat x 3,
// phi^{n+1/2}, the accumulator.  The low part of phi stays a per-thread load.
constexpr int CP_N = 5;                  // point fields
constexpr int CP_PT = TX * CH_K3_TY;     // reals per field-plane
// UPTS (with USUM): stage 1 takes the face sums the same way, each with the
// face above the cell: s_x boxes of (TX + 4) x CH_K3_TY, s_y TX x (CH_K3_TY + 1),
// s_z TX x CH_K3_TY of planes k and k + 1, in three slots (pmaps: s_x, s_y, s_z)
constexpr int US_X = (TX + 4) * CH_K3_TY, US_Y = TX * (CH_K3_TY + 1), US_Z = TX * CH_K3_TY;
constexpr int US_SLOT = US_X + US_Y + US_Z;

template <typename real, int ISO, int CONS, int RING, bool USUM, bool PTS, bool UPTS>
__global__ void __launch_bounds__(CH_NTHR) ch3d_kernel(const __grid_constant__ Maps<5> maps,
                                                    const __grid_constant__ Maps<5> pmaps,
                                                    const __grid_constant__ KParams<real> P,
                                                    const CHArgs<real> A, const int kchunk, int* err) {
  constexpr int NRAW = CONS ? 5 : 2;
  using G = RingGeom<real, CH_K3_SY>;
  extern __shared__ __align__(128) unsigned char smraw[];
  Ring<real, NRAW, RING, CH_K3_SY> R;
  unsigned char* sbase = smem_base128(smraw);
  R.bar = reinterpret_cast<uint64_t*>(sbase);
  R.raw = reinterpret_cast<real*>(sbase + 128);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * CH_K3_TY;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(kbeg + kchunk, P.n[2]);
  const int nx = P.n[0], ny = P.n[1];
  const bool edge_tile = i0 == 0 || i0 + TX + 1 > nx || j0 == 0 || j0 + CH_K3_TY + 1 > ny;
  const int i = i0 + tx, ja = j0 + CH_CPT * ty;
  bool act[CH_CPT];
#pragma unroll
  for (int r = 0; r < CH_CPT; ++r) act[r] = i < nx && ja + r < ny;
  auto fix = [&](int f, int ci, int cj, int kk) -> real {
    switch (f) {
      case C_PHI: return ld_cen(A.phis, P, ci, cj, kk);
      case C_MU: return ld_cen(A.mus, P, ci, cj, kk);
      case C_UH + 0: return ld_cvec<0>(A.uh[0], P, ci, cj, kk);
      case C_UH + 1: return ld_cvec<1>(A.uh[1], P, ci, cj, kk);
      default: return ld_cvec<2>(A.uh[2], P, ci, cj, kk);
    }
  };
  // point planes (PTS): two slots after the ring, their barriers after the ring's
  const int tid = ty * TX + tx;
  uint64_t* pbar = R.bar + 8;
  real* pts = R.raw + (size_t)RING * NRAW * G::PE;
  const bool need_acc = (A.scheme == 4 && A.stage >= 2) || (A.phi_lo && A.scheme == 2 && A.stage == 2);
  int pissued = kbeg - 1;  // thread 0: last point plane issued
  auto pissue = [&](int kk) {
    if (kk >= kend) return;
    uint64_t* b = &pbar[(kk - kbeg) & 1];
    real* dst = pts + (size_t)((kk - kbeg) & 1) * CP_N * CP_PT;
    mbar_arrive_expect_tx(b, (uint32_t)((need_acc ? 5 : 4) * CP_PT * sizeof(real)));
#pragma unroll
    for (int f = 0; f < 4; ++f) tma_load_3d(dst + f * CP_PT, &pmaps.m[f], i0, j0, kk, b);
    if (need_acc) tma_load_3d(dst + 4 * CP_PT, &pmaps.m[4], i0, j0, kk, b);
    pissued = kk;
  };
  // after a ring timeout: let this block's point copies in flight land
  auto pdrain = [&](int from) {
    if (PTS && tid == 0)
      for (int kk = from; kk <= pissued; ++kk)
        mbar_wait_bounded(&pbar[(kk - kbeg) & 1], ((kk - kbeg) >> 1) & 1, WAIT_CYCLES / 2);
  };
  // UPTS: the face-sum point planes kbeg .. klast
  const int klast = min(kend, P.n[2] - 1);
  int uissued = kbeg - 1;  // thread 0: last face-sum plane issued
  auto uslot = [&](int kk) { return (kk - kbeg) % 3; };
  auto upar = [&](int kk) { return (uint32_t)(((kk - kbeg) / 3) & 1); };
  auto uissue = [&](int kk) {
    if (kk > klast) return;
    uint64_t* b = &pbar[uslot(kk)];
    real* dst = pts + (size_t)uslot(kk) * US_SLOT;
    mbar_arrive_expect_tx(b, (uint32_t)(US_SLOT * sizeof(real)));
    tma_load_3d(dst, &pmaps.m[0], i0, j0, kk, b);
    tma_load_3d(dst + US_X, &pmaps.m[1], i0, j0, kk, b);
    tma_load_3d(dst + US_X + US_Y, &pmaps.m[2], i0, j0, kk, b);
    uissued = kk;
  };
  auto udrain = [&](int from) {
    if (UPTS && tid == 0)
      for (int kk = from; kk <= uissued; ++kk) mbar_wait_bounded(&pbar[uslot(kk)], upar(kk), WAIT_CYCLES / 2);
  };
  if ((PTS || UPTS) && tid == 0) {
    mbar_init(&pbar[0], 1);
    mbar_init(&pbar[1], 1);
    mbar_init(&pbar[2], 1);
  }
  R.start(P, maps.m, kbeg, kend, i0, j0, (P.wait_fault & WF_CH_RING) != 0);
  if (PTS && tid == 0) pissue(kbeg);
  if (UPTS && tid == 0) {
    uissue(kbeg);
    uissue(kbeg + 1);
  }
  if (!ring_acquire<real, NRAW, RING, CH_K3_SY, CH_NTHR>(R, P, maps.m, kbeg - 1, false, edge_tile, fix)) { R.fail(err, kbeg - 1); pdrain(kbeg); udrain(kbeg); return; }
  if (!ring_acquire<real, NRAW, RING, CH_K3_SY, CH_NTHR>(R, P, maps.m, kbeg, false, edge_tile, fix)) { R.fail(err, kbeg); pdrain(kbeg); udrain(kbeg); return; }
  bool pfail = false;  // a point-plane wait of this thread gave up
  // test switch: the first point-plane wait completes, then reports a timeout
  const bool plose = (P.wait_fault & WF_CH_POINTS) != 0;
  if (UPTS && (!mbar_wait_bounded(&pbar[uslot(kbeg)], upar(kbeg), WAIT_CYCLES) || plose)) {
    atomicExch(err, ERR_TMA_TIMEOUT);
    pfail = true;
  }
  const real* smr = reinterpret_cast<const real*>(smraw);
  const int raw0 = (int)(R.raw - smr), cell0 = G::at(tx + 1, CH_CPT * ty + 1);
  for (int k = kbeg; k < kend; ++k) {
    CHPoint<real> c[CH_CPT];
    if (PTS || UPTS) {
#pragma unroll
      for (int r = 0; r < CH_CPT; ++r)
        c[r].pnl = (A.phi_lo && act[r]) ? A.phi_lo[lin(P, i, ja + r, k)] : real(0);
    } else {
#pragma unroll
      for (int r = 0; r < CH_CPT; ++r)
        if (act[r]) ch_point_load<real, 3, USUM>(P, A, i, ja + r, k, c[r]);
    }
    if (!ring_acquire<real, NRAW, RING, CH_K3_SY, CH_NTHR>(R, P, maps.m, k + 1, true, edge_tile, fix)) { R.fail(err, k + 1); pdrain(k); udrain(k + 1); return; }
    if (UPTS) {
      // every thread is past plane k - 1: its slot takes plane k + 2
      if (tid == 0) uissue(k + 2);
      if (k + 1 <= klast && !mbar_wait_bounded(&pbar[uslot(k + 1)], upar(k + 1), WAIT_CYCLES)) {
        atomicExch(err, ERR_TMA_TIMEOUT);
        pfail = true;
      }
      const real* sb = pts + (size_t)uslot(k) * US_SLOT;
      const real* sz1p = pts + (size_t)uslot(k + 1) * US_SLOT + US_X + US_Y;
#pragma unroll
      for (int r = 0; r < CH_CPT; ++r) {
        const int row = CH_CPT * ty + r, j = ja + r;
        const real sx0 = sb[row * (TX + 4) + tx];
        real sx1 = sb[row * (TX + 4) + tx + 1];
        const real sy0 = sb[US_X + row * TX + tx];
        real sy1 = sb[US_X + (row + 1) * TX + tx];
        const real sz0 = sb[US_X + US_Y + row * TX + tx];
        real sz1 = k + 1 <= klast ? sz1p[row * TX + tx] : real(0);
        // the face above the cell on a periodic axis's far end is face 0 (a
        // wall face beyond the domain reads zero, as the box fill gives it)
        if (act[r]) {
          if (P.bc[0] == BC_PERIODIC && i + 1 == P.n[0]) sx1 = A.usum[0][lin(P, 0, j, k)];
          if (P.bc[1] == BC_PERIODIC && j + 1 == P.n[1]) sy1 = A.usum[1][lin(P, i, 0, k)];
          if (P.bc[2] == BC_PERIODIC && k + 1 == P.n[2]) sz1 = A.usum[2][lin(P, i, j, 0)];
        }
        c[r].uh[0] = real(0.25) * (sx0 + sx1);
        c[r].uh[1] = real(0.25) * (sy0 + sy1);
        c[r].uh[2] = real(0.25) * (sz0 + sz1);
      }
    }
    if (PTS) {
      // every thread is past plane k - 1: its slot takes plane k + 1
      if (tid == 0) pissue(k + 1);
      if (!mbar_wait_bounded(&pbar[(k - kbeg) & 1], ((k - kbeg) >> 1) & 1, WAIT_CYCLES) || (plose && k == kbeg)) {
        atomicExch(err, ERR_TMA_TIMEOUT);
        pfail = true;
      }
      const real* pp = pts + (size_t)((k - kbeg) & 1) * CP_N * CP_PT + (CH_CPT * ty) * TX + tx;
#pragma unroll
      for (int r = 0; r < CH_CPT; ++r) {
#pragma unroll
        for (int a = 0; a < 3; ++a) c[r].uh[a] = pp[a * CP_PT + r * TX];
        c[r].pn = pp[3 * CP_PT + r * TX];
        c[r].acc = pp[4 * CP_PT + r * TX];
      }
    }
    if (edge_tile || k + 1 >= P.n[2]) __syncthreads();  // out-of-domain writes seen by all
    real L[CH_CPT], ph0[CH_CPT];
#pragma unroll
    for (int r = 0; r < CH_CPT; ++r) {
      RawTile<real, NRAW, CH_K3_SY> S;
      S.sm = smr;
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz) S.r[dz + 1] = raw0 + R.slot(k + dz) * NRAW * G::PE + cell0 + r * G::BX;
      L[r] = ch_rate<real, 3, ISO>(S, P, A, c[r]);
      ph0[r] = S(C_PHI, 0, 0, 0);
      if (USUM) c[r].pn = ph0[r];  // stage 1: phi^{n+1/2} = phi_s
    }
    // stores after both cells, so that nothing separates their shared loads
#pragma unroll
    for (int r = 0; r < CH_CPT; ++r)
      if (act[r]) ch_finish<real, 3>(P, A, lin(P, i, ja + r, k), c[r], L[r], ph0[r]);
  }
  // a point-plane wait of thread 0 gave up (the error word is set): let the
  // last copies into each slot land before the block exits; a phase that
  // never completed also holds the bytes of the copies issued after it
  if ((PTS || UPTS) && tid == 0 && pfail) {
    if (PTS)
      for (int kk = pissued; kk >= kbeg && kk > pissued - 2; --kk)
        mbar_wait_bounded(&pbar[(kk - kbeg) & 1], ((kk - kbeg) >> 1) & 1, WAIT_CYCLES / 2);
    if (UPTS)
      for (int kk = uissued; kk >= kbeg && kk > uissued - 3; --kk)
        mbar_wait_bounded(&pbar[uslot(kk)], upar(kk), WAIT_CYCLES / 2);
  }
}

template <typename real, int ISO, int RING>
__global__ void __launch_bounds__(MU_NTHR) mu3d_kernel(const __grid_constant__ Maps<1> maps,
                                                    const __grid_constant__ KParams<real> P,
                                                    const real* __restrict__ phi, real* __restrict__ mu,
                                                    const int kchunk, int* err) {
  using G = RingGeom<real, MU_K3_SY>;
  extern __shared__ __align__(128) unsigned char smraw[];
  Ring<real, 1, RING, MU_K3_SY> R;
  unsigned char* sbase = smem_base128(smraw);
  R.bar = reinterpret_cast<uint64_t*>(sbase);
  R.raw = reinterpret_cast<real*>(sbase + 128);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * MU_K3_TY;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(kbeg + kchunk, P.n[2]);
  const int nx = P.n[0], ny = P.n[1];
  const bool edge_tile = i0 == 0 || i0 + TX + 1 > nx || j0 == 0 || j0 + MU_K3_TY + 1 > ny;
  const int i = i0 + tx, ja = j0 + MU_CPT * ty;
  bool act[MU_CPT];
#pragma unroll
  for (int r = 0; r < MU_CPT; ++r) act[r] = i < nx && ja + r < ny;
  auto fix = [&](int, int ci, int cj, int kk) -> real { return ld_cen(phi, P, ci, cj, kk); };
  R.start(P, maps.m, kbeg, kend, i0, j0, (P.wait_fault & WF_MU_RING) != 0);
  if (!ring_acquire<real, 1, RING, MU_K3_SY, MU_NTHR>(R, P, maps.m, kbeg - 1, false, edge_tile, fix)) { R.fail(err, kbeg - 1); return; }
  if (!ring_acquire<real, 1, RING, MU_K3_SY, MU_NTHR>(R, P, maps.m, kbeg, false, edge_tile, fix)) { R.fail(err, kbeg); return; }
  const real* smr = reinterpret_cast<const real*>(smraw);
  const int raw0 = (int)(R.raw - smr), cell0 = G::at(tx + 1, MU_CPT * ty + 1);
  for (int k = kbeg; k < kend; ++k) {
    if (!ring_acquire<real, 1, RING, MU_K3_SY, MU_NTHR>(R, P, maps.m, k + 1, true, edge_tile, fix)) { R.fail(err, k + 1); return; }
    if (edge_tile || k + 1 >= P.n[2]) __syncthreads();  // out-of-domain writes seen by all
    real m[MU_CPT];
#pragma unroll
    for (int r = 0; r < MU_CPT; ++r) {
      RawTile<real, 1, MU_K3_SY> S;
      S.sm = smr;
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz) S.r[dz + 1] = raw0 + R.slot(k + dz) * G::PE + cell0 + r * G::BX;
      const real f = S(0, 0, 0, 0);
      // the Laplacian as shell sums: mu is not conserved, and the form takes
      // 7 % less time than the difference form the CH rate needs
      m[r] = fma(P.a4 * f, fma(f, f, real(-1)), -(P.kappa * lap_iso_shells<real, 3, ISO>(S, P, 0)));
    }
#pragma unroll
    for (int r = 0; r < MU_CPT; ++r)
      if (act[r]) mu[lin(P, i, ja + r, k)] = m[r];
  }
}

// plane slots of the CH and mu rings (power of two): more slots keep more TMA
// copies in flight, fewer leave shared memory for more resident blocks
#ifndef GPE2P_CH_RING
#define GPE2P_CH_RING 4
#endif
template <typename real>
constexpr int ch_ring() { return GPE2P_CH_RING; }

template <typename real, int DIM>
__global__ void center_velocity_kernel(const KParams<real> P, const real* u00, const real* u01,
                                       const real* u02, const real* u10, const real* u11, const real* u12,
                                       real* uh0, real* uh1, real* uh2) {
  const long long n = (long long)P.n[0] * P.n[1] * P.n[2];
  for (long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x; d < n;
       d += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(d % P.n[0]);
    const int j = (int)((d / P.n[0]) % P.n[1]);
    const int k = (int)(d / ((long long)P.n[0] * P.n[1]));
    const long long id = lin(P, i, j, k);
    uh0[id] = real(0.25) * ((ld_face<0>(u00, P, i, j, k) + ld_face<0>(u00, P, i + 1, j, k)) +
                            (ld_face<0>(u10, P, i, j, k) + ld_face<0>(u10, P, i + 1, j, k)));
    uh1[id] = real(0.25) * ((ld_face<1>(u01, P, i, j, k) + ld_face<1>(u01, P, i, j + 1, k)) +
                            (ld_face<1>(u11, P, i, j, k) + ld_face<1>(u11, P, i, j + 1, k)));
    if (DIM == 3)
      uh2[id] = real(0.25) * ((ld_face<2>(u02, P, i, j, k) + ld_face<2>(u02, P, i, j, k + 1)) +
                              (ld_face<2>(u12, P, i, j, k) + ld_face<2>(u12, P, i, j, k + 1)));
  }
}

template <typename real>
static size_t ch2d_smem() {
  return sizeof(real) * (size_t)C_N * PL;
}

template <typename real, int DIM, int ISO>
static cudaError_t ch_go(const KParams<real>& P, const CHArgs<real>& A, int kchunk, cudaStream_t s,
                         const Maps<5>* maps, int* err, const Maps<5>* pmaps, const Maps<5>* umaps) {
  dim3 blk(TX, TY, 1);
  dim3 grd((P.n[0] + TX - 1) / TX, (P.n[1] + TY - 1) / TY, DIM == 3 ? (P.n[2] + kchunk - 1) / kchunk : 1);
  cudaError_t e;
  if constexpr (DIM == 3) {
    blk.y = CH_TY;
    grd.y = (P.n[1] + CH_K3_TY - 1) / CH_K3_TY;
    constexpr int RING = ch_ring<real>();
    if (A.conservative) {
      const size_t sm = ring_smem_bytes<real, 5, 0, RING, CH_K3_SY>();
      e = cudaFuncSetAttribute(ch3d_kernel<real, ISO, 1, RING, false, false, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      ch3d_kernel<real, ISO, 1, RING, false, false, false><<<grd, blk, sm, s>>>(*maps, *maps, P, A, kchunk, err);
    } else if (A.compute_uh && A.usum[0] && A.phin == A.phis && umaps) {
      const size_t sm = ring_smem_bytes<real, 2, 0, RING, CH_K3_SY>() + sizeof(real) * (size_t)3 * US_SLOT;
      e = cudaFuncSetAttribute(ch3d_kernel<real, ISO, 0, RING, true, false, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      ch3d_kernel<real, ISO, 0, RING, true, false, true><<<grd, blk, sm, s>>>(*maps, *umaps, P, A, kchunk, err);
    } else if (A.compute_uh && A.usum[0] && A.phin == A.phis) {
      const size_t sm = ring_smem_bytes<real, 2, 0, RING, CH_K3_SY>();
      e = cudaFuncSetAttribute(ch3d_kernel<real, ISO, 0, RING, true, false, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      ch3d_kernel<real, ISO, 0, RING, true, false, false><<<grd, blk, sm, s>>>(*maps, *maps, P, A, kchunk, err);
    } else if (!A.compute_uh && A.stage != 0 && pmaps) {
      const size_t sm = ring_smem_bytes<real, 2, 0, RING, CH_K3_SY>() + sizeof(real) * (size_t)2 * CP_N * CP_PT;
      e = cudaFuncSetAttribute(ch3d_kernel<real, ISO, 0, RING, false, true, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      ch3d_kernel<real, ISO, 0, RING, false, true, false><<<grd, blk, sm, s>>>(*maps, *pmaps, P, A, kchunk, err);
    } else {
      const size_t sm = ring_smem_bytes<real, 2, 0, RING, CH_K3_SY>();
      e = cudaFuncSetAttribute(ch3d_kernel<real, ISO, 0, RING, false, false, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      ch3d_kernel<real, ISO, 0, RING, false, false, false><<<grd, blk, sm, s>>>(*maps, *maps, P, A, kchunk, err);
    }
  } else {
    const size_t sm = ch2d_smem<real>();
    blk.y = TY / 2;  // two cells per thread
    e = cudaFuncSetAttribute(ch2d_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    ch2d_kernel<real><<<grd, blk, sm, s>>>(P, A);
  }
  return cudaGetLastError();
}

template <typename real, int DIM>
cudaError_t launch_ch_stage(const KParams<real>& P, const CHArgs<real>& A, int iso, int kchunk,
                            cudaStream_t s, const Maps<5>* maps, int* err, const Maps<5>* pmaps,
                            const Maps<5>* umaps) {
  if constexpr (DIM == 2) {
    return ch_go<real, DIM, 9>(P, A, kchunk, s, maps, err, nullptr, nullptr);
  } else {
    switch (iso) {
      case 15: return ch_go<real, DIM, 15>(P, A, kchunk, s, maps, err, pmaps, umaps);
      case 19: return ch_go<real, DIM, 19>(P, A, kchunk, s, maps, err, pmaps, umaps);
      default: return ch_go<real, DIM, 27>(P, A, kchunk, s, maps, err, pmaps, umaps);
    }
  }
}

template <typename real, int DIM, int ISO>
static cudaError_t mu_go(const KParams<real>& P, const real* phi, real* mu, int kchunk, cudaStream_t s,
                         const Maps<1>* maps, int* err) {
  dim3 blk(TX, TY, 1);
  dim3 grd((P.n[0] + TX - 1) / TX, (P.n[1] + TY - 1) / TY, DIM == 3 ? (P.n[2] + kchunk - 1) / kchunk : 1);
  if constexpr (DIM == 3) {
    blk.y = MU_TY;
    grd.y = (P.n[1] + MU_K3_TY - 1) / MU_K3_TY;
    constexpr int RING = ch_ring<real>();
    const size_t sm = ring_smem_bytes<real, 1, 0, RING, MU_K3_SY>();
    cudaError_t e = cudaFuncSetAttribute(mu3d_kernel<real, ISO, RING>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    mu3d_kernel<real, ISO, RING><<<grd, blk, sm, s>>>(*maps, P, phi, mu, kchunk, err);
  } else {
    blk.y = TY / 2;  // two cells per thread
    mu2d_kernel<real><<<grd, blk, 0, s>>>(P, phi, mu);
  }
  return cudaGetLastError();
}

template <typename real, int DIM>
cudaError_t launch_mu(const KParams<real>& P, const real* phi, real* mu, int iso, int kchunk, cudaStream_t s,
                      const Maps<1>* maps, int* err) {
  if constexpr (DIM == 2) {
    return mu_go<real, DIM, 9>(P, phi, mu, kchunk, s, maps, err);
  } else {
    switch (iso) {
      case 15: return mu_go<real, DIM, 15>(P, phi, mu, kchunk, s, maps, err);
      case 19: return mu_go<real, DIM, 19>(P, phi, mu, kchunk, s, maps, err);
      default: return mu_go<real, DIM, 27>(P, phi, mu, kchunk, s, maps, err);
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
  template cudaError_t launch_ch_stage<R, D>(const KParams<R>&, const CHArgs<R>&, int, int, cudaStream_t,   \
                                             const Maps<5>*, int*, const Maps<5>*, const Maps<5>*);        \
  template cudaError_t launch_mu<R, D>(const KParams<R>&, const R*, R*, int, int, cudaStream_t, const Maps<1>*, \
                                       int*);                                                              \
  template cudaError_t launch_center_velocity<R, D>(const KParams<R>&, const R* const[3], const R* const[3], \
                                                    R* const[3], cudaStream_t);
GPE2P_CH_INST(float, 2)
GPE2P_CH_INST(float, 3)
GPE2P_CH_INST(double, 2)
GPE2P_CH_INST(double, 3)
#undef GPE2P_CH_INST

}  // namespace gpe2p
