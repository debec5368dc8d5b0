// ring3d.cuh -- the z-marching plane pipeline shared by the 3D stencil kernels.
//
// A block owns a TX x TY column of cells and a range of z-planes.  Each plane
// of every input field, with a one-cell halo in x and y, arrives in shared
// memory by one TMA copy per field (a box of BX x SY elements starting at
// x = i0 - A so that the start is 16-byte aligned); RING slots let several
// planes be in flight while the block computes plane k from planes k-1, k and
// k+1.  Cells of the staged region that lie outside the domain (the halo of
// boundary tiles, and the ghost planes k = -1 and k = nz, which are not copied)
// are then overwritten by the threads with the boundary rules of
// gpe2p_dev.cuh.
#pragma once

#include "gpe2p_dev.cuh"
#include "tma.cuh"

namespace gpe2p {

// kinds of staged fields, for the ghost rules
enum { K_CEN = 0, K_FACE0 = 1, K_FACE1 = 2, K_FACE2 = 3, K_CVEC0 = 4, K_CVEC1 = 5, K_CVEC2 = 6 };

template <typename real>
__device__ __forceinline__ real ld_kind(int kind, const real* __restrict__ f, const KParams<real>& P, int i,
                                        int j, int k) {
  switch (kind) {
    case K_FACE0: return ld_face<0>(f, P, i, j, k);
    case K_FACE1: return ld_face<1>(f, P, i, j, k);
    case K_FACE2: return ld_face<2>(f, P, i, j, k);
    case K_CVEC0: return ld_cvec<0>(f, P, i, j, k);
    case K_CVEC1: return ld_cvec<1>(f, P, i, j, k);
    case K_CVEC2: return ld_cvec<2>(f, P, i, j, k);
    default: return ld_cen(f, P, i, j, k);
  }
}

// SYv: rows of a staged plane (the tile's rows plus the two halo rows)
template <typename real, int SYv = SY>
struct RingGeom {
  static constexpr int A = 16 / (int)sizeof(real);     // alignment of the box start, elements
  static constexpr int BX = TX + 2 * A;                // box width
  static constexpr int ROWS = SYv;
  static constexpr int PE = ((BX * SYv * (int)sizeof(real) + 127) / 128) * 128 / (int)sizeof(real);
  static constexpr uint32_t BOX_BYTES = BX * SYv * sizeof(real);
  // element (lx, ly) of the staged region (lx, ly in [0, SX) x [0, SYv)): global
  // cell (i0 - 1 + lx, j0 - 1 + ly)
  __device__ __forceinline__ static int at(int lx, int ly) { return ly * BX + lx + A - 1; }
};

template <int NMAP>
struct Maps {
  CUtensorMap m[NMAP];
};

// The pipeline state of one block.  NRAW fields are staged per plane; RING is
// a power of two so that slots and phases are masks and shifts.
template <typename real, int NRAW, int RING, int SYv = SY>
struct Ring {
  static_assert((RING & (RING - 1)) == 0 && RING >= 4, "RING must be a power of two >= 4");
  static constexpr int LOG2 = RING == 4 ? 2 : (RING == 8 ? 3 : 4);
  using G = RingGeom<real, SYv>;
  uint64_t* bar;  // RING barriers
  real* raw;      // RING x NRAW x PE
  int first, last;  // planes kbeg-1 .. kend (inclusive)
  int i0, j0;
  int issued;       // last plane issued
  bool lose_first;  // test switch: report the wait for the first plane as timed out
  __device__ __forceinline__ int slot(int kk) const { return (int)((unsigned)(kk - first) & (RING - 1)); }
  __device__ __forceinline__ uint32_t parity(int kk) const { return ((unsigned)(kk - first) >> LOG2) & 1u; }
  __device__ __forceinline__ real* plane(int kk, int f) const { return raw + ((size_t)slot(kk) * NRAW + f) * G::PE; }

  // thread 0: start the copies of plane kk (or, for a ghost plane, just arrive)
  __device__ __forceinline__ void issue(const KParams<real>& P, const CUtensorMap* maps, int kk) {
    uint64_t* b = &bar[slot(kk)];
    if (kk >= 0 && kk < P.n[2]) {
      mbar_arrive_expect_tx(b, NRAW * G::BOX_BYTES);
#pragma unroll
      for (int f = 0; f < NRAW; ++f) tma_load_3d(plane(kk, f), &maps[f], i0 - G::A, j0 - 1, kk, b);
    } else {
      mbar_arrive(b);
    }
    issued = kk;
  }

  // lose: the test switch of the timeout path (the wait for the first plane
  // still completes, so no copy is left in flight, and then reports a timeout)
  __device__ __forceinline__ void start(const KParams<real>& P, const CUtensorMap* maps, int kbeg, int kend,
                                        int i0_, int j0_, bool lose = false) {
    lose_first = lose;
    first = kbeg - 1;
    last = kend;
    i0 = i0_;
    j0 = j0_;
    issued = first - 1;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      for (int s = 0; s < RING; ++s) mbar_init(&bar[s], 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const int upto = min(last, first + RING - 1);
      for (int kk = first; kk <= upto; ++kk) issue(P, maps, kk);
    }
    issued = min(last, first + RING - 1);
  }

  // all threads: wait for plane kk; false (block-uniform) on timeout
  __device__ __forceinline__ bool wait(int kk) {
    const bool ok = mbar_wait_bounded(&bar[slot(kk)], parity(kk), WAIT_CYCLES) && !(lose_first && kk == first);
    return !__syncthreads_or(!ok);
  }

  // thread 0, after the wait for plane kk (every thread is then done with
  // plane kk - 3): start plane kk - 3 + RING in the freed slot
  __device__ __forceinline__ void refill(const KParams<real>& P, const CUtensorMap* maps, int kk) {
    const int nk = kk - 3 + RING;
    if (nk <= last && nk > issued) issue(P, maps, nk);
  }

  // after a timeout: record it, let this block's copies in flight land, return
  __device__ __forceinline__ void fail(int* err, int from) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      atomicExch(err, ERR_TMA_TIMEOUT);
      for (int kk = from; kk <= issued; ++kk) mbar_wait_bounded(&bar[slot(kk)], parity(kk), WAIT_CYCLES / 2);
    }
  }
};

// the staged cells of a plane that can lie outside the domain: all of them on
// a ghost plane, else the one-cell perimeter of the staged region (SYv rows)
template <int SYv = SY>
constexpr int perim() { return 2 * SX + 2 * (SYv - 2); }
constexpr int PERIM = perim<SY>();
template <int SYv = SY>
__device__ __forceinline__ void perim_cell(int q, int& lx, int& ly) {
  if (q < SX) { lx = q; ly = 0; }
  else if (q < 2 * SX) { lx = q - SX; ly = SYv - 1; }
  else if (q < 2 * SX + SYv - 2) { lx = 0; ly = q - 2 * SX + 1; }
  else { lx = SX - 1; ly = q - 2 * SX - (SYv - 2) + 1; }
}

// shared-memory bytes of a kernel with NRAW staged and NDER derived fields
// (derived fields keep four planes, indexed by the plane number mod 4):
// 128 bytes of slack to align the base, 128 for the barriers, then the planes
template <typename real, int NRAW, int NDER, int RING, int SYv = SY>
constexpr size_t ring_smem_bytes() {
  return 256 + sizeof(real) * (size_t)RingGeom<real, SYv>::PE * (RING * NRAW + 4 * NDER);
}

// the 128-byte aligned start of the dynamic shared memory
__device__ __forceinline__ unsigned char* smem_base128(unsigned char* p) {
  const uint32_t off = smem_u32(p);
  return p + ((128u - (off & 127u)) & 127u);
}

}  // namespace gpe2p
