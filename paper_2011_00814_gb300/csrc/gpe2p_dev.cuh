// gpe2p_dev.cuh -- device-side building blocks of the two-phase GPE step:
// kernel parameters, boundary index maps, material laws and the shared-memory
// tile that every stencil kernel stages its halo in.
//
// Grid convention (Sec. 3, staggered-grid figure): cell (i,j,k) centre at
// ((i+1/2)dx, (j+1/2)dx, (k+1/2)dx); the velocity component along axis c is
// stored on the low face of the cell along c.  Arrays are x-fastest.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gpe2p {

enum { BC_PERIODIC = 0, BC_NOSLIP = 1, BC_FREESLIP = 2 };

// Tile of one thread block: TX x TY cells in (x, y); 3D kernels march the tile
// along z through a window of three planes kept in shared memory.
constexpr int TX = 32;
constexpr int TY = 8;
constexpr int SX = TX + 2;       // with a one-cell halo on each side
constexpr int SY = TY + 2;
constexpr int PL = SX * SY;      // elements of one staged plane
constexpr int NTHR = TX * TY;

template <typename real>
struct KParams {
  int n[3];            // cells per axis; n[2] = 1 in 2D
  int bc[3];           // boundary per axis; axis 2 is periodic in 2D
  long long sy, sz;    // element strides of y and z
  real dt, inv_dx, inv_dx2, inv_2dx, cs2;
  real rhoL, rhoG, etaL, etaG, rho_ref;
  real rho_m, rho_d, eta_m, eta_d;  // (L + G)/2 and (L - G)/2 of density and viscosity
  real sigma, M, a4, kappa;  // a4 = 4a with a = 3/(4W); kappa = 3W/8
  real g[3];
  int bulk, pavg;
  int axisym;          // 1: axisymmetric (r, z) form, 2D: x = r with the axis at x = 0, y = z
  // isotropic stencils (Eqs. 1st-der-iso, laplacian-iso)
  real w1, w2, w3;     // weights of the shells |e|^2 = 1, 2, 3 (0 if absent)
  real lap_c, grad_c;  // 6/dx^2 and 3/dx
  // host-set test switch of the 3D kernels' timeout paths (bits WF_*): the
  // first wait of the chosen kind completes, then is treated as timed out
  int wait_fault;
};

// bits of KParams::wait_fault
enum { WF_FLOW_RING = 1, WF_CH_RING = 2, WF_MU_RING = 4, WF_CH_POINTS = 8 };

// ---------------------------------------------------------------------------
// boundary maps (ghost layer of one cell); arguments in [-1, n]
// ---------------------------------------------------------------------------

__device__ __forceinline__ int wrap1(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

__device__ __forceinline__ int mirror_cen(int x, int n) {
  return x < 0 ? -1 - x : (x >= n ? 2 * n - 1 - x : x);
}

template <typename real>
__device__ __forceinline__ long long lin(const KParams<real>& P, int i, int j, int k) {
  return (long long)i + (long long)j * P.sy + (long long)k * P.sz;
}

// cell-centred scalar (p, phi, mu): even ghosts on walls
template <typename real>
__device__ __forceinline__ real ld_cen(const real* __restrict__ f, const KParams<real>& P, int i, int j,
                                       int k) {
  i = P.bc[0] == BC_PERIODIC ? wrap1(i, P.n[0]) : mirror_cen(i, P.n[0]);
  j = P.bc[1] == BC_PERIODIC ? wrap1(j, P.n[1]) : mirror_cen(j, P.n[1]);
  k = P.bc[2] == BC_PERIODIC ? wrap1(k, P.n[2]) : mirror_cen(k, P.n[2]);
  return f[lin(P, i, j, k)];
}

// velocity component C on low faces: zero on the wall faces 0 and n and odd
// beyond them along C; odd (no-slip) or even (free-slip) across the other walls,
// and even across the axis of the axisymmetric form (a symmetry line at x = 0)
template <int C, typename real>
__device__ __forceinline__ real ld_face(const real* __restrict__ f, const KParams<real>& P, int i, int j,
                                        int k) {
  int x[3] = {i, j, k};
  bool neg = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int n = P.n[a];
    if (P.bc[a] == BC_PERIODIC) {
      x[a] = wrap1(x[a], n);
    } else if (a == C) {
      if (x[a] < 0) { x[a] = -x[a]; neg = !neg; }
      if (x[a] == 0 || x[a] >= n) return real(0);
    } else {
      if (x[a] < 0) { x[a] = -1 - x[a]; if (P.bc[a] == BC_NOSLIP && !(a == 0 && P.axisym)) neg = !neg; }
      else if (x[a] >= n) { x[a] = 2 * n - 1 - x[a]; if (P.bc[a] == BC_NOSLIP) neg = !neg; }
    }
  }
  const real v = f[lin(P, x[0], x[1], x[2])];
  return neg ? -v : v;
}

// cell-centred vector component C (the time-averaged CH velocity): odd across
// a wall normal to C, even across the others
template <int C, typename real>
__device__ __forceinline__ real ld_cvec(const real* __restrict__ f, const KParams<real>& P, int i, int j,
                                        int k) {
  int x[3] = {i, j, k};
  bool neg = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int n = P.n[a];
    if (P.bc[a] == BC_PERIODIC) {
      x[a] = wrap1(x[a], n);
    } else {
      if (x[a] < 0) { x[a] = -1 - x[a]; if (a == C) neg = !neg; }
      else if (x[a] >= n) { x[a] = 2 * n - 1 - x[a]; if (a == C) neg = !neg; }
    }
  }
  const real v = f[lin(P, x[0], x[1], x[2])];
  return neg ? -v : v;
}

// ---------------------------------------------------------------------------
// material laws, Eq. density-viscosity-op-two-phase
// ---------------------------------------------------------------------------

// both laws are linear in phi, (1 + phi)/2 L + (1 - phi)/2 G = (L + G)/2 + phi (L - G)/2,
// evaluated as one fused multiply-add with the two coefficients formed on the host
template <typename real>
__device__ __forceinline__ real rho_of(const KParams<real>& P, real phi) {
  return fma(P.rho_d, phi, P.rho_m);
}
template <typename real>
__device__ __forceinline__ real eta_of(const KParams<real>& P, real phi) {
  return fma(P.eta_d, phi, P.eta_m);
}

// an add and a multiply that the compiler never fuses with a neighbouring
// operation: where a sum of two products could be contracted into a fused
// multiply-add either way, the operator code spells out the fusion it wants
// with fma() and these, so that every kernel that inlines the same operator
// code rounds alike
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// division: the FP32 path uses the fast approximate quotient (2 ulp), the
// FP64 path the IEEE one
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }

// ---------------------------------------------------------------------------
// shared-memory tile: NF fields x NPL planes x (SX*SY)
// ---------------------------------------------------------------------------

template <typename real, int NPL>
struct Tile {
  static constexpr int PAVG = -1;  // pressure averaging decided at run time
  const real* sm;
  int c;                 // index of the thread's cell within a plane
  int s0, sm1, sp1;      // plane slots of k, k-1, k+1
  __device__ __forceinline__ real operator()(int f, int dx, int dy, int dz) const {
    const int s = dz < 0 ? sm1 : (dz > 0 ? sp1 : s0);
    return sm[(f * NPL + s) * PL + c + dy * SX + dx];
  }
};

__device__ __forceinline__ int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

// isotropic lattice weight of the shell |e|^2 = s
template <typename real>
__device__ __forceinline__ real shell_w(const KParams<real>& P, int s) {
  return s == 1 ? P.w1 : (s == 2 ? P.w2 : P.w3);
}

}  // namespace gpe2p
