// gpe2p_launch.h -- argument blocks and launchers of the device kernels
// (internal to the library; the public interface is include/gpe2p.h).
#pragma once

#include <cuda_runtime.h>

#include "gpe2p_dev.cuh"
#include "ring3d.cuh"

namespace gpe2p {

// 3D ring kernels (flow stage, CH stage, mu): each thread computes two cells
// adjacent in y, so a block of TX x T threads has a tile of 2T rows and
// stages planes of 2T + 2 rows.
//
// the 3D flow stage's block: TX x FLOW_TY threads, FLOW_K3_TY = 2 FLOW_TY rows
// of cells, FLOW_MINB resident blocks per SM (registers: 128 per thread, so
// 16 warps per SM at any block height).  Four warps per block rather than
// eight: the per-plane barrier then holds back half as many warps, which
// measured 0.645 against 0.684 ms per stage on the 256x256x512 bubble.
#ifndef GPE2P_FLOW_TY
#define GPE2P_FLOW_TY 4
#endif
constexpr int FLOW_TY = GPE2P_FLOW_TY;
constexpr int FLOW_NTHR = TX * FLOW_TY;
constexpr int FLOW_K3_TY = 2 * FLOW_TY;
constexpr int FLOW_K3_SY = FLOW_K3_TY + 2;
constexpr int FLOW_MINB = 16 / FLOW_TY;

// the blocks of the 3D CH stage and of mu, likewise (2 CH_TY and MU_CPT MU_TY
// rows of cells), and the blocks of each that fit on an SM: the FP32 CH stage
// is held by shared memory (its ring and point planes) to nine blocks of four
// warps, mu by threads to 64 warps.  Four
// warps per CH block measured 0.552 against 0.576 ms for stage 1 (the other
// stages unchanged).  A mu thread takes MU_CPT = 4 cells in y, so that its
// plane wait, barrier and addressing serve four cells: 0.094 against 0.114
// ms per sweep with two.  Four cells per CH thread measured no faster (the
// larger tile halves the resident blocks).
#ifndef GPE2P_CH_TY
#define GPE2P_CH_TY 4
#endif
#ifndef GPE2P_MU_TY
#define GPE2P_MU_TY 4
#endif
#ifndef GPE2P_CH_CPT
#define GPE2P_CH_CPT 2
#endif
constexpr int CH_TY = GPE2P_CH_TY;
constexpr int CH_CPT = GPE2P_CH_CPT;   // cells per CH thread, adjacent in y
constexpr int CH_NTHR = TX * CH_TY;
constexpr int CH_K3_TY = CH_CPT * CH_TY;
constexpr int CH_K3_SY = CH_K3_TY + 2;
constexpr int CH_RESIDENT = CH_CPT == 2 && CH_TY == 4 ? 9 : 40 / CH_TY;
#ifndef GPE2P_MU_CPT
#define GPE2P_MU_CPT 4
#endif
constexpr int MU_TY = GPE2P_MU_TY;
constexpr int MU_CPT = GPE2P_MU_CPT;   // cells per mu thread, adjacent in y
constexpr int MU_NTHR = TX * MU_TY;
constexpr int MU_K3_TY = MU_CPT * MU_TY;
constexpr int MU_K3_SY = MU_K3_TY + 2;
constexpr int MU_RESIDENT = 64 / MU_TY;

// one flow stage: out = a q0 + b (q + dt L(q))   (Eq. tvd-rk3)
template <typename real>
struct FlowArgs {
  const real* q0[4];   // p, u, v, w at t^n (read at the cell only)
  const real* q[4];    // stage input (read with halo)
  real* out[4];
  const real* phi;     // frozen at t^{n+1/2}
  const real* mu;
  real a, b;
  real* usum[3];       // 3D mode 2 (last stage): if set, also u0_c + u^{n+1}_c on every face
};

// one Cahn-Hilliard stage (Eqs. che, tvd-rk2, rk4) or its rate
template <typename real>
struct CHArgs {
  const real* phis;    // stage state phi_s (read with halo)
  const real* mus;     // mu(phi_s) (read with halo)
  const real* phin;    // phi^{n+1/2} (read at the cell)
  real* out;           // stage output (phi_{s+1} or phi^{n+3/2}) or the rate
  real* acc;           // RK4 accumulator a + 2b + 2c
  real* uh[3];         // time-centred cell velocity (written when compute_uh)
  const real* u0[3];   // face velocity at t^n      (read when compute_uh)
  const real* u1[3];   // face velocity at t^{n+1}  (read when compute_uh)
  const real* usum[3]; // if set (3D): u0 + u1 per face, read instead of u0 and u1
  int scheme;          // 2 or 4
  int stage;           // 1..scheme; 0 = write the rate L only
  int compute_uh;      // 1: build uhat (Eq. u-center-2d) from u0, u1 and store it
  int conservative;    // 1: -div(uhat phi) instead of -uhat.grad(phi)
  // low part of phi^{n+1/2} (phi = phin + phi_lo): when set, the final stage
  // forms phi^{n+3/2} in FP64 and stores it back as this high/low pair
  real* phi_lo = nullptr;
};

// 3D launches read their haloed inputs through TMA tensor maps (one per
// staged field, in the order the kernel stages them) and report a timed-out
// copy in *err; 2D launches ignore both.
template <typename real, int DIM>
cudaError_t launch_flow_stage(const KParams<real>& P, const FlowArgs<real>& A, int mode, int kchunk,
                              cudaStream_t s, const Maps<6>* maps, int* err);

template <typename real, int DIM>
// pmaps (3D advective stages after the first, else nullptr): uhat x 3,
// phi^{n+1/2} and the accumulator as boxes of a block's own cells, which the
// kernel then brings in by TMA instead of loading them per cell
// umaps (3D advective stage 1 with A.usum, else nullptr): the face sums
// s_x, s_y, s_z as boxes of a block's cells and the faces above them
cudaError_t launch_ch_stage(const KParams<real>& P, const CHArgs<real>& A, int iso, int kchunk,
                            cudaStream_t s, const Maps<5>* maps, int* err, const Maps<5>* pmaps = nullptr,
                            const Maps<5>* umaps = nullptr);

// mu = 4 a phi (phi^2 - 1) - kappa lap_iso phi   (Eq. chem-pot)
template <typename real, int DIM>
cudaError_t launch_mu(const KParams<real>& P, const real* phi, real* mu, int iso, int kchunk,
                      cudaStream_t s, const Maps<1>* maps, int* err);

// uhat_a = 1/4 [(u0_a + u0_a(+e_a)) + (u1_a + u1_a(+e_a))]   (Eq. u-center-2d)
template <typename real, int DIM>
cudaError_t launch_center_velocity(const KParams<real>& P, const real* const u0[3], const real* const u1[3],
                                   real* const uh[3], cudaStream_t s);

// FP64 diagnostics: out[0] sum phi, out[1] kinetic energy (per unit volume
// element), out[2] max |u|, out[3] NaN/Inf flag (as 0/1).  partial must hold
// 4 * nblocks doubles.
template <typename real, int DIM>
cudaError_t launch_diag(const KParams<real>& P, const real* p, const real* const U[3], const real* phi,
                        const real* phi_lo,
                        double* partial, int nblocks, double* out, cudaStream_t s);

// FP64 <-> working precision copies with the wall faces of component c zeroed (c < 0: none)
template <typename real>
cudaError_t launch_from_double(const KParams<real>& P, const double* src, real* dst, int c, long long n,
                               cudaStream_t s);
// the same for phi, also reducing the integral of |src| times vol into out[0]
// (partial: 4 doubles per block, at most nblocks blocks)
template <typename real>
cudaError_t launch_from_double_abs(const KParams<real>& P, const double* src, real* dst, double* partial,
                                   int nblocks, double vol, double* out, cudaStream_t s);
template <typename real>
cudaError_t launch_to_double(const KParams<real>& P, const real* src, double* dst, long long n, cudaStream_t s,
                             const real* lo = nullptr);

// 2D state <-> network tensor [ny][nx][nch] (phi, u, v, p[, rho/rho_L]); see pack.cu
constexpr int kDistanceBlocks = 304;
template <typename real>
cudaError_t launch_pack(const KParams<real>& P, const real* const f[4], float* out, int nch, const float* mean,
                        const float* scale, cudaStream_t s);
template <typename real>
cudaError_t launch_unpack(const KParams<real>& P, real* const f[4], const float* in, int nch, const float* mean,
                          const float* scale, cudaStream_t s);
// the interface displacement between the state's phi and the tensor's phi
// channel (see pack.cu); part: kDistanceBlocks * 4 doubles; out: 3 doubles (device)
template <typename real>
cudaError_t launch_interface_distance(const KParams<real>& P, const real* phi, const float* in, int nch,
                                      const float* mean, const float* scale, double* part, double* out,
                                      cudaStream_t s);
// part: kDistanceBlocks * 8 doubles; out: 8 doubles (device)
template <typename real>
cudaError_t launch_distance(const KParams<real>& P, const real* const f[4], const float* in, int nch, const float* mean,
                            const float* scale, double* part, double* out, cudaStream_t s);

}  // namespace gpe2p
