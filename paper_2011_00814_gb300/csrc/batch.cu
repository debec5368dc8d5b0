// batch.cu -- many independent 2D problems of uneven sizes advanced together.
//
// Every instance has its own parameters (Sec. 2, Sec. 4) and its own state;
// all instances step together.  The tiles of all instances form one work
// table of (instance, tile) items.  A step is the sequence of the 2D sweeps
// of the method (three flow stages, Eq. tvd-rk3; the CH stages of
// Eq. tvd-rk2 with mu recomputed, Eq. chem-pot), each sweep covering every
// item, and it runs in one of two forms:
//   persistent: one cooperative launch per step; the blocks walk the work
//               table sweep by sweep and meet at a grid barrier between
//               sweeps (a bounded wait: after the limit the block records an
//               error and returns);
//   per sweep:  one launch per sweep over the whole table.
// Both are captured into CUDA graphs.  The tile shape and the form are chosen
// by timing the candidates when the batch is created (the autotuner).  The
// per-tile arithmetic is the same device code as the single-instance 2D
// kernels (flow_ops.cuh, ch_ops.cuh), so an instance of a batch follows the
// single-instance path bit for bit.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gpe2p.h"
#include "batch.h"
#include "ch_ops.cuh"
#include "flow_ops.cuh"
#include "gpe2p_dev.cuh"
#include "gpe2p_launch.h"

namespace gpe2p {

// ---------------------------------------------------------------------------
// device side
// ---------------------------------------------------------------------------

template <typename real>
struct BInst {
  KParams<real> P;
  real* Q[3][3];   // (p, u, v) of the three stage sets
  real* phi;       // phi^{n+1/2}
  real* mu;        // mu(phi^{n+1/2})
  real* phis;      // CH stage state
  real* mus;       // mu of the stage state
  real* uh[2];     // time-centred cell velocity
  real* us[2];     // u^n + u^{n+1} per face (advective form), left by the last flow stage
  int conservative;
};

struct BItem {
  int inst, i0, j0;
};

struct BarrierState {
  unsigned count;
  unsigned gen;
};

enum {
  SW_FLOW1 = 0, SW_FLOW2, SW_FLOW3, SW_UH, SW_CH1, SW_MU1, SW_CH2, SW_MU2, SW_N
};

// the centre velocity of the tile's cells for the conservative form (no halo)
template <typename real, int TXv, int TYv>
__device__ __forceinline__ void uh2d_tile(const KParams<real>& P, const real* u0, const real* v0, const real* u1,
                                          const real* v1, real* uh0, real* uh1, int i0, int j0) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int i = i0 + tid % TXv, j = j0 + 2 * (tid / TXv) + r;
    if (i < P.n[0] && j < P.n[1]) {
      const long long id = lin(P, i, j, 0);
      uh0[id] =
          real(0.25) * ((u0[id] + face_next<0>(u0, P, i, j, 0, id)) + (u1[id] + face_next<0>(u1, P, i, j, 0, id)));
      uh1[id] =
          real(0.25) * ((v0[id] + face_next<1>(v0, P, i, j, 0, id)) + (v1[id] + face_next<1>(v1, P, i, j, 0, id)));
    }
  }
}

template <typename real, int TXv, int TYv>
__device__ __forceinline__ void do_sweep(int sw, const BInst<real>& b, const BItem& it, int cur, real* sm) {
  const int s1 = 1 - cur, s2 = 2;
  if (sw <= SW_FLOW3) {
    FlowArgs<real> A;
    const int qin = sw == SW_FLOW1 ? cur : (sw == SW_FLOW2 ? s1 : s2);
    const int qout = sw == SW_FLOW2 ? s2 : s1;
    for (int f = 0; f < 3; ++f) {
      A.q0[f] = b.Q[cur][f];
      A.q[f] = b.Q[qin][f];
      A.out[f] = b.Q[qout][f];
    }
    A.q0[3] = A.q[3] = nullptr;
    A.out[3] = nullptr;
    A.phi = b.phi;
    A.mu = b.mu;
    const bool sums = sw == SW_FLOW3 && !b.conservative;
    A.usum[0] = sums ? b.us[0] : nullptr;
    A.usum[1] = sums ? b.us[1] : nullptr;
    A.usum[2] = nullptr;
    if (sw == SW_FLOW1) {
      A.a = real(0);
      A.b = real(1);
      flow2d_tile<real, 1, TXv, TYv>(b.P, A, it.i0, it.j0, sm);
    } else {
      A.a = sw == SW_FLOW2 ? real(0.75) : real(1.0 / 3.0);
      A.b = sw == SW_FLOW2 ? real(0.25) : real(2.0 / 3.0);
      flow2d_tile<real, 2, TXv, TYv>(b.P, A, it.i0, it.j0, sm);
    }
    return;
  }
  if (sw == SW_UH) {
    if (b.conservative)
      uh2d_tile<real, TXv, TYv>(b.P, b.Q[cur][1], b.Q[cur][2], b.Q[s1][1], b.Q[s1][2], b.uh[0], b.uh[1], it.i0,
                                it.j0);
    return;
  }
  if (sw == SW_MU1 || sw == SW_MU2) {
    if (sw == SW_MU1) mu2d_tile<real, TXv, TYv>(b.P, b.phis, b.mus, it.i0, it.j0, sm);
    else mu2d_tile<real, TXv, TYv>(b.P, b.phi, b.mu, it.i0, it.j0, sm);
    return;
  }
  CHArgs<real> C;
  C.uh[0] = b.uh[0];
  C.uh[1] = b.uh[1];
  C.uh[2] = nullptr;
  C.u0[0] = b.Q[cur][1];
  C.u0[1] = b.Q[cur][2];
  C.u1[0] = b.Q[s1][1];
  C.u1[1] = b.Q[s1][2];
  C.u0[2] = C.u1[2] = nullptr;
  C.scheme = 2;
  C.conservative = b.conservative;
  C.acc = nullptr;
  C.phin = b.phi;
  C.usum[0] = b.conservative ? nullptr : b.us[0];
  C.usum[1] = b.conservative ? nullptr : b.us[1];
  C.usum[2] = nullptr;
  C.phi_lo = nullptr;
  if (sw == SW_CH1) {
    C.stage = 1;
    C.phis = b.phi;
    C.mus = b.mu;
    C.out = b.phis;
    C.compute_uh = !b.conservative;
  } else {
    C.stage = 2;
    C.phis = b.phis;
    C.mus = b.mus;
    C.out = b.phi;
    C.compute_uh = 0;
  }
  ch2d_tile<real, TXv, TYv>(b.P, C, it.i0, it.j0, sm);
}

// all blocks of a cooperative launch meet here; false (block-uniform) if the
// wait ran past its limit.  With skip set the block does not arrive (a
// host-side fault injection used by the tests) and waits like the others.
__device__ __forceinline__ bool grid_barrier(BarrierState* bs, unsigned nblocks, long long limit, bool skip) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    volatile unsigned* gen = &bs->gen;
    const unsigned g = *gen;
    __threadfence();
    bool last = false;
    if (!skip) last = atomicAdd(&bs->count, 1u) + 1u == nblocks;
    if (last) {
      bs->count = 0u;
      __threadfence();
      atomicAdd(&bs->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > limit) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  return __syncthreads_and(ok) != 0;
}

constexpr int ERR_BARRIER_TIMEOUT = 2;

template <typename real, int TXv, int TYv>
__global__ void __launch_bounds__(TXv* TYv / 2) batch_persistent_kernel(const BInst<real>* __restrict__ insts,
                                                                     const BItem* __restrict__ items, int nitems,
                                                                     int cur, int any_cons, BarrierState* bs,
                                                                     long long limit, int skip_block, int* err) {
  extern __shared__ __align__(16) unsigned char smraw[];
  real* sm = reinterpret_cast<real*>(smraw);
  for (int sw = 0; sw < SW_N; ++sw) {
    if (sw == SW_UH && !any_cons) continue;
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
      const BItem it = items[w];
      do_sweep<real, TXv, TYv>(sw, insts[it.inst], it, cur, sm);
    }
    if (sw < SW_N - 1) {
      if (!grid_barrier(bs, gridDim.x, limit, (int)blockIdx.x == skip_block)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) atomicExch(err, ERR_BARRIER_TIMEOUT);
        return;
      }
    }
  }
}

// one sweep SW over the work table, a tile per block: the sweep is a template
// parameter, so that each sweep's kernel has the registers of its own tile
// code (the flow stages need the most) and the others keep their occupancy
template <typename real, int TXv, int TYv, int SW>
__global__ void __launch_bounds__(TXv* TYv / 2) batch_sweep_kernel(const BInst<real>* __restrict__ insts,
                                                                const BItem* __restrict__ items, int cur) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const BItem it = items[blockIdx.x];
  do_sweep<real, TXv, TYv>(SW, insts[it.inst], it, cur, reinterpret_cast<real*>(smraw));
}

template <typename real, int TXv, int TYv>
constexpr size_t batch_smem() {
  return sizeof(real) * (size_t)F_N * (TXv + 2) * (TYv + 2);  // the largest staged set (flow)
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

struct Shape {
  int tx, ty;
};
const Shape kShapes[] = {{32, 8}, {64, 4}, {16, 16}};
constexpr int kNumShapes = 3;

long long pitch_of(int nx) { return ((long long)nx + 31) / 32 * 32; }

template <typename real>
KParams<real> kp2(const gpe2p_params& p) {
  KParams<real> P{};
  P.n[0] = p.nx;
  P.n[1] = p.ny;
  P.n[2] = 1;
  P.bc[0] = p.bc[0];
  P.bc[1] = p.bc[1];
  P.bc[2] = BC_PERIODIC;
  P.sy = pitch_of(p.nx);
  P.sz = pitch_of(p.nx) * p.ny;
  P.dt = (real)p.dt;
  P.inv_dx = (real)(1.0 / p.dx);
  P.inv_dx2 = (real)(1.0 / (p.dx * p.dx));
  P.inv_2dx = (real)(1.0 / (2.0 * p.dx));
  P.cs2 = (real)(p.cs * p.cs);
  P.rhoL = (real)p.rhoL;
  P.rhoG = (real)p.rhoG;
  P.etaL = (real)p.etaL;
  P.etaG = (real)p.etaG;
  P.rho_m = (real)(0.5 * (p.rhoL + p.rhoG));
  P.rho_d = (real)(0.5 * (p.rhoL - p.rhoG));
  P.eta_m = (real)(0.5 * (p.etaL + p.etaG));
  P.eta_d = (real)(0.5 * (p.etaL - p.etaG));
  P.rho_ref = (real)p.rho_ref;
  P.sigma = (real)p.sigma;
  P.M = (real)p.M;
  P.a4 = (real)(4.0 * (3.0 / (4.0 * p.W)));
  P.kappa = (real)(3.0 * p.W / 8.0);
  for (int c = 0; c < 3; ++c) P.g[c] = (real)p.g[c];
  P.bulk = p.bulk_visc;
  P.pavg = p.p_average;
  P.axisym = p.axisym;
  P.w1 = (real)(1.0 / 9.0);
  P.w2 = (real)(1.0 / 36.0);
  P.w3 = real(0);
  P.lap_c = (real)(6.0 / (p.dx * p.dx));
  P.grad_c = (real)(3.0 / p.dx);
  return P;
}

}  // namespace

struct BatchCtx {
  int n = 0;
  int esize = 4;
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<gpe2p_params> prm;
  std::vector<long long> ncell;        // cells per instance
  std::vector<size_t> field_off;       // byte offset of each instance's first field
  size_t field_bytes_max = 0;
  char* base = nullptr;
  void* insts_dev = nullptr;           // BInst<real>[n]
  std::vector<char> insts_host;        // the same, on the host
  BItem* items_dev[kNumShapes] = {};   // work tables per tile shape
  int nitems[kNumShapes] = {};
  BarrierState* bar = nullptr;
  int* err = nullptr;
  double* d_stage = nullptr;
  double* d_part = nullptr;
  double* d_out = nullptr;
  double* h_out = nullptr;
  int nblk = 0;
  int any_cons = 0;
  int cur = 0;
  long long step = 0;
  bool initialized = false;
  // autotuned configuration
  int shape = 0;
  int persistent = 0;
  int grid_persistent[kNumShapes] = {};
  bool persistent_ok = true;
  double tuned_ms = 0.0;
  double cand_ms[kNumShapes][2] = {};
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  long long wait_limit = WAIT_LIMIT_DEFAULT;
  int skip_block = -1;
  std::string err_text;
};

// field roles inside an instance block
enum { BF_Q = 0, BF_PHI = 9, BF_MU = 10, BF_PHIS = 11, BF_MUS = 12, BF_UH = 13, BF_US = 15, BF_N = 17 };

template <typename real>
static void fill_insts(BatchCtx* b) {
  b->insts_host.assign(sizeof(BInst<real>) * b->n, 0);
  BInst<real>* I = reinterpret_cast<BInst<real>*>(b->insts_host.data());
  for (int k = 0; k < b->n; ++k) {
    const gpe2p_params& p = b->prm[k];
    const size_t fb = ((size_t)pitch_of(p.nx) * p.ny * b->esize + 255) / 256 * 256;
    char* c = b->base + b->field_off[k];
    auto fld = [&](int r) { return (real*)(c + (size_t)r * fb); };
    I[k].P = kp2<real>(p);
    for (int s = 0; s < 3; ++s)
      for (int f = 0; f < 3; ++f) I[k].Q[s][f] = fld(BF_Q + 3 * s + f);
    I[k].phi = fld(BF_PHI);
    I[k].mu = fld(BF_MU);
    I[k].phis = fld(BF_PHIS);
    I[k].mus = fld(BF_MUS);
    I[k].uh[0] = fld(BF_UH);
    I[k].uh[1] = fld(BF_UH + 1);
    I[k].us[0] = fld(BF_US);
    I[k].us[1] = fld(BF_US + 1);
    I[k].conservative = p.ch_advection;
  }
}

template <typename real, int TXv, int TYv>
static cudaError_t enqueue_batch_shape(BatchCtx* b, int si, int persistent, int cur) {
  const size_t smem = batch_smem<real, TXv, TYv>();
  const BInst<real>* insts = (const BInst<real>*)b->insts_dev;
  cudaError_t e;
  if (persistent) {
    e = cudaMemsetAsync(b->bar, 0, sizeof(BarrierState), b->stream);
    if (e != cudaSuccess) return e;
    const BItem* items = b->items_dev[si];
    int nitems = b->nitems[si];
    int anyc = b->any_cons;
    long long lim = b->wait_limit;
    int skip = b->skip_block;
    void* args[] = {(void*)&insts, (void*)&items, (void*)&nitems, (void*)&cur, (void*)&anyc,
                    (void*)&b->bar, (void*)&lim, (void*)&skip, (void*)&b->err};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid_persistent[si]);
    cfg.blockDim = dim3(TXv * TYv / 2);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelExC(&cfg, (const void*)batch_persistent_kernel<real, TXv, TYv>, args);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  const unsigned grid = (unsigned)b->nitems[si], nt = TXv * TYv / 2;
  const BItem* items = b->items_dev[si];
  cudaStream_t st = b->stream;
  batch_sweep_kernel<real, TXv, TYv, SW_FLOW1><<<grid, nt, smem, st>>>(insts, items, cur);
  batch_sweep_kernel<real, TXv, TYv, SW_FLOW2><<<grid, nt, smem, st>>>(insts, items, cur);
  batch_sweep_kernel<real, TXv, TYv, SW_FLOW3><<<grid, nt, smem, st>>>(insts, items, cur);
  if (b->any_cons) batch_sweep_kernel<real, TXv, TYv, SW_UH><<<grid, nt, smem, st>>>(insts, items, cur);
  batch_sweep_kernel<real, TXv, TYv, SW_CH1><<<grid, nt, smem, st>>>(insts, items, cur);
  batch_sweep_kernel<real, TXv, TYv, SW_MU1><<<grid, nt, smem, st>>>(insts, items, cur);
  batch_sweep_kernel<real, TXv, TYv, SW_CH2><<<grid, nt, smem, st>>>(insts, items, cur);
  batch_sweep_kernel<real, TXv, TYv, SW_MU2><<<grid, nt, smem, st>>>(insts, items, cur);
  static_assert(SW_N == 8, "the per-sweep form launches every sweep above, in order");
  return cudaGetLastError();
}

template <typename real>
static cudaError_t enqueue_batch(BatchCtx* b, int si, int persistent, int cur) {
  switch (si) {
    case 0: return enqueue_batch_shape<real, 32, 8>(b, si, persistent, cur);
    case 1: return enqueue_batch_shape<real, 64, 4>(b, si, persistent, cur);
    default: return enqueue_batch_shape<real, 16, 16>(b, si, persistent, cur);
  }
}

static cudaError_t enqueue_any(BatchCtx* b, int si, int persistent, int cur) {
  return b->esize == 4 ? enqueue_batch<float>(b, si, persistent, cur) : enqueue_batch<double>(b, si, persistent, cur);
}

template <typename real, int TXv, int TYv>
static cudaError_t prepare_shape(BatchCtx* b, int si) {
  const size_t smem = batch_smem<real, TXv, TYv>();
  cudaError_t e = cudaFuncSetAttribute(batch_persistent_kernel<real, TXv, TYv>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const void* sweeps[SW_N] = {(const void*)batch_sweep_kernel<real, TXv, TYv, SW_FLOW1>,
                              (const void*)batch_sweep_kernel<real, TXv, TYv, SW_FLOW2>,
                              (const void*)batch_sweep_kernel<real, TXv, TYv, SW_FLOW3>,
                              (const void*)batch_sweep_kernel<real, TXv, TYv, SW_UH>,
                              (const void*)batch_sweep_kernel<real, TXv, TYv, SW_CH1>,
                              (const void*)batch_sweep_kernel<real, TXv, TYv, SW_MU1>,
                              (const void*)batch_sweep_kernel<real, TXv, TYv, SW_CH2>,
                              (const void*)batch_sweep_kernel<real, TXv, TYv, SW_MU2>};
  for (int w = 0; w < SW_N; ++w)
    if ((e = cudaFuncSetAttribute(sweeps[w], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
  // the work table of this tile shape: the tiles of every instance in order
  std::vector<BItem> items;
  for (int k = 0; k < b->n; ++k)
    for (int j0 = 0; j0 < b->prm[k].ny; j0 += TYv)
      for (int i0 = 0; i0 < b->prm[k].nx; i0 += TXv) items.push_back({k, i0, j0});
  b->nitems[si] = (int)items.size();
  // the persistent grid: as many blocks as can be resident at once
  int per_sm = 0, nsm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel<real, TXv, TYv>, TXv * TYv / 2,
                                                    smem);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->dev);
  if (e != cudaSuccess) return e;
  long long g = (long long)per_sm * nsm;
  if (g > b->nitems[si]) g = b->nitems[si];
  if (g < 1) g = 1;
  b->grid_persistent[si] = (int)g;
  e = cudaMalloc((void**)&b->items_dev[si], items.size() * sizeof(BItem));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(b->items_dev[si], items.data(), items.size() * sizeof(BItem), cudaMemcpyHostToDevice);
}

template <typename real>
static cudaError_t prepare_all(BatchCtx* b) {
  cudaError_t e;
  if ((e = prepare_shape<real, 32, 8>(b, 0)) != cudaSuccess) return e;
  if ((e = prepare_shape<real, 64, 4>(b, 1)) != cudaSuccess) return e;
  return prepare_shape<real, 16, 16>(b, 2);
}

static cudaError_t build_graphs_batch(BatchCtx* b) {
  for (int c = 0; c < 2; ++c) {
    if (b->gexec[c]) {
      cudaGraphExecDestroy(b->gexec[c]);
      b->gexec[c] = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    cudaError_t e1 = enqueue_any(b, b->shape, b->persistent, c);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return e1 != cudaSuccess ? e1 : e2;
    }
    e = cudaGraphInstantiate(&b->gexec[c], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// time every candidate on the (zero) state, keep the fastest, zero the state again
static cudaError_t autotune(BatchCtx* b, size_t state_bytes) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return e;
  double best = 1e30;
  for (int si = 0; si < kNumShapes; ++si) {
    for (int pers = 0; pers < 2; ++pers) {
      b->cand_ms[si][pers] = -1.0;
      if (pers && !b->persistent_ok) continue;
      b->shape = si;
      b->persistent = pers;
      e = build_graphs_batch(b);
      if (e != cudaSuccess) {
        cudaGetLastError();
        if (pers) b->persistent_ok = false;
        continue;
      }
      const int reps = 4;
      for (int r = 0; r < 1 + reps; ++r) {
        if (r == 1) cudaEventRecord(e0, b->stream);
        if ((e = cudaGraphLaunch(b->gexec[r & 1], b->stream)) != cudaSuccess) break;
      }
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) return e;
      int errw = 0;
      cudaMemcpy(&errw, b->err, sizeof(int), cudaMemcpyDeviceToHost);
      if (errw != 0) {  // a barrier that timed out: the persistent form is not usable here
        cudaMemset(b->err, 0, sizeof(int));
        b->persistent_ok = false;
        continue;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      b->cand_ms[si][pers] = ms / reps;
      if (ms / reps < best) {
        best = ms / reps;
        b->tuned_ms = best;
      }
    }
  }
  // pick the best recorded candidate
  int bs = 0, bp = 0;
  double bm = 1e30;
  for (int si = 0; si < kNumShapes; ++si)
    for (int pers = 0; pers < 2; ++pers)
      if (b->cand_ms[si][pers] > 0.0 && b->cand_ms[si][pers] < bm) {
        bm = b->cand_ms[si][pers];
        bs = si;
        bp = pers;
      }
  b->shape = bs;
  b->persistent = bp;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if ((e = cudaMemsetAsync(b->base, 0, state_bytes, b->stream)) != cudaSuccess) return e;
  if ((e = build_graphs_batch(b)) != cudaSuccess) return e;
  return cudaStreamSynchronize(b->stream);
}

int batch_create(const gpe2p_params* p, int n, void* stream, BatchCtx** out, std::string& why) {
  *out = nullptr;
  if (n < 1 || n > 65536) { why = "n must lie in [1, 65536]"; return GPE2P_EINVAL; }
  for (int k = 0; k < n; ++k) {
    if (p[k].dim != 2) { why = "batched instances must be 2D"; return GPE2P_EINVAL; }
    if (p[k].precision != p[0].precision) { why = "all instances must share one precision"; return GPE2P_EINVAL; }
    if (p[k].ch_scheme != 2) { why = "batched instances use TVD-RK2 for the CH step (ch_scheme = 2)"; return GPE2P_EINVAL; }
  }
  BatchCtx* b = new BatchCtx();
  b->n = n;
  b->esize = p[0].precision == 32 ? 4 : 8;
  b->prm.assign(p, p + n);
  cudaError_t e = cudaGetDevice(&b->dev);
  if (e == cudaSuccess && stream) b->stream = (cudaStream_t)stream;
  else if (e == cudaSuccess) {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = true;
  }
  if (e != cudaSuccess) {
    why = std::string("CUDA set-up: ") + cudaGetErrorString(e);
    batch_destroy(b);
    return GPE2P_ECUDA;
  }
  // memory: BF_N fields per instance, then the staging, reduction, barrier
  size_t off = 0;
  long long maxcell = 0;
  for (int k = 0; k < n; ++k) {
    if (p[k].ch_advection) b->any_cons = 1;
    const size_t fb = ((size_t)pitch_of(p[k].nx) * p[k].ny * b->esize + 255) / 256 * 256;
    b->field_off.push_back(off);
    off += fb * BF_N;
    b->ncell.push_back((long long)p[k].nx * p[k].ny);
    if (b->ncell.back() > maxcell) maxcell = b->ncell.back();
  }
  const size_t state_bytes = off;
  const size_t stage_b = ((size_t)maxcell * sizeof(double) + 255) / 256 * 256;
  const long long nb = (maxcell + 255) / 256;
  b->nblk = (int)(nb < 152 * 8 ? nb : 152 * 8);
  const size_t part_b = ((size_t)b->nblk * 4 * sizeof(double) + 255) / 256 * 256;
  const size_t total = state_bytes + stage_b + part_b + 256 + 256;
  e = cudaMalloc((void**)&b->base, total);
  if (e != cudaSuccess) {
    why = std::string("device allocation: ") + cudaGetErrorString(e);
    batch_destroy(b);
    return GPE2P_ENOMEM;
  }
  b->d_stage = (double*)(b->base + state_bytes);
  b->d_part = (double*)(b->base + state_bytes + stage_b);
  b->d_out = (double*)(b->base + state_bytes + stage_b + part_b);
  b->err = (int*)(b->d_out + 4);
  b->bar = (BarrierState*)(b->base + state_bytes + stage_b + part_b + 256);
  if (b->esize == 4) fill_insts<float>(b);
  else fill_insts<double>(b);
  e = cudaMalloc(&b->insts_dev, b->insts_host.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(b->insts_dev, b->insts_host.data(), b->insts_host.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->base, 0, total);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_out, 5 * sizeof(double));
  if (e == cudaSuccess) e = b->esize == 4 ? prepare_all<float>(b) : prepare_all<double>(b);
  if (e == cudaSuccess) e = autotune(b, state_bytes);
  if (e != cudaSuccess) {
    why = std::string("batch set-up: ") + cudaGetErrorString(e);
    batch_destroy(b);
    return GPE2P_ECUDA;
  }
  *out = b;
  return GPE2P_OK;
}

void batch_destroy(BatchCtx* b) {
  if (!b) return;
  cudaSetDevice(b->dev);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int c = 0; c < 2; ++c)
    if (b->gexec[c]) cudaGraphExecDestroy(b->gexec[c]);
  for (int s = 0; s < kNumShapes; ++s)
    if (b->items_dev[s]) cudaFree(b->items_dev[s]);
  if (b->insts_dev) cudaFree(b->insts_dev);
  if (b->base) cudaFree(b->base);
  if (b->h_out) cudaFreeHost(b->h_out);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

template <typename real>
static cudaError_t batch_init_impl(BatchCtx* b, int k, const double* const src[4]) {
  const BInst<real>* I = reinterpret_cast<const BInst<real>*>(b->insts_host.data());
  const KParams<real>& P = I[k].P;
  real* dst[4] = {I[k].Q[b->cur][0], I[k].Q[b->cur][1], I[k].Q[b->cur][2], I[k].phi};
  const int comp[4] = {-1, 0, 1, -1};
  cudaError_t e;
  for (int f = 0; f < 4; ++f) {
    e = cudaMemcpyAsync(b->d_stage, src[f], (size_t)b->ncell[k] * sizeof(double), cudaMemcpyHostToDevice,
                        b->stream);
    if (e != cudaSuccess) return e;
    if ((e = launch_from_double<real>(P, b->d_stage, dst[f], comp[f], b->ncell[k], b->stream)) != cudaSuccess)
      return e;
  }
  if ((e = launch_mu<real, 2>(P, I[k].phi, I[k].mu, 9, 1, b->stream, nullptr, b->err)) != cudaSuccess) return e;
  return cudaStreamSynchronize(b->stream);
}

int batch_init(BatchCtx* b, int k, const double* phi, const double* u, const double* v, const double* p,
               std::string& why) {
  if (k < 0 || k >= b->n) { why = "instance index out of range"; return GPE2P_EINVAL; }
  if (!phi || !u || !v || !p) { why = "a required field is NULL"; return GPE2P_EINVAL; }
  cudaSetDevice(b->dev);
  const double* src[4] = {p, u, v, phi};
  cudaError_t e = b->esize == 4 ? batch_init_impl<float>(b, k, src) : batch_init_impl<double>(b, k, src);
  if (e != cudaSuccess) { why = std::string("init: ") + cudaGetErrorString(e); return GPE2P_ECUDA; }
  b->initialized = true;
  b->step = 0;
  return GPE2P_OK;
}

template <typename real>
static cudaError_t batch_read_impl(BatchCtx* b, int k, double* const dst[5]) {
  const BInst<real>* I = reinterpret_cast<const BInst<real>*>(b->insts_host.data());
  const KParams<real>& P = I[k].P;
  const int c = b->cur;
  const real* src[5] = {I[k].Q[c][0], I[k].Q[c][1], I[k].Q[c][2], I[k].phi, I[k].mu};
  cudaError_t e;
  for (int f = 0; f < 5; ++f) {
    if (!dst[f]) continue;
    if ((e = launch_to_double<real>(P, src[f], b->d_stage, b->ncell[k], b->stream)) != cudaSuccess) return e;
    e = cudaMemcpyAsync(dst[f], b->d_stage, (size_t)b->ncell[k] * sizeof(double), cudaMemcpyDeviceToHost,
                        b->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaStreamSynchronize(b->stream);
}

int batch_read(BatchCtx* b, int k, double* phi, double* u, double* v, double* p, double* mu, std::string& why) {
  if (k < 0 || k >= b->n) { why = "instance index out of range"; return GPE2P_EINVAL; }
  cudaSetDevice(b->dev);
  double* dst[5] = {p, u, v, phi, mu};
  cudaError_t e = b->esize == 4 ? batch_read_impl<float>(b, k, dst) : batch_read_impl<double>(b, k, dst);
  if (e != cudaSuccess) { why = std::string("read: ") + cudaGetErrorString(e); return GPE2P_ECUDA; }
  return GPE2P_OK;
}

int batch_step(BatchCtx* b, std::string& why) {
  if (!b->initialized) { why = "step before any instance was initialised"; return GPE2P_ESTATE; }
  cudaSetDevice(b->dev);
  cudaError_t e = cudaGraphLaunch(b->gexec[b->cur], b->stream);
  if (e != cudaSuccess) { why = std::string("graph launch: ") + cudaGetErrorString(e); return GPE2P_ECUDA; }
  b->cur = 1 - b->cur;
  b->step += 1;
  return GPE2P_OK;
}

template <typename real>
static cudaError_t batch_diag_impl(BatchCtx* b, int k) {
  const BInst<real>* I = reinterpret_cast<const BInst<real>*>(b->insts_host.data());
  const int c = b->cur;
  const real* U[3] = {I[k].Q[c][1], I[k].Q[c][2], I[k].Q[c][2]};
  return launch_diag<real, 2>(I[k].P, I[k].Q[c][0], U, I[k].phi, nullptr, b->d_part, b->nblk, b->d_out,
                              b->stream);
}

int batch_diag(BatchCtx* b, int k, gpe2p_diag* d, std::string& why) {
  cudaSetDevice(b->dev);
  gpe2p_diag acc{};
  const int k0 = k < 0 ? 0 : k, k1 = k < 0 ? b->n : k + 1;
  if (k >= b->n) { why = "instance index out of range"; return GPE2P_EINVAL; }
  for (int q = k0; q < k1; ++q) {
    cudaError_t e = b->esize == 4 ? batch_diag_impl<float>(b, q) : batch_diag_impl<double>(b, q);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->h_out, b->d_out, 4 * sizeof(double) + sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) { why = std::string("diagnostics: ") + cudaGetErrorString(e); return GPE2P_ECUDA; }
    int errw = 0;
    std::memcpy(&errw, b->h_out + 4, sizeof(int));
    if (errw != 0) {
      why = "a grid barrier or device-side copy did not complete within its bounded wait";
      return GPE2P_ETIMEOUT;
    }
    acc.int_phi += b->h_out[0];
    acc.kinetic += b->h_out[1];
    acc.umax = b->h_out[2] > acc.umax ? b->h_out[2] : acc.umax;
    if (b->h_out[3] != 0.0 || !std::isfinite(b->h_out[0]) || !std::isfinite(b->h_out[1])) acc.nan_flag = 1;
  }
  acc.step = b->step;
  acc.t = (double)b->step * b->prm[k0].dt;
  *d = acc;
  return GPE2P_OK;
}

int batch_config(BatchCtx* b, int* tile_x, int* tile_y, int* persistent, double* ms) {
  if (tile_x) *tile_x = kShapes[b->shape].tx;
  if (tile_y) *tile_y = kShapes[b->shape].ty;
  if (persistent) *persistent = b->persistent;
  if (ms) *ms = b->tuned_ms;
  return GPE2P_OK;
}

int batch_fault(BatchCtx* b, int what, long long value, std::string& why) {
  cudaSetDevice(b->dev);
  if (what == GPE2P_FAULT_SKIP_BARRIER) {
    b->skip_block = (int)value;
  } else if (what == GPE2P_FAULT_WAIT_LIMIT) {
    if (value <= 0) { why = "wait limit must be positive"; return GPE2P_EINVAL; }
    b->wait_limit = value;
  } else if (what == GPE2P_FAULT_FORCE_PERSISTENT) {
    if (!b->persistent_ok) { why = "the persistent form is not available on this device"; return GPE2P_EINVAL; }
    b->persistent = value ? 1 : 0;
  } else if (what == GPE2P_FAULT_CLEAR) {
    b->skip_block = -1;
    b->wait_limit = WAIT_LIMIT_DEFAULT;
    if (cudaMemsetAsync(b->err, 0, sizeof(int), b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
      why = "clearing the error word failed";
      return GPE2P_ECUDA;
    }
  } else {
    why = "unknown fault-injection switch";
    return GPE2P_EINVAL;
  }
  cudaError_t e = build_graphs_batch(b);
  if (e != cudaSuccess) { why = std::string("graph rebuild: ") + cudaGetErrorString(e); return GPE2P_ECUDA; }
  return GPE2P_OK;
}

template <typename real>
int batch_instance(BatchCtx* b, int k, KParams<real>* P, real* f[5], int* iso) {
  if (k < 0 || k >= b->n || (int)sizeof(real) != b->esize) return GPE2P_EINVAL;
  const BInst<real>* I = reinterpret_cast<const BInst<real>*>(b->insts_host.data());
  const int c = b->cur;
  *P = I[k].P;
  f[0] = I[k].phi;
  f[1] = I[k].Q[c][1];
  f[2] = I[k].Q[c][2];
  f[3] = I[k].Q[c][0];
  f[4] = I[k].mu;
  *iso = b->prm[k].iso;
  return GPE2P_OK;
}
template int batch_instance<float>(BatchCtx*, int, KParams<float>*, float* [5], int*);
template int batch_instance<double>(BatchCtx*, int, KParams<double>*, double* [5], int*);

void batch_mark_initialized(BatchCtx* b) { b->initialized = true; }
int* batch_err(BatchCtx* b) { return b->err; }
int batch_dev(const BatchCtx* b) { return b->dev; }
int batch_esize(const BatchCtx* b) { return b->esize; }

cudaStream_t batch_stream(const BatchCtx* b) { return b->stream; }

long long batch_cells(const BatchCtx* b) {
  long long s = 0;
  for (long long c : b->ncell) s += c;
  return s;
}

int batch_size(const BatchCtx* b) { return b->n; }
int batch_dim(const BatchCtx*) { return 2; }

}  // namespace gpe2p
