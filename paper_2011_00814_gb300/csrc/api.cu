// api.cu -- host side of the C ABI declared in include/gpe2p.h: parameter
// validation, explicit stability limits, device state, the step as a
// sequence of kernels captured into CUDA graphs, host I/O and diagnostics.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/gpe2p.h"
#include "batch.h"
#include "gpe2p_launch.h"

using namespace gpe2p;

namespace {

thread_local std::string g_create_error;

enum { FLD_P = 0, FLD_U = 1, FLD_V = 2, FLD_W = 3 };

}  // namespace

struct gpe2p_ctx {
  gpe2p_params prm;
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  long long ncell = 0;
  int esize = 8;
  char* base = nullptr;         // one device allocation holds the whole state
  void* Q[3][4] = {};           // three sets of (p, u, v, w): q^n, stage, stage
  void* phi = nullptr;          // phi^{n+1/2}
  void* mu = nullptr;           // mu(phi^{n+1/2})
  void* phis[2] = {};           // CH stage states
  void* mus = nullptr;          // mu of a CH stage state
  void* acc = nullptr;          // RK4 accumulator
  void* uh[3] = {};             // time-centred cell velocity
  void* usum[3] = {};           // u^n + u^{n+1} per face (3D advective steps)
  double* d_stage = nullptr;    // one FP64 field for host transfers
  double* d_part = nullptr;     // reduction scratch: 4 doubles per block
  double* d_out = nullptr;      // 4 reduced values
  double* h_out = nullptr;      // pinned copy of d_out (and the error word)
  int* d_err = nullptr;         // device error word (a timed-out TMA copy)
  long long pitch = 0;          // row pitch of every field, elements
  int nblk = 0;
  // TMA tensor maps of the 3D kernels (one per staged field)
  Maps<6> flow_maps[3];         // stage input Q[set] (p, u, v, w), phi, mu
  Maps<5> ch_maps[3];           // (phi, mu), (phis0, mus), (phis1, mus), each with uhat
  Maps<1> mu_maps[3];           // phi, phis0, phis1
  Maps<5> pt_maps;              // uhat x 3, phi, acc: point boxes of a CH block's cells
  Maps<5> us_maps;              // face sums s_x, s_y, s_z with the faces above a CH block's cells
  int cur = 0;                  // which Q set holds q^n (0 or 1)
  long long step = 0;
  int kchunk = 8;                // z-chunk of the flow stage
  int kchunk_ch = 8;             // ... of the CH stage
  int kchunk_mu = 8;             // ... of mu
  bool initialized = false;
  bool have_graph = false;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  BatchCtx* batch = nullptr;    // set for a batch of 2D instances
  double* d_dist = nullptr;     // state-distance scratch (allocated on first use)
  double* h_dist = nullptr;
  // precision policy of the phi accumulation (FP32 problems): low part of phi
  // when the compensated (FP64) accumulation is on; the mode; the drift
  // threshold of the automatic switch and its reference values
  void* phi_lo = nullptr;
  int acc_mode = GPE2P_PHI_ACC_AUTO;
  double drift_thr = 1e-10;
  double int_phi0 = 0.0, abs_phi0 = 0.0, last_drift = 0.0;
  long long switched_at = -1;
  int wait_fault = 0;           // test switch of the 3D kernels' timeout paths (WF_* bits)
  std::string err;
};

static int fail(gpe2p_ctx* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

static int cuda_fail(gpe2p_ctx* h, cudaError_t e, const char* what) {
  return fail(h, GPE2P_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call, what)                            \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

// ---------------------------------------------------------------------------
// validation and stability limits
// ---------------------------------------------------------------------------

static bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

static int validate(const gpe2p_params* p, std::string& why) {
  if (!p) { why = "params is NULL"; return GPE2P_EINVAL; }
  if (p->dim != 2 && p->dim != 3) { why = "dim must be 2 or 3"; return GPE2P_EINVAL; }
  const int nz = p->dim == 3 ? p->nz : 1;
  if (p->nx < 1 || p->ny < 1 || nz < 1 || p->nx > 65536 || p->ny > 65536 || nz > 65536) {
    why = "nx, ny, nz must lie in [1, 65536]";
    return GPE2P_EINVAL;
  }
  if ((double)p->nx * p->ny * nz > 4.0e9) { why = "more than 4e9 cells"; return GPE2P_EINVAL; }
  if (!finite_pos(p->dx) || !finite_pos(p->dt) || !finite_pos(p->cs)) {
    why = "dx, dt and cs must be finite and positive";
    return GPE2P_EINVAL;
  }
  if (!finite_pos(p->rhoL) || !finite_pos(p->rhoG)) { why = "densities must be positive"; return GPE2P_EINVAL; }
  if (!std::isfinite(p->etaL) || !std::isfinite(p->etaG) || p->etaL < 0 || p->etaG < 0) {
    why = "viscosities must be finite and non-negative";
    return GPE2P_EINVAL;
  }
  if (!std::isfinite(p->sigma) || p->sigma < 0 || !std::isfinite(p->M) || p->M < 0) {
    why = "sigma and M must be finite and non-negative";
    return GPE2P_EINVAL;
  }
  if (!finite_pos(p->W)) { why = "W must be finite and positive"; return GPE2P_EINVAL; }
  if (!std::isfinite(p->rho_ref) || !std::isfinite(p->g[0]) || !std::isfinite(p->g[1]) ||
      !std::isfinite(p->g[2])) {
    why = "rho_ref and g must be finite";
    return GPE2P_EINVAL;
  }
  for (int a = 0; a < p->dim; ++a)
    if (p->bc[a] < 0 || p->bc[a] > 2) { why = "bc must be PERIODIC, NOSLIP or FREESLIP"; return GPE2P_EINVAL; }
  if (p->precision != 32 && p->precision != 64) { why = "precision must be 32 or 64"; return GPE2P_EINVAL; }
  if (p->ch_scheme != 2 && p->ch_scheme != 4) { why = "ch_scheme must be 2 or 4"; return GPE2P_EINVAL; }
  if (p->dim == 2 && p->iso != 9) { why = "2D needs iso = 9 (D2Q9)"; return GPE2P_EINVAL; }
  if (p->dim == 3 && p->iso != 15 && p->iso != 19 && p->iso != 27) {
    why = "3D needs iso = 15, 19 or 27";
    return GPE2P_EINVAL;
  }
  if ((p->bulk_visc | p->p_average | p->ch_advection | p->check_stability) & ~1) {
    why = "bulk_visc, p_average, ch_advection and check_stability are 0 or 1";
    return GPE2P_EINVAL;
  }
  if (p->diag_every < 0) { why = "diag_every must be >= 0"; return GPE2P_EINVAL; }
  if (p->axisym & ~1) { why = "axisym is 0 or 1"; return GPE2P_EINVAL; }
  if (p->axisym) {
    if (p->dim != 2) { why = "axisym needs dim = 2 (x = r, y = z)"; return GPE2P_EINVAL; }
    if (p->bc[0] == GPE2P_PERIODIC) {
      why = "axisym: bc[0] is the outer radial wall and must be NOSLIP or FREESLIP";
      return GPE2P_EINVAL;
    }
    if (p->ch_advection) { why = "axisym takes the advective CH form (ch_advection = 0)"; return GPE2P_EINVAL; }
    if (p->g[0] != 0.0) { why = "axisym: the body force must act along the axis (g[0] = 0)"; return GPE2P_EINVAL; }
  }
  return GPE2P_OK;
}

// largest magnitude of the isotropic Laplacian symbol (times dx^2), by scan
static double iso_lambda_max(int dim, int iso) {
  double w0, w1, w2 = 0.0, w3 = 0.0;
  if (iso == 9) { w0 = 4.0 / 9; w1 = 1.0 / 9; w2 = 1.0 / 36; }
  else if (iso == 15) { w0 = 2.0 / 9; w1 = 1.0 / 9; w3 = 1.0 / 72; }
  else if (iso == 19) { w0 = 1.0 / 3; w1 = 1.0 / 18; w2 = 1.0 / 36; }
  else { w0 = 8.0 / 27; w1 = 2.0 / 27; w2 = 1.0 / 54; w3 = 1.0 / 216; }
  const int N = 24;
  double best = 0.0;
  for (int a = 0; a <= N; ++a)
    for (int b = 0; b <= N; ++b)
      for (int c = 0; c <= (dim == 3 ? N : 0); ++c) {
        const double t[3] = {M_PI * a / N, M_PI * b / N, M_PI * c / N};
        double s = 0.0;
        for (int ez = (dim == 3 ? -1 : 0); ez <= (dim == 3 ? 1 : 0); ++ez)
          for (int ey = -1; ey <= 1; ++ey)
            for (int ex = -1; ex <= 1; ++ex) {
              const int sh = ex * ex + ey * ey + ez * ez;
              const double w = sh == 0 ? 0.0 : (sh == 1 ? w1 : (sh == 2 ? w2 : w3));
              s += w * std::cos(t[0] * ex + t[1] * ey + t[2] * ez);
            }
        const double lam = 6.0 * (s - (1.0 - w0));
        if (-lam > best) best = -lam;
      }
  return best;
}

extern "C" int gpe2p_stability_limits(const gpe2p_params* p, double out[3]) {
  std::string why;
  int rc = validate(p, why);
  if (rc != GPE2P_OK) return fail(nullptr, rc, why);
  if (!out) return fail(nullptr, GPE2P_EINVAL, "out is NULL");
  const int d = p->dim;
  const double dx = p->dx;
  // acoustic: omega^2 = cs^2 (4/dx^2) sum_a sin^2(t_a/2) A_a(t), A_a the
  // product of the transverse averaging factors (4 + 2 cos t)/6
  double amax = 0.0;
  const int N = 32;
  for (int a = 0; a <= N; ++a)
    for (int b = 0; b <= N; ++b)
      for (int c = 0; c <= (d == 3 ? N : 0); ++c) {
        const double t[3] = {M_PI * a / N, M_PI * b / N, M_PI * c / N};
        double s = 0.0;
        for (int x = 0; x < d; ++x) {
          double A = 1.0;
          if (p->p_average)
            for (int y = 0; y < d; ++y)
              if (y != x) A *= (4.0 + 2.0 * std::cos(t[y])) / 6.0;
          const double sn = std::sin(t[x] / 2.0);
          s += sn * sn * A;
        }
        if (s > amax) amax = s;
      }
  const double omega = p->cs * 2.0 / dx * std::sqrt(amax);
  out[0] = std::sqrt(3.0) / omega;
  // viscous: the stress operator of a uniform state has the symbol
  // nu [sum_t s_t^2 I + (1 + bulk) s s^T], s_t = 2 i sin(t_t/2) / dx, whose
  // largest eigenvalue magnitude, (2 + bulk) nu sum_t |s_t|^2 on longitudinal
  // modes, peaks at (2 + bulk) nu 4 d / dx^2 for t = (pi, ..., pi); the
  // pressure diffusion's nu 4 d / dx^2 lies below it.  nu = eta / rho is
  // largest in one of the two phases (a ratio of linear laws is monotone).
  const double nuL = p->etaL / p->rhoL, nuG = p->etaG / p->rhoG;
  const double nu = nuL > nuG ? nuL : nuG;
  const double lv = nu * (2.0 + (p->bulk_visc ? 1.0 : 0.0)) * 4.0 * d / (dx * dx);
  out[1] = lv > 0.0 ? 2.5127 / lv : INFINITY;  // RK3 real-axis limit
  // Cahn-Hilliard: |z| = dt M lam (8a + kappa lam) with f'' <= 8a on |phi| <= 1
  const double a = 3.0 / (4.0 * p->W), kappa = 3.0 * p->W / 8.0;
  const double lam = iso_lambda_max(d, p->iso) / (dx * dx);
  const double lc = p->M * lam * (8.0 * a + kappa * lam);
  const double lim = p->ch_scheme == 2 ? 2.0 : 2.7853;  // RK2 / RK4 real-axis limits
  out[2] = lc > 0.0 ? lim / lc : INFINITY;
  return GPE2P_OK;
}

// ---------------------------------------------------------------------------
// kernel parameters
// ---------------------------------------------------------------------------

static long long row_pitch(int nx) { return ((long long)nx + 31) / 32 * 32; }

template <typename real>
static KParams<real> kparams(const gpe2p_params& p) {
  KParams<real> P{};
  P.n[0] = p.nx;
  P.n[1] = p.ny;
  P.n[2] = p.dim == 3 ? p.nz : 1;
  P.bc[0] = p.bc[0];
  P.bc[1] = p.bc[1];
  P.bc[2] = p.dim == 3 ? p.bc[2] : BC_PERIODIC;
  P.sy = row_pitch(p.nx);
  P.sz = row_pitch(p.nx) * p.ny;
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
  const double a = 3.0 / (4.0 * p.W);
  P.a4 = (real)(4.0 * a);
  P.kappa = (real)(3.0 * p.W / 8.0);
  for (int c = 0; c < 3; ++c) P.g[c] = (real)p.g[c];
  P.bulk = p.bulk_visc;
  P.pavg = p.p_average;
  P.axisym = p.axisym;
  double w0, w1, w2 = 0.0, w3 = 0.0;
  if (p.iso == 9) { w0 = 4.0 / 9.0; w1 = 1.0 / 9.0; w2 = 1.0 / 36.0; }
  else if (p.iso == 15) { w0 = 2.0 / 9.0; w1 = 1.0 / 9.0; w3 = 1.0 / 72.0; }
  else if (p.iso == 19) { w0 = 1.0 / 3.0; w1 = 1.0 / 18.0; w2 = 1.0 / 36.0; }
  else { w0 = 8.0 / 27.0; w1 = 2.0 / 27.0; w2 = 1.0 / 54.0; w3 = 1.0 / 216.0; }
  P.w1 = (real)w1;
  P.w2 = (real)w2;
  P.w3 = (real)w3;
  P.lap_c = (real)(6.0 / (p.dx * p.dx));
  P.grad_c = (real)(3.0 / p.dx);
  return P;
}

// ---------------------------------------------------------------------------
// one step: three flow stages, then the CH stages
// ---------------------------------------------------------------------------

// Per-launch timing hook of gpe2p_profile_steps: when set, an event is
// recorded before the first launch and after every launch of a step.
struct ProfHook {
  cudaEvent_t* ev = nullptr;
  int n = 0;
  int max = 0;
  const char** names = nullptr;
};

template <typename real, int DIM>
static cudaError_t enqueue_step(gpe2p_ctx* h, int cur, ProfHook* hook = nullptr) {
  KParams<real> P = kparams<real>(h->prm);
  P.wait_fault = h->wait_fault;
  cudaStream_t s = h->stream;
  auto mark = [&](const char* name) -> cudaError_t {
    if (!hook) return cudaSuccess;
    if (hook->n >= hook->max) return cudaErrorInvalidValue;
    hook->names[hook->n] = name;
    return cudaEventRecord(hook->ev[++hook->n], s);
  };
  if (hook) {
    hook->n = 0;
    cudaError_t e0 = cudaEventRecord(hook->ev[0], s);
    if (e0 != cudaSuccess) return e0;
  }
  const int s1 = 1 - cur, s2 = 2;
  auto q = [&](int set, int f) { return (real*)h->Q[set][f]; };
  FlowArgs<real> A{};
  for (int f = 0; f < 4; ++f) {
    A.q0[f] = q(cur, f);
    A.q[f] = q(cur, f);
    A.out[f] = q(s1, f);
  }
  A.phi = (const real*)h->phi;
  A.mu = (const real*)h->mu;
  A.a = real(0);
  A.b = real(1);
  cudaError_t e = launch_flow_stage<real, DIM>(P, A, 1, h->kchunk, s, &h->flow_maps[cur], h->d_err);
  if (e != cudaSuccess || (e = mark("flow_stage1")) != cudaSuccess) return e;
  for (int f = 0; f < 4; ++f) { A.q[f] = q(s1, f); A.out[f] = q(s2, f); }
  A.a = real(0.75);
  A.b = real(0.25);
  if ((e = launch_flow_stage<real, DIM>(P, A, 2, h->kchunk, s, &h->flow_maps[s1], h->d_err)) != cudaSuccess)
    return e;
  if ((e = mark("flow_stage2")) != cudaSuccess) return e;
  for (int f = 0; f < 4; ++f) { A.q[f] = q(s2, f); A.out[f] = q(s1, f); }
  A.a = real(1.0 / 3.0);
  A.b = real(2.0 / 3.0);
  // advective steps: the last stage also leaves u^n + u^{n+1} per face
  const bool usum = !h->prm.ch_advection;
  if (usum)
    for (int a = 0; a < 3; ++a) A.usum[a] = (real*)h->usum[a];
  if ((e = launch_flow_stage<real, DIM>(P, A, 2, h->kchunk, s, &h->flow_maps[s2], h->d_err)) != cudaSuccess)
    return e;
  if ((e = mark("flow_stage3")) != cudaSuccess) return e;

  // Cahn-Hilliard step with the time-centred velocity of Eq. u-center-2d
  CHArgs<real> C{};
  for (int a = 0; a < 3; ++a) {
    C.uh[a] = (real*)h->uh[a];
    C.u0[a] = q(cur, 1 + a);
    C.u1[a] = q(s1, 1 + a);
    C.usum[a] = usum ? (const real*)h->usum[a] : nullptr;
  }
  C.scheme = h->prm.ch_scheme;
  C.conservative = h->prm.ch_advection;
  C.acc = (real*)h->acc;
  C.phin = (const real*)h->phi;
  C.phi_lo = (real*)h->phi_lo;
  if (C.conservative) {
    const real* u0[3] = {C.u0[0], C.u0[1], C.u0[2]};
    const real* u1[3] = {C.u1[0], C.u1[1], C.u1[2]};
    real* uh[3] = {C.uh[0], C.uh[1], C.uh[2]};
    if ((e = launch_center_velocity<real, DIM>(P, u0, u1, uh, s)) != cudaSuccess) return e;
    if ((e = mark("center_velocity")) != cudaSuccess) return e;
  }
  real* phi = (real*)h->phi;
  real* mu = (real*)h->mu;
  real* F0 = (real*)h->phis[0];
  real* F1 = (real*)h->phis[1];
  real* MS = (real*)h->mus;
  const int iso = h->prm.iso;
  auto ch = [&](const real* phis) {
    const int mi = phis == phi ? 0 : (phis == F0 ? 1 : 2);
    return launch_ch_stage<real, DIM>(P, C, iso, h->kchunk_ch, s, &h->ch_maps[mi], h->d_err, &h->pt_maps,
                                      &h->us_maps);
  };
  auto mu_of = [&](const real* f, real* out) {
    const int mi = f == phi ? 0 : (f == F0 ? 1 : 2);
    return launch_mu<real, DIM>(P, f, out, iso, h->kchunk_mu, s, &h->mu_maps[mi], h->d_err);
  };
  if (C.scheme == 2) {
    C.stage = 1; C.phis = phi; C.mus = mu; C.out = F0; C.compute_uh = !C.conservative;
    if ((e = ch(C.phis)) != cudaSuccess || (e = mark("ch_stage")) != cudaSuccess) return e;
    if ((e = mu_of(F0, MS)) != cudaSuccess || (e = mark("mu")) != cudaSuccess) return e;
    C.stage = 2; C.phis = F0; C.mus = MS; C.out = phi; C.compute_uh = 0;
    if ((e = ch(C.phis)) != cudaSuccess || (e = mark("ch_stage")) != cudaSuccess) return e;
  } else {
    C.stage = 1; C.phis = phi; C.mus = mu; C.out = F0; C.compute_uh = !C.conservative;
    if ((e = ch(C.phis)) != cudaSuccess || (e = mark("ch_stage")) != cudaSuccess) return e;
    if ((e = mu_of(F0, MS)) != cudaSuccess || (e = mark("mu")) != cudaSuccess) return e;
    C.stage = 2; C.phis = F0; C.mus = MS; C.out = F1; C.compute_uh = 0;
    if ((e = ch(C.phis)) != cudaSuccess || (e = mark("ch_stage")) != cudaSuccess) return e;
    if ((e = mu_of(F1, MS)) != cudaSuccess || (e = mark("mu")) != cudaSuccess) return e;
    C.stage = 3; C.phis = F1; C.mus = MS; C.out = F0;
    if ((e = ch(C.phis)) != cudaSuccess || (e = mark("ch_stage")) != cudaSuccess) return e;
    if ((e = mu_of(F0, MS)) != cudaSuccess || (e = mark("mu")) != cudaSuccess) return e;
    C.stage = 4; C.phis = F0; C.mus = MS; C.out = phi;
    if ((e = ch(C.phis)) != cudaSuccess || (e = mark("ch_stage")) != cudaSuccess) return e;
  }
  if ((e = mu_of(phi, mu)) != cudaSuccess) return e;
  return mark("mu");
}

static cudaError_t enqueue(gpe2p_ctx* h, int cur, ProfHook* hook = nullptr) {
  if (h->esize == 4)
    return h->prm.dim == 2 ? enqueue_step<float, 2>(h, cur, hook) : enqueue_step<float, 3>(h, cur, hook);
  return h->prm.dim == 2 ? enqueue_step<double, 2>(h, cur, hook) : enqueue_step<double, 3>(h, cur, hook);
}

static int build_graphs(gpe2p_ctx* h) {
  for (int c = 0; c < 2; ++c) {
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed), "begin capture");
    cudaError_t e = enqueue(h, c);
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(h, e, "enqueue step");
    }
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "end capture");
    e = cudaGraphInstantiate(&h->gexec[c], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
  }
  h->have_graph = true;
  return GPE2P_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// TMA tensor maps of the 3D kernels
// ---------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// a field as a 3D tensor (x, y, z) with padded rows; box = one staged plane of
// `rows` rows (width: the staged row with its halo, or bx0 elements when given)
static bool encode_map(gpe2p_ctx* h, CUtensorMap* m, void* base, int rows, int bx0 = 0) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const int es = h->esize;
  cuuint64_t dims[3] = {(cuuint64_t)h->prm.nx, (cuuint64_t)h->prm.ny, (cuuint64_t)h->prm.nz};
  cuuint64_t strides[2] = {(cuuint64_t)(h->pitch * es), (cuuint64_t)(h->pitch * h->prm.ny * es)};
  const int bx = bx0 > 0 ? bx0 : (es == 4 ? RingGeom<float>::BX : RingGeom<double>::BX);
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, base, dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static int build_maps(gpe2p_ctx* h) {
  bool ok = true;
  for (int s = 0; s < 3; ++s) {
    for (int f = 0; f < 4; ++f) ok = ok && encode_map(h, &h->flow_maps[s].m[f], h->Q[s][f], FLOW_K3_SY);
    ok = ok && encode_map(h, &h->flow_maps[s].m[4], h->phi, FLOW_K3_SY);
    ok = ok && encode_map(h, &h->flow_maps[s].m[5], h->mu, FLOW_K3_SY);
  }
  void* phis[3] = {h->phi, h->phis[0], h->phis[1]};
  void* mus[3] = {h->mu, h->mus, h->mus};
  for (int c = 0; c < 3; ++c) {
    ok = ok && encode_map(h, &h->ch_maps[c].m[0], phis[c], CH_K3_SY);
    ok = ok && encode_map(h, &h->ch_maps[c].m[1], mus[c], CH_K3_SY);
    for (int a = 0; a < 3; ++a) ok = ok && encode_map(h, &h->ch_maps[c].m[2 + a], h->uh[a], CH_K3_SY);
    ok = ok && encode_map(h, &h->mu_maps[c].m[0], phis[c], MU_K3_SY);
  }
  for (int a = 0; a < 3; ++a) ok = ok && encode_map(h, &h->pt_maps.m[a], h->uh[a], CH_K3_TY, TX);
  ok = ok && encode_map(h, &h->us_maps.m[0], h->usum[0], CH_K3_TY, TX + 4);
  ok = ok && encode_map(h, &h->us_maps.m[1], h->usum[1], CH_K3_TY + 1, TX);
  ok = ok && encode_map(h, &h->us_maps.m[2], h->usum[2], CH_K3_TY, TX);
  h->us_maps.m[3] = h->us_maps.m[4] = h->us_maps.m[2];
  ok = ok && encode_map(h, &h->pt_maps.m[3], h->phi, CH_K3_TY, TX);
  ok = ok && encode_map(h, &h->pt_maps.m[4], h->acc, CH_K3_TY, TX);
  if (!ok) return fail(h, GPE2P_ECUDA, "cuTensorMapEncodeTiled failed or is unavailable");
  return GPE2P_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" int gpe2p_create(const gpe2p_params* p, void* stream, gpe2p_handle* out) {
  std::string why;
  if (!out) return fail(nullptr, GPE2P_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(p, why);
  if (rc != GPE2P_OK) return fail(nullptr, rc, why);
  if (p->check_stability) {
    double lim[3];
    gpe2p_stability_limits(p, lim);
    const char* nm[3] = {"acoustic", "viscous", "Cahn-Hilliard"};
    for (int i = 0; i < 3; ++i)
      if (p->dt > lim[i] * (1.0 + 1e-12)) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "dt = %.6g exceeds the %s limit %.6g", p->dt, nm[i], lim[i]);
        return fail(nullptr, GPE2P_EUNSTABLE, buf);
      }
  }
  gpe2p_ctx* h = new (std::nothrow) gpe2p_ctx();
  if (!h) return fail(nullptr, GPE2P_ENOMEM, "host allocation failed");
  h->prm = *p;
  if (h->prm.dim == 2) { h->prm.nz = 1; h->prm.bc[2] = GPE2P_PERIODIC; }
  h->esize = p->precision == 32 ? 4 : 8;
  h->ncell = (long long)h->prm.nx * h->prm.ny * h->prm.nz;
  cudaError_t e = cudaGetDevice(&h->dev);
  if (e != cudaSuccess) {
    delete h;
    return fail(nullptr, GPE2P_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  }
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete h;
      return fail(nullptr, GPE2P_ECUDA, std::string("stream create: ") + cudaGetErrorString(e));
    }
    h->own_stream = true;
  }
  // layout: 12 velocity/pressure fields, phi, mu, 2 stage phi, mus, acc, 3 uhat,
  // 3 face-velocity sums;
  // every field has rows padded to a multiple of 32 elements (TMA strides)
  h->pitch = row_pitch(h->prm.nx);
  const size_t fb = align256((size_t)h->pitch * h->prm.ny * h->prm.nz * h->esize);
  const int nfield = 12 + 2 + 2 + 1 + 1 + 3 + 3;
  const size_t stage_b = align256((size_t)h->ncell * sizeof(double));
  const long long nb_blocks = (h->ncell + 255) / 256;
  h->nblk = (int)(nb_blocks < 152 * 8 ? nb_blocks : 152 * 8);
  const size_t part_b = align256((size_t)h->nblk * 4 * sizeof(double));
  const size_t out_b = align256(4 * sizeof(double) + sizeof(int));
  const size_t total = fb * nfield + stage_b + part_b + out_b;
  e = cudaMalloc((void**)&h->base, total);
  if (e != cudaSuccess) {
    gpe2p_destroy(h);
    return fail(nullptr, GPE2P_ENOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
  }
  char* c = h->base;
  for (int s = 0; s < 3; ++s)
    for (int f = 0; f < 4; ++f) { h->Q[s][f] = c; c += fb; }
  h->phi = c; c += fb;
  h->mu = c; c += fb;
  h->phis[0] = c; c += fb;
  h->phis[1] = c; c += fb;
  h->mus = c; c += fb;
  h->acc = c; c += fb;
  for (int a = 0; a < 3; ++a) { h->uh[a] = c; c += fb; }
  for (int a = 0; a < 3; ++a) { h->usum[a] = c; c += fb; }
  h->d_stage = (double*)c; c += stage_b;
  h->d_part = (double*)c; c += part_b;
  h->d_out = (double*)c;
  h->d_err = (int*)(h->d_out + 4);
  e = cudaMemsetAsync(h->base, 0, total, h->stream);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h->h_out, 5 * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    gpe2p_destroy(h);
    return fail(nullptr, GPE2P_ECUDA, std::string("set-up: ") + cudaGetErrorString(e));
  }
  if (h->prm.dim == 3) {
    int rc = build_maps(h);
    if (rc != GPE2P_OK) {
      std::string why = h->err;
      gpe2p_destroy(h);
      return fail(nullptr, rc, why);
    }
  }
  // z-chunks of the marching kernels: a block marches kc planes after a
  // prologue of two, and the blocks run in waves of the resident slots; take
  // the kc in [4, 64] that minimises waves x (kc + 2), the time of the slowest
  // SM.  Resident blocks per SM (registers and shared memory, as ncu reports
  // them): flow stage FLOW_MINB, CH stage CH_RESIDENT, mu MU_RESIDENT.
  if (h->prm.dim == 3) {
    const long long bx = (h->prm.nx + TX - 1) / TX;
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->dev);
    auto pick = [&](int per_sm, int rows) {
      const long long bxy = bx * ((h->prm.ny + rows - 1) / rows);
      const long long slots = (long long)per_sm * nsm;
      long long best_kc = 4, best = -1;
      for (long long kc = 4; kc <= 64 && kc <= h->prm.nz; ++kc) {
        const long long nb = bxy * ((h->prm.nz + kc - 1) / kc);
        const long long cost = ((nb + slots - 1) / slots) * (kc + 2);
        if (best < 0 || cost < best) { best = cost; best_kc = kc; }
      }
      return (int)(best_kc > h->prm.nz ? h->prm.nz : best_kc);
    };
    h->kchunk = pick(FLOW_MINB, FLOW_K3_TY);
    h->kchunk_ch = pick(CH_RESIDENT, CH_K3_TY);
    h->kchunk_mu = pick(MU_RESIDENT, MU_K3_TY);
  } else {
    h->kchunk = h->kchunk_ch = h->kchunk_mu = 1;
  }
  *out = h;
  return GPE2P_OK;
}

static size_t field_bytes(const gpe2p_ctx* h) {
  return (size_t)h->pitch * h->prm.ny * (h->prm.dim == 3 ? h->prm.nz : 1) * h->esize;
}

static int diag_impl(gpe2p_ctx* h, gpe2p_diag* d);

// start the compensated accumulation of phi: a zero low part; the step graphs
// are rebuilt at the next step
static int phi_acc_on(gpe2p_ctx* h) {
  if (h->phi_lo || h->esize != 4) return GPE2P_OK;
  CK(h, cudaMalloc(&h->phi_lo, field_bytes(h)), "low part of phi");
  CK(h, cudaMemsetAsync(h->phi_lo, 0, field_bytes(h), h->stream), "low part of phi");
  for (int c = 0; c < 2; ++c)
    if (h->gexec[c]) { cudaGraphExecDestroy(h->gexec[c]); h->gexec[c] = nullptr; }
  h->have_graph = false;
  h->switched_at = h->step;
  return GPE2P_OK;
}

// the automatic policy: switch to the compensated accumulation once the
// relative drift of the phi integral passes the threshold
static int phi_acc_check(gpe2p_ctx* h, const gpe2p_diag& d) {
  if (h->esize != 4 || h->batch || !(h->abs_phi0 > 0.0)) return GPE2P_OK;
  h->last_drift = std::fabs(d.int_phi - h->int_phi0) / h->abs_phi0;
  if (h->acc_mode == GPE2P_PHI_ACC_AUTO && !h->phi_lo && h->last_drift > h->drift_thr) return phi_acc_on(h);
  return GPE2P_OK;
}

// The address at which the device can dereference a caller's host array, or
// nullptr.  Pinned host memory (cudaHostAlloc, cudaHostRegister) is mapped
// into the device's address space; the conversion kernels then read or write
// it in place over the host link, with no FP64 staging copy in HBM and no
// second pass.  Pageable memory (nullptr) goes through the staging buffer and
// the copy engines.
static const void* device_view(const void* host) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// one field from the caller's dense FP64 array into the padded working array
// (comp: the velocity component whose wall faces are zeroed, -1 none; with
// abs, phi: also the integral of |phi_0|, the reference of the conservation
// drift, into d_out[0], from the same single read of the FP64 input)
template <typename real>
static cudaError_t put_field(gpe2p_ctx* h, const double* src, void* dst, int comp, bool abs = false) {
  const KParams<real> P = kparams<real>(h->prm);
  const double* dsrc = static_cast<const double*>(device_view(src));
  if (!dsrc) {
    cudaError_t e = cudaMemcpyAsync(h->d_stage, src, (size_t)h->ncell * sizeof(double), cudaMemcpyHostToDevice,
                                    h->stream);
    if (e != cudaSuccess) return e;
    dsrc = h->d_stage;
  }
  if (!abs) return launch_from_double<real>(P, dsrc, (real*)dst, comp, h->ncell, h->stream);
  const double dx = h->prm.dx, vol = h->prm.dim == 3 ? dx * dx * dx : dx * dx;
  return launch_from_double_abs<real>(P, dsrc, (real*)dst, h->d_part, h->nblk, vol, h->d_out, h->stream);
}

template <typename real>
static cudaError_t init_impl(gpe2p_ctx* h, const double* phi, const double* u, const double* v, const double* w,
                             const double* p) {
  const double* src[4] = {p, u, v, w};
  cudaError_t e;
  for (int f = 0; f < 1 + h->prm.dim; ++f)
    if ((e = put_field<real>(h, src[f], h->Q[0][f], f - 1)) != cudaSuccess) return e;
  if ((e = put_field<real>(h, phi, h->phi, -1, true)) != cudaSuccess) return e;
  const KParams<real> P = kparams<real>(h->prm);
  if (h->prm.dim == 2)
    e = launch_mu<real, 2>(P, (real*)h->phi, (real*)h->mu, h->prm.iso, h->kchunk, h->stream, nullptr, h->d_err);
  else
    e = launch_mu<real, 3>(P, (real*)h->phi, (real*)h->mu, h->prm.iso, h->kchunk_mu, h->stream, &h->mu_maps[0],
                           h->d_err);
  if (e != cudaSuccess) return e;
  // the integrals of |phi_0| and phi_0 (d_out[0], d_out[1]) and the error word after it
  if ((e = cudaMemcpyAsync(h->h_out, h->d_out, 4 * sizeof(double) + sizeof(int), cudaMemcpyDeviceToHost,
                           h->stream)) != cudaSuccess)
    return e;
  return cudaStreamSynchronize(h->stream);
}

extern "C" int gpe2p_init_fields(gpe2p_handle h, const double* phi, const double* u, const double* v,
                                 const double* w, const double* p) {
  if (!h) return fail(nullptr, GPE2P_EINVAL, "handle is NULL");
  if (h->batch) return fail(h, GPE2P_EINVAL, "a batch handle: use the per-instance calls");
  if (!phi || !u || !v || !p || (h->prm.dim == 3 && !w)) return fail(h, GPE2P_EINVAL, "a required field is NULL");
  CK(h, cudaSetDevice(h->dev), "set device");
  h->cur = 0;
  // a new state starts with a clear error word (a wait that timed out on the old one)
  CK(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream), "init_fields");
  cudaError_t e = h->esize == 4 ? init_impl<float>(h, phi, u, v, w, p) : init_impl<double>(h, phi, u, v, w, p);
  if (e != cudaSuccess) return cuda_fail(h, e, "init_fields");
  if (h->phi_lo) CK(h, cudaMemsetAsync(h->phi_lo, 0, field_bytes(h), h->stream), "init_fields");
  h->step = 0;
  h->initialized = true;
  h->abs_phi0 = h->h_out[0];
  int errw = 0;
  std::memcpy(&errw, h->h_out + 4, sizeof(int));
  if (errw != 0) return fail(h, GPE2P_ETIMEOUT, "a device-side copy did not complete within its bounded wait");
  // the reference of the conservation drift: the integral of phi_0 as stored,
  // summed by the conversion pass
  h->int_phi0 = h->h_out[1];
  h->last_drift = 0.0;
  h->switched_at = -1;
  return GPE2P_OK;
}

static int diag_impl(gpe2p_ctx* h, gpe2p_diag* d) {
  cudaError_t e;
  const int cur = h->cur;
  if (h->esize == 4) {
    const KParams<float> P = kparams<float>(h->prm);
    const float* U[3] = {(float*)h->Q[cur][1], (float*)h->Q[cur][2], (float*)h->Q[cur][3]};
    const float* lo = (const float*)h->phi_lo;
    e = h->prm.dim == 2 ? launch_diag<float, 2>(P, (float*)h->Q[cur][0], U, (float*)h->phi, lo, h->d_part,
                                                h->nblk, h->d_out, h->stream)
                        : launch_diag<float, 3>(P, (float*)h->Q[cur][0], U, (float*)h->phi, lo, h->d_part,
                                                h->nblk, h->d_out, h->stream);
  } else {
    const KParams<double> P = kparams<double>(h->prm);
    const double* U[3] = {(double*)h->Q[cur][1], (double*)h->Q[cur][2], (double*)h->Q[cur][3]};
    e = h->prm.dim == 2 ? launch_diag<double, 2>(P, (double*)h->Q[cur][0], U, (double*)h->phi, nullptr,
                                                 h->d_part, h->nblk, h->d_out, h->stream)
                        : launch_diag<double, 3>(P, (double*)h->Q[cur][0], U, (double*)h->phi, nullptr,
                                                 h->d_part, h->nblk, h->d_out, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics");
  CK(h, cudaMemcpyAsync(h->h_out, h->d_out, 4 * sizeof(double) + sizeof(int), cudaMemcpyDeviceToHost, h->stream),
     "diag copy");
  CK(h, cudaStreamSynchronize(h->stream), "diag sync");
  int errw = 0;
  std::memcpy(&errw, h->h_out + 4, sizeof(int));
  if (errw != 0) return fail(h, GPE2P_ETIMEOUT, "a device-side copy did not complete within its bounded wait");
  d->int_phi = h->h_out[0];
  d->kinetic = h->h_out[1];
  d->umax = h->h_out[2];
  d->nan_flag = h->h_out[3] != 0.0 || !std::isfinite(h->h_out[0]) || !std::isfinite(h->h_out[1]);
  d->step = h->step;
  d->t = (double)h->step * h->prm.dt;
  return GPE2P_OK;
}

extern "C" int gpe2p_step(gpe2p_handle h) {
  if (!h) return fail(nullptr, GPE2P_EINVAL, "handle is NULL");
  if (h->batch) {
    std::string why;
    const int rc = batch_step(h->batch, why);
    return rc == GPE2P_OK ? rc : fail(h, rc, why);
  }
  if (!h->initialized) return fail(h, GPE2P_ESTATE, "gpe2p_step before gpe2p_init_fields");
  CK(h, cudaSetDevice(h->dev), "set device");
  if (!h->have_graph) {
    int rc = build_graphs(h);
    if (rc != GPE2P_OK) return rc;
  }
  CK(h, cudaGraphLaunch(h->gexec[h->cur], h->stream), "graph launch");
  h->cur = 1 - h->cur;
  h->step += 1;
  return GPE2P_OK;
}

static int any_diag(gpe2p_ctx* h, gpe2p_diag* d) {
  if (h->batch) {
    std::string why;
    const int rc = batch_diag(h->batch, -1, d, why);
    return rc == GPE2P_OK ? rc : fail(h, rc, why);
  }
  const int rc = diag_impl(h, d);
  if (rc != GPE2P_OK) return rc;
  return phi_acc_check(h, *d);
}

extern "C" int gpe2p_advance(gpe2p_handle h, long long nsteps, gpe2p_diag* last) {
  if (!h) return fail(nullptr, GPE2P_EINVAL, "handle is NULL");
  if (nsteps < 0) return fail(h, GPE2P_EINVAL, "nsteps < 0");
  if (!h->initialized && !h->batch) return fail(h, GPE2P_ESTATE, "gpe2p_advance before gpe2p_init_fields");
  gpe2p_diag d{};
  for (long long s = 0; s < nsteps; ++s) {
    int rc = gpe2p_step(h);
    if (rc != GPE2P_OK) return rc;
    if (h->prm.diag_every > 0 && (s + 1) % h->prm.diag_every == 0 && s + 1 < nsteps) {
      rc = any_diag(h, &d);
      if (rc != GPE2P_OK) return rc;
      if (d.nan_flag) {
        if (last) *last = d;
        return fail(h, GPE2P_EDIVERGED, "NaN/Inf in the state at step " + std::to_string(h->step));
      }
    }
  }
  int rc = any_diag(h, &d);
  if (rc != GPE2P_OK) return rc;
  if (last) *last = d;
  if (d.nan_flag) return fail(h, GPE2P_EDIVERGED, "NaN/Inf in the state at step " + std::to_string(d.step));
  return GPE2P_OK;
}

extern "C" int gpe2p_diagnostics(gpe2p_handle h, gpe2p_diag* out) {
  if (!h || !out) return fail(h, GPE2P_EINVAL, "NULL argument");
  if (h->batch) return any_diag(h, out);
  if (!h->initialized) return fail(h, GPE2P_ESTATE, "diagnostics before gpe2p_init_fields");
  CK(h, cudaSetDevice(h->dev), "set device");
  return any_diag(h, out);
}

extern "C" int gpe2p_set_phi_accumulation(gpe2p_handle h, int mode, double threshold) {
  if (!h) return fail(nullptr, GPE2P_EINVAL, "handle is NULL");
  if (h->batch) return fail(h, GPE2P_EINVAL, "a batch handle accumulates phi in its working precision");
  if (mode != GPE2P_PHI_ACC_FP32 && mode != GPE2P_PHI_ACC_COMPENSATED && mode != GPE2P_PHI_ACC_AUTO)
    return fail(h, GPE2P_EINVAL, "mode must be GPE2P_PHI_ACC_FP32, _COMPENSATED or _AUTO");
  if (!(threshold > 0.0) || !std::isfinite(threshold)) return fail(h, GPE2P_EINVAL, "threshold must be positive");
  CK(h, cudaSetDevice(h->dev), "set device");
  h->acc_mode = mode;
  h->drift_thr = threshold;
  if (mode == GPE2P_PHI_ACC_COMPENSATED) return phi_acc_on(h);
  if (mode == GPE2P_PHI_ACC_FP32 && h->phi_lo) {
    CK(h, cudaStreamSynchronize(h->stream), "phi accumulation");
    cudaFree(h->phi_lo);
    h->phi_lo = nullptr;
    for (int c = 0; c < 2; ++c)
      if (h->gexec[c]) { cudaGraphExecDestroy(h->gexec[c]); h->gexec[c] = nullptr; }
    h->have_graph = false;
  }
  return GPE2P_OK;
}

extern "C" int gpe2p_phi_accumulation(gpe2p_handle h, int* mode, int* active, double* drift,
                                      long long* switched_at) {
  if (!h) return fail(nullptr, GPE2P_EINVAL, "handle is NULL");
  if (mode) *mode = h->acc_mode;
  if (active) *active = h->phi_lo != nullptr;
  if (drift) *drift = h->last_drift;
  if (switched_at) *switched_at = h->switched_at;
  return GPE2P_OK;
}

template <typename real>
static cudaError_t get_field(gpe2p_ctx* h, const void* src, double* dst, const void* lo = nullptr) {
  cudaError_t e;
  double* ddst = static_cast<double*>(const_cast<void*>(device_view(dst)));
  if (sizeof(real) == 8 && h->pitch == h->prm.nx && !lo) {
    e = cudaMemcpyAsync(dst, src, (size_t)h->ncell * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  } else if (ddst) {
    // pinned destination: the conversion kernel writes the host array in place
    e = launch_to_double<real>(kparams<real>(h->prm), (const real*)src, ddst, h->ncell, h->stream,
                               (const real*)lo);
  } else {
    e = launch_to_double<real>(kparams<real>(h->prm), (const real*)src, h->d_stage, h->ncell, h->stream,
                               (const real*)lo);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dst, h->d_stage, (size_t)h->ncell * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  }
  return e;
}

static cudaError_t get_any(gpe2p_ctx* h, const void* src, double* dst, const void* lo = nullptr) {
  return h->esize == 4 ? get_field<float>(h, src, dst, lo) : get_field<double>(h, src, dst, lo);
}

extern "C" int gpe2p_read_fields(gpe2p_handle h, double* phi, double* u, double* v, double* w, double* p,
                                 double* mu) {
  if (!h) return fail(nullptr, GPE2P_EINVAL, "handle is NULL");
  if (h->batch) return fail(h, GPE2P_EINVAL, "a batch handle: use the per-instance calls");
  if (!h->initialized) return fail(h, GPE2P_ESTATE, "read_fields before gpe2p_init_fields");
  CK(h, cudaSetDevice(h->dev), "set device");
  double* dst[6] = {p, u, v, h->prm.dim == 3 ? w : nullptr, phi, mu};
  const void* src[6] = {h->Q[h->cur][0], h->Q[h->cur][1], h->Q[h->cur][2], h->Q[h->cur][3], h->phi, h->mu};
  for (int f = 0; f < 6; ++f)
    if (dst[f]) CK(h, get_any(h, src[f], dst[f], f == 4 ? h->phi_lo : nullptr), "read_fields");
  CK(h, cudaStreamSynchronize(h->stream), "read_fields sync");
  return GPE2P_OK;
}

template <typename real, int DIM>
static cudaError_t rates_impl(gpe2p_ctx* h) {
  const KParams<real> P = kparams<real>(h->prm);
  const int cur = h->cur;
  FlowArgs<real> A{};
  for (int f = 0; f < 4; ++f) {
    A.q0[f] = (const real*)h->Q[cur][f];
    A.q[f] = (const real*)h->Q[cur][f];
    A.out[f] = (real*)h->Q[2][f];
  }
  A.phi = (const real*)h->phi;
  A.mu = (const real*)h->mu;
  cudaError_t e = launch_flow_stage<real, DIM>(P, A, 0, h->kchunk, h->stream, &h->flow_maps[cur], h->d_err);
  if (e != cudaSuccess) return e;
  CHArgs<real> C{};
  for (int a = 0; a < 3; ++a) {
    C.uh[a] = (real*)h->uh[a];
    C.u0[a] = (const real*)h->Q[cur][1 + a];
    C.u1[a] = (const real*)h->Q[cur][1 + a];
  }
  C.conservative = h->prm.ch_advection;
  if (C.conservative) {
    const real* u0[3] = {C.u0[0], C.u0[1], C.u0[2]};
    real* uh[3] = {C.uh[0], C.uh[1], C.uh[2]};
    if ((e = launch_center_velocity<real, DIM>(P, u0, u0, uh, h->stream)) != cudaSuccess) return e;
  }
  C.scheme = h->prm.ch_scheme;
  C.stage = 0;
  C.compute_uh = !C.conservative;
  C.phis = (const real*)h->phi;
  C.mus = (const real*)h->mu;
  C.phin = (const real*)h->phi;
  C.out = (real*)h->phis[0];
  return launch_ch_stage<real, DIM>(P, C, h->prm.iso, h->kchunk_ch, h->stream, &h->ch_maps[0], h->d_err);
}

extern "C" int gpe2p_eval_rates(gpe2p_handle h, double* Lp, double* Lu, double* Lv, double* Lw, double* Lphi) {
  if (!h) return fail(nullptr, GPE2P_EINVAL, "handle is NULL");
  if (h->batch) return fail(h, GPE2P_EINVAL, "a batch handle: use the per-instance calls");
  if (!h->initialized) return fail(h, GPE2P_ESTATE, "eval_rates before gpe2p_init_fields");
  CK(h, cudaSetDevice(h->dev), "set device");
  cudaError_t e;
  if (h->esize == 4) e = h->prm.dim == 2 ? rates_impl<float, 2>(h) : rates_impl<float, 3>(h);
  else e = h->prm.dim == 2 ? rates_impl<double, 2>(h) : rates_impl<double, 3>(h);
  if (e != cudaSuccess) return cuda_fail(h, e, "eval_rates");
  double* dst[5] = {Lp, Lu, Lv, h->prm.dim == 3 ? Lw : nullptr, Lphi};
  const void* src[5] = {h->Q[2][0], h->Q[2][1], h->Q[2][2], h->Q[2][3], h->phis[0]};
  for (int f = 0; f < 5; ++f)
    if (dst[f]) CK(h, get_any(h, src[f], dst[f]), "eval_rates copy");
  CK(h, cudaStreamSynchronize(h->stream), "eval_rates sync");
  return GPE2P_OK;
}

extern "C" int gpe2p_profile_steps(gpe2p_handle h, int nsteps, double* ms, int max_launches, int* nlaunches,
                                   char* names, int names_len) {
  if (!h || !ms || !nlaunches || nsteps < 1 || max_launches < 1) return fail(h, GPE2P_EINVAL, "bad argument");
  if (h->batch) return fail(h, GPE2P_EINVAL, "a batch handle has no per-launch profile");
  if (!h->initialized) return fail(h, GPE2P_ESTATE, "profile_steps before gpe2p_init_fields");
  if (nsteps > 64) return fail(h, GPE2P_EINVAL, "at most 64 profiled steps");
  CK(h, cudaSetDevice(h->dev), "set device");
  // One untimed step, then the timed ones, all enqueued back to back with
  // their own events: each step's first event then waits on the GPU for the
  // previous step's last kernel, so no launch is charged with the host's
  // enqueue time (a wait for the GPU between steps would leave it idle while
  // the next step's first launch is being issued).
  const int cap = 32;
  const int nst = nsteps + 1;
  std::vector<cudaEvent_t> ev((size_t)nst * (cap + 1), nullptr);
  const char* nm[cap];
  int rc = GPE2P_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) { rc = cuda_fail(h, cudaGetLastError(), "event create"); break; }
  for (int i = 0; i < max_launches; ++i) ms[i] = 0.0;
  int n = 0;
  for (int s = 0; s < nst && rc == GPE2P_OK; ++s) {
    ProfHook hook;
    hook.ev = &ev[(size_t)s * (cap + 1)];
    hook.max = cap;
    hook.names = nm;
    cudaError_t e = enqueue(h, h->cur, &hook);
    if (e != cudaSuccess) { rc = cuda_fail(h, e, "profile step"); break; }
    h->cur = 1 - h->cur;
    h->step += 1;
    n = hook.n;
  }
  if (rc == GPE2P_OK) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_fail(h, e, "profile step");
  }
  for (int s = 1; s < nst && rc == GPE2P_OK; ++s) {
    const cudaEvent_t* se = &ev[(size_t)s * (cap + 1)];
    for (int i = 0; i < n && i < max_launches; ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, se[i], se[i + 1]);
      ms[i] += (double)t / nsteps;
    }
  }
  *nlaunches = n;
  if (names && names_len > 0) {
    std::string all;
    for (int i = 0; i < n; ++i) { if (i) all += ","; all += nm[i]; }
    std::snprintf(names, (size_t)names_len, "%s", all.c_str());
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  return rc;
}

extern "C" int gpe2p_field_ptr(gpe2p_handle h, int which, void** dptr, long long* row_pitch) {
  if (!h || !dptr) return fail(h, GPE2P_EINVAL, "NULL argument");
  if (h->batch) return fail(h, GPE2P_EINVAL, "a batch handle: use the per-instance calls");
  if (row_pitch) *row_pitch = h->pitch;
  if (which < 0 || which > 6 || (which == 3 && h->prm.dim == 2)) return fail(h, GPE2P_EINVAL, "bad field index");
  void* src[7] = {h->Q[h->cur][0], h->Q[h->cur][1], h->Q[h->cur][2], h->Q[h->cur][3], h->phi, h->mu, h->phi_lo};
  *dptr = src[which];
  return GPE2P_OK;
}

extern "C" const char* gpe2p_last_error(gpe2p_handle h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

extern "C" void gpe2p_destroy(gpe2p_handle h) {
  if (!h) return;
  if (h->batch) {
    batch_destroy(h->batch);
    if (h->d_dist) cudaFree(h->d_dist);
    if (h->h_dist) cudaFreeHost(h->h_dist);
    delete h;
    return;
  }
  cudaSetDevice(h->dev);
  // let the handle's work in flight finish before its memory goes
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->d_dist) cudaFree(h->d_dist);
  if (h->h_dist) cudaFreeHost(h->h_dist);
  if (h->phi_lo) cudaFree(h->phi_lo);
  for (int c = 0; c < 2; ++c)
    if (h->gexec[c]) cudaGraphExecDestroy(h->gexec[c]);
  if (h->base) cudaFree(h->base);
  if (h->h_out) cudaFreeHost(h->h_out);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

// ---------------------------------------------------------------------------
// batches of 2D problems
// ---------------------------------------------------------------------------

extern "C" int gpe2p_create_batch(const gpe2p_params* p, int n, void* stream, gpe2p_handle* out) {
  if (!out || !p) return fail(nullptr, GPE2P_EINVAL, "NULL argument");
  *out = nullptr;
  if (n < 1) return fail(nullptr, GPE2P_EINVAL, "n must be >= 1");
  for (int k = 0; k < n; ++k) {
    std::string why;
    int rc = validate(&p[k], why);
    if (rc != GPE2P_OK) return fail(nullptr, rc, "instance " + std::to_string(k) + ": " + why);
    if (p[k].check_stability) {
      double lim[3];
      gpe2p_stability_limits(&p[k], lim);
      for (int i = 0; i < 3; ++i)
        if (p[k].dt > lim[i] * (1.0 + 1e-12))
          return fail(nullptr, GPE2P_EUNSTABLE, "instance " + std::to_string(k) + ": dt beyond a stability limit");
    }
  }
  gpe2p_ctx* h = new (std::nothrow) gpe2p_ctx();
  if (!h) return fail(nullptr, GPE2P_ENOMEM, "host allocation failed");
  h->prm = p[0];
  std::string why;
  const int rc = batch_create(p, n, stream, &h->batch, why);
  if (rc != GPE2P_OK) {
    delete h;
    return fail(nullptr, rc, why);
  }
  cudaGetDevice(&h->dev);
  *out = h;
  return GPE2P_OK;
}

extern "C" int gpe2p_init_instance(gpe2p_handle h, int inst, const double* phi, const double* u, const double* v,
                                   const double*, const double* p) {
  if (!h || !h->batch) return fail(h, GPE2P_EINVAL, "not a batch handle");
  std::string why;
  const int rc = batch_init(h->batch, inst, phi, u, v, p, why);
  return rc == GPE2P_OK ? rc : fail(h, rc, why);
}

extern "C" int gpe2p_read_instance(gpe2p_handle h, int inst, double* phi, double* u, double* v, double*, double* p,
                                   double* mu) {
  if (!h || !h->batch) return fail(h, GPE2P_EINVAL, "not a batch handle");
  std::string why;
  const int rc = batch_read(h->batch, inst, phi, u, v, p, mu, why);
  return rc == GPE2P_OK ? rc : fail(h, rc, why);
}

extern "C" int gpe2p_diagnostics_instance(gpe2p_handle h, int inst, gpe2p_diag* out) {
  if (!h || !h->batch || !out) return fail(h, GPE2P_EINVAL, "not a batch handle or NULL output");
  if (inst < 0) return fail(h, GPE2P_EINVAL, "instance index out of range");
  std::string why;
  const int rc = batch_diag(h->batch, inst, out, why);
  return rc == GPE2P_OK ? rc : fail(h, rc, why);
}

extern "C" int gpe2p_batch_config(gpe2p_handle h, int* tile_x, int* tile_y, int* persistent, double* ms_per_step) {
  if (!h || !h->batch) return fail(h, GPE2P_EINVAL, "not a batch handle");
  return batch_config(h->batch, tile_x, tile_y, persistent, ms_per_step);
}

static_assert((int)GPE2P_LOSE_FLOW_RING == (int)WF_FLOW_RING && (int)GPE2P_LOSE_CH_RING == (int)WF_CH_RING &&
                  (int)GPE2P_LOSE_MU_RING == (int)WF_MU_RING && (int)GPE2P_LOSE_CH_POINTS == (int)WF_CH_POINTS,
              "the header's bits are the kernels' bits");

extern "C" int gpe2p_set_fault_injection(gpe2p_handle h, int what, long long value) {
  if (!h) return fail(nullptr, GPE2P_EINVAL, "handle is NULL");
  if (!h->batch) {
    // a single problem: the switch of the 3D kernels' timeout paths
    if (what == GPE2P_FAULT_LOSE_COPY) {
      if (h->prm.dim != 3) return fail(h, GPE2P_EINVAL, "GPE2P_FAULT_LOSE_COPY applies to 3D problems");
      if (value < 0 || value > 15) return fail(h, GPE2P_EINVAL, "GPE2P_FAULT_LOSE_COPY takes bits 1, 2, 4, 8");
      h->wait_fault = (int)value;
    } else if (what == GPE2P_FAULT_CLEAR) {
      h->wait_fault = 0;
      CK(h, cudaSetDevice(h->dev), "set device");
      CK(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream), "clear error word");
      CK(h, cudaStreamSynchronize(h->stream), "clear error word");
    } else {
      return fail(h, GPE2P_EINVAL, "a single problem takes GPE2P_FAULT_LOSE_COPY or GPE2P_FAULT_CLEAR");
    }
    for (int c = 0; c < 2; ++c)
      if (h->gexec[c]) { cudaGraphExecDestroy(h->gexec[c]); h->gexec[c] = nullptr; }
    h->have_graph = false;
    return GPE2P_OK;
  }
  if (what == GPE2P_FAULT_LOSE_COPY) return fail(h, GPE2P_EINVAL, "GPE2P_FAULT_LOSE_COPY applies to 3D problems");
  std::string why;
  const int rc = batch_fault(h->batch, what, value, why);
  return rc == GPE2P_OK ? rc : fail(h, rc, why);
}

// ---------------------------------------------------------------------------
// the state of a 2D problem as a network tensor
// ---------------------------------------------------------------------------

// the fields (phi, u, v, p, mu) of the single problem or of batch instance inst
template <typename real>
static int state_of(gpe2p_ctx* h, int inst, KParams<real>* P, real* f[5], int* iso, int** err) {
  if (h->batch) {
    *err = batch_err(h->batch);
    return batch_instance<real>(h->batch, inst, P, f, iso);
  }
  *P = kparams<real>(h->prm);
  const int c = h->cur;
  f[0] = (real*)h->phi;
  f[1] = (real*)h->Q[c][1];
  f[2] = (real*)h->Q[c][2];
  f[3] = (real*)h->Q[c][0];
  f[4] = (real*)h->mu;
  *iso = h->prm.iso;
  *err = h->d_err;
  return GPE2P_OK;
}

enum PackOp { OP_PACK, OP_UNPACK, OP_DISTANCE, OP_IFACE };

template <typename real>
static cudaError_t pack_op(gpe2p_ctx* h, int inst, PackOp op, float* t, int nch, const float* mean,
                           const float* scale, cudaStream_t s, int* rc) {
  KParams<real> P;
  real* f[5];
  int iso = 9;
  int* err = nullptr;
  *rc = state_of<real>(h, inst, &P, f, &iso, &err);
  if (*rc != GPE2P_OK) return cudaSuccess;
  if (op == OP_PACK) return launch_pack<real>(P, f, t, nch, mean, scale, s);
  if (op == OP_DISTANCE) return launch_distance<real>(P, f, t, nch, mean, scale, h->d_dist, h->d_dist + 8 * kDistanceBlocks, s);
  if (op == OP_IFACE)
    return launch_interface_distance<real>(P, f[0], t, nch, mean, scale, h->d_dist, h->d_dist + 8 * kDistanceBlocks, s);
  cudaError_t e = launch_unpack<real>(P, f, t, nch, mean, scale, s);
  if (e != cudaSuccess) return e;
  return launch_mu<real, 2>(P, f[0], f[4], iso, 1, s, nullptr, err);
}

static int pack_any(gpe2p_handle h, int inst, PackOp op, float* t, int nch, const float* mean, const float* scale,
                    double* dist) {
  if (!h || !t) return fail(h, GPE2P_EINVAL, "NULL argument");
  if (nch != 4 && nch != 5) return fail(h, GPE2P_EINVAL, "nch must be 4 or 5");
  for (int c = 0; c < nch; ++c)
    if ((scale && (!(scale[c] != 0.0f) || !std::isfinite(scale[c]))) || (mean && !std::isfinite(mean[c])))
      return fail(h, GPE2P_EINVAL, "mean and scale must be finite, scale nonzero");
  if (!h->batch && h->prm.dim != 2) return fail(h, GPE2P_EINVAL, "the tensor form is defined for 2D problems");
  if (h->batch && (inst < 0 || inst >= batch_size(h->batch))) return fail(h, GPE2P_EINVAL, "instance index out of range");
  if (!h->batch && !h->initialized && op != OP_UNPACK) return fail(h, GPE2P_ESTATE, "state used before gpe2p_init_fields");
  const int dev = h->batch ? batch_dev(h->batch) : h->dev;
  const int esize = h->batch ? batch_esize(h->batch) : h->esize;
  cudaStream_t s = h->batch ? batch_stream(h->batch) : h->stream;
  CK(h, cudaSetDevice(dev), "set device");
  if ((op == OP_DISTANCE || op == OP_IFACE) && !h->d_dist) {
    CK(h, cudaMalloc((void**)&h->d_dist, (8 * kDistanceBlocks + 8) * sizeof(double)), "distance scratch");
    CK(h, cudaMallocHost((void**)&h->h_dist, 8 * sizeof(double)), "distance scratch");
  }
  int rc = GPE2P_OK;
  cudaError_t e = esize == 4 ? pack_op<float>(h, inst, op, t, nch, mean, scale, s, &rc)
                             : pack_op<double>(h, inst, op, t, nch, mean, scale, s, &rc);
  if (rc != GPE2P_OK) return fail(h, rc, "instance index out of range");
  if (e != cudaSuccess)
    return cuda_fail(h, e, op == OP_PACK ? "pack" : op == OP_UNPACK ? "unpack" : op == OP_IFACE ? "interface distance"
                                                                                              : "distance");
  if (op == OP_UNPACK) {
    if (h->batch) batch_mark_initialized(h->batch);
    else h->initialized = true;
    if (!h->batch && h->phi_lo) CK(h, cudaMemsetAsync(h->phi_lo, 0, field_bytes(h), s), "unpack");
  }
  if (op == OP_DISTANCE || op == OP_IFACE) {
    const int nout = op == OP_DISTANCE ? 8 : 3;
    CK(h, cudaMemcpyAsync(h->h_dist, h->d_dist + 8 * kDistanceBlocks, nout * sizeof(double), cudaMemcpyDeviceToHost, s),
       "distance");
    CK(h, cudaStreamSynchronize(s), "distance");
    std::memcpy(dist, h->h_dist, nout * sizeof(double));
  }
  return GPE2P_OK;
}

extern "C" int gpe2p_pack_state(gpe2p_handle h, int inst, float* tensor, int nch, const float* mean,
                                const float* scale) {
  return pack_any(h, inst, OP_PACK, tensor, nch, mean, scale, nullptr);
}

extern "C" int gpe2p_unpack_state(gpe2p_handle h, int inst, const float* tensor, int nch, const float* mean,
                                  const float* scale) {
  return pack_any(h, inst, OP_UNPACK, const_cast<float*>(tensor), nch, mean, scale, nullptr);
}

extern "C" int gpe2p_state_distance(gpe2p_handle h, int inst, const float* tensor, int nch, const float* mean,
                                    const float* scale, double* out) {
  if (!out) return fail(h, GPE2P_EINVAL, "NULL argument");
  return pack_any(h, inst, OP_DISTANCE, const_cast<float*>(tensor), nch, mean, scale, out);
}

extern "C" int gpe2p_interface_distance(gpe2p_handle h, int inst, const float* tensor, int nch, const float* mean,
                                        const float* scale, double* out) {
  if (!out) return fail(h, GPE2P_EINVAL, "NULL argument");
  return pack_any(h, inst, OP_IFACE, const_cast<float*>(tensor), nch, mean, scale, out);
}
