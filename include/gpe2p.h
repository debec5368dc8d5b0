/*
 * gpe2p.h -- C ABI of the GB300 two-phase general-pressure-equation solver.
 *
 * Method: Huang, "A fully explicit method for two-phase incompressible flows
 * based on the general pressure equation" (arXiv 2011.00814).  One time step
 * is the TVD-RK3 update (Eq. tvd-rk3) of pressure and velocity on the
 * staggered grid of Sec. 3, with the pressure equation of
 * Eq. gpe-pressure-two-phase, the momentum equation of
 * Eq. gpe-momentum-two-phase-const-bf (stress with bulk viscosity,
 * Eq. vis-stress-two-phase; surface tension -sigma phi grad mu; gravity
 * (rho - rho_ref) g), phi and mu frozen at t^{n+1/2}; followed by one
 * Cahn-Hilliard step (Eqs. che, chem-pot) with the isotropic stencils of
 * Eqs. 1st-der-iso and laplacian-iso, TVD-RK2 (Eq. tvd-rk2) or RK4
 * (Eq. rk4), advected by the time-centred cell velocity of Eq. u-center-2d.
 *
 * Layout (all host and device arrays): one array of nx*ny*nz values per field,
 * x fastest, then y, then z (nz = 1 in 2D).  p, phi and mu are cell averages
 * at cell centres; the velocity component along axis c is stored on the face
 * of each cell on its LOW side along c (u[i,j] at x = i dx, v[i,j] at
 * y = j dx).  On a wall axis the face with index 0 is the wall itself: its
 * normal velocity is zero and is never updated; the opposite wall face
 * (index n) is implicit.  Boundary ghosts: p, phi, mu even; tangential
 * velocity odd (no-slip) or even (free-slip).
 *
 * p is the pressure deviation from the uniform reference pressure (only its
 * differences enter the method, Sec. 4), so the solver stores and returns it
 * as given; a run started from p = 0 holds p - p_ref.
 *
 * Errors: every call returns a gpe2p_status; nothing aborts.  The text of the
 * last error of a handle is returned by gpe2p_last_error.  A handle is not
 * thread-safe: calls on one handle must not run concurrently.
 * Ownership: the handle owns all device memory it allocates (released by
 * gpe2p_destroy); host arrays passed in stay owned by the caller and are only
 * accessed during the call.
 */
#ifndef GPE2P_H
#define GPE2P_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GPE2P_OK = 0,
  GPE2P_EINVAL = 1,     /* bad argument (size, parameter, pointer, dimension) */
  GPE2P_EUNSTABLE = 2,  /* dt beyond an explicit stability limit (check_stability = 1) */
  GPE2P_ENOMEM = 3,     /* device or pinned host allocation failed */
  GPE2P_ECUDA = 4,      /* a CUDA runtime call or kernel launch failed */
  GPE2P_EDIVERGED = 5,  /* NaN/Inf found in the state by the diagnostics */
  GPE2P_ETIMEOUT = 6,   /* a bounded device-side wait gave up */
  GPE2P_ESTATE = 7      /* call out of order (e.g. step before init_fields) */
} gpe2p_status;

enum { GPE2P_PERIODIC = 0, GPE2P_NOSLIP = 1, GPE2P_FREESLIP = 2 };

/* Parameters of one problem (Sec. 2, Sec. 4).  Physical units are the
 * caller's; the method is dimensional. */
typedef struct {
  int dim;                 /* 2 or 3 */
  int nx, ny, nz;          /* cells per axis, each in [1, 65536]; nz = 1 in 2D */
  double dx, dt, cs;       /* mesh size, time step, sound speed c_s (Eq. gpe-pressure) */
  double rhoL, rhoG;       /* densities at phi = +1 / -1 (Eq. density-viscosity-op-two-phase) */
  double etaL, etaG;       /* dynamic viscosities at phi = +1 / -1 */
  double rho_ref;          /* reference density of the hydrostatic split (Sec. 2) */
  double sigma;            /* physical surface tension; F_ST = -sigma phi grad mu */
  double M;                /* mobility of Eq. che */
  double W;                /* interface width: a = 3/(4W), kappa = 3W/8 (Eq. chem-pot) */
  double g[3];             /* constant body force per unit mass */
  int bc[3];               /* per axis (both sides): GPE2P_PERIODIC / NOSLIP / FREESLIP */
  int precision;           /* 32 (FP32 storage and arithmetic) or 64 */
  int ch_scheme;           /* 2: TVD-RK2 (Eq. tvd-rk2), 4: classic RK4 (Eq. rk4) */
  int iso;                 /* isotropic stencil lattice: 9 (2D), 15, 19, 27 (3D) */
  int bulk_visc;           /* 1: eta_b = eta (Sec. 2, the paper's choice); 0: eta_b = 0 */
  int p_average;           /* 1: averaged pressure in grad p (Eqs. gradp-u-*), 0: plain */
  int ch_advection;        /* 0: u.grad(phi) as in Eq. che; 1: div(u phi) (conservative) */
  int check_stability;     /* 1: gpe2p_create refuses dt beyond gpe2p_stability_limits */
  int diag_every;          /* gpe2p_advance: check for NaN/Inf every this many steps (0: at the end) */
  int axisym;              /* 1: the axisymmetric form (Sec. 2, Eqs. gpe-pressure-two-phase-axisym,
                            * gpe-momentum-two-phase-axisym-z/-r, che-axisym, div-v-axisym,
                            * chem-pot-axisym), dim = 2 only: x is the radius r, y the axis
                            * coordinate z, u = u_r, v = u_z; cell column i is centred at
                            * r = (i + 1/2) dx.  The low-x side is the axis, a symmetry line
                            * (u_r = 0, every other ghost even) whatever bc[0] says; bc[0] is
                            * the outer wall (NOSLIP or FREESLIP; PERIODIC is refused).  Needs
                            * ch_advection = 0 and g[0] = 0.  The stability limits and the
                            * diagnostics stay those of the planar (x, y) grid (on small test
                            * grids the limits held for the axisymmetric operator's spectrum
                            * too); int_phi and kinetic sum over the (r, z) plane, not over
                            * the volume. */
} gpe2p_params;

typedef struct gpe2p_ctx *gpe2p_handle;

/* Scalar diagnostics of the current state (FP64 reductions in any precision). */
typedef struct {
  double int_phi;     /* sum over cells of phi dx^dim */
  double kinetic;     /* 1/2 sum over faces of rho_face u^2 dx^dim */
  double umax;        /* max over faces of |velocity component| */
  int nan_flag;       /* 1 if any of p, phi or a velocity component is NaN or Inf */
  long long step;     /* steps taken since gpe2p_init_fields */
  double t;           /* step * dt */
} gpe2p_diag;

/* Explicit stability limits of dt for the parameters: out[0] acoustic
 * (RK3 imaginary-axis limit sqrt 3 against the staggered acoustic operator,
 * with the pressure averaging), out[1] viscous (RK3 real-axis limit against
 * the largest shear + bulk viscous and pressure-diffusion eigenvalue),
 * out[2] Cahn-Hilliard (RK2/RK4 real-axis limit against M lam (8a + kappa lam),
 * lam the largest magnitude of the isotropic Laplacian symbol).  Host-only;
 * needs no GPU.  Returns GPE2P_EINVAL on bad parameters. */
int gpe2p_stability_limits(const gpe2p_params *p, double out_dt_max[3]);

/* Validates p, allocates the device state on the current CUDA device and
 * creates the handle.  stream: a cudaStream_t to run on, or NULL for a
 * stream the handle creates (non-blocking).  The state is undefined until
 * gpe2p_init_fields. */
int gpe2p_create(const gpe2p_params *p, void *stream, gpe2p_handle *out);

/* Sets the state from host arrays (nx*ny*nz doubles each, layout above):
 * phi, u, v and p are required, w is required in 3D and ignored in 2D.
 * Arrays in pinned host memory (cudaHostAlloc, cudaHostRegister) are read in
 * place by the device through their mapped address; pageable arrays are
 * copied through a staging buffer.  Either way the call returns after the
 * last read.
 * Wall faces of the normal velocity are set to zero.  mu is computed from
 * phi (Eq. chem-pot); phi is taken as phi^{1/2} of the time-staggered scheme
 * (Sec. 3).  Resets the step counter.  Synchronises the handle's stream. */
int gpe2p_init_fields(gpe2p_handle h, const double *phi, const double *u, const double *v,
                      const double *w, const double *p);

/* Advances one full step (flow TVD-RK3 + CH step), asynchronously on the
 * handle's stream.  The first call on a handle captures the step into CUDA
 * graphs and should come before any capture the caller runs on the stream. */
int gpe2p_step(gpe2p_handle h);

/* Advances nsteps full steps by replaying the captured step graphs; checks
 * for NaN/Inf every diag_every steps and at the end (GPE2P_EDIVERGED if
 * found: the state is left as it was at that check and stays readable).
 * If last != NULL it receives the diagnostics at the end.  Synchronises. */
int gpe2p_advance(gpe2p_handle h, long long nsteps, gpe2p_diag *last);

/* Copies the state to host arrays (nx*ny*nz doubles each).  Any pointer
 * may be NULL to skip that field; w is ignored in 2D.  Pinned host arrays
 * are written in place by the device (FP32 states: the conversion to FP64
 * writes them directly).  Synchronises. */
int gpe2p_read_fields(gpe2p_handle h, double *phi, double *u, double *v, double *w, double *p,
                      double *mu);

/* Diagnostics of the current state (see gpe2p_diag).  Synchronises. */
int gpe2p_diagnostics(gpe2p_handle h, gpe2p_diag *out);

/* Semi-discrete rates of the current state, for operator-level checks:
 * Lp, Lu, Lv, Lw the right-hand sides of the flow equations
 * (Eq. p-u-v-semidiscrete-2d; zero on wall faces) and Lphi the CH rate
 * -uhat.grad(phi) + M lap(mu) (Eq. che) with uhat the cell average of the
 * current face velocities.  Host arrays of nx*ny*nz doubles; any may be
 * NULL; Lw is ignored in 2D.  Synchronises. */
int gpe2p_eval_rates(gpe2p_handle h, double *Lp, double *Lu, double *Lv, double *Lw, double *Lphi);

/* Measurement aid: advances nsteps + 1 full steps (1 <= nsteps <= 64)
 * launched eagerly (not from the graphs) and back to back, timing every
 * kernel launch of the last nsteps with CUDA events on the handle's stream
 * (the first step only fills the queue, so that no launch is charged with
 * the time the host takes to issue it).  ms[i] receives the mean duration in
 * milliseconds of the i-th launch of a step (i < max_launches), *nlaunches
 * the launches per step, names (if not NULL) a comma-separated list of their
 * kernel names, truncated to names_len bytes.  The state advances exactly as
 * with gpe2p_advance.  Synchronises. */
int gpe2p_profile_steps(gpe2p_handle h, int nsteps, double *ms, int max_launches, int *nlaunches,
                        char *names, int names_len);

/* Measurement aid (the paper has no counterpart): the rate of fused
 * multiply-adds of the current device in the given precision (32 or 64),
 * in floating-point operations per second (two per multiply-add), written to
 * *flops_per_s; *ms (may be NULL) receives the duration of the timed launch.
 * Independent chains of multiply-adds in every thread of a grid of eight
 * 256-thread blocks per SM, sized to run about 50 ms, the best of three
 * launches after a calibration launch, timed with CUDA events on stream (a
 * cudaStream_t, NULL for the legacy default stream).  The FP64 path of the
 * step is bound by this FP64 rate rather than by memory bandwidth.
 * Allocates nothing; synchronises the stream.  GPE2P_EINVAL for a NULL
 * pointer or another precision, GPE2P_ECUDA if a launch fails. */
int gpe2p_fma_rate(int precision, double *flops_per_s, double *ms, void *stream);

/* Measurement aid (the paper has no counterpart): the issue rate of the
 * tensor cores as the surrogate's convolutions use them.  On one SM, lane 0
 * of `issuers` warps (1, 2 or 4) each issues back-to-back tcgen05.mma
 * (kind::f16, BF16 operands from shared memory, FP32 accumulator in tensor
 * memory, M = 128, N = n in {32, 64, 128, 256}, K = 16) into its own
 * accumulator, n * issuers <= 512 columns.  *cycles_per_mma receives the SM
 * clock cycles per MMA of the whole SM (the slowest issuer's elapsed cycles
 * over all issuers' MMAs), the best of three launches after a warm-up, on
 * stream (a cudaStream_t, NULL for the legacy default stream).  128 n 16
 * multiply-adds over this figure is the SM's multiply-add rate at that N.
 * Allocates nothing; synchronises the stream.  GPE2P_EINVAL for a NULL
 * pointer or another n or issuer count, GPE2P_ETIMEOUT if the bounded wait
 * for the MMAs gave up, GPE2P_ECUDA if a launch or copy fails. */
int gpe2p_mma_rate(int n, int issuers, double *cycles_per_mma, void *stream);

/* Device pointer of a field of the current state, in the handle's precision
 * (float or double): which = 0 p, 1 u, 2 v, 3 w, 4 phi, 5 mu, 6 the low part
 * of phi under the compensated accumulation (phi = field 4 + field 6; see
 * gpe2p_set_phi_accumulation), for which *dptr is NULL while that
 * accumulation is not active.  On the device
 * every field is stored x-fastest with rows padded to *row_pitch elements
 * (a multiple of 32; row (j, k) starts at element (k ny + j) row_pitch);
 * row_pitch may be NULL.  Valid until the next call that advances,
 * re-initialises or destroys the handle. */
int gpe2p_field_ptr(gpe2p_handle h, int which, void **dptr, long long *row_pitch);

/* ---- batches of independent 2D problems ------------------------------ */

/* Creates one handle for n independent 2D problems p[0..n-1] (uneven sizes,
 * their own physical parameters and boundaries; one precision; TVD-RK2 for
 * the CH step).  All instances advance together: gpe2p_step and
 * gpe2p_advance run every sweep of the method over the tiles of all
 * instances, either as one cooperative persistent launch per step whose
 * blocks meet at a bounded grid barrier between sweeps, or as one launch per
 * sweep; both are captured into CUDA graphs.  The tile shape and the form
 * are chosen at creation by timing each candidate on the zero state (the
 * state is zeroed again afterwards).  gpe2p_diagnostics of a batch sums
 * int_phi and kinetic over the instances and takes the max of umax and the
 * NaN flags; gpe2p_init_fields and gpe2p_read_fields do not apply to a batch
 * (GPE2P_EINVAL): use the per-instance calls below. */
int gpe2p_create_batch(const gpe2p_params *p, int n, void *stream, gpe2p_handle *out);

/* Sets instance inst of a batch from host arrays (nx*ny doubles each, the
 * layout of the single-problem calls; w is ignored) and computes its mu.
 * Resets the batch's step counter.  Synchronises. */
int gpe2p_init_instance(gpe2p_handle h, int inst, const double *phi, const double *u, const double *v,
                        const double *w, const double *p);

/* Copies instance inst of a batch to host arrays; NULL pointers are skipped. */
int gpe2p_read_instance(gpe2p_handle h, int inst, double *phi, double *u, double *v, double *w, double *p,
                        double *mu);

/* Diagnostics of one instance of a batch. */
int gpe2p_diagnostics_instance(gpe2p_handle h, int inst, gpe2p_diag *out);

/* The configuration the autotuner chose for a batch: tile shape, 1 for the
 * persistent form (0: one launch per sweep), and its measured ms per step. */
int gpe2p_batch_config(gpe2p_handle h, int *tile_x, int *tile_y, int *persistent, double *ms_per_step);

/* Host-side fault injection and test switches (rebuilds the step graphs).
 * A batch takes GPE2P_FAULT_SKIP_BARRIER (value = block index that never
 * arrives at the grid barrier; -1 none), GPE2P_FAULT_WAIT_LIMIT (barrier wait
 * limit in SM clock cycles), GPE2P_FAULT_FORCE_PERSISTENT (1: persistent
 * form, 0: one launch per sweep) and GPE2P_FAULT_CLEAR (defaults, and clears
 * the error word).  A barrier wait that runs out makes every block return and
 * the next diagnostics report GPE2P_ETIMEOUT; the state is then undefined.
 * A single 3D problem takes GPE2P_FAULT_LOSE_COPY, value a mask of
 * GPE2P_LOSE_* bits: in every block of the chosen kernels the first wait of
 * that kind for a plane copy (which still completes, so that no copy is left
 * in flight) is reported as timed out, as if the copy had been lost; the
 * block then records the error, waits for its other copies and returns, and
 * the next diagnostics report GPE2P_ETIMEOUT.  GPE2P_FAULT_CLEAR (value
 * ignored) turns it off and clears the error word; gpe2p_init_fields also
 * clears the error word.  No fault reaches the GPU: only the kernels' own
 * bounded-wait bookkeeping is exercised. */
enum { GPE2P_FAULT_SKIP_BARRIER = 1, GPE2P_FAULT_WAIT_LIMIT = 2, GPE2P_FAULT_FORCE_PERSISTENT = 3,
       GPE2P_FAULT_CLEAR = 4, GPE2P_FAULT_LOSE_COPY = 5 };
/* bits of GPE2P_FAULT_LOSE_COPY: the plane rings of the flow stage, of the CH
 * stages and of mu, and the CH stages' point planes */
enum { GPE2P_LOSE_FLOW_RING = 1, GPE2P_LOSE_CH_RING = 2, GPE2P_LOSE_MU_RING = 4, GPE2P_LOSE_CH_POINTS = 8 };
int gpe2p_set_fault_injection(gpe2p_handle h, int what, long long value);

/* ---- precision policy of the phi accumulation --------------------------
 * FP32 problems store phi^{n+1/2} in FP32.  The Cahn-Hilliard update
 * conserves the phi integral exactly in exact arithmetic with the
 * conservative advection form (and with the diffusion part of Eq. che in
 * either form); FP32 rounding of phi + dt L makes the integral drift.  With
 * the compensated accumulation on, phi is held as an FP32 high/low pair and
 * the final RK stage of each step forms phi^{n+3/2} in FP64 (about 48
 * significant bits), while the stencils keep reading the FP32 high part.
 * Modes: GPE2P_PHI_ACC_FP32 (off), GPE2P_PHI_ACC_COMPENSATED (on),
 * GPE2P_PHI_ACC_AUTO (the default: switched on for the rest of the run at
 * the first diagnostics -- gpe2p_diagnostics, the end of gpe2p_advance and
 * every diag_every steps inside it -- at which the relative drift
 * |int phi - int phi_0| / int |phi_0| exceeds threshold, 1e-10 by default).
 * The drift is measured from the state set by gpe2p_init_fields.  The low
 * part is included in gpe2p_read_fields and in the diagnostics.  FP64
 * problems and batches ignore the policy.  The paper has no counterpart. */
enum { GPE2P_PHI_ACC_FP32 = 0, GPE2P_PHI_ACC_COMPENSATED = 1, GPE2P_PHI_ACC_AUTO = 2 };
int gpe2p_set_phi_accumulation(gpe2p_handle h, int mode, double threshold);
/* The mode, whether the compensated accumulation is active, the last
 * measured relative drift and the step at which it was switched on (-1:
 * not switched since gpe2p_init_fields).  Any pointer may be NULL. */
int gpe2p_phi_accumulation(gpe2p_handle h, int *mode, int *active, double *drift, long long *switched_at);

/* ---- the learned surrogate ------------------------------------------- */
/* A convolutional U-Net on the periodic 2D grid that learns to advance the
 * state over many solver steps (the paper has no learned component): levels
 * l = 0..L-1 with channels[l] (multiples of 16) at resolution H/2^l;
 * encoder l: [2x2 average pooling if l > 0] conv3x3 + SiLU, conv3x3 + SiLU;
 * decoder l = L-2..0: nearest 2x upsampling, conv3x3 + SiLU, concatenation
 * with the encoder output of level l, conv3x3 + SiLU, conv3x3 + SiLU; a 1x1
 * head to out_ch channels.  Convolutions pad circularly.  BF16 weights and
 * activations, FP32 accumulation on the tensor cores, FP32 master weights,
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).  Tensors are FP32
 * device arrays in NHWC order [batch][H][W][channels]. */
typedef struct gpe2p_net *gpe2p_net_handle;

/* Creates the network with seeded He-uniform weights (zero biases, a head
 * scaled by 0.01).  in_ch, out_ch in [1, 16]; H, W multiples of
 * 2^(levels-1); max_batch bounds the batch of every call. */
int gpe2p_net_create(int levels, const int *channels, int in_ch, int out_ch, int H, int W, int max_batch,
                     unsigned long long seed, void *stream, gpe2p_net_handle *out);
/* Number of FP32 parameters (the layout: per convolution, in the order
 * encoder 0..L-1 (a, b), then decoder L-2..0 (up, a, b): weights
 * [cout][tap][cin] with tap = 3(dy+1) + (dx+1), then bias [cout]; then the
 * head weights [out_ch][channels[0]] and bias [out_ch]). */
long long gpe2p_net_num_params(gpe2p_net_handle n);
int gpe2p_net_get_params(gpe2p_net_handle n, float *host, long long count);
/* Sets the master weights (and resets the Adam moments). */
int gpe2p_net_set_params(gpe2p_net_handle n, const float *host, long long count);
/* Input normalisation and output map (host arrays of in_ch, in_ch and
 * out_ch floats; NULL for 0, 1, 1): the network sees
 * (x[c] - in_mean[c]) / in_scale[c] and returns
 * y[c] = (residual ? x[c] : 0) + out_scale[c] * head[c], so that with
 * residual = 1 it predicts the increment of its first out_ch input
 * channels; the loss below is then taken on (y - t) / out_scale.  Defaults
 * 0, 1, 1, residual 0.  residual needs out_ch <= in_ch. */
int gpe2p_net_set_normalization(gpe2p_net_handle n, const float *in_mean, const float *in_scale,
                                const float *out_scale, int residual);
/* y[batch][H][W][out_ch] = net(x[batch][H][W][in_ch]); device pointers; asynchronous. */
int gpe2p_net_forward(gpe2p_net_handle n, const float *x, float *y, int batch);
/* Loss = mean over all outputs of ((net(x) - t) / out_scale)^2 and its gradient with
 * respect to the master weights, copied to grad (host, num_params floats)
 * if not NULL.  Synchronises. */
int gpe2p_net_gradients(gpe2p_net_handle n, const float *x, const float *t, int batch, float *grad, float *loss);
/* One training step: the loss above, its gradient and one Adam update with
 * learning rate lr.  The loss is copied to *loss if not NULL (which
 * synchronises).  */
int gpe2p_net_train_step(gpe2p_net_handle n, const float *x, const float *t, int batch, float lr, float *loss);
/* Kernels of the 3x3 forward and data-gradient convolutions: 1 (default)
 * tcgen05.mma with the accumulator in tensor memory, 0 the warp-level
 * mma.sync kernels.  Both compute the same products (FP32 accumulation in a
 * different order). */
int gpe2p_net_set_backend(gpe2p_net_handle n, int tcgen05);
/* Host-side test switch of the tcgen05 convolutions (the forward graph is
 * rebuilt).  GPE2P_FAULT_LOSE_COPY with value 1: in every CTA of those
 * kernels the first wait for a filled pipeline stage, whose copies have in
 * fact all landed, is reported as timed out; the CTA's other roles give up
 * their waits, it lets any copy or MMA in flight finish, frees its tensor
 * memory, records the error word and returns, and gpe2p_net_sync then
 * reports GPE2P_ETIMEOUT (the outputs of those calls are undefined); value 0
 * turns it off.  GPE2P_FAULT_CLEAR turns it off and clears the error word.
 * No fault reaches the GPU.  GPE2P_EINVAL for other kinds or values. */
int gpe2p_net_fault(gpe2p_net_handle n, int what, int value);
/* Waits for the network's stream and reports GPE2P_ETIMEOUT if a tensor-core
 * kernel gave up a bounded wait since the handle was created or the error
 * word was last cleared (the outputs of that call are then undefined).  gpe2p_net_gradients and
 * gpe2p_net_train_step (with a loss pointer) report it too. */
int gpe2p_net_sync(gpe2p_net_handle n);
/* Multiply-add FLOPs (x2) of one forward pass of a batch. */
double gpe2p_net_flops(gpe2p_net_handle n, int batch);
const char *gpe2p_net_last_error(gpe2p_net_handle n);
void gpe2p_net_destroy(gpe2p_net_handle n);

/* ---- the state as a network tensor --------------------------------------
 * The learned surrogate (a network that advances the state over many
 * steps) reads and writes the state of a 2D problem as a
 * device array tensor[ny][nx][nch] of floats, nch = 4 or 5, with the
 * channels 0 phi, 1 u, 2 v, 3 p (the velocity components of the cell's low
 * faces, p the stored deviation from rho_ref c_s^2) and, for nch = 5,
 * 4 rho(phi)/rho_L (the density law of Sec. 2).  Element (j, i, c) holds
 * (field_c at cell (i, j) - mean[c]) / scale[c]; mean and scale are host
 * arrays of nch floats (scale nonzero), or NULL for 0 and 1.  inst is the
 * instance of a batch handle and is ignored for a single problem.  The
 * paper has no counterpart of these calls.  All are ordered on the
 * handle's stream; only gpe2p_state_distance waits for it. */
int gpe2p_pack_state(gpe2p_handle h, int inst, float *tensor, int nch, const float *mean, const float *scale);
/* The inverse: sets phi, u, v, p to mean[c] + scale[c] * tensor (channel 4
 * is not read; wall faces of the normal velocity stay zero) and recomputes
 * mu from phi (the chemical-potential equation).  The step counter is kept. */
int gpe2p_unpack_state(gpe2p_handle h, int inst, const float *tensor, int nch, const float *mean,
                       const float *scale);
/* FP64 sums over the cells, for c = 0..3 (phi, u, v, p):
 * out[2c] = sum (field_c - (mean[c] + scale[c] tensor_c))^2 and
 * out[2c+1] = sum field_c^2 (out: 8 doubles on the host).  A per-handle
 * scratch of about 20 KB is allocated on the first call.  Deterministic. */
int gpe2p_state_distance(gpe2p_handle h, int inst, const float *tensor, int nch, const float *mean,
                         const float *scale, double *out);

/* The displacement of the phi = 0 interface, in cells, between the state's
 * phi (the reference phi_b; instance inst of a batch) and the phi channel of
 * a network tensor, phi_a = mean[0] + scale[0] tensor[j][i][0]:
 * out[0] = max over the cells with |phi_b| < 1/2 of |phi_a - phi_b| /
 * |grad phi_b|, out[1] = sum |phi_a - phi_b| / sum |grad phi_b| over all
 * cells (for the equilibrium profile tanh(2d/W) the mean normal
 * displacement), out[2] = the number of cells with |phi_b| < 1/2 (host
 * array of 3 doubles).  grad phi_b by central differences in cell units, with
 * the boundaries' ghost rules.  The paper has no counterpart: the learned
 * surrogate's check compares one network call with the solver by it.  FP64
 * sums in a fixed order (deterministic); shares the scratch of
 * gpe2p_state_distance.  Synchronises. */
int gpe2p_interface_distance(gpe2p_handle h, int inst, const float *tensor, int nch, const float *mean,
                             const float *scale, double *out);

/* Largest number of cells gpe2p_diagnostics_noalloc accepts. */
#define GPE2P_NOALLOC_MAX_CELLS 67108864LL

/* The paper has no counterpart to this entry point: it serves callers that
 * cannot allocate device memory when they need the diagnostics (inside a
 * CUDA-graph capture or a custom memory pool, a device handed over to
 * another allocator, a loop that must not block in cudaMalloc).  It computes
 * the four values of gpe2p_diagnostics (sum of phi dx^dim, kinetic energy,
 * max |velocity component|, NaN/Inf flag as 0.0/1.0, in that order) of a
 * state the caller holds on the current device and writes them to out, a
 * caller-owned device array of 4 doubles.
 *   p, u, v, w, phi: device arrays in the precision p->precision (32: float,
 *   64: double), in the layout of gpe2p_field_ptr with rows of row_pitch
 *   elements (>= nx); w may be NULL in 2D.  Only the dim, nx, ny, nz, dx,
 *   rhoL, rhoG, bc and precision members of *p are used.
 *   phi_lo: the low part of phi in the same layout and precision (field 6 of
 *   gpe2p_field_ptr, while the compensated accumulation is active), or NULL
 *   for none.  With it, the phi integral and each cell's density take
 *   phi + phi_lo, as gpe2p_diagnostics does.
 *   stream: a cudaStream_t, or NULL for the legacy default stream.  The call
 *   is asynchronous; out is valid once the stream has reached it.
 * It allocates nothing: its scratch is a fixed device array of 512 KiB in the
 * library, held by every GPU that loads the library until the process
 * exits.  The first call on a device (with that device current) looks up
 * that array's device address, so it should come before any stream capture;
 * calls made while their stream is not capturing look it up again, so the
 * call stays valid after a device reset.  All calls share the array: calls
 * whose work overlaps on the GPU race.
 * Returns GPE2P_EINVAL for a NULL pointer, bad parameters or more than
 * GPE2P_NOALLOC_MAX_CELLS cells, GPE2P_ECUDA if a launch fails; it records
 * no error text. */
int gpe2p_diagnostics_noalloc(const gpe2p_params *p, const void *pfield, const void *u, const void *v,
                              const void *w, const void *phi, const void *phi_lo, long long row_pitch,
                              double *out, void *stream);

/* Text of the handle's last error ("" if none); with h == NULL, the last
 * error of a failed gpe2p_create on this thread. */
const char *gpe2p_last_error(gpe2p_handle h);

/* Releases the handle and its device memory.  NULL is ignored. */
void gpe2p_destroy(gpe2p_handle h);

#ifdef __cplusplus
}
#endif

#endif /* GPE2P_H */
