/*
 * gpe2p_oracle.c -- plain CPU FP64 oracle of the two-phase GPE method
 * (Huang, arXiv 2011.00814: general pressure equation + Cahn-Hilliard,
 * staggered grid, TVD-RK3 flow marching).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header, table or constant
 * with the CUDA path.
 *
 * Every routine is a plain loop over cells that evaluates the paper's discrete
 * formulas in the order the paper writes them, in double precision.  Build with
 * -ffp-contract=off so that no multiply-add is fused behind the reader's back.
 *
 * Grid (Sec. 3, staggered-grid figure): cell (i,j,k) has its centre at
 * ((i+1/2)dx, (j+1/2)dx, (k+1/2)dx).  p, phi, mu, rho, eta live at centres.
 * The velocity component along axis c is stored on the face of cell (i,j,k)
 * on its LOW side along c (u[i,j] at x = i dx, v[i,j] at y = j dx).  This
 * placement is the one forced by the divergence (Eq. div-v-discretization,
 * u_{i+1,j}-u_{i,j} spans cell i) and by the surface-tension and pressure
 * gradient terms (Eqs. st-u-discretization, gradp-u-discretization, which put
 * u_{i,j} between cells i-1 and i).  All arrays are nx*ny*nz doubles, x fastest.
 *
 * Boundaries (the paper names them but never writes their discrete form; the
 * reading taken here): on a wall the normal velocity face is zero and is never
 * updated; ghosts of the normal component are odd about the wall face, ghosts
 * of a tangential component are odd (no-slip) or even (free-slip) about the
 * wall; ghosts of p, phi, mu (hence rho, eta, nu) are even (zero normal
 * gradient, 90 degree contact angle, no diffusive flux through the wall).
 *
 * Axisymmetric form (Eqs. gpe-pressure-two-phase-axisym,
 * gpe-momentum-two-phase-axisym-z and -r, che-axisym, div-v-axisym,
 * chem-pot-axisym), axisym = 1, 2D only: x is the radius r and y the axis
 * coordinate z, so u is u_r and v is u_z; cell i is centred at
 * r = (i + 1/2) dx and the u face i lies at r = i dx.  The low-x side is the
 * axis: u_r = 0 on it and every ghost across it is even (a symmetry line,
 * whatever bc[0] says); bc[0] applies to the outer wall only.  The terms the
 * axisymmetric equations add to the planar ones are evaluated as printed,
 * with the derivatives by central differences at the point where the
 * equation lives and the viscosity on a face as the mean of the two cells it
 * separates (the same mean the planar scheme takes for the density there).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PERIODIC 0
#define ORC_NOSLIP 1
#define ORC_FREESLIP 2

typedef struct {
  int dim;            /* 2 or 3 */
  int nx, ny, nz;     /* cells; nz = 1 in 2D */
  double dx, dt, cs;  /* mesh size, time step, sound speed */
  double rhoL, rhoG, etaL, etaG, rho_ref;
  double sigma, M, W; /* surface tension, mobility, interface width */
  double g[3];        /* body force per unit mass */
  int bc[3];          /* per axis, both sides: periodic / no-slip / free-slip */
  int ch_scheme;      /* 2: TVD-RK2, 4: classic RK4 */
  int iso;            /* lattice for isotropic CH stencils: 9, 15, 19, 27 */
  int bulk_visc;      /* 1: eta_b = eta (Sec. 2), 0: eta_b = 0 */
  int p_average;      /* 1: averaged pressure in grad p (Eqs. gradp-u-*) */
  int ch_advection;   /* 0: u.grad(phi) as in Eq. che; 1: div(u phi) */
  int axisym;         /* 1: axisymmetric (r, z) form, x = r, y = z (2D only) */
} orc_par;

/* ------------------------------------------------------------------ */
/* index maps with the boundary reading above                          */
/* ------------------------------------------------------------------ */

static int nlen(const orc_par *P, int a) { return a == 0 ? P->nx : (a == 1 ? P->ny : P->nz); }

static size_t lin(const orc_par *P, const int x[3]) {
  return (size_t)x[0] + (size_t)P->nx * ((size_t)x[1] + (size_t)P->ny * (size_t)x[2]);
}

/* value of a cell-centred field at a (possibly ghost) cell */
static double cen(const orc_par *P, const double *f, int i, int j, int k) {
  int x[3] = {i, j, k};
  for (int a = 0; a < P->dim; ++a) {
    int n = nlen(P, a);
    if (P->bc[a] == ORC_PERIODIC) {
      x[a] %= n;
      if (x[a] < 0) x[a] += n;
    } else {
      if (x[a] < 0) x[a] = -1 - x[a];
      else if (x[a] >= n) x[a] = 2 * n - 1 - x[a];
    }
  }
  return f[lin(P, x)];
}

/* value of velocity component c (stored on low faces along c) at a face */
static double fac(const orc_par *P, const double *f, int c, int i, int j, int k) {
  int x[3] = {i, j, k};
  double s = 1.0;
  for (int a = 0; a < P->dim; ++a) {
    int n = nlen(P, a);
    if (P->bc[a] == ORC_PERIODIC) {
      x[a] %= n;
      if (x[a] < 0) x[a] += n;
    } else if (a == c) {
      /* odd about a wall face; a mirrored index can land on the opposite
       * wall face (n = 1), which is zero as well */
      if (x[a] < 0) { x[a] = -x[a]; s = -s; }
      else if (x[a] > n) { x[a] = 2 * n - x[a]; s = -s; }
      if (x[a] == 0 || x[a] == n) return 0.0;
    } else {
      /* the axis (low x of the axisymmetric form) mirrors tangential
       * components evenly */
      int axis = P->axisym && a == 0;
      if (x[a] < 0) { x[a] = -1 - x[a]; if (P->bc[a] == ORC_NOSLIP && !axis) s = -s; }
      else if (x[a] >= n) { x[a] = 2 * n - 1 - x[a]; if (P->bc[a] == ORC_NOSLIP) s = -s; }
    }
  }
  return s * f[lin(P, x)];
}

/* cell-centred vector component c (the averaged CH velocity): odd across a
 * wall normal to c, even across the other walls */
static double cvec(const orc_par *P, const double *f, int c, int i, int j, int k) {
  int x[3] = {i, j, k};
  double s = 1.0;
  for (int a = 0; a < P->dim; ++a) {
    int n = nlen(P, a);
    if (P->bc[a] == ORC_PERIODIC) {
      x[a] %= n;
      if (x[a] < 0) x[a] += n;
    } else {
      if (x[a] < 0) { x[a] = -1 - x[a]; if (a == c) s = -s; }
      else if (x[a] >= n) { x[a] = 2 * n - 1 - x[a]; if (a == c) s = -s; }
    }
  }
  return s * f[lin(P, x)];
}

/* is the face of component c at cell x a wall face (never updated)? */
static int wall_face(const orc_par *P, int c, const int x[3]) {
  return P->bc[c] != ORC_PERIODIC && x[c] == 0;
}

/* ------------------------------------------------------------------ */
/* material laws, Eq. density-viscosity-op-two-phase                    */
/* ------------------------------------------------------------------ */

static double rho_of(const orc_par *P, double phi) {
  return 0.5 * (P->rhoL * (1.0 + phi) + P->rhoG * (1.0 - phi));
}
static double eta_of(const orc_par *P, double phi) {
  return 0.5 * (P->etaL * (1.0 + phi) + P->etaG * (1.0 - phi));
}
static double nu_of(const orc_par *P, double phi) { return eta_of(P, phi) / rho_of(P, phi); }

static double rho_at(const orc_par *P, const double *phi, const int x[3], const int o[3]) {
  return rho_of(P, cen(P, phi, x[0] + o[0], x[1] + o[1], x[2] + o[2]));
}
static double eta_at(const orc_par *P, const double *phi, const int x[3], const int o[3]) {
  return eta_of(P, cen(P, phi, x[0] + o[0], x[1] + o[1], x[2] + o[2]));
}
static double nu_at(const orc_par *P, const double *phi, const int x[3], const int o[3]) {
  return nu_of(P, cen(P, phi, x[0] + o[0], x[1] + o[1], x[2] + o[2]));
}
static double p_at(const orc_par *P, const double *p, const int x[3], const int o[3]) {
  return cen(P, p, x[0] + o[0], x[1] + o[1], x[2] + o[2]);
}
static double u_at(const orc_par *P, const double *const U[3], int c, const int x[3], const int o[3]) {
  return fac(P, U[c], c, x[0] + o[0], x[1] + o[1], x[2] + o[2]);
}

/* radius of the centre of cell column i and of the u face i (axisymmetric form) */
static double r_cell(const orc_par *P, int i) { return (i + 0.5) * P->dx; }
static double r_face(const orc_par *P, int i) { return i * P->dx; }

/* velocity divergence at a (possibly ghost) cell, Eq. div-v-discretization;
 * the axisymmetric form adds u_r / r (Eq. div-v-axisym) with u_r at the cell
 * centre the mean of its two faces */
static double divu(const orc_par *P, const double *const U[3], const int x[3], const int o[3]) {
  double d = 0.0;
  for (int a = 0; a < P->dim; ++a) {
    int op[3] = {o[0], o[1], o[2]};
    op[a] += 1;
    d += u_at(P, U, a, x, op) - u_at(P, U, a, x, o);
  }
  double div = d / P->dx;
  if (P->axisym) {
    int op[3] = {o[0] + 1, o[1], o[2]};
    double ur = 0.5 * (u_at(P, U, 0, x, o) + u_at(P, U, 0, x, op));
    div += ur / r_cell(P, x[0] + o[0]);
  }
  return div;
}

/* averaged pressure of the cell at x+o, for the gradient along axis c
 * (Eq. gradp-u-discretization in 2D, Eq. gradp-u-p-ave-3d in 3D) */
static double pbar(const orc_par *P, const double *p, int c, const int x[3], const int o[3]) {
  if (!P->p_average) return p_at(P, p, x, o);
  if (P->dim == 2) {
    int t = 1 - c;
    int op[3] = {o[0], o[1], o[2]}, om[3] = {o[0], o[1], o[2]};
    op[t] += 1;
    om[t] -= 1;
    return (4.0 * p_at(P, p, x, o) + p_at(P, p, x, op) + p_at(P, p, x, om)) / 6.0;
  }
  int t1 = (c + 1) % 3, t2 = (c + 2) % 3;
  int a1p[3] = {o[0], o[1], o[2]}, a1m[3] = {o[0], o[1], o[2]};
  int a2p[3] = {o[0], o[1], o[2]}, a2m[3] = {o[0], o[1], o[2]};
  a1p[t1] += 1; a1m[t1] -= 1; a2p[t2] += 1; a2m[t2] -= 1;
  int pp[3] = {o[0], o[1], o[2]}, mm[3] = {o[0], o[1], o[2]};
  int mp[3] = {o[0], o[1], o[2]}, pm[3] = {o[0], o[1], o[2]};
  pp[t1] += 1; pp[t2] += 1;
  mm[t1] -= 1; mm[t2] -= 1;
  mp[t1] -= 1; mp[t2] += 1;
  pm[t1] += 1; pm[t2] -= 1;
  return (16.0 * p_at(P, p, x, o)
          + 4.0 * (p_at(P, p, x, a1p) + p_at(P, p, x, a1m) + p_at(P, p, x, a2p) + p_at(P, p, x, a2m))
          + (p_at(P, p, x, pp) + p_at(P, p, x, mm) + p_at(P, p, x, mp) + p_at(P, p, x, pm))) / 36.0;
}

/* ------------------------------------------------------------------ */
/* semi-discrete flow operators L_p, L_u, L_v, L_w                      */
/* (Eqs. gpe-pressure-two-phase, gpe-momentum-two-phase-const-bf and    */
/*  the discretisations div-v, diff-p, conv-u, u-stress a-d, st-u,      */
/*  gradp-u, gradp-u-p-ave-3d; Eq. p-u-v-semidiscrete-2d)               */
/* ------------------------------------------------------------------ */

/* pressure rate at cell x:  -rho c_s^2 div u + div(nu grad p) */
static double Lp_cell(const orc_par *P, const double *p, const double *const U[3],
                      const double *phi, const int x[3]) {
  const int o0[3] = {0, 0, 0};
  double dx2 = P->dx * P->dx;
  double diff = 0.0;
  for (int a = 0; a < P->dim; ++a) {
    int op[3] = {0, 0, 0}, om[3] = {0, 0, 0};
    op[a] = 1;
    om[a] = -1;
    double nup = 0.5 * (nu_at(P, phi, x, o0) + nu_at(P, phi, x, op));
    double num = 0.5 * (nu_at(P, phi, x, o0) + nu_at(P, phi, x, om));
    diff += (nup * (p_at(P, p, x, op) - p_at(P, p, x, o0))
             - num * (p_at(P, p, x, o0) - p_at(P, p, x, om))) / dx2;
  }
  if (P->axisym) {
    /* + (nu / r) dp/dr at the cell centre, Eq. gpe-pressure-two-phase-axisym */
    const int xp[3] = {1, 0, 0}, xm[3] = {-1, 0, 0};
    double dpdr = (p_at(P, p, x, xp) - p_at(P, p, x, xm)) / (2.0 * P->dx);
    diff += nu_at(P, phi, x, o0) / r_cell(P, x[0]) * dpdr;
  }
  return -rho_at(P, phi, x, o0) * P->cs * P->cs * divu(P, U, x, o0) + diff;
}

/* rate of velocity component c on the low-c face of cell x */
static double Lvel_face(const orc_par *P, int c, const double *p, const double *const U[3],
                        const double *phi, const double *mu, const int x[3]) {
  const double dx = P->dx, dx2 = P->dx * P->dx;
  const int o0[3] = {0, 0, 0};
  int cm[3] = {0, 0, 0}, cp[3] = {0, 0, 0};
  cm[c] = -1;
  cp[c] = 1;

  /* density on the face: mean of the two cells it separates */
  double rb = 0.5 * (rho_at(P, phi, x, cm) + rho_at(P, phi, x, o0));

  /* pressure gradient with the averaged pressure */
  double gradp = (pbar(P, p, c, x, o0) - pbar(P, p, c, x, cm)) / dx;

  /* d/dc [eta d u_c/dc], face viscosity = the cell between the two faces */
  double t_cc = (eta_at(P, phi, x, o0) * (u_at(P, U, c, x, cp) - u_at(P, U, c, x, o0))
                 - eta_at(P, phi, x, cm) * (u_at(P, U, c, x, o0) - u_at(P, U, c, x, cm))) / dx2;

  /* transverse terms d/dt [eta d u_c/dt] and d/dt [eta d u_t/dc] with the
   * corner viscosity = mean of the four cells around the edge */
  double t_tr = 0.0;
  double conv_tr = 0.0;
  for (int t = 0; t < P->dim; ++t) {
    if (t == c) continue;
    int tp[3] = {0, 0, 0}, tm[3] = {0, 0, 0}, ctp[3] = {0, 0, 0}, ctm[3] = {0, 0, 0};
    tp[t] = 1;
    tm[t] = -1;
    ctp[c] = -1; ctp[t] = 1;
    ctm[c] = -1; ctm[t] = -1;
    double etp = (eta_at(P, phi, x, o0) + eta_at(P, phi, x, tp) + eta_at(P, phi, x, cm)
                  + eta_at(P, phi, x, ctp)) / 4.0;
    double etm = (eta_at(P, phi, x, o0) + eta_at(P, phi, x, tm) + eta_at(P, phi, x, cm)
                  + eta_at(P, phi, x, ctm)) / 4.0;
    double t_tt = (etp * (u_at(P, U, c, x, tp) - u_at(P, U, c, x, o0))
                   - etm * (u_at(P, U, c, x, o0) - u_at(P, U, c, x, tm))) / dx2;
    double t_tc = (etp * (u_at(P, U, t, x, tp) - u_at(P, U, t, x, ctp))
                   - etm * (u_at(P, U, t, x, o0) - u_at(P, U, t, x, cm))) / dx2;
    t_tr += t_tt + t_tc;
    /* transverse velocity averaged onto the face (Eq. conv-u-discretization) */
    double ubar = (u_at(P, U, t, x, o0) + u_at(P, U, t, x, cm) + u_at(P, U, t, x, tp)
                   + u_at(P, U, t, x, ctp)) / 4.0;
    conv_tr += ubar * (u_at(P, U, c, x, tp) - u_at(P, U, c, x, tm)) / (2.0 * dx);
  }

  /* bulk-viscosity term d/dc [eta_b div u], eta_b = eta, centred on the face */
  double t_b = 0.0;
  if (P->bulk_visc)
    t_b = (eta_at(P, phi, x, o0) * divu(P, U, x, o0) - eta_at(P, phi, x, cm) * divu(P, U, x, cm)) / dx;

  /* surface tension -sigma phi d mu/dc on the face */
  double st = -P->sigma * (cen(P, phi, x[0], x[1], x[2]) + cen(P, phi, x[0] + cm[0], x[1] + cm[1], x[2] + cm[2]))
              * (cen(P, mu, x[0], x[1], x[2]) - cen(P, mu, x[0] + cm[0], x[1] + cm[1], x[2] + cm[2])) / (2.0 * dx);

  double grav = (rb - P->rho_ref) * P->g[c];

  /* the axisymmetric extra viscous terms, viscosity on the face = mean of
   * its two cells:
   *   u_r (Eq. gpe-momentum-two-phase-axisym-r): (eta / r) (du_r/dr - u_r / r)
   *   u_z (Eq. gpe-momentum-two-phase-axisym-z): (eta / r) du_z/dr */
  double t_axi = 0.0;
  if (P->axisym) {
    double eta_f = 0.5 * (eta_at(P, phi, x, cm) + eta_at(P, phi, x, o0));
    const int xp[3] = {1, 0, 0}, xm[3] = {-1, 0, 0};
    double dudr = (u_at(P, U, c, x, xp) - u_at(P, U, c, x, xm)) / (2.0 * dx);
    if (c == 0) {
      double r = r_face(P, x[0]);
      t_axi = eta_f / r * (dudr - u_at(P, U, 0, x, o0) / r);
    } else {
      t_axi = eta_f / r_cell(P, x[0]) * dudr;
    }
  }

  double force = -gradp + 2.0 * t_cc + t_tr + t_b + st + grav + t_axi;

  double conv = u_at(P, U, c, x, o0) * (u_at(P, U, c, x, cp) - u_at(P, U, c, x, cm)) / (2.0 * dx) + conv_tr;

  return force / rb - conv;
}

static size_t ncells(const orc_par *P) { return (size_t)P->nx * P->ny * (P->dim == 3 ? P->nz : 1); }

#define FOR_CELLS(P)                                      \
  for (int kk = 0; kk < ((P)->dim == 3 ? (P)->nz : 1); ++kk) \
    for (int jj = 0; jj < (P)->ny; ++jj)                  \
      for (int ii = 0; ii < (P)->nx; ++ii)

/* all flow rates; Lw/w may be NULL in 2D */
void orc_flow_rhs(const orc_par *P, const double *p, const double *u, const double *v, const double *w,
                  const double *phi, const double *mu, double *Lp, double *Lu, double *Lv, double *Lw) {
  const double *U[3] = {u, v, w};
  double *L[3] = {Lu, Lv, Lw};
  int nk = P->dim == 3 ? P->nz : 1;
#pragma omp parallel for
  for (int kk = 0; kk < nk; ++kk)
    for (int jj = 0; jj < P->ny; ++jj)
      for (int ii = 0; ii < P->nx; ++ii) {
        int x[3] = {ii, jj, kk};
        size_t id = lin(P, x);
        Lp[id] = Lp_cell(P, p, U, phi, x);
        for (int c = 0; c < P->dim; ++c)
          L[c][id] = wall_face(P, c, x) ? 0.0 : Lvel_face(P, c, p, U, phi, mu, x);
      }
}

/* ------------------------------------------------------------------ */
/* isotropic stencils (Eqs. 1st-der-iso, laplacian-iso) with the        */
/* standard lattice weights of D2Q9, D3Q15, D3Q19, D3Q27                */
/* ------------------------------------------------------------------ */

typedef struct { int n; int e[27][3]; double w[27]; } orc_lattice;

/* builds the lattice from its shells: rest, axis (|e|^2=1), edge (2), corner (3) */
static void lattice(const orc_par *P, orc_lattice *L) {
  double w0, w1, w2, w3;
  int use2, use3;
  switch (P->iso) {
    case 9:  w0 = 4.0 / 9.0; w1 = 1.0 / 9.0; w2 = 1.0 / 36.0; w3 = 0.0; use2 = 1; use3 = 0; break;
    case 15: w0 = 2.0 / 9.0; w1 = 1.0 / 9.0; w2 = 0.0; w3 = 1.0 / 72.0; use2 = 0; use3 = 1; break;
    case 19: w0 = 1.0 / 3.0; w1 = 1.0 / 18.0; w2 = 1.0 / 36.0; w3 = 0.0; use2 = 1; use3 = 0; break;
    default: w0 = 8.0 / 27.0; w1 = 2.0 / 27.0; w2 = 1.0 / 54.0; w3 = 1.0 / 216.0; use2 = 1; use3 = 1; break;
  }
  int d = P->dim;
  L->n = 0;
  for (int ez = (d == 3 ? -1 : 0); ez <= (d == 3 ? 1 : 0); ++ez)
    for (int ey = -1; ey <= 1; ++ey)
      for (int ex = -1; ex <= 1; ++ex) {
        int s = ex * ex + ey * ey + ez * ez;
        double w;
        if (s == 0) w = w0;
        else if (s == 1) w = w1;
        else if (s == 2) { if (!use2) continue; w = w2; }
        else { if (!use3) continue; w = w3; }
        L->e[L->n][0] = ex; L->e[L->n][1] = ey; L->e[L->n][2] = ez;
        L->w[L->n] = w;
        L->n++;
      }
}

static double rest_weight(const orc_lattice *L) {
  for (int q = 0; q < L->n; ++q)
    if (L->e[q][0] == 0 && L->e[q][1] == 0 && L->e[q][2] == 0) return L->w[q];
  return 0.0;
}

static double lap_iso_at(const orc_par *P, const orc_lattice *L, const double *f, const int x[3]) {
  double s = 0.0;
  for (int q = 0; q < L->n; ++q) {
    if (L->e[q][0] == 0 && L->e[q][1] == 0 && L->e[q][2] == 0) continue;
    s += L->w[q] * cen(P, f, x[0] + L->e[q][0], x[1] + L->e[q][1], x[2] + L->e[q][2]);
  }
  return 6.0 / (P->dx * P->dx) * (s - (1.0 - rest_weight(L)) * cen(P, f, x[0], x[1], x[2]));
}

static double grad_iso_at(const orc_par *P, const orc_lattice *L, const double *f, int a, const int x[3]) {
  double s = 0.0;
  for (int q = 0; q < L->n; ++q) {
    if (L->e[q][a] == 0) continue;
    s += L->w[q] * L->e[q][a] * cen(P, f, x[0] + L->e[q][0], x[1] + L->e[q][1], x[2] + L->e[q][2]);
  }
  return 3.0 / P->dx * s;
}

void orc_lap_iso(const orc_par *P, const double *f, double *out) {
  orc_lattice L;
  lattice(P, &L);
  FOR_CELLS(P) {
    int x[3] = {ii, jj, kk};
    out[lin(P, x)] = lap_iso_at(P, &L, f, x);
  }
}

void orc_grad_iso(const orc_par *P, const double *f, double *gx, double *gy, double *gz) {
  orc_lattice L;
  lattice(P, &L);
  double *G[3] = {gx, gy, gz};
  FOR_CELLS(P) {
    int x[3] = {ii, jj, kk};
    for (int a = 0; a < P->dim; ++a) G[a][lin(P, x)] = grad_iso_at(P, &L, f, a, x);
  }
}

/* chemical potential, Eq. chem-pot: mu = 4 a phi (phi^2 - 1) - kappa lap phi,
 * a = 3 sigma_ref / (4 W), kappa = 3 sigma_ref W / 8, sigma_ref = 1 */
void orc_mu(const orc_par *P, const double *phi, double *mu) {
  orc_lattice L;
  lattice(P, &L);
  double a = 3.0 / (4.0 * P->W), kappa = 3.0 * P->W / 8.0;
  int nk = P->dim == 3 ? P->nz : 1;
#pragma omp parallel for
  for (int kk = 0; kk < nk; ++kk)
    for (int jj = 0; jj < P->ny; ++jj)
      for (int ii = 0; ii < P->nx; ++ii) {
        int x[3] = {ii, jj, kk};
        double f = phi[lin(P, x)];
        double lap = lap_iso_at(P, &L, phi, x);
        /* Eq. chem-pot-axisym: the Laplacian gains (1/r) dphi/dr */
        if (P->axisym) lap += grad_iso_at(P, &L, phi, 0, x) / r_cell(P, ii);
        mu[lin(P, x)] = 4.0 * a * f * (f * f - 1.0) - kappa * lap;
      }
}

/* CH rate, Eq. che: -uhat . grad_iso phi + M lap_iso mu
 * (ch_advection = 1: -div_iso(uhat phi) instead of the advective form) */
void orc_ch_rhs(const orc_par *P, const double *phi, const double *mu, const double *uh,
                const double *vh, const double *wh, double *Lphi) {
  orc_lattice L;
  lattice(P, &L);
  const double *UH[3] = {uh, vh, wh};
  int nk = P->dim == 3 ? P->nz : 1;
#pragma omp parallel for
  for (int kk = 0; kk < nk; ++kk)
    for (int jj = 0; jj < P->ny; ++jj)
      for (int ii = 0; ii < P->nx; ++ii) {
        int x[3] = {ii, jj, kk};
        double adv = 0.0;
        for (int a = 0; a < P->dim; ++a) {
          if (P->ch_advection == 0) {
            adv += UH[a][lin(P, x)] * grad_iso_at(P, &L, phi, a, x);
          } else {
            double s = 0.0;
            for (int q = 0; q < L.n; ++q) {
              if (L.e[q][a] == 0) continue;
              int y0 = x[0] + L.e[q][0], y1 = x[1] + L.e[q][1], y2 = x[2] + L.e[q][2];
              s += L.w[q] * L.e[q][a] * cvec(P, UH[a], a, y0, y1, y2) * cen(P, phi, y0, y1, y2);
            }
            adv += 3.0 / P->dx * s;
          }
        }
        double lap = lap_iso_at(P, &L, mu, x);
        /* Eq. che-axisym: the Laplacian of mu gains (1/r) dmu/dr */
        if (P->axisym) lap += grad_iso_at(P, &L, mu, 0, x) / r_cell(P, ii);
        Lphi[lin(P, x)] = -adv + P->M * lap;
      }
}

/* ------------------------------------------------------------------ */
/* one full time step (Sec. 3): TVD-RK3 (Eq. tvd-rk3) on p and the      */
/* velocity with phi, mu frozen at t^{n+1/2}; then the CH step from     */
/* phi^{n+1/2} to phi^{n+3/2} with the time-averaged cell-centre        */
/* velocity of Eq. u-center-2d frozen, TVD-RK2 (Eq. tvd-rk2) or RK4     */
/* (Eq. rk4), mu recomputed from phi at every stage.                    */
/* ------------------------------------------------------------------ */

static void ch_step(const orc_par *P, double *phi, double *mu, const double *const UH[3]) {
  size_t n = ncells(P);
  double *Lf = malloc(n * sizeof(double));
  double *f1 = malloc(n * sizeof(double));
  double *m1 = malloc(n * sizeof(double));
  if (P->ch_scheme == 4) {
    double *acc = malloc(n * sizeof(double));
    /* a = dt L(phi) */
    orc_ch_rhs(P, phi, mu, UH[0], UH[1], UH[2], Lf);
    for (size_t i = 0; i < n; ++i) { double a = P->dt * Lf[i]; acc[i] = a; f1[i] = phi[i] + 0.5 * a; }
    /* b = dt L(phi + a/2) */
    orc_mu(P, f1, m1);
    orc_ch_rhs(P, f1, m1, UH[0], UH[1], UH[2], Lf);
    for (size_t i = 0; i < n; ++i) { double b = P->dt * Lf[i]; acc[i] += 2.0 * b; f1[i] = phi[i] + 0.5 * b; }
    /* c = dt L(phi + b/2) */
    orc_mu(P, f1, m1);
    orc_ch_rhs(P, f1, m1, UH[0], UH[1], UH[2], Lf);
    for (size_t i = 0; i < n; ++i) { double c = P->dt * Lf[i]; acc[i] += 2.0 * c; f1[i] = phi[i] + c; }
    /* d = dt L(phi + c) */
    orc_mu(P, f1, m1);
    orc_ch_rhs(P, f1, m1, UH[0], UH[1], UH[2], Lf);
    for (size_t i = 0; i < n; ++i) { double d = P->dt * Lf[i]; phi[i] = phi[i] + (acc[i] + d) / 6.0; }
    free(acc);
  } else {
    orc_ch_rhs(P, phi, mu, UH[0], UH[1], UH[2], Lf);
    for (size_t i = 0; i < n; ++i) f1[i] = phi[i] + P->dt * Lf[i];
    orc_mu(P, f1, m1);
    orc_ch_rhs(P, f1, m1, UH[0], UH[1], UH[2], Lf);
    for (size_t i = 0; i < n; ++i) phi[i] = 0.5 * phi[i] + 0.5 * (f1[i] + P->dt * Lf[i]);
  }
  orc_mu(P, phi, mu);
  free(Lf);
  free(f1);
  free(m1);
}

/* time-averaged cell-centre velocity, Eq. u-center-2d, for every axis */
static void center_velocity(const orc_par *P, const double *const U0[3], const double *const U1[3], double *UH[3]) {
  FOR_CELLS(P) {
    int x[3] = {ii, jj, kk};
    for (int a = 0; a < P->dim; ++a) {
      int o[3] = {0, 0, 0};
      o[a] = 1;
      UH[a][lin(P, x)] = 0.25 * ((u_at(P, U0, a, x, (int[3]){0, 0, 0}) + u_at(P, U0, a, x, o))
                                 + (u_at(P, U1, a, x, (int[3]){0, 0, 0}) + u_at(P, U1, a, x, o)));
    }
  }
}

int orc_step(const orc_par *P, double *p, double *u, double *v, double *w, double *phi, double *mu,
             long long nsteps) {
  size_t n = ncells(P);
  int d = P->dim;
  double *q0[4], *qa[4], *qb[4], *Lq[4], *uh[3];
  for (int f = 0; f < 4; ++f) {
    q0[f] = malloc(n * sizeof(double));
    qa[f] = malloc(n * sizeof(double));
    qb[f] = malloc(n * sizeof(double));
    Lq[f] = malloc(n * sizeof(double));
    if (!q0[f] || !qa[f] || !qb[f] || !Lq[f]) return 1;
  }
  for (int a = 0; a < 3; ++a) uh[a] = calloc(n, sizeof(double));
  double *Q[4] = {p, u, v, w};
  int nf = 1 + d;

  for (long long s = 0; s < nsteps; ++s) {
    for (int f = 0; f < nf; ++f) memcpy(q0[f], Q[f], n * sizeof(double));
    /* stage 1: q1 = q^n + dt L(q^n) */
    orc_flow_rhs(P, q0[0], q0[1], q0[2], d == 3 ? q0[3] : NULL, phi, mu, Lq[0], Lq[1], Lq[2], Lq[3]);
    for (int f = 0; f < nf; ++f)
      for (size_t i = 0; i < n; ++i) qa[f][i] = q0[f][i] + P->dt * Lq[f][i];
    /* stage 2: q2 = 3/4 q^n + 1/4 (q1 + dt L(q1)) */
    orc_flow_rhs(P, qa[0], qa[1], qa[2], d == 3 ? qa[3] : NULL, phi, mu, Lq[0], Lq[1], Lq[2], Lq[3]);
    for (int f = 0; f < nf; ++f)
      for (size_t i = 0; i < n; ++i) qb[f][i] = 0.75 * q0[f][i] + 0.25 * (qa[f][i] + P->dt * Lq[f][i]);
    /* stage 3: q^{n+1} = 1/3 q^n + 2/3 (q2 + dt L(q2)) */
    orc_flow_rhs(P, qb[0], qb[1], qb[2], d == 3 ? qb[3] : NULL, phi, mu, Lq[0], Lq[1], Lq[2], Lq[3]);
    for (int f = 0; f < nf; ++f)
      for (size_t i = 0; i < n; ++i) Q[f][i] = q0[f][i] / 3.0 + 2.0 / 3.0 * (qb[f][i] + P->dt * Lq[f][i]);

    const double *U0[3] = {q0[1], q0[2], d == 3 ? q0[3] : NULL};
    const double *U1[3] = {u, v, d == 3 ? w : NULL};
    center_velocity(P, U0, U1, uh);
    const double *UH[3] = {uh[0], uh[1], uh[2]};
    ch_step(P, phi, mu, UH);
  }
  for (int f = 0; f < 4; ++f) { free(q0[f]); free(qa[f]); free(qb[f]); free(Lq[f]); }
  for (int a = 0; a < 3; ++a) free(uh[a]);
  return 0;
}

/* diagnostics: out[0] = sum phi dx^d, out[1] = kinetic energy
 * 1/2 sum over faces of rho_face u^2 dx^d, out[2] = max |velocity component|,
 * out[3] = 1 if any field holds a NaN or Inf */
void orc_diag(const orc_par *P, const double *p, const double *u, const double *v, const double *w,
              const double *phi, double out[4]) {
  const double *U[3] = {u, v, w};
  double vol = P->dim == 3 ? P->dx * P->dx * P->dx : P->dx * P->dx;
  double sphi = 0.0, ke = 0.0, umax = 0.0;
  int bad = 0;
  FOR_CELLS(P) {
    int x[3] = {ii, jj, kk};
    size_t id = lin(P, x);
    sphi += phi[id];
    if (!isfinite(phi[id]) || !isfinite(p[id])) bad = 1;
    for (int c = 0; c < P->dim; ++c) {
      int cm[3] = {0, 0, 0};
      cm[c] = -1;
      double uc = U[c][id];
      double rb = 0.5 * (rho_at(P, phi, x, cm) + rho_at(P, phi, x, (int[3]){0, 0, 0}));
      ke += 0.5 * rb * uc * uc;
      if (fabs(uc) > umax) umax = fabs(uc);
      if (!isfinite(uc)) bad = 1;
    }
  }
  out[0] = sphi * vol;
  out[1] = ke * vol;
  out[2] = umax;
  out[3] = bad;
}

/* the lattice the oracle uses, for the moment-condition tests:
 * returns the number of velocities, fills e (n x 3) and w (n) */
int orc_lattice_table(const orc_par *P, int *e, double *w) {
  orc_lattice L;
  lattice(P, &L);
  for (int q = 0; q < L.n; ++q) {
    e[3 * q] = L.e[q][0]; e[3 * q + 1] = L.e[q][1]; e[3 * q + 2] = L.e[q][2];
    w[q] = L.w[q];
  }
  return L.n;
}
