/*
 * FP64 CPU oracle for one Godunov finite-volume Runge-Kutta step of 3D adiabatic
 * Newtonian hydrodynamics (AthenaK, arXiv 2409.16053, Section 3 and Section 3.1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this
 * file: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.
 * It shares no code, header or constant table with the CUDA path.
 *
 * Design: plain, slow, obviously correct.  The whole domain is ONE periodic grid
 * (no MeshBlocks): a MeshBlock mesh with exact ghost exchange computes the same
 * arithmetic per cell, so this is the plain definition the GPU's blocked layout and
 * its ghost fill must reproduce.  Every face flux is computed from scratch, one face
 * at a time, in the order the method states: primitives, reconstruction, Riemann
 * solver, flux divergence, RK stage update.  Built with -ffp-contract=off so each
 * line rounds as written.
 *
 * Arrays are double[5][n3][n2][n1] with x1 fastest; the 5 components are
 * U = (rho, M1, M2, M3, E) or W = (rho, v1, v2, v3, u_g).
 *
 * Readings of places where the paper defers to its references (all restated in the
 * design notes):
 *   - PLM limiter: van Leer harmonic mean of the one-sided differences.
 *   - PPM4: Colella & Woodward (1984) uniform-grid interface values and limiter,
 *     no flattening, no contact steepening.
 *   - PPMX: the fourth-order interface values of PPM with the extremum-preserving
 *     interface limiter of Colella & Sekora (2008) and the cell limiter of
 *     McCorquodale & Colella (2011), curvature constant C = 1.25, on the five-cell
 *     stencil (3 ghost cells): the third-derivative smoothness test of the latter,
 *     which needs seven cells, is not applied.
 *   - WENO-Z: Borges, Carmona, Costa & Don (2008): the three third-order candidate
 *     interface values of Jiang & Shu (1996) with their smoothness indicators, weights
 *     alpha_k = d_k (1 + tau5 / (beta_k + eps)), tau5 = |beta_0 - beta_2|, ideal weights
 *     (1, 6, 3)/10, eps = 1e-40; on primitives, 3 ghost cells.
 *   - HLLC: Toro (2009) ch. 10, PVRS wave-speed estimate bounded outward by the
 *     Davis speeds, star states of the standard form, ties at S_L = 0 / S* = 0
 *     resolved to the left.
 *   - LLF (Rusanov): Toro (2009) Sec. 10.5.1 with the single speed
 *     S+ = max(|u_L| + c_L, |u_R| + c_R).
 *   - HLLE: the HLL flux (Toro Eq. 10.21) with Einfeldt's speeds
 *     S_L = min(u_L - c_L, u~ - c~), S_R = max(u_R + c_R, u~ + c~) from the Roe averages
 *     (Toro Sec. 10.5.1, Eqs. 10.49-10.53), taken as b- = min(S_L, 0), b+ = max(S_R, 0).
 *   - SSP-RK2 (Heun) and SSP-RK3 (Shu-Osher) coefficients, each stage evaluated as
 *     a*U0 + b*(U + dt*L(U)).
 *   - Floors: rho < 1e-12 or u_g < 1e-15 in the primitive recovery are clamped and
 *     counted (the paper gives no hydro floor values).
 *   - FOFC (Section 3, first-order flux correction): after a stage's update, a cell
 *     whose density or internal energy is not positive gets LLF fluxes of the
 *     piecewise-constant states on all its faces, and the stage is recomputed with them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NVAR 5
#define ORC_RHO_FLOOR 1.0e-12
#define ORC_UG_FLOOR 1.0e-15

#define ORC_PLM 0
#define ORC_PPM4 1
#define ORC_WENOZ 2
#define ORC_PPMX 3

#define ORC_HLLC 0
#define ORC_HLLE 1
#define ORC_LLF 2

typedef struct {
  int64_t n[3];     /* cells per dimension of the periodic grid */
  double dx[3];     /* uniform cell widths (Section 2: uniform Cartesian only) */
  double gamma;     /* ratio of specific heats of the gamma-law EOS */
  int32_t recon;    /* ORC_PLM, ORC_PPM4, ORC_WENOZ or ORC_PPMX */
  int32_t riemann;  /* ORC_HLLC, ORC_HLLE or ORC_LLF */
  int32_t fofc;     /* 1: first-order flux correction in every RK stage */
  int32_t pad;
} orc_grid;

static int64_t wrap(int64_t i, int64_t n) {
  int64_t r = i % n;
  return r < 0 ? r + n : r;
}

static int64_t cell(const orc_grid* g, int64_t i, int64_t j, int64_t k) {
  return (wrap(k, g->n[2]) * g->n[1] + wrap(j, g->n[1])) * g->n[0] + wrap(i, g->n[0]);
}

/* ---------------------------------------------------------------------------------
 * Conserved -> primitive, Section 3.1 Eq. (4): rho = U0, v = M/rho,
 * E = u_g + rho v^2/2  =>  u_g = E - (M.M)/(2 rho).  Floors are a reading (counted).
 * ------------------------------------------------------------------------------- */
void orc_cons_to_prim(const double u[5], double w[5], int64_t* nfloor) {
  double rho = u[0];
  if (!(rho >= ORC_RHO_FLOOR)) {
    rho = ORC_RHO_FLOOR;
    *nfloor += 1;
  }
  double v1 = u[1] / rho;
  double v2 = u[2] / rho;
  double v3 = u[3] / rho;
  double ug = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / rho;
  if (!(ug >= ORC_UG_FLOOR)) {
    ug = ORC_UG_FLOOR;
    *nfloor += 1;
  }
  w[0] = rho;
  w[1] = v1;
  w[2] = v2;
  w[3] = v3;
  w[4] = ug;
}

/* Primitive -> conserved, Section 3.1 Eq. (4). */
void orc_prim_to_cons(const double w[5], double u[5]) {
  u[0] = w[0];
  u[1] = w[0] * w[1];
  u[2] = w[0] * w[2];
  u[3] = w[0] * w[3];
  u[4] = w[4] + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
}

/* ---------------------------------------------------------------------------------
 * PLM (Section 3: piecewise linear reconstruction on primitives).  Reading: van Leer
 * harmonic-mean limiter.  Given the three cell values q(i-1), q(i), q(i+1), returns
 * the limited slope of cell i; the face states are q(i) -/+ slope/2.
 * ------------------------------------------------------------------------------- */
double orc_plm_slope(double qm, double q0, double qp) {
  double dl = q0 - qm;
  double dr = qp - q0;
  double prod = dl * dr;
  if (prod > 0.0) return 2.0 * prod / (dl + dr);
  return 0.0;
}

/* ---------------------------------------------------------------------------------
 * PPM4 (Section 3: "original" PPM limiters of Colella & Woodward 1984), uniform grid.
 * Given q(i-2..i+2) returns the left (x_{i-1/2}) and right (x_{i+1/2}) edge values of
 * the parabola in cell i after monotonization.
 * ------------------------------------------------------------------------------- */
static double ppm_limited_slope(double qm, double q0, double qp) {
  /* CW84 Eq. (1.7)-(1.8): centred slope, limited to twice the one-sided ones, zero at
   * extrema. */
  double d = 0.5 * (qp - qm);
  double dl = q0 - qm;
  double dr = qp - q0;
  if (dl * dr <= 0.0) return 0.0;
  double m = fabs(d);
  if (2.0 * fabs(dl) < m) m = 2.0 * fabs(dl);
  if (2.0 * fabs(dr) < m) m = 2.0 * fabs(dr);
  return d > 0.0 ? m : -m;
}

void orc_ppm4_edges(const double q[5], double* qlo, double* qhi) {
  /* q[0..4] = q(i-2), q(i-1), q(i), q(i+1), q(i+2) */
  double sm1 = ppm_limited_slope(q[0], q[1], q[2]);
  double s0 = ppm_limited_slope(q[1], q[2], q[3]);
  double sp1 = ppm_limited_slope(q[2], q[3], q[4]);
  /* CW84 Eq. (1.6) on a uniform grid: interface values. */
  double alo = 0.5 * (q[1] + q[2]) - (s0 - sm1) / 6.0;
  double ahi = 0.5 * (q[2] + q[3]) - (sp1 - s0) / 6.0;
  double a = q[2];
  /* CW84 Eq. (1.10): monotonize the parabola. */
  if ((ahi - a) * (a - alo) <= 0.0) {
    alo = a;
    ahi = a;
  } else {
    double da = ahi - alo;
    double a6 = 6.0 * (a - 0.5 * (alo + ahi));
    if (da * a6 > da * da) {
      alo = 3.0 * a - 2.0 * ahi;
    } else if (-da * da > da * a6) {
      ahi = 3.0 * a - 2.0 * alo;
    }
  }
  *qlo = alo;
  *qhi = ahi;
}

/* ---------------------------------------------------------------------------------
 * PPMX (Section 3: PPM with extremum-preserving limiters).  Given q(i-2..i+2) returns
 * the left (x_{i-1/2}) and right (x_{i+1/2}) edge values of cell i.
 * ------------------------------------------------------------------------------- */
#define PPMX_C 1.25

static int ppmx_same_sign3(double x, double y, double z) {
  return (x > 0.0 && y > 0.0 && z > 0.0) || (x < 0.0 && y < 0.0 && z < 0.0);
}

/* Interface value between cells b and c of the four cells a, b, c, d.  The fourth-order
 * value; if it does not lie between b and c, its second difference is limited by those
 * of the neighbouring cells (Colella & Sekora 2008). */
static double ppmx_interface(double a, double b, double c, double d) {
  double f = 7.0 / 12.0 * (b + c) - 1.0 / 12.0 * (a + d);
  if ((f - b) * (c - f) < 0.0) {
    double d2 = 3.0 * ((b + c) - 2.0 * f); /* the interface's own second difference */
    double d2l = (a + c) - 2.0 * b;        /* second difference of cell b */
    double d2r = (b + d) - 2.0 * c;        /* second difference of cell c */
    double lim = 0.0;
    if (ppmx_same_sign3(d2, d2l, d2r)) {
      double m = fabs(d2);
      if (PPMX_C * fabs(d2l) < m) m = PPMX_C * fabs(d2l);
      if (PPMX_C * fabs(d2r) < m) m = PPMX_C * fabs(d2r);
      lim = d2 > 0.0 ? m : -m;
    }
    f = 0.5 * (b + c) - lim / 6.0;
  }
  return f;
}

void orc_ppmx_edges(const double q[5], double* qlo, double* qhi) {
  /* q[0..4] = q(i-2), q(i-1), q(i), q(i+1), q(i+2) */
  double alo = ppmx_interface(q[0], q[1], q[2], q[3]);
  double ahi = ppmx_interface(q[1], q[2], q[3], q[4]);
  double a = q[2];
  double dp = ahi - a; /* rise of the parabola from the mean to the right edge */
  double dm = a - alo; /* rise from the left edge to the mean */
  if (dp * dm <= 0.0 || (q[3] - a) * (a - q[1]) <= 0.0) {
    /* An extremum: of the parabola inside the cell, or of the cell means.  Compare
     * the parabola's second derivative, 6 (a_lo + a_hi - 2 a), with the second
     * differences of cells i-1, i, i+1 (McCorquodale & Colella 2011). */
    double d2 = 6.0 * ((alo + ahi) - 2.0 * a);
    double d2c = (q[1] + q[3]) - 2.0 * a;
    double d2l = (q[0] + a) - 2.0 * q[1];
    double d2r = (a + q[4]) - 2.0 * q[3];
    double r = 0.0; /* ratio of the limited to the parabola's second derivative */
    int limit = 1;
    if (ppmx_same_sign3(d2, d2c, d2l) && ppmx_same_sign3(d2, d2c, d2r)) {
      double m = PPMX_C * fabs(d2c);
      if (PPMX_C * fabs(d2l) < m) m = PPMX_C * fabs(d2l);
      if (PPMX_C * fabs(d2r) < m) m = PPMX_C * fabs(d2r);
      if (m >= fabs(d2))
        limit = 0; /* the curvature is consistent with the neighbours' */
      else
        r = m / fabs(d2);
    }
    if (limit) {
      if (dp * dm < 0.0) {
        /* extremum inside the cell: scale the curvature by r */
        alo = a - r * dm;
        ahi = a + r * dp;
      } else if (fabs(dm) >= 2.0 * fabs(dp)) {
        alo = a - 2.0 * (1.0 - r) * dp - r * dm;
      } else if (fabs(dp) >= 2.0 * fabs(dm)) {
        ahi = a + 2.0 * (1.0 - r) * dm + r * dp;
      }
    }
  } else {
    /* monotone: keep the parabola's extremum out of the cell (Colella & Woodward) */
    if (fabs(dm) >= 2.0 * fabs(dp))
      alo = a - 2.0 * dp;
    else if (fabs(dp) >= 2.0 * fabs(dm))
      ahi = a + 2.0 * dm;
  }
  *qlo = alo;
  *qhi = ahi;
}

/* ---------------------------------------------------------------------------------
 * WENO-Z (Section 3: one of the reconstructions of the hydro module).  Given
 * q(i-2..i+2) returns the values at x_{i-1/2} (from the right) and x_{i+1/2} (from the
 * left) in cell i.
 * ------------------------------------------------------------------------------- */
static double wenoz_value(double a, double b, double c, double d, double e) {
  /* value at the interface between c and d from cells a, b, c, d, e (c is the cell) */
  double p0 = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
  double p1 = (-b + 5.0 * c + 2.0 * d) / 6.0;
  double p2 = (2.0 * c + 5.0 * d - e) / 6.0;
  double b0 = 13.0 / 12.0 * (a - 2.0 * b + c) * (a - 2.0 * b + c) +
              0.25 * (a - 4.0 * b + 3.0 * c) * (a - 4.0 * b + 3.0 * c);
  double b1 = 13.0 / 12.0 * (b - 2.0 * c + d) * (b - 2.0 * c + d) + 0.25 * (b - d) * (b - d);
  double b2 = 13.0 / 12.0 * (c - 2.0 * d + e) * (c - 2.0 * d + e) +
              0.25 * (3.0 * c - 4.0 * d + e) * (3.0 * c - 4.0 * d + e);
  double tau = fabs(b0 - b2);
  const double eps = 1e-40;
  double a0 = 0.1 * (1.0 + tau / (b0 + eps));
  double a1 = 0.6 * (1.0 + tau / (b1 + eps));
  double a2 = 0.3 * (1.0 + tau / (b2 + eps));
  return (a0 * p0 + a1 * p1 + a2 * p2) / (a0 + a1 + a2);
}

void orc_wenoz_edges(const double q[5], double* qlo, double* qhi) {
  *qhi = wenoz_value(q[0], q[1], q[2], q[3], q[4]);
  *qlo = wenoz_value(q[4], q[3], q[2], q[1], q[0]);
}

/* ---------------------------------------------------------------------------------
 * HLLC Riemann solver (Section 3, Toro ch. 10).  Inputs are primitive states with the
 * normal velocity in component 1 and the two transverse ones in 2 and 3:
 * w = (rho, u, v, w, u_g).  Output: the flux of (rho, rho u, rho v, rho w, E) through a
 * face normal to the sweep direction, Section 3.1 Eq. (4).
 * ------------------------------------------------------------------------------- */
static void phys_flux(const double w[5], double p, double e, double f[5]) {
  double mn = w[0] * w[1];
  f[0] = mn;
  f[1] = mn * w[1] + p;
  f[2] = mn * w[2];
  f[3] = mn * w[3];
  f[4] = (e + p) * w[1];
}

/* PVRS pressure estimate p_pv (Toro Sec. 9.3 and Sec. 10.5.2): the star pressure of
 * the Riemann problem linearised about the mean state, with sound speeds
 * c_K = sqrt(gamma p_K / rho_K). */
double orc_pvrs_pressure(const double wl[5], const double wr[5], double gamma) {
  double rl = wl[0], ul = wl[1];
  double rr = wr[0], ur = wr[1];
  double pl = (gamma - 1.0) * wl[4];
  double pr = (gamma - 1.0) * wr[4];
  double cl = sqrt(gamma * pl / rl);
  double cr = sqrt(gamma * pr / rr);
  return 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr);
}

/* Shock factor q_K (Toro Sec. 10.5.2): a wave of side K with star pressure p* above p_K
 * is a shock, with speed S_L = u_L - c_L q_L (left) or S_R = u_R + c_R q_R (right) and
 * q_K = sqrt(1 + (gamma + 1) / (2 gamma) (p* / p_K - 1)); otherwise q_K = 1. */
double orc_shock_factor(double pstar, double pk, double gamma) {
  if (pstar > pk) return sqrt(1.0 + (gamma + 1.0) / (2.0 * gamma) * (pstar / pk - 1.0));
  return 1.0;
}

/* HLLC wave-speed estimates S_L, S_R: the pressure-based speeds of Toro Sec. 10.5.2
 * with p* = max(0, p_pv), bounded outward by the Davis speeds. */
void orc_hllc_speeds(const double wl[5], const double wr[5], double gamma, double* sl_out,
                     double* sr_out) {
  double ul = wl[1], ur = wr[1];
  double pl = (gamma - 1.0) * wl[4];
  double pr = (gamma - 1.0) * wr[4];
  double cl = sqrt(gamma * pl / wl[0]);
  double cr = sqrt(gamma * pr / wr[0]);
  double ppv = orc_pvrs_pressure(wl, wr, gamma);
  double pstar = ppv > 0.0 ? ppv : 0.0;
  double ql = orc_shock_factor(pstar, pl, gamma);
  double qr = orc_shock_factor(pstar, pr, gamma);
  double sl = ul - cl * ql;
  double sr = ur + cr * qr;
  /* Reading: in strongly colliding supersonic flow the PVRS estimates can cross
   * (S_L > S_R); bounding them outward by the Davis speeds u_R - c_R and u_L + c_L
   * keeps S_L < S_R, and changes nothing where the PVRS speeds already bracket them. */
  if (ur - cr < sl) sl = ur - cr;
  if (ul + cl > sr) sr = ul + cl;
  *sl_out = sl;
  *sr_out = sr;
}

void orc_hllc(const double wl[5], const double wr[5], double gamma, double f[5]) {
  double rl = wl[0], ul = wl[1];
  double rr = wr[0], ur = wr[1];
  double pl = (gamma - 1.0) * wl[4];
  double pr = (gamma - 1.0) * wr[4];
  double el = wl[4] + 0.5 * rl * (wl[1] * wl[1] + wl[2] * wl[2] + wl[3] * wl[3]);
  double er = wr[4] + 0.5 * rr * (wr[1] * wr[1] + wr[2] * wr[2] + wr[3] * wr[3]);
  double sl, sr;
  orc_hllc_speeds(wl, wr, gamma, &sl, &sr);

  /* Toro Eq. (10.37): contact speed. */
  double sstar = (pr - pl + rl * ul * (sl - ul) - rr * ur * (sr - ur)) /
                 (rl * (sl - ul) - rr * (sr - ur));

  double fl[5], fr[5];
  phys_flux(wl, pl, el, fl);
  phys_flux(wr, pr, er, fr);

  if (sl >= 0.0) {
    memcpy(f, fl, sizeof(fl));
    return;
  }
  if (sr <= 0.0) {
    memcpy(f, fr, sizeof(fr));
    return;
  }
  /* Toro Eq. (10.38)-(10.39): star state of the side the face lies in. */
  const double* w = (sstar >= 0.0) ? wl : wr;
  double s = (sstar >= 0.0) ? sl : sr;
  double p = (sstar >= 0.0) ? pl : pr;
  double e = (sstar >= 0.0) ? el : er;
  const double* fk = (sstar >= 0.0) ? fl : fr;
  double rk = w[0], uk = w[1];
  double fac = rk * (s - uk) / (s - sstar);
  double ustar[5], uk5[5];
  ustar[0] = fac;
  ustar[1] = fac * sstar;
  ustar[2] = fac * w[2];
  ustar[3] = fac * w[3];
  ustar[4] = fac * (e / rk + (sstar - uk) * (sstar + p / (rk * (s - uk))));
  uk5[0] = rk;
  uk5[1] = rk * uk;
  uk5[2] = rk * w[2];
  uk5[3] = rk * w[3];
  uk5[4] = e;
  for (int n = 0; n < NVAR; ++n) f[n] = fk[n] + s * (ustar[n] - uk5[n]);
}

/* Conserved state of a primitive face state (same layout as the flux). */
static void face_cons(const double w[5], double e, double u[5]) {
  u[0] = w[0];
  u[1] = w[0] * w[1];
  u[2] = w[0] * w[2];
  u[3] = w[0] * w[3];
  u[4] = e;
}

/* LLF (Rusanov): F = (F_L + F_R) / 2 - S+ (U_R - U_L) / 2. */
void orc_llf(const double wl[5], const double wr[5], double gamma, double f[5]) {
  double pl = (gamma - 1.0) * wl[4];
  double pr = (gamma - 1.0) * wr[4];
  double el = wl[4] + 0.5 * wl[0] * (wl[1] * wl[1] + wl[2] * wl[2] + wl[3] * wl[3]);
  double er = wr[4] + 0.5 * wr[0] * (wr[1] * wr[1] + wr[2] * wr[2] + wr[3] * wr[3]);
  double cl = sqrt(gamma * pl / wl[0]);
  double cr = sqrt(gamma * pr / wr[0]);
  double al = fabs(wl[1]) + cl, ar = fabs(wr[1]) + cr;
  double smax = al > ar ? al : ar;
  double fl[5], fr[5], ul[5], ur[5];
  phys_flux(wl, pl, el, fl);
  phys_flux(wr, pr, er, fr);
  face_cons(wl, el, ul);
  face_cons(wr, er, ur);
  for (int n = 0; n < NVAR; ++n) f[n] = 0.5 * (fl[n] + fr[n]) - 0.5 * smax * (ur[n] - ul[n]);
}

/* Roe averages of two primitive states (Toro Sec. 10.5.1, Eqs. 10.49-10.53): weights
 * sqrt(rho), total enthalpy H = (E + p) / rho; returns the averaged normal velocity u~
 * and sound speed c~ = sqrt((gamma - 1) (H~ - |v~|^2 / 2)), taken as 0 where the
 * square is not positive. */
void orc_roe_average(const double wl[5], const double wr[5], double gamma, double* un,
                     double* cb_out) {
  double rl = wl[0], rr = wr[0];
  double pl = (gamma - 1.0) * wl[4];
  double pr = (gamma - 1.0) * wr[4];
  double el = wl[4] + 0.5 * rl * (wl[1] * wl[1] + wl[2] * wl[2] + wl[3] * wl[3]);
  double er = wr[4] + 0.5 * rr * (wr[1] * wr[1] + wr[2] * wr[2] + wr[3] * wr[3]);
  double sl = sqrt(rl), sr = sqrt(rr);
  double ub[3], hb, q2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    ub[a] = (sl * wl[1 + a] + sr * wr[1 + a]) / (sl + sr);
    q2 += ub[a] * ub[a];
  }
  hb = (sl * (el + pl) / rl + sr * (er + pr) / rr) / (sl + sr);
  double cb2 = (gamma - 1.0) * (hb - 0.5 * q2);
  *un = ub[0];
  *cb_out = cb2 > 0.0 ? sqrt(cb2) : 0.0;
}

/* Einfeldt's HLLE speeds S_L = min(u_L - c_L, u~ - c~), S_R = max(u_R + c_R, u~ + c~). */
void orc_hlle_speeds(const double wl[5], const double wr[5], double gamma, double* sl_out,
                     double* sr_out) {
  double pl = (gamma - 1.0) * wl[4];
  double pr = (gamma - 1.0) * wr[4];
  double cl = sqrt(gamma * pl / wl[0]);
  double cr = sqrt(gamma * pr / wr[0]);
  double ub, cb;
  orc_roe_average(wl, wr, gamma, &ub, &cb);
  double sL = wl[1] - cl, sR = wr[1] + cr;
  if (ub - cb < sL) sL = ub - cb;
  if (ub + cb > sR) sR = ub + cb;
  *sl_out = sL;
  *sr_out = sR;
}

/* HLLE: HLL flux with Einfeldt's wave speeds from the Roe averages. */
void orc_hlle(const double wl[5], const double wr[5], double gamma, double f[5]) {
  double rl = wl[0], rr = wr[0];
  double pl = (gamma - 1.0) * wl[4];
  double pr = (gamma - 1.0) * wr[4];
  double el = wl[4] + 0.5 * rl * (wl[1] * wl[1] + wl[2] * wl[2] + wl[3] * wl[3]);
  double er = wr[4] + 0.5 * rr * (wr[1] * wr[1] + wr[2] * wr[2] + wr[3] * wr[3]);
  double sL, sR;
  orc_hlle_speeds(wl, wr, gamma, &sL, &sR);
  double bm = sL < 0.0 ? sL : 0.0;
  double bp = sR > 0.0 ? sR : 0.0;
  double fl[5], fr[5], ul[5], ur[5];
  phys_flux(wl, pl, el, fl);
  phys_flux(wr, pr, er, fr);
  face_cons(wl, el, ul);
  face_cons(wr, er, ur);
  for (int n = 0; n < NVAR; ++n)
    f[n] = (bp * fl[n] - bm * fr[n] + bp * bm * (ur[n] - ul[n])) / (bp - bm);
}

void orc_riemann(int solver, const double wl[5], const double wr[5], double gamma,
                 double f[5]) {
  if (solver == ORC_LLF)
    orc_llf(wl, wr, gamma, f);
  else if (solver == ORC_HLLE)
    orc_hlle(wl, wr, gamma, f);
  else
    orc_hllc(wl, wr, gamma, f);
}

/* ---------------------------------------------------------------------------------
 * Right-hand side L(U) = -div F of Section 3 Eq. (1) (S = 0) on the periodic grid.
 * For each direction d, the face between cells c - e_d and c gets its left state from
 * the reconstruction in cell c - e_d and its right state from that in cell c; the
 * Riemann solver (HLLC, HLLE or LLF) gives the flux; then L -= (F(c + e_d) - F(c)) / dx_d, summed x1, x2, x3 in turn.
 * ------------------------------------------------------------------------------- */
static void face_states(const orc_grid* g, const double* W, int d, int64_t i, int64_t j,
                        int64_t k, double wl[5], double wr[5]) {
  int64_t e[3] = {0, 0, 0};
  e[d] = 1;
  int64_t N = g->n[0] * g->n[1] * g->n[2];
  /* Permutation into (rho, normal, transverse 1, transverse 2, u_g): cyclic. */
  int perm[5] = {0, 1 + d, 1 + (d + 1) % 3, 1 + (d + 2) % 3, 4};
  for (int n = 0; n < NVAR; ++n) {
    int v = perm[n];
    const double* q = W + (int64_t)v * N;
    if (g->recon == ORC_PLM) {
      double qm2 = q[cell(g, i - 2 * e[0], j - 2 * e[1], k - 2 * e[2])];
      double qm1 = q[cell(g, i - e[0], j - e[1], k - e[2])];
      double q0 = q[cell(g, i, j, k)];
      double qp1 = q[cell(g, i + e[0], j + e[1], k + e[2])];
      /* left state: upper edge of cell c - e_d; right state: lower edge of cell c */
      wl[n] = qm1 + 0.5 * orc_plm_slope(qm2, qm1, q0);
      wr[n] = q0 - 0.5 * orc_plm_slope(qm1, q0, qp1);
    } else {
      double s[6];
      for (int m = 0; m < 6; ++m) {
        int64_t o = m - 3;
        s[m] = q[cell(g, i + o * e[0], j + o * e[1], k + o * e[2])];
      }
      double lo, hi, lo2, hi2;
      if (g->recon == ORC_WENOZ) {
        orc_wenoz_edges(&s[0], &lo, &hi);  /* cell c - e_d, stencil c-3e..c+e */
        orc_wenoz_edges(&s[1], &lo2, &hi2); /* cell c, stencil c-2e..c+2e */
      } else if (g->recon == ORC_PPMX) {
        orc_ppmx_edges(&s[0], &lo, &hi);
        orc_ppmx_edges(&s[1], &lo2, &hi2);
      } else {
        orc_ppm4_edges(&s[0], &lo, &hi);
        orc_ppm4_edges(&s[1], &lo2, &hi2);
      }
      (void)lo;
      (void)hi2;
      wl[n] = hi;
      wr[n] = lo2;
    }
  }
}

/* flag != NULL: a face with a flagged cell on either side gets the LLF flux of the two
 * cells' own (piecewise-constant) states instead of the reconstructed one (FOFC). */
static int64_t rhs_impl(const orc_grid* g, const double* U, double* L,
                        const unsigned char* flag) {
  int64_t N = g->n[0] * g->n[1] * g->n[2];
  int64_t nfloor = 0;
  double* W = (double*)malloc(sizeof(double) * NVAR * N);
  double* F = (double*)malloc(sizeof(double) * NVAR * N);
  if (!W || !F) {
    free(W);
    free(F);
    return -1;
  }
#pragma omp parallel for reduction(+ : nfloor)
  for (int64_t c = 0; c < N; ++c) {
    double u[5], w[5];
    for (int n = 0; n < NVAR; ++n) u[n] = U[n * N + c];
    orc_cons_to_prim(u, w, &nfloor);
    for (int n = 0; n < NVAR; ++n) W[n * N + c] = w[n];
  }
  for (int64_t c = 0; c < NVAR * N; ++c) L[c] = 0.0;

  for (int d = 0; d < 3; ++d) {
    int perm[5] = {0, 1 + d, 1 + (d + 1) % 3, 1 + (d + 2) % 3, 4};
    /* F[.][c] = flux through the lower face of cell c in direction d */
#pragma omp parallel for
    for (int64_t k = 0; k < g->n[2]; ++k)
      for (int64_t j = 0; j < g->n[1]; ++j)
        for (int64_t i = 0; i < g->n[0]; ++i) {
          double wl[5], wr[5], f[5];
          int64_t c = cell(g, i, j, k);
          int64_t cm = cell(g, i - (d == 0), j - (d == 1), k - (d == 2));
          if (flag && (flag[c] || flag[cm])) {
            for (int n = 0; n < NVAR; ++n) {
              wl[n] = W[(int64_t)perm[n] * N + cm];
              wr[n] = W[(int64_t)perm[n] * N + c];
            }
            orc_llf(wl, wr, g->gamma, f);
          } else {
            face_states(g, W, d, i, j, k, wl, wr);
            orc_riemann(g->riemann, wl, wr, g->gamma, f);
          }
          for (int n = 0; n < NVAR; ++n) F[(int64_t)perm[n] * N + c] = f[n];
        }
#pragma omp parallel for
    for (int64_t k = 0; k < g->n[2]; ++k)
      for (int64_t j = 0; j < g->n[1]; ++j)
        for (int64_t i = 0; i < g->n[0]; ++i) {
          int64_t c = cell(g, i, j, k);
          int64_t cp = cell(g, i + (d == 0), j + (d == 1), k + (d == 2));
          for (int n = 0; n < NVAR; ++n)
            L[n * N + c] -= (F[n * N + cp] - F[n * N + c]) / g->dx[d];
        }
  }
  free(W);
  free(F);
  return nfloor;
}

int64_t orc_rhs(const orc_grid* g, const double* U, double* L) {
  return rhs_impl(g, U, L, NULL);
}

/* L(U) with the first-order LLF flux on every face next to a flagged cell (flag: one
 * byte per cell, x1 fastest). */
int64_t orc_rhs_flagged(const orc_grid* g, const double* U, double* L,
                        const unsigned char* flag) {
  return rhs_impl(g, U, L, flag);
}

/* ---------------------------------------------------------------------------------
 * One SSP-RK step (Section 3, method of lines with SSP-RK; reading of the standard
 * coefficients).  Stage s: U <- a_s*U0 + b_s*(U + dt*L(U)).  Returns the number of
 * floors applied, or -1 on allocation failure.
 * ------------------------------------------------------------------------------- */
int64_t orc_rk_step_fofc(const orc_grid* g, double* U, double dt, int rk, int64_t* nfofc) {
  static const double a2[2] = {0.0, 0.5}, b2[2] = {1.0, 0.5};
  static const double a3[3] = {0.0, 0.75, 1.0 / 3.0}, b3[3] = {1.0, 0.25, 2.0 / 3.0};
  const double* a = (rk == 3) ? a3 : a2;
  const double* b = (rk == 3) ? b3 : b2;
  int ns = (rk == 3) ? 3 : 2;
  int64_t NC = g->n[0] * g->n[1] * g->n[2];
  int64_t N = NVAR * NC;
  double* U0 = (double*)malloc(sizeof(double) * N);
  double* L = (double*)malloc(sizeof(double) * N);
  unsigned char* flag = g->fofc ? (unsigned char*)malloc(NC) : NULL;
  if (!U0 || !L || (g->fofc && !flag)) {
    free(U0);
    free(L);
    free(flag);
    return -1;
  }
  memcpy(U0, U, sizeof(double) * N);
  int64_t nfloor = 0, nflag = 0;
  for (int s = 0; s < ns; ++s) {
    int64_t nf = orc_rhs(g, U, L);
    if (nf < 0) {
      nfloor = -1;
      break;
    }
    nfloor += nf;
    if (g->fofc) {
      /* tentative update; flag cells whose density or internal energy is not positive */
      int64_t nst = 0;
#pragma omp parallel for reduction(+ : nst)
      for (int64_t c = 0; c < NC; ++c) {
        double u[5];
        for (int n = 0; n < NVAR; ++n)
          u[n] = a[s] * U0[n * NC + c] + b[s] * (U[n * NC + c] + dt * L[n * NC + c]);
        double ug = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0];
        flag[c] = !(u[0] > 0.0) || !(ug > 0.0);
        nst += flag[c];
      }
      if (nst) {
        nflag += nst;
        if (rhs_impl(g, U, L, flag) < 0) {
          nfloor = -1;
          break;
        }
      }
    }
#pragma omp parallel for
    for (int64_t c = 0; c < N; ++c) U[c] = a[s] * U0[c] + b[s] * (U[c] + dt * L[c]);
  }
  free(U0);
  free(L);
  free(flag);
  if (nfofc) *nfofc = nflag;
  return nfloor;
}

int64_t orc_rk_step(const orc_grid* g, double* U, double dt, int rk) {
  return orc_rk_step_fofc(g, U, dt, rk, NULL);
}

/* ---------------------------------------------------------------------------------
 * CFL time step, Section 3 Eq. (3): dt = CFL * min over cells and dimensions of
 * dx_d / lambda_max,d with lambda_max,d = |v_d| + c_s, c_s = sqrt(gamma p / rho).
 * ------------------------------------------------------------------------------- */
double orc_new_dt(const orc_grid* g, const double* U, double cfl) {
  int64_t N = g->n[0] * g->n[1] * g->n[2];
  double dtmin = INFINITY;
#pragma omp parallel for reduction(min : dtmin)
  for (int64_t c = 0; c < N; ++c) {
    double u[5], w[5];
    int64_t nf = 0;
    for (int n = 0; n < NVAR; ++n) u[n] = U[n * N + c];
    orc_cons_to_prim(u, w, &nf);
    double p = (g->gamma - 1.0) * w[4];
    double cs = sqrt(g->gamma * p / w[0]);
    for (int d = 0; d < 3; ++d) {
      double dtd = g->dx[d] / (fabs(w[1 + d]) + cs);
      if (dtd < dtmin) dtmin = dtd;
    }
  }
  return cfl * dtmin;
}

/* ---------------------------------------------------------------------------------
 * Exact Riemann solver for the gamma-law Euler equations (Toro ch. 4), used only to
 * pin the scheme on shock tubes.  Solves f_L(p) + f_R(p) + (u_R - u_L) = 0 by Newton
 * iteration, then samples the self-similar solution at xi = x/t.
 * ------------------------------------------------------------------------------- */
static void pressure_fn(double p, double rk, double pk, double ck, double gamma, double* f,
                        double* fd) {
  if (p > pk) { /* shock: Rankine-Hugoniot */
    double A = 2.0 / ((gamma + 1.0) * rk);
    double B = (gamma - 1.0) / (gamma + 1.0) * pk;
    double q = sqrt(A / (p + B));
    *f = (p - pk) * q;
    *fd = q * (1.0 - 0.5 * (p - pk) / (p + B));
  } else { /* rarefaction: isentropic */
    double ex = (gamma - 1.0) / (2.0 * gamma);
    *f = 2.0 * ck / (gamma - 1.0) * (pow(p / pk, ex) - 1.0);
    *fd = 1.0 / (rk * ck) * pow(p / pk, -(gamma + 1.0) / (2.0 * gamma));
  }
}

/* Star-region pressure and velocity.  Returns 0, or -1 if a vacuum forms. */
int orc_exact_star(const double wl[3], const double wr[3], double gamma, double* pstar,
                   double* ustar) {
  /* wl, wr = (rho, u, p) */
  double rl = wl[0], ul = wl[1], pl = wl[2];
  double rr = wr[0], ur = wr[1], pr = wr[2];
  double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
  if (2.0 / (gamma - 1.0) * (cl + cr) <= ur - ul) return -1;
  double p = 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr);
  if (p < 1e-8 * (pl < pr ? pl : pr)) p = 1e-8 * (pl < pr ? pl : pr);
  for (int it = 0; it < 200; ++it) {
    double fl, fdl, fr, fdr;
    pressure_fn(p, rl, pl, cl, gamma, &fl, &fdl);
    pressure_fn(p, rr, pr, cr, gamma, &fr, &fdr);
    double pn = p - (fl + fr + ur - ul) / (fdl + fdr);
    if (pn < 0.0) pn = 0.5 * p;
    double change = fabs(pn - p) / (0.5 * (pn + p));
    p = pn;
    if (change < 1e-15) break;
  }
  double fl, fdl, fr, fdr;
  pressure_fn(p, rl, pl, cl, gamma, &fl, &fdl);
  pressure_fn(p, rr, pr, cr, gamma, &fr, &fdr);
  *pstar = p;
  *ustar = 0.5 * (ul + ur) + 0.5 * (fr - fl);
  return 0;
}

/* Sample the exact solution at xi = x/t; out = (rho, u, p). */
int orc_exact_sample(const double wl[3], const double wr[3], double gamma, double xi,
                     double out[3]) {
  double ps, us;
  if (orc_exact_star(wl, wr, gamma, &ps, &us) != 0) return -1;
  double g1 = (gamma - 1.0) / (gamma + 1.0);
  if (xi <= us) { /* left of the contact */
    double rl = wl[0], ul = wl[1], pl = wl[2];
    double cl = sqrt(gamma * pl / rl);
    if (ps > pl) { /* left shock */
      double sl = ul - cl * sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl +
                                 (gamma - 1.0) / (2.0 * gamma));
      if (xi <= sl) {
        out[0] = rl; out[1] = ul; out[2] = pl;
      } else {
        out[0] = rl * (ps / pl + g1) / (g1 * ps / pl + 1.0);
        out[1] = us; out[2] = ps;
      }
    } else { /* left rarefaction */
      double rs = rl * pow(ps / pl, 1.0 / gamma);
      double cs = cl * pow(ps / pl, (gamma - 1.0) / (2.0 * gamma));
      double head = ul - cl, tail = us - cs;
      if (xi <= head) {
        out[0] = rl; out[1] = ul; out[2] = pl;
      } else if (xi >= tail) {
        out[0] = rs; out[1] = us; out[2] = ps;
      } else { /* inside the fan */
        double u = 2.0 / (gamma + 1.0) * (cl + 0.5 * (gamma - 1.0) * ul + xi);
        double c = 2.0 / (gamma + 1.0) * (cl + 0.5 * (gamma - 1.0) * (ul - xi));
        out[0] = rl * pow(c / cl, 2.0 / (gamma - 1.0));
        out[1] = u;
        out[2] = pl * pow(c / cl, 2.0 * gamma / (gamma - 1.0));
      }
    }
  } else { /* right of the contact */
    double rr = wr[0], ur = wr[1], pr = wr[2];
    double cr = sqrt(gamma * pr / rr);
    if (ps > pr) { /* right shock */
      double sr = ur + cr * sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr +
                                 (gamma - 1.0) / (2.0 * gamma));
      if (xi >= sr) {
        out[0] = rr; out[1] = ur; out[2] = pr;
      } else {
        out[0] = rr * (ps / pr + g1) / (g1 * ps / pr + 1.0);
        out[1] = us; out[2] = ps;
      }
    } else { /* right rarefaction */
      double rs = rr * pow(ps / pr, 1.0 / gamma);
      double cs = cr * pow(ps / pr, (gamma - 1.0) / (2.0 * gamma));
      double head = ur + cr, tail = us + cs;
      if (xi >= head) {
        out[0] = rr; out[1] = ur; out[2] = pr;
      } else if (xi <= tail) {
        out[0] = rs; out[1] = us; out[2] = ps;
      } else {
        double u = 2.0 / (gamma + 1.0) * (-cr + 0.5 * (gamma - 1.0) * ur + xi);
        double c = 2.0 / (gamma + 1.0) * (cr - 0.5 * (gamma - 1.0) * (ur - xi));
        out[0] = rr * pow(c / cr, 2.0 / (gamma - 1.0));
        out[1] = u;
        out[2] = pr * pow(c / cr, 2.0 * gamma / (gamma - 1.0));
      }
    }
  }
  return 0;
}

/* Thread count the OpenMP runtime will use (reported with CPU timings). */
int orc_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
