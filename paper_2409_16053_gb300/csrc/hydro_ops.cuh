// Device operations of the hydro stage: primitive recovery, reconstruction and the
// HLLC Riemann solver, in two arithmetic forms.
//
//   FP64 form  -- every operation in double precision.
//   mixed form -- primitive recovery and everything on the conserved state in double
//                 precision; reconstruction, Riemann solver and flux arithmetic in
//                 single precision on deviations from a background state (rho_b,
//                 u_g,b), so that FP32 keeps its relative precision on small
//                 perturbations: W' = (rho - rho_b, v1, v2, v3, u_g - u_g,b).  The
//                 background pressure is left out of the normal momentum flux; a
//                 constant flux cancels exactly in the divergence.
//
// Sources: Section 3, Eq. (1) and Section 3.1, Eq. (4) of AthenaK (arXiv 2409.16053)
// for the equations; PLM with the van Leer harmonic limiter, PPM4 after Colella &
// Woodward (1984) and HLLC after Toro (2009) ch. 10 (PVRS wave-speed estimate bounded
// outward by the Davis speeds), as readings of the methods the paper names.
#pragma once

#include <cuda_runtime.h>

namespace ak {

// Background state of the mixed form and EOS constants, passed by value.
struct Bg {
  double rho, ug;        // FP64 background subtracted before the FP32 arithmetic
  float rho_f, ug_f;     // the same, rounded
  double gamma;
  float gamma_f;
};

// ------------------------------------------------------------------------------
// Reconstruction (Section 3: on primitive variables).
// ------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R plm_slope(R qm, R q0, R qp) {
  // van Leer harmonic mean of the one-sided differences; zero at extrema
  R dl = q0 - qm;
  R dr = qp - q0;
  R prod = dl * dr;
  return prod > R(0) ? R(2) * prod / (dl + dr) : R(0);
}

template <typename R>
__device__ __forceinline__ R ppm_slope(R qm, R q0, R qp) {
  // centred difference limited to twice the one-sided ones, zero at extrema (CW84)
  R dl = q0 - qm;
  R dr = qp - q0;
  if (dl * dr <= R(0)) return R(0);
  R d = R(0.5) * (qp - qm);
  R m = fabs(d);
  R tl = R(2) * fabs(dl);
  R tr = R(2) * fabs(dr);
  m = tl < m ? tl : m;
  m = tr < m ? tr : m;
  return d > R(0) ? m : -m;
}

// Edge values (lower, upper) of the monotonized parabola of the middle cell of
// q[0..4] (CW84 interface values on a uniform grid and their monotonization).
template <typename R>
__device__ __forceinline__ void ppm_edges(R q0, R q1, R q2, R q3, R q4, R& lo, R& hi) {
  R sm = ppm_slope(q0, q1, q2);
  R sc = ppm_slope(q1, q2, q3);
  R sp = ppm_slope(q2, q3, q4);
  R a_lo = R(0.5) * (q1 + q2) - (sc - sm) / R(6);
  R a_hi = R(0.5) * (q2 + q3) - (sp - sc) / R(6);
  R a = q2;
  if ((a_hi - a) * (a - a_lo) <= R(0)) {
    a_lo = a;
    a_hi = a;
  } else {
    R da = a_hi - a_lo;
    R a6 = R(6) * (a - R(0.5) * (a_lo + a_hi));
    if (da * a6 > da * da) {
      a_lo = R(3) * a - R(2) * a_hi;
    } else if (-da * da > da * a6) {
      a_hi = R(3) * a - R(2) * a_lo;
    }
  }
  lo = a_lo;
  hi = a_hi;
}

// ------------------------------------------------------------------------------
// HLLC, FP64 form.  w = (rho, u_n, u_t1, u_t2, u_g); f = flux of
// (rho, M_n, M_t1, M_t2, E).
// ------------------------------------------------------------------------------
__device__ __forceinline__ void hllc_fp64(const double* wl, const double* wr, double gamma,
                                          double* f) {
  const double gm1 = gamma - 1.0;
  const double rl = wl[0], ul = wl[1], rr = wr[0], ur = wr[1];
  const double pl = gm1 * wl[4];
  const double pr = gm1 * wr[4];
  const double el = wl[4] + 0.5 * rl * (ul * ul + wl[2] * wl[2] + wl[3] * wl[3]);
  const double er = wr[4] + 0.5 * rr * (ur * ur + wr[2] * wr[2] + wr[3] * wr[3]);
  const double cl = sqrt(gamma * pl / rl);
  const double cr = sqrt(gamma * pr / rr);

  // pressure estimate of the linearised (PVRS) solver, then shock-aware speeds
  double ps = 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr);
  ps = ps > 0.0 ? ps : 0.0;
  const double kq = (gamma + 1.0) / (2.0 * gamma);
  double ql = 1.0, qr = 1.0;
  if (ps > pl) ql = sqrt(1.0 + kq * (ps / pl - 1.0));
  if (ps > pr) qr = sqrt(1.0 + kq * (ps / pr - 1.0));
  double sl = ul - cl * ql;
  double sr = ur + cr * qr;
  sl = (ur - cr < sl) ? ur - cr : sl;
  sr = (ul + cl > sr) ? ul + cl : sr;

  const double ml = rl * (sl - ul);  // mass flux through the left wave (frame of S_L)
  const double mr = rr * (sr - ur);
  const double sstar = (pr - pl + ul * ml - ur * mr) / (ml - mr);

  const bool left = sstar >= 0.0;
  const double* w = left ? wl : wr;
  const double rk = w[0], uk = w[1];
  const double pk = left ? pl : pr;
  const double ek = left ? el : er;
  const double mn = rk * uk;
  double fk[5];
  fk[0] = mn;
  fk[1] = mn * uk + pk;
  fk[2] = mn * w[2];
  fk[3] = mn * w[3];
  fk[4] = (ek + pk) * uk;
  if (sl >= 0.0 || sr <= 0.0) {
    // supersonic: the upwind physical flux (S_L >= 0 takes the left state)
    const bool up_left = sl >= 0.0;
    const double* wu = up_left ? wl : wr;
    const double pu = up_left ? pl : pr;
    const double eu = up_left ? el : er;
    const double mu = wu[0] * wu[1];
    f[0] = mu;
    f[1] = mu * wu[1] + pu;
    f[2] = mu * wu[2];
    f[3] = mu * wu[3];
    f[4] = (eu + pu) * wu[1];
    return;
  }
  const double s = left ? sl : sr;
  const double fac = rk * (s - uk) / (s - sstar);
  double us[5];
  us[0] = fac;
  us[1] = fac * sstar;
  us[2] = fac * w[2];
  us[3] = fac * w[3];
  us[4] = fac * (ek / rk + (sstar - uk) * (sstar + pk / (rk * (s - uk))));
  f[0] = fk[0] + s * (us[0] - rk);
  f[1] = fk[1] + s * (us[1] - mn);
  f[2] = fk[2] + s * (us[2] - rk * w[2]);
  f[3] = fk[3] + s * (us[3] - rk * w[3]);
  f[4] = fk[4] + s * (us[4] - ek);
}

// ------------------------------------------------------------------------------
// HLLC, mixed form.  w = (rho - rho_b, u_n, u_t1, u_t2, u_g - u_g,b) in FP32.
// Returns F - (0, p_b, 0, 0, 0).  Every difference of two O(1) quantities is formed
// from the deviations, so that a perturbation of relative size 1e-6 keeps ~7 digits.
// ------------------------------------------------------------------------------
__device__ __forceinline__ void hllc_mixed(const float* wl, const float* wr, const Bg& bg,
                                           float* f) {
  const float g = bg.gamma_f;
  const float gm1 = g - 1.0f;
  const float rl = bg.rho_f + wl[0], rr = bg.rho_f + wr[0];
  const float ul = wl[1], ur = wr[1];
  const float dpl = gm1 * wl[4], dpr = gm1 * wr[4];     // p - p_b
  const float pb = gm1 * bg.ug_f;
  const float pl = pb + dpl, pr = pb + dpr;             // full pressures
  const float kel = 0.5f * rl * (ul * ul + wl[2] * wl[2] + wl[3] * wl[3]);
  const float ker = 0.5f * rr * (ur * ur + wr[2] * wr[2] + wr[3] * wr[3]);
  const float hl = kel + g / gm1 * pl;                  // E + p
  const float hr = ker + g / gm1 * pr;
  const float cl = sqrtf(g * pl / rl);
  const float cr = sqrtf(g * pr / rr);

  // PVRS estimate as a deviation from p_b; p* = max(0, p_b + dps)
  float dps = 0.5f * (dpl + dpr) - 0.125f * (ur - ul) * (rl + rr) * (cl + cr);
  dps = (pb + dps > 0.0f) ? dps : -pb;
  const float kq = (g + 1.0f) / (2.0f * g);
  float ql = 1.0f, qr = 1.0f;
  if (dps > dpl) ql = sqrtf(1.0f + kq * (dps - dpl) / pl);
  if (dps > dpr) qr = sqrtf(1.0f + kq * (dps - dpr) / pr);
  float sl = ul - cl * ql;
  float sr = ur + cr * qr;
  sl = (ur - cr < sl) ? ur - cr : sl;
  sr = (ul + cl > sr) ? ul + cl : sr;

  const float ml = rl * (sl - ul);
  const float mr = rr * (sr - ur);
  const float sstar = (dpr - dpl + ul * ml - ur * mr) / (ml - mr);

  if (sl >= 0.0f || sr <= 0.0f) {
    const bool up_left = sl >= 0.0f;
    const float* wu = up_left ? wl : wr;
    const float ru = up_left ? rl : rr;
    const float mu = ru * wu[1];
    f[0] = mu;
    f[1] = mu * wu[1] + (up_left ? dpl : dpr);
    f[2] = mu * wu[2];
    f[3] = mu * wu[3];
    f[4] = (up_left ? hl : hr) * wu[1];
    return;
  }
  const bool left = sstar >= 0.0f;
  const float* w = left ? wl : wr;
  const float rk = left ? rl : rr;
  const float uk = w[1];
  const float s = left ? sl : sr;
  const float pk = left ? pl : pr;
  const float ek = (left ? kel : ker) + (bg.ug_f + w[4]);
  const float mn = rk * uk;
  const float inv = 1.0f / (s - sstar);
  const float fac = rk * (s - uk) * inv;
  const float drho = rk * (sstar - uk) * inv;           // U*_rho - rho_K
  const float dmn = fac * sstar - mn;                   // U*_Mn - M_n
  const float de = drho / rk * ek + fac * (sstar - uk) * (sstar + pk / (rk * (s - uk)));
  f[0] = mn + s * drho;
  f[1] = mn * uk + (left ? dpl : dpr) + s * dmn;
  f[2] = mn * w[2] + s * drho * w[2];
  f[3] = mn * w[3] + s * drho * w[3];
  f[4] = (left ? hl : hr) * uk + s * de;
}

}  // namespace ak
