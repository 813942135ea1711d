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

#include "fastmath.cuh"

namespace ak {

// Background state of the mixed form and EOS constants, passed by value.
struct Bg {
  double rho, ug;        // FP64 background subtracted before the FP32 arithmetic
  float rho_f, ug_f;     // the same, rounded
  double gamma;
  float gamma_f;
  double kq;             // (gamma + 1) / (2 gamma), for the shock speed factor
  double gm1;            // gamma - 1
  float ug_floor_f;      // u_g floor minus u_g,b, rounded (mixed form)
};

// ------------------------------------------------------------------------------
// Reconstruction (Section 3: on primitive variables).
// ------------------------------------------------------------------------------
// One fused multiply-add in the reconstruction's own precision (the library compiles
// without implicit contraction: every fma is written out).
__device__ __forceinline__ float fmar(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return fma(a, b, c); }

// van Leer harmonic mean of the one-sided differences; zero at extrema.
// FP64: the harmonic mean with a Newton-refined reciprocal (no IEEE division)
__device__ __forceinline__ double plm_slope(double qm, double q0, double qp) {
  const double dl = q0 - qm;
  const double dr = qp - q0;
  const double prod = dl * dr;
  return prod > 0.0 ? (prod + prod) * rcp64(dl + dr) : 0.0;
}

// FP32: the harmonic mean with the hardware reciprocal refined once in FP32
__device__ __forceinline__ float plm_slope(float qm, float q0, float qp) {
  const float dl = q0 - qm;
  const float dr = qp - q0;
  const float prod = dl * dr;
  if (!(prod > 0.0f)) return 0.0f;
  const float s = dl + dr;
  float r = rcp_approx_f32(s);
  r = fmaf(r, fmaf(-s, r, 1.0f), r);
  return (prod + prod) * r;
}

// Half of the van Leer slope, dl dr / (dl + dr): the offset of the face values from the
// cell value.  In FP64 it skips the doubling and halving of plm_slope (same bits: both
// are exact scalings by two).
__device__ __forceinline__ double plm_half_slope(double qm, double q0, double qp) {
  const double dl = q0 - qm;
  const double dr = qp - q0;
  const double prod = dl * dr;
  return dpos(prod) ? prod * rcp64(dl + dr) : 0.0;
}
__device__ __forceinline__ float plm_half_slope(float qm, float q0, float qp) {
  return 0.5f * plm_slope(qm, q0, qp);
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
  const R sixth = R(1) / R(6);
  R a_lo = fmar(sm - sc, sixth, R(0.5) * (q1 + q2));
  R a_hi = fmar(sc - sp, sixth, R(0.5) * (q2 + q3));
  R a = q2;
  if ((a_hi - a) * (a - a_lo) <= R(0)) {
    a_lo = a;
    a_hi = a;
  } else {
    R da = a_hi - a_lo;
    R a6 = R(6) * fmar(R(-0.5), a_lo + a_hi, a);
    if (da * a6 > da * da) {
      a_lo = fmar(R(3), a, R(-2) * a_hi);
    } else if (-da * da > da * a6) {
      a_hi = fmar(R(3), a, R(-2) * a_lo);
    }
  }
  lo = a_lo;
  hi = a_hi;
}

// ------------------------------------------------------------------------------
// HLLC, FP64 form.  w = (rho, u_n, u_t1, u_t2, u_g); f = flux of
// (rho, M_n, M_t1, M_t2, E).
// ------------------------------------------------------------------------------
__device__ __forceinline__ void hllc_fp64(const double* wl, const double* wr, const Bg& bg,
                                          double* f) {
  // Comparisons run on the integer pipe (dgt/dpos/dnonneg) and powers of two scale
  // by exponent arithmetic (dscale): only the arithmetic itself uses the FP64 unit.
  const double gamma = bg.gamma;
  const double gm1 = bg.gm1;
  const double rl = wl[0], ul = wl[1], rr = wr[0], ur = wr[1];
  const double pl = gm1 * wl[4];
  const double pr = gm1 * wr[4];
  // c = sqrt(gamma p / rho) = (gamma p) / sqrt(gamma p rho)
  const double gpl = gamma * pl, gpr = gamma * pr;
  const double cl = gpl * rsqrt64(gpl * rl);
  const double cr = gpr * rsqrt64(gpr * rr);

  // pressure estimate of the linearised (PVRS) solver, then shock-aware speeds
  double ps = fma(-dscale_down((ur - ul) * (rl + rr), 3, 0.125), cl + cr,
                  dscale_down(pl + pr, 1, 0.5));
  ps = dpos(ps) ? ps : 0.0;
  const double kq = bg.kq;
  double ql = 1.0, qr = 1.0;
  if (dgt_pos(ps, pl)) ql = sqrt64(fma(kq * (ps - pl), rcp64(pl), 1.0));
  if (dgt_pos(ps, pr)) qr = sqrt64(fma(kq * (ps - pr), rcp64(pr), 1.0));
  double sl = fma(-cl, ql, ul);
  double sr = fma(cr, qr, ur);
  const double dl = ur - cr, dr = ul + cl;
  sl = dgt(sl, dl) ? dl : sl;
  sr = dgt(dr, sr) ? dr : sr;

  const bool sup_l = dnonneg(sl), sup_r = !dpos(sr);
  if (sup_l || sup_r) {
    // supersonic: the upwind physical flux (S_L >= 0 takes the left state)
    const double* wu = sup_l ? wl : wr;
    const double pu = sup_l ? pl : pr;
    const double ru = wu[0], uu = wu[1];
    const double eu = fma(dscale(ru, -1), fma(uu, uu, fma(wu[2], wu[2], wu[3] * wu[3])), wu[4]);
    const double mu = ru * uu;
    f[0] = mu;
    f[1] = fma(mu, uu, pu);
    f[2] = mu * wu[2];
    f[3] = mu * wu[3];
    f[4] = (eu + pu) * uu;
    return;
  }
  const double ml = rl * (sl - ul);  // mass flux through the left wave (frame of S_L)
  const double mr = rr * (sr - ur);
  const double sstar = fma(ul, ml, fma(-ur, mr, pr - pl)) * rcp64(ml - mr);

  const bool left = dnonneg(sstar);
  const double* w = left ? wl : wr;
  const double rk = w[0], uk = w[1];
  const double pk = left ? pl : pr;
  const double mk = left ? ml : mr;  // rho_K (S_K - u_K)
  const double s = left ? sl : sr;
  const double ek = fma(dscale(rk, -1), fma(uk, uk, fma(w[2], w[2], w[3] * w[3])), w[4]);
  const double mn = rk * uk;
  const double inv = rcp64(s - sstar);
  const double fac = mk * inv;       // rho*_K
  // E*_K = fac (E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K))))
  //      = E_K (S_K - u_K)/(S_K - S*) + (S* - u_K)(fac S* + p_K/(S_K - S*))
  const double us4 = fma(sstar - uk, fma(fac, sstar, pk * inv), ek * ((s - uk) * inv));
  const double mt = fma(s, fac - rk, mn);  // M_n + S_K (rho*_K - rho_K)
  f[0] = mt;
  f[1] = fma(s, fma(fac, sstar, -mn), fma(mn, uk, pk));
  f[2] = mt * w[2];
  f[3] = mt * w[3];
  f[4] = fma(s, us4 - ek, (ek + pk) * uk);
}

// ------------------------------------------------------------------------------
// HLLC, mixed form.  w = (rho - rho_b, u_n, u_t1, u_t2, u_g - u_g,b) in FP32.
// Returns F - (0, p_b, 0, 0, 0).  Every difference of two O(1) quantities is formed
// from the deviations, so that a perturbation of relative size 1e-6 keeps ~7 digits.
// ------------------------------------------------------------------------------
__device__ __forceinline__ float sqrt_fast(float x) { return x * rsqrt_approx_f32(x); }

__device__ __forceinline__ void hllc_mixed(const float* wl, const float* wr, const Bg& bg,
                                           float* f) {
  const float g = bg.gamma_f;
  const float gm1 = g - 1.0f;
  const float gg = g * rcp_approx_f32(gm1);             // gamma / (gamma - 1)
  const float rl = bg.rho_f + wl[0], rr = bg.rho_f + wr[0];
  const float ul = wl[1], ur = wr[1];
  const float dpl = gm1 * wl[4], dpr = gm1 * wr[4];     // p - p_b
  const float pb = gm1 * bg.ug_f;
  const float pl = pb + dpl, pr = pb + dpr;             // full pressures
  const float kel = 0.5f * rl * fmaf(ul, ul, fmaf(wl[2], wl[2], wl[3] * wl[3]));
  const float ker = 0.5f * rr * fmaf(ur, ur, fmaf(wr[2], wr[2], wr[3] * wr[3]));
  const float hl = fmaf(gg, pl, kel);                   // E + p
  const float hr = fmaf(gg, pr, ker);
  const float gpl = g * pl, gpr = g * pr;
  const float cl = gpl * rsqrt_approx_f32(gpl * rl);   // sqrt(gamma p / rho)
  const float cr = gpr * rsqrt_approx_f32(gpr * rr);

  // PVRS estimate as a deviation from p_b; p* = max(0, p_b + dps)
  float dps = fmaf(-0.125f * (ur - ul) * (rl + rr), cl + cr, 0.5f * (dpl + dpr));
  dps = (pb + dps > 0.0f) ? dps : -pb;
  const float kq = (g + 1.0f) * rcp_approx_f32(2.0f * g);
  float ql = 1.0f, qr = 1.0f;
  if (dps > dpl) ql = sqrt_fast(fmaf(kq * (dps - dpl), rcp_approx_f32(pl), 1.0f));
  if (dps > dpr) qr = sqrt_fast(fmaf(kq * (dps - dpr), rcp_approx_f32(pr), 1.0f));
  float sl = fmaf(-cl, ql, ul);
  float sr = fmaf(cr, qr, ur);
  sl = (ur - cr < sl) ? ur - cr : sl;
  sr = (ul + cl > sr) ? ul + cl : sr;

  if (sl >= 0.0f || sr <= 0.0f) {
    const bool up_left = sl >= 0.0f;
    const float* wu = up_left ? wl : wr;
    const float ru = up_left ? rl : rr;
    const float mu = ru * wu[1];
    f[0] = mu;
    f[1] = fmaf(mu, wu[1], up_left ? dpl : dpr);
    f[2] = mu * wu[2];
    f[3] = mu * wu[3];
    f[4] = (up_left ? hl : hr) * wu[1];
    return;
  }
  const float ml = rl * (sl - ul);
  const float mr = rr * (sr - ur);
  const float sstar = fmaf(ul, ml, fmaf(-ur, mr, dpr - dpl)) * rcp_approx_f32(ml - mr);
  const bool left = sstar >= 0.0f;
  const float* w = left ? wl : wr;
  const float rk = left ? rl : rr;
  const float mk = left ? ml : mr;                      // rho_K (S_K - u_K)
  const float uk = w[1];
  const float s = left ? sl : sr;
  const float pk = left ? pl : pr;
  const float ek = (left ? kel : ker) + (bg.ug_f + w[4]);
  const float mn = rk * uk;
  const float inv = rcp_approx_f32(s - sstar);
  const float fac = mk * inv;
  const float drho = rk * (sstar - uk) * inv;           // U*_rho - rho_K
  const float dmn = fmaf(fac, sstar, -mn);              // U*_Mn - M_n
  // E*_K - E_K = (S* - u_K) ((E_K + p_K) / (S_K - S*) + rho*_K S*)
  const float de = (sstar - uk) * fmaf(fac, sstar, (ek + pk) * inv);
  const float mt = fmaf(s, drho, mn);                   // M_n + S_K (U*_rho - rho_K)
  f[0] = mt;
  f[1] = fmaf(s, dmn, fmaf(mn, uk, left ? dpl : dpr));
  f[2] = mt * w[2];
  f[3] = mt * w[3];
  f[4] = fmaf(s, de, (left ? hl : hr) * uk);
}

}  // namespace ak
