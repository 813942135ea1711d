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
// Woodward (1984), PPMX after Colella & Sekora (2008) and McCorquodale & Colella (2011), HLLC after Toro (2009) ch. 10 (PVRS wave-speed estimate bounded
// outward by the Davis speeds), HLLE (HLL with Einfeldt's Roe-average speeds, Toro
// Sec. 10.5.1) and LLF (Rusanov), as readings of the methods the paper names.
#pragma once

#include <cuda_runtime.h>

#include "fastmath.cuh"
#include "lanes.cuh"

namespace ak {

// Background state of the mixed form and EOS constants, passed by value.
struct Bg {
  double rho, ug;        // FP64 background subtracted before the FP32 arithmetic
  float rho_f, ug_f;     // the same, rounded
  double gamma;
  float gamma_f;
  float gamma_l;         // gamma - gamma_f, rounded: gamma split into two floats
  double kq;             // (gamma + 1) / (2 gamma), for the shock speed factor
  double kq1;            // 1 - kq
  double gm1;            // gamma - 1
  float ug_floor_f;      // mixed form: u_g floor minus u_g,b, rounded
  double rho_min;        // mixed form: density floor
  float gm1_f;           // gamma - 1, gamma / (gamma - 1), (gamma + 1) / (2 gamma) and
  float gg_f;            // p_b = (gamma - 1) u_g,b, rounded (mixed form)
  float kq_f;
  float pb_f;
  int rsolver;           // AK_HLLC, AK_HLLE or AK_LLF
  int recon;             // AK_PLM, AK_PPM4, AK_WENOZ or AK_PPMX
};

// ------------------------------------------------------------------------------
// Reconstruction (Section 3: on primitive variables).
// ------------------------------------------------------------------------------
// One fused multiply-add in the reconstruction's own precision (the library compiles
// without implicit contraction: every fma is written out).
__device__ __forceinline__ float fmar(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return fma(a, b, c); }

// FP64 PPM4 with the sign tests, minima and exact halvings on the integer pipe.  The
// limited slope is carried as half its value,
//   h = sgn(dq) min(|qp - qm| / 4, |q0 - qm|, |qp - q0|)  (0 at extrema),
// so the interface value 0.5 (q_i + q_i+1) - (S_i+1 - S_i) / 6 is
// fma(h_i - h_i+1, 1/3, 0.5 (q_i + q_i+1)); the monotonization keeps the products of CW84.
__device__ __forceinline__ double ppm_half_slope_fp64(double qm, double q0, double qp) {
  const double dl = q0 - qm, dr = qp - q0;
  const long long bl = __double_as_longlong(dl), br = __double_as_longlong(dr);
  if ((bl ^ br) < 0 || (bl << 1) == 0 || (br << 1) == 0) return 0.0;  // extremum or flat
  const double s = qp - qm;
  const long long mask = 0x7fffffffffffffffll;
  long long m = __double_as_longlong(dscale_down(s, 2)) & mask;       // |qp - qm| / 4
  m = (bl & mask) < m ? (bl & mask) : m;
  m = (br & mask) < m ? (br & mask) : m;
  return __longlong_as_double(m | (bl & ~mask));                       // sign of dl (= dr)
}

// FP64 CW84 interface value between cells of values ql, qr and half slopes hl, hr
__device__ __forceinline__ double ppm_interface_fp64(double ql, double qr, double hl, double hr) {
  return fma(hl - hr, 1.0 / 3.0, dscale_down(ql + qr, 1));
}

// CW84 monotonization of a cell's interface values a_lo, a_hi around its value a.  CW84's
// tests (a_hi - a_lo) 6 (a - (a_lo + a_hi)/2) > (a_hi - a_lo)^2 and its mirror, divided by
// a_hi - a_lo (whose sign is that of dh = a_hi - a once a lies between the two), compare
// each interface value with the value that puts the parabola's extremum on the opposite
// edge: u = 3a - 2 a_hi = a - 2 dh replaces a_lo where a_lo lies beyond u as seen from a,
// w = 3a - 2 a_lo = a + 2 dlo replaces a_hi likewise (the two cannot both apply).  Four
// FP64 operations instead of ten; the results differ from the product form only where a
// test is decided by rounding, where both choices agree to rounding.
__device__ __forceinline__ void ppm_monotonize_fp64(double a_lo, double a_hi, double a,
                                                    double& lo, double& hi) {
  const double dh = a_hi - a, dlo = a - a_lo;
  const long long bh = __double_as_longlong(dh), bo = __double_as_longlong(dlo);
  if ((bh ^ bo) < 0 || (bh << 1) == 0 || (bo << 1) == 0) {  // (a_hi - a)(a - a_lo) <= 0
    lo = a;
    hi = a;
    return;
  }
  const double u = fma(-2.0, dh, a), w = fma(2.0, dlo, a);
  if (bh > 0) {  // a_lo < a < a_hi
    lo = dgt(u, a_lo) ? u : a_lo;
    hi = dgt(a_hi, w) ? w : a_hi;
  } else {       // a_hi < a < a_lo
    lo = dgt(a_lo, u) ? u : a_lo;
    hi = dgt(w, a_hi) ? w : a_hi;
  }
}

__device__ __forceinline__ void ppm_edges_fp64(double q0, double q1, double q2, double q3,
                                               double q4, double& lo, double& hi) {
  const double hm = ppm_half_slope_fp64(q0, q1, q2);
  const double hc = ppm_half_slope_fp64(q1, q2, q3);
  const double hp = ppm_half_slope_fp64(q2, q3, q4);
  ppm_monotonize_fp64(ppm_interface_fp64(q1, q2, hm, hc), ppm_interface_fp64(q2, q3, hc, hp), q2,
                      lo, hi);
}

// PPMX: PPM with extremum-preserving limiters.  The fourth-order interface value
//   f = 7/12 (q_i + q_i+1) - 1/12 (q_i-1 + q_i+2);
// if f is not between q_i and q_i+1, its second difference 3 (q_i + q_i+1 - 2 f) is
// limited by those of cells i and i+1 (Colella & Sekora 2008) and
// f = (q_i + q_i+1) / 2 - lim / 6.  In a cell at an extremum (of the parabola, or of the
// cell values) the parabola's second derivative 6 (lo + hi - 2 q) is compared with
// C x the second differences of cells i-1, i, i+1 (C = 1.25) and its deviations from the
// mean are scaled by their ratio r (McCorquodale & Colella 2011); elsewhere the
// overshooting edge is pulled in as in Colella & Woodward.  Five-cell stencil: the
// seven-cell third-derivative test of the latter paper is not applied.  Same
// operations and order in both precisions; -fmad=false keeps each rounding as written.
template <typename R>
__device__ __forceinline__ bool same_sign3(R x, R y, R z) {
  return (x > R(0) && y > R(0) && z > R(0)) || (x < R(0) && y < R(0) && z < R(0));
}
template <typename R>
__device__ __forceinline__ R ppmx_interface(R a, R b, R c, R d) {
  const R C = R(1.25);
  R f = R(7.0 / 12.0) * (b + c) - R(1.0 / 12.0) * (a + d);
  if ((f - b) * (c - f) < R(0)) {
    const R d2 = R(3) * ((b + c) - R(2) * f);
    const R d2l = (a + c) - R(2) * b;
    const R d2r = (b + d) - R(2) * c;
    R lim = R(0);
    if (same_sign3(d2, d2l, d2r)) {
      const R m = fmin(fabs(d2), fmin(C * fabs(d2l), C * fabs(d2r)));
      lim = d2 > R(0) ? m : -m;
    }
    f = R(0.5) * (b + c) - lim / R(6);
  }
  return f;
}
template <typename R>
__device__ __forceinline__ void ppmx_edges(R q0, R q1, R q2, R q3, R q4, R& lo, R& hi) {
  const R C = R(1.25);
  R alo = ppmx_interface(q0, q1, q2, q3);
  R ahi = ppmx_interface(q1, q2, q3, q4);
  const R a = q2, dp = ahi - a, dm = a - alo;
  if (dp * dm <= R(0) || (q3 - a) * (a - q1) <= R(0)) {
    const R d2 = R(6) * ((alo + ahi) - R(2) * a);
    const R d2c = (q1 + q3) - R(2) * a;
    const R d2l = (q0 + a) - R(2) * q1;
    const R d2r = (a + q4) - R(2) * q3;
    R r = R(0);
    bool limit = true;
    if (same_sign3(d2, d2c, d2l) && same_sign3(d2, d2c, d2r)) {
      const R m = C * fmin(fabs(d2c), fmin(fabs(d2l), fabs(d2r)));
      if (m >= fabs(d2))
        limit = false;
      else
        r = m / fabs(d2);
    }
    if (limit) {
      if (dp * dm < R(0)) {
        alo = a - r * dm;
        ahi = a + r * dp;
      } else if (fabs(dm) >= R(2) * fabs(dp)) {
        alo = a - R(2) * (R(1) - r) * dp - r * dm;
      } else if (fabs(dp) >= R(2) * fabs(dm)) {
        ahi = a + R(2) * (R(1) - r) * dm + r * dp;
      }
    }
  } else if (fabs(dm) >= R(2) * fabs(dp)) {
    alo = a - R(2) * dp;
  } else if (fabs(dp) >= R(2) * fabs(dm)) {
    ahi = a + R(2) * dm;
  }
  lo = alo;
  hi = ahi;
}

// WENO-Z value at the face between c and d of the cells a, b, c, d, e (c the cell), in
// FP64 with IEEE division and the plain left-to-right order of the definition: the
// candidates (2a - 7b + 11c)/6, (-b + 5c + 2d)/6, (2c + 5d - e)/6, the indicators
// 13/12 (second difference)^2 + 1/4 (first difference)^2, tau5 = |beta_0 - beta_2| and
// the weights d_k (1 + tau5 / (beta_k + eps)).  The FP64 form uses it for both faces
// (the lower one on the mirrored stencil): in extreme flows, where a reconstructed
// pressure sits at zero, the last bit of these weights decides which faces FOFC
// corrects.  The FP32 form uses wenoz_edges below.
__device__ __forceinline__ double wenoz_value_fp64(double a, double b, double c, double d,
                                                   double e) {
  const double p0 = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
  const double p1 = (-b + 5.0 * c + 2.0 * d) / 6.0;
  const double p2 = (2.0 * c + 5.0 * d - e) / 6.0;
  const double s0 = a - 2.0 * b + c, t0 = a - 4.0 * b + 3.0 * c;
  const double s1 = b - 2.0 * c + d, t1 = b - d;
  const double s2 = c - 2.0 * d + e, t2 = 3.0 * c - 4.0 * d + e;
  const double b0 = 13.0 / 12.0 * s0 * s0 + 0.25 * t0 * t0;
  const double b1 = 13.0 / 12.0 * s1 * s1 + 0.25 * t1 * t1;
  const double b2 = 13.0 / 12.0 * s2 * s2 + 0.25 * t2 * t2;
  const double tau = fabs(b0 - b2);
  const double eps = 1e-40;
  const double a0 = 0.1 * (1.0 + tau / (b0 + eps));
  const double a1 = 0.6 * (1.0 + tau / (b1 + eps));
  const double a2 = 0.3 * (1.0 + tau / (b2 + eps));
  return (a0 * p0 + a1 * p1 + a2 * p2) / (a0 + a1 + a2);
}

// WENO-Z (Borges et al. 2008) values at both faces of the middle cell of q0..q4: the
// three third-order candidates of Jiang & Shu (1996), their smoothness indicators
// beta_k, tau5 = |beta_0 - beta_2| and weights alpha_k = d_k (1 + tau5 / (beta_k + eps))
// with d = (1, 6, 3)/10.  The lower face uses the mirrored stencil, whose indicators are
// beta_2, beta_1, beta_0.  eps = 1e-40 in FP64; 1e-30 in FP32, where 1e-40 would be
// subnormal (and flushed by the hardware reciprocal).
__device__ __forceinline__ double rcp_w(double x) { return rcp64(x); }
__device__ __forceinline__ float rcp_w(float x) {
  float r = rcp_approx_f32(x);
  return fmaf(r, fmaf(-x, r, 1.0f), r);
}
template <typename R>
__device__ __forceinline__ void wenoz_edges(R a, R b, R c, R d, R e, R& lo, R& hi) {
  const R sixth = R(1) / R(6), c13 = R(13) / R(12), q = R(0.25);
  const R eps = sizeof(R) == 8 ? R(1e-40) : R(1e-30);
  const R t0 = fmar(R(-2), b, a + c), u0 = fmar(R(-4), b, fmar(R(3), c, a));
  const R t1 = fmar(R(-2), c, b + d), u1 = b - d;
  const R t2 = fmar(R(-2), d, c + e), u2 = fmar(R(3), c, fmar(R(-4), d, e));
  const R b0 = fmar(c13, t0 * t0, q * (u0 * u0));
  const R b1 = fmar(c13, t1 * t1, q * (u1 * u1));
  const R b2 = fmar(c13, t2 * t2, q * (u2 * u2));
  const R tau = fabs(b0 - b2);
  const R r0 = tau * rcp_w(b0 + eps), r1 = tau * rcp_w(b1 + eps), r2 = tau * rcp_w(b2 + eps);
  // upper face (candidates toward d, e)
  {
    const R p0 = fmar(R(2), a, fmar(R(-7), b, R(11) * c)) * sixth;
    const R p1 = fmar(R(5), c, fmar(R(2), d, -b)) * sixth;
    const R p2 = fmar(R(2), c, fmar(R(5), d, -e)) * sixth;
    const R a0 = fmar(R(0.1), r0, R(0.1)), a1 = fmar(R(0.6), r1, R(0.6)),
            a2 = fmar(R(0.3), r2, R(0.3));
    hi = fmar(a0, p0, fmar(a1, p1, a2 * p2)) * rcp_w(a0 + a1 + a2);
  }
  // lower face: the mirrored stencil e, d, c, b, a
  {
    const R p0 = fmar(R(2), e, fmar(R(-7), d, R(11) * c)) * sixth;
    const R p1 = fmar(R(5), c, fmar(R(2), b, -d)) * sixth;
    const R p2 = fmar(R(2), c, fmar(R(5), b, -a)) * sixth;
    const R a0 = fmar(R(0.1), r2, R(0.1)), a1 = fmar(R(0.6), r1, R(0.6)),
            a2 = fmar(R(0.3), r0, R(0.3));
    lo = fmar(a0, p0, fmar(a1, p1, a2 * p2)) * rcp_w(a0 + a1 + a2);
  }
}

// NANCHK (the FP64 solvers of the reconstructions that can overshoot, WENO-Z and PPMX):
// the wave-speed tests use IEEE comparisons written as in the definition (a test with a
// NaN operand is false), instead of the integer-pipe ones, which order a NaN like a large
// number.  A face state with rho p < 0 has a NaN sound speed; the IEEE tests then pick
// the same branch -- an upwind flux, or a NaN flux that leaves the cells next to the
// face not a number for FOFC to flag -- as the definition does.

// ------------------------------------------------------------------------------
// HLLC, FP64 form.  w = (rho, u_n, u_t1, u_t2, u_g); f = flux of
// (rho, M_n, M_t1, M_t2, E).
// ------------------------------------------------------------------------------
template <bool NANCHK = false>
__device__ __forceinline__ void hllc_fp64(const double* wl, const double* wr, const Bg& bg,
                                          double* f) {
  // Comparisons run on the integer pipe (dgt/dpos/dnonneg) and powers of two scale
  // by exponent arithmetic (dscale): only the arithmetic itself uses the FP64 unit.
  const double gamma = bg.gamma;
  const double gm1 = bg.gm1;
  const double rl = wl[0], ul = wl[1], rr = wr[0], ur = wr[1];
  const double pl = gm1 * wl[4];
  const double pr = gm1 * wr[4];
  // c = sqrt(gamma p / rho) from split mantissas, with gamma split into two floats: no
  // FP64 instruction
  const double cl = sqrt_gratio64(pl, rl, gamma, bg.gamma_f, bg.gamma_l);
  const double cr = sqrt_gratio64(pr, rr, gamma, bg.gamma_f, bg.gamma_l);

  // pressure estimate of the linearised (PVRS) solver, then shock-aware speeds
  double ps = fma(-dscale_down((ur - ul) * (rl + rr), 3), cl + cr, dscale_down(pl + pr, 1));
  const double kq = bg.kq;
  double ql = 1.0, qr = 1.0;
  double sl, sr;
  bool sup_l, sup_r;
  if constexpr (NANCHK) {
    ps = ps > 0.0 ? ps : 0.0;
    if (ps > pl) ql = sqrt64(fma(kq * (ps - pl), rcp64(pl), 1.0));
    if (ps > pr) qr = sqrt64(fma(kq * (ps - pr), rcp64(pr), 1.0));
    sl = fma(-cl, ql, ul);
    sr = fma(cr, qr, ur);
    if (ur - cr < sl) sl = ur - cr;
    if (ul + cl > sr) sr = ul + cl;
    sup_l = sl >= 0.0;
    sup_r = !sup_l && sr <= 0.0;
  } else {
    // q_K = sqrt(1 + kq (p* / p_K - 1)) = sqrt((kq p* + (1 - kq) p_K) / p_K), kq p* shared
    ps = dpos(ps) ? ps : 0.0;
    const double kps = kq * ps;
    if (dgt_pos(ps, pl)) ql = sqrt_ratio64(fma(bg.kq1, pl, kps), pl);
    if (dgt_pos(ps, pr)) qr = sqrt_ratio64(fma(bg.kq1, pr, kps), pr);
    sl = fma(-cl, ql, ul);
    sr = fma(cr, qr, ur);
    const double dl = ur - cr, dr = ul + cl;
    sl = dgt(sl, dl) ? dl : sl;
    sr = dgt(dr, sr) ? dr : sr;
    sup_l = dnonneg(sl);
    sup_r = !dpos(sr);
  }
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

  const bool left = NANCHK ? sstar >= 0.0 : dnonneg(sstar);
  const double* w = left ? wl : wr;
  const double rk = w[0], uk = w[1];
  const double pk = left ? pl : pr;
  const double mk = left ? ml : mr;  // rho_K (S_K - u_K)
  const double s = left ? sl : sr;
  const double ek = fma(dscale(rk, -1), fma(uk, uk, fma(w[2], w[2], w[3] * w[3])), w[4]);
  const double mn = rk * uk;
  const double inv = rcp64(s - sstar);
  const double fac = mk * inv;       // rho*_K
  // E*_K = fac (E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))), so that
  // E*_K - E_K = (S* - u_K) ((E_K + p_K)/(S_K - S*) + rho*_K S*) in closed form,
  // and the star momentum flux is F*_rho S* + p* with p* = p_K + rho_K (S_K - u_K)(S* - u_K)
  const double su = sstar - uk;
  const double ep = ek + pk;
  const double de = su * fma(fac, sstar, ep * inv);
  const double mt = fma(s, fac - rk, mn);  // M_n + S_K (rho*_K - rho_K)
  f[0] = mt;
  f[1] = fma(mt, sstar, fma(mk, su, pk));
  f[2] = mt * w[2];
  f[3] = mt * w[3];
  f[4] = fma(s, de, ep * uk);
}

// ------------------------------------------------------------------------------
// LLF (Rusanov), FP64 form: F = (F_L + F_R)/2 - S+ (U_R - U_L)/2,
// S+ = max(|u_L| + c_L, |u_R| + c_R).
// ------------------------------------------------------------------------------
template <bool NANCHK = false>
__device__ __forceinline__ void llf_fp64(const double* wl, const double* wr, const Bg& bg,
                                         double* f) {
  const double gamma = bg.gamma, gm1 = bg.gm1;
  const double rl = wl[0], ul = wl[1], rr = wr[0], ur = wr[1];
  const double pl = gm1 * wl[4], pr = gm1 * wr[4];
  const double cl = sqrt_gratio64(pl, rl, gamma, bg.gamma_f, bg.gamma_l);
  const double cr = sqrt_gratio64(pr, rr, gamma, bg.gamma_f, bg.gamma_l);
  const double al = fabs(ul) + cl, ar = fabs(ur) + cr;
  const double sm = NANCHK ? -(al > ar ? al : ar) : -(dgt_pos(al, ar) ? al : ar);
  const double el = fma(dscale(rl, -1), fma(ul, ul, fma(wl[2], wl[2], wl[3] * wl[3])), wl[4]);
  const double er = fma(dscale(rr, -1), fma(ur, ur, fma(wr[2], wr[2], wr[3] * wr[3])), wr[4]);
  const double ml = rl * ul, mr = rr * ur;
  f[0] = dscale_down(fma(sm, rr - rl, ml + mr), 1);
  f[1] = dscale_down(fma(sm, mr - ml, fma(ml, ul, pl) + fma(mr, ur, pr)), 1);
  f[2] = dscale_down(fma(sm, fma(rr, wr[2], -(rl * wl[2])), fma(ml, wl[2], mr * wr[2])), 1);
  f[3] = dscale_down(fma(sm, fma(rr, wr[3], -(rl * wl[3])), fma(ml, wl[3], mr * wr[3])), 1);
  f[4] = dscale_down(fma(sm, er - el, fma(el + pl, ul, (er + pr) * ur)), 1);
}

// ------------------------------------------------------------------------------
// HLLE, FP64 form: the HLL flux (b+ F_L - b- F_R + b+ b- (U_R - U_L)) / (b+ - b-) with
// b- = min(S_L, 0), b+ = max(S_R, 0), S_L = min(u_L - c_L, u~ - c~),
// S_R = max(u_R + c_R, u~ + c~) from the Roe averages (weights sqrt(rho)).
// ------------------------------------------------------------------------------
template <bool NANCHK = false>
__device__ __forceinline__ void hlle_fp64(const double* wl, const double* wr, const Bg& bg,
                                          double* f) {
  const double gamma = bg.gamma, gm1 = bg.gm1;
  const double rl = wl[0], ul = wl[1], rr = wr[0], ur = wr[1];
  const double pl = gm1 * wl[4], pr = gm1 * wr[4];
  const double cl = sqrt_gratio64(pl, rl, gamma, bg.gamma_f, bg.gamma_l);
  const double cr = sqrt_gratio64(pr, rr, gamma, bg.gamma_f, bg.gamma_l);
  const double el = fma(dscale(rl, -1), fma(ul, ul, fma(wl[2], wl[2], wl[3] * wl[3])), wl[4]);
  const double er = fma(dscale(rr, -1), fma(ur, ur, fma(wr[2], wr[2], wr[3] * wr[3])), wr[4]);
  const double isl = rsqrt64(rl), isr = rsqrt64(rr);  // 1 / sqrt(rho)
  const double sl = rl * isl, sr = rr * isr;          // sqrt(rho)
  const double iw = rcp64(sl + sr);
  const double ub = fma(sl, ul, sr * ur) * iw;
  const double vb = fma(sl, wl[2], sr * wr[2]) * iw;
  const double wb = fma(sl, wl[3], sr * wr[3]) * iw;
  const double hb = fma(el + pl, isl, (er + pr) * isr) * iw;  // Roe-averaged (E + p)/rho
  const double cb2 = gm1 * fma(-0.5, fma(ub, ub, fma(vb, vb, wb * wb)), hb);
  double sL = ul - cl, sR = ur + cr, bm, bp;
  if constexpr (NANCHK) {
    const double cb = cb2 > 0.0 ? sqrt64(cb2) : 0.0;
    if (ub - cb < sL) sL = ub - cb;
    if (ub + cb > sR) sR = ub + cb;
    bm = sL < 0.0 ? sL : 0.0;
    bp = sR > 0.0 ? sR : 0.0;
  } else {
    const double cb = dpos(cb2) ? sqrt64(cb2) : 0.0;
    const double ea = ub - cb, eb = ub + cb;
    sL = dgt(sL, ea) ? ea : sL;
    sR = dgt(eb, sR) ? eb : sR;
    bm = dnonneg(sL) ? 0.0 : sL;
    bp = dpos(sR) ? sR : 0.0;
  }
  const double ib = rcp64(bp - bm);
  const double bpm = bp * bm;
  const double ml = rl * ul, mr = rr * ur;
  f[0] = fma(bp, ml, fma(-bm, mr, bpm * (rr - rl))) * ib;
  f[1] = fma(bp, fma(ml, ul, pl), fma(-bm, fma(mr, ur, pr), bpm * (mr - ml))) * ib;
  f[2] = fma(bp, ml * wl[2], fma(-bm, mr * wr[2], bpm * fma(rr, wr[2], -(rl * wl[2])))) * ib;
  f[3] = fma(bp, ml * wl[3], fma(-bm, mr * wr[3], bpm * fma(rr, wr[3], -(rl * wl[3])))) * ib;
  f[4] = fma(bp, (el + pl) * ul, fma(-bm, (er + pr) * ur, bpm * (er - el))) * ib;
}

// ------------------------------------------------------------------------------
// Mixed form, FP32 on deviations, written once over the lane-generic operations of
// lanes.cuh: V = float solves one problem, V = float2 two at once with the same bits.
// ------------------------------------------------------------------------------
// PLM, van Leer: face values q0 -+ dl dr / (dl + dr) (zero slope at extrema); the
// reciprocal is the hardware seed refined once in FP32
template <typename V>
__device__ __forceinline__ void plm_edges_v(V qm, V q0, V qp, V& lo, V& hi) {
  const V zero = vset<V>(0.0f);
  const V dl = vsub(q0, qm);
  const V dr = vsub(qp, q0);
  const V prod = vmul(dl, dr);
  const V s = vadd(dl, dr);
  V r = vrcp(s);
  r = vfma(r, vfma(vneg(s), r, vset<V>(1.0f)), r);
  const V h = vsel(vgt(prod, zero), vmul(prod, r), zero);
  lo = vsub(q0, h);
  hi = vadd(q0, h);
}

// FP64 PLM face values from the one-sided differences dl = q0 - qm, dr = qp - q0:
// q0 -+ dl dr / (dl + dr), each a single fused multiply-add of dl dr and the
// Newton-refined reciprocal (zero slope where dl dr <= 0).
__device__ __forceinline__ void plm_edges_fp64(double dl, double dr, double q0, double& lo,
                                               double& hi) {
  const double prod = dl * dr;
  const bool pos = dpos(prod);
  const double p = pos ? prod : 0.0;
  const double r = pos ? rcp64(dl + dr) : 0.0;
  lo = fma(-p, r, q0);
  hi = fma(p, r, q0);
}

// CW84 limited slope: centred difference bounded by twice the one-sided ones, zero at an
// extremum.  min(|d|, 2|dl|, 2|dr|) with the sign of d: where d = 0 the one-sided
// differences have opposite signs (or one is zero), so the sign of a zero never reaches
// the result.
template <typename V>
__device__ __forceinline__ V ppm_slope_v(V qm, V q0, V qp) {
  const V zero = vset<V>(0.0f), two = vset<V>(2.0f);
  const V dl = vsub(q0, qm);
  const V dr = vsub(qp, q0);
  const V d = vmul(vset<V>(0.5f), vsub(qp, qm));
  const V m = vmin(vmin(vabs(d), vmul(two, vabs(dl))), vmul(two, vabs(dr)));
  return vsel(vgt(vmul(dl, dr), zero), vcopysign(m, d), zero);
}

// CW84 fourth-order interface value between cells of values ql, qr and limited slopes
// sl, sr
template <typename V>
__device__ __forceinline__ V ppm_interface_v(V ql, V qr, V sl, V sr) {
  return vfma(vsub(sl, sr), vset<V>(1.0f / 6.0f), vmul(vset<V>(0.5f), vadd(ql, qr)));
}

// CW84 monotonization of a cell's interface values a_lo, a_hi around its value a, in the
// comparison form of ppm_monotonize_fp64: where a lies between them, a_lo is moved to
// u = a - 2 (a_hi - a) and a_hi to w = a + 2 (a - a_lo) where they lie beyond those
// values, as seen from a (the larger or smaller of the two, by the direction of the rise)
template <typename V>
__device__ __forceinline__ void ppm_monotonize_v(V a_lo, V a_hi, V a, V& lo, V& hi) {
  const V zero = vset<V>(0.0f);
  const V dh = vsub(a_hi, a), dlo = vsub(a, a_lo);
  const auto flat = vnot(vgt(vmul(dh, dlo), zero));
  const V u = vfma(vset<V>(-2.0f), dh, a), w = vfma(vset<V>(2.0f), dlo, a);
  const auto rise = vgt(dh, zero);
  const V n_lo = vsel(rise, vmax(a_lo, u), vmin(a_lo, u));
  const V n_hi = vsel(rise, vmin(a_hi, w), vmax(a_hi, w));
  lo = vsel(flat, a, n_lo);
  hi = vsel(flat, a, n_hi);
}

// CW84 interface values of the middle cell of q0..q4 and their monotonization
template <typename V>
__device__ __forceinline__ void ppm_edges_v(V q0, V q1, V q2, V q3, V q4, V& lo, V& hi) {
  const V sm = ppm_slope_v(q0, q1, q2);
  const V sc = ppm_slope_v(q1, q2, q3);
  const V sp = ppm_slope_v(q2, q3, q4);
  ppm_monotonize_v(ppm_interface_v(q1, q2, sm, sc), ppm_interface_v(q2, q3, sc, sp), q2, lo, hi);
}

// HLLC, mixed form.  w = (rho - rho_b, u_n, u_t1, u_t2, u_g - u_g,b) in FP32.  Returns
// F - (0, p_b, 0, 0, 0).  Every difference of two O(1) quantities is formed from the
// deviations, so that a perturbation of relative size 1e-6 keeps ~7 digits.  Without
// branches: the star state of the upwind side K is always formed, and its jump term is
// switched off (S_K -> 0) when the fan is supersonic, which leaves the physical flux F_K.
template <typename V>
__device__ __forceinline__ void hllc_mixed(const V* wl, const V* wr, const Bg& bg, V* f) {
  const V zero = vset<V>(0.0f), one = vset<V>(1.0f), half = vset<V>(0.5f);
  const V g = vset<V>(bg.gamma_f), gm1 = vset<V>(bg.gm1_f), gg = vset<V>(bg.gg_f);
  const V pb = vset<V>(bg.pb_f);
  V rl = vadd(vset<V>(bg.rho_f), wl[0]), rr = vadd(vset<V>(bg.rho_f), wr[0]);
  const V ul = wl[1], ur = wr[1];
  const V dpl = vmul(gm1, wl[4]), dpr = vmul(gm1, wr[4]);  // p - p_b
  const V pl = vadd(pb, dpl), pr = vadd(pb, dpr);          // full pressures
  const V kel = vmul(vmul(half, rl), vfma(ul, ul, vfma(wl[2], wl[2], vmul(wl[3], wl[3]))));
  const V ker = vmul(vmul(half, rr), vfma(ur, ur, vfma(wr[2], wr[2], vmul(wr[3], wr[3]))));
  const V hl = vfma(gg, pl, kel);                          // E + p
  const V hr = vfma(gg, pr, ker);
  const V gpl = vmul(g, pl), gpr = vmul(g, pr);
  const V cl = vmul(vabs(gpl), vrsqrt(vmul(gpl, rl)));           // sqrt(gamma p / rho)
  const V cr = vmul(vabs(gpr), vrsqrt(vmul(gpr, rr)));

  // PVRS estimate as a deviation from p_b; p* = max(0, p_b + dps)
  // (p_b + dps > 0 exactly when dps > -p_b: a sum of two floats keeps the sign of its
  // exact value)
  V dps = vfma(vmul(vmul(vset<V>(-0.125f), vsub(ur, ul)), vadd(rl, rr)), vadd(cl, cr),
               vmul(half, vadd(dpl, dpr)));
  dps = vmax(dps, vneg(pb));
  const V kq = vset<V>(bg.kq_f);
  const V al = vfma(vmul(kq, vsub(dps, dpl)), vrcp(pl), one);
  const V ar = vfma(vmul(kq, vsub(dps, dpr)), vrcp(pr), one);
  const V ql = vsel(vgt(dps, dpl), vmul(al, vrsqrt(al)), one);
  const V qr = vsel(vgt(dps, dpr), vmul(ar, vrsqrt(ar)), one);
  V sl = vfma(vneg(cl), ql, ul);
  V sr = vfma(cr, qr, ur);
  sl = vmin(sl, vsub(ur, cr));                             // Davis bounds
  sr = vmax(sr, vadd(ul, cl));

  const auto sup_l = vge(sl, zero);                        // S_L >= 0
  const auto sup_r = vge(zero, sr);                        // S_R <= 0
  const V ml = vmul(rl, vsub(sl, ul));
  const V mr = vmul(rr, vsub(sr, ur));
  const V sstar = vmul(vfma(ul, ml, vfma(vneg(ur), mr, vsub(dpr, dpl))), vrcp(vsub(ml, mr)));
  const auto left = vor(sup_l, vand(vnot(sup_r), vge(sstar, zero)));
  const auto sub = vnot(vor(sup_l, sup_r));
  const V rk = vsel(left, rl, rr), uk = vsel(left, ul, ur);
  const V w2 = vsel(left, wl[2], wr[2]), w3 = vsel(left, wl[3], wr[3]);
  const V dpk = vsel(left, dpl, dpr), pk = vsel(left, pl, pr), hk = vsel(left, hl, hr);
  const V mk = vsel(left, ml, mr);                         // rho_K (S_K - u_K)
  const V s = vsel(left, sl, sr);
  const V ek = vadd(vsel(left, kel, ker), vadd(vset<V>(bg.ug_f), vsel(left, wl[4], wr[4])));
  const V mn = vmul(rk, uk);
  const V inv = vrcp(vsub(s, sstar));
  const V fac = vmul(mk, inv);
  const V su = vsub(sstar, uk);
  // U*_rho - rho_K, U*_Mn - M_n, and E*_K - E_K = (S* - u_K) ((E_K + p_K)/(S_K - S*) + rho*_K S*)
  const V drho = vsel(sub, vmul(vmul(rk, su), inv), zero);
  const V dmn = vsel(sub, vfma(fac, sstar, vneg(mn)), zero);
  const V de = vsel(sub, vmul(su, vfma(fac, sstar, vmul(vadd(ek, pk), inv))), zero);
  const V se = vsel(sub, s, zero);
  const V mt = vfma(se, drho, mn);                         // M_n + S_K (U*_rho - rho_K)
  f[0] = mt;
  f[1] = vfma(se, dmn, vfma(mn, uk, dpk));
  f[2] = vmul(mt, w2);
  f[3] = vmul(mt, w3);
  f[4] = vfma(se, de, vmul(hk, uk));
}

__device__ __forceinline__ float sqrt_fast(float x) { return x * rsqrt_approx_f32(x); }

// State jumps U_R - U_L of the mixed form from the deviations, each written so that no
// O(1) quantities are subtracted: M_R - M_L = rho_R (v_R - v_L) + (rho_R - rho_L) v_L and
// E_R - E_L = (k_R - k_L) + (u_g,R - u_g,L), k_R - k_L = (rho_R (|v_R|^2 - |v_L|^2) +
// (rho_R - rho_L) |v_L|^2) / 2.
template <typename V>
__device__ __forceinline__ void jumps_mixed(const V* wl, const V* wr, V rr, V* d) {
  d[0] = vsub(wr[0], wl[0]);
  V dv2 = vset<V>(0.0f), vl2 = vset<V>(0.0f);
#pragma unroll
  for (int a = 1; a < 4; ++a) {
    const V dv = vsub(wr[a], wl[a]);
    d[a] = vfma(rr, dv, vmul(d[0], wl[a]));
    dv2 = vfma(dv, vadd(wr[a], wl[a]), dv2);
    vl2 = vfma(wl[a], wl[a], vl2);
  }
  d[4] = vadd(vmul(vset<V>(0.5f), vfma(rr, dv2, vmul(d[0], vl2))), vsub(wr[4], wl[4]));
}

// Physical fluxes of one face state in the mixed form (background pressure left out of
// the normal momentum flux): (m, m u + dp, m v, m w, h u) with m = rho u, h = E + p.
template <typename V>
__device__ __forceinline__ void pflux_mixed(const V* w, V rho, V dp, V h, V* f) {
  const V m = vmul(rho, w[1]);
  f[0] = m;
  f[1] = vfma(m, w[1], dp);
  f[2] = vmul(m, w[2]);
  f[3] = vmul(m, w[3]);
  f[4] = vmul(h, w[1]);
}

// LLF, mixed form.  Returns F - (0, p_b, 0, 0, 0).
template <typename V>
__device__ __forceinline__ void llf_mixed(const V* wl, const V* wr, const Bg& bg, V* f) {
  const V half = vset<V>(0.5f);
  const V g = vset<V>(bg.gamma_f), gm1 = vset<V>(bg.gm1_f), gg = vset<V>(bg.gg_f);
  const V pb = vset<V>(bg.pb_f);
  V rl = vadd(vset<V>(bg.rho_f), wl[0]), rr = vadd(vset<V>(bg.rho_f), wr[0]);
  const V dpl = vmul(gm1, wl[4]), dpr = vmul(gm1, wr[4]);
  const V pl = vadd(pb, dpl), pr = vadd(pb, dpr);
  const V kel = vmul(vmul(half, rl), vfma(wl[1], wl[1], vfma(wl[2], wl[2], vmul(wl[3], wl[3]))));
  const V ker = vmul(vmul(half, rr), vfma(wr[1], wr[1], vfma(wr[2], wr[2], vmul(wr[3], wr[3]))));
  const V gpl = vmul(g, pl), gpr = vmul(g, pr);
  const V cl = vmul(vabs(gpl), vrsqrt(vmul(gpl, rl)));
  const V cr = vmul(vabs(gpr), vrsqrt(vmul(gpr, rr)));
  const V al = vadd(vabs(wl[1]), cl), ar = vadd(vabs(wr[1]), cr);
  const V sm = vneg(vsel(vgt(al, ar), al, ar));
  V fl[5], fr[5], d[5];
  pflux_mixed(wl, rl, dpl, vfma(gg, pl, kel), fl);
  pflux_mixed(wr, rr, dpr, vfma(gg, pr, ker), fr);
  jumps_mixed(wl, wr, rr, d);
#pragma unroll
  for (int n = 0; n < 5; ++n) f[n] = vmul(half, vfma(sm, d[n], vadd(fl[n], fr[n])));
}

// HLLE, mixed form (Roe averages and wave speeds in FP32).  Returns F - (0, p_b, 0, 0, 0).
template <typename V>
__device__ __forceinline__ void hlle_mixed(const V* wl, const V* wr, const Bg& bg, V* f) {
  const V zero = vset<V>(0.0f), half = vset<V>(0.5f);
  const V g = vset<V>(bg.gamma_f), gm1 = vset<V>(bg.gm1_f), gg = vset<V>(bg.gg_f);
  const V pb = vset<V>(bg.pb_f);
  V rl = vadd(vset<V>(bg.rho_f), wl[0]), rr = vadd(vset<V>(bg.rho_f), wr[0]);
  const V ul = wl[1], ur = wr[1];
  const V dpl = vmul(gm1, wl[4]), dpr = vmul(gm1, wr[4]);
  const V pl = vadd(pb, dpl), pr = vadd(pb, dpr);
  const V kel = vmul(vmul(half, rl), vfma(ul, ul, vfma(wl[2], wl[2], vmul(wl[3], wl[3]))));
  const V ker = vmul(vmul(half, rr), vfma(ur, ur, vfma(wr[2], wr[2], vmul(wr[3], wr[3]))));
  const V hl = vfma(gg, pl, kel), hr = vfma(gg, pr, ker);  // E + p
  const V gpl = vmul(g, pl), gpr = vmul(g, pr);
  const V cl = vmul(vabs(gpl), vrsqrt(vmul(gpl, rl)));
  const V cr = vmul(vabs(gpr), vrsqrt(vmul(gpr, rr)));
  const V isl = vrsqrt(rl), isr = vrsqrt(rr);              // 1 / sqrt(rho)
  const V iw = vrcp(vadd(vmul(rl, isl), vmul(rr, isr)));   // 1 / (sqrt(rho_L) + sqrt(rho_R))
  const V sl = vmul(rl, isl), sr = vmul(rr, isr);
  const V ub = vmul(vfma(sl, ul, vmul(sr, ur)), iw);
  const V vb = vmul(vfma(sl, wl[2], vmul(sr, wr[2])), iw);
  const V wb = vmul(vfma(sl, wl[3], vmul(sr, wr[3])), iw);
  const V hb = vmul(vfma(hl, isl, vmul(hr, isr)), iw);
  const V cb2 = vmul(gm1, vfma(vset<V>(-0.5f), vfma(ub, ub, vfma(vb, vb, vmul(wb, wb))), hb));
  const V cb = vsel(vgt(cb2, zero), vmul(cb2, vrsqrt(cb2)), zero);
  V sL = vsub(ul, cl), sR = vadd(ur, cr);
  const V ea = vsub(ub, cb), eb = vadd(ub, cb);
  sL = vsel(vgt(sL, ea), ea, sL);
  sR = vsel(vgt(eb, sR), eb, sR);
  const V bm = vsel(vge(sL, zero), zero, sL);
  const V bp = vsel(vgt(sR, zero), sR, zero);
  const V ib = vrcp(vsub(bp, bm));
  const V bpm = vmul(bp, bm);
  V fl[5], fr[5], d[5];
  pflux_mixed(wl, rl, dpl, hl, fl);
  pflux_mixed(wr, rr, dpr, hr, fr);
  jumps_mixed(wl, wr, rr, d);
#pragma unroll
  for (int n = 0; n < 5; ++n)
    f[n] = vmul(vfma(bp, fl[n], vfma(vneg(bm), fr[n], vmul(bpm, d[n]))), ib);
}

}  // namespace ak
