// First-order flux correction (FOFC, Section 3): after a stage, a cell whose density or
// internal energy would not be positive gets, on all its faces, the LLF flux of the
// piecewise-constant states of the two cells instead of the reconstructed flux.
//
// The stage kernels flag such cells (fofc_flag) while they write the stage's output; a
// cell whose tentative state is not a number (a high-order flux through a face with a
// negative reconstructed pressure) is flagged too, and the stage kernel saves its U0.
// This kernel then
//   (a) redoes each flagged cell's update from the stage input, its saved U0 and L of
//       the LLF fluxes of its six faces, in the stage kernels' order of operations;
//   (b) corrects each unflagged cell next to a flagged one by b dt (the stage's weight
//       of dt L) times the change of L from its faces next to flagged cells,
//       dL = sum_faces -+ (F_LLF - F_high) / dx_d; F_high is recomputed from the stage
//       input with the stage kernels' own device code, so it equals the flux the stage
//       used (and is a number: a cell next to a face without one is flagged itself).
// Each cell is written by exactly one thread -- a flagged cell by its own list entry, an
// unflagged one by the entry of the lowest-numbered flagged cell next to it -- so the
// result does not depend on thread order.  One CTA runs it; flagged cells are rare.
//
// Refined meshes (the paper applies FOFC before the level flux correction): a face
// between a fine cell and a coarser leaf is the fine block's face, computed from the
// fine block's data (its ghost cell there is the prolongated coarse value); it turns
// first-order when the fine cell or the coarse cell is flagged.  The coarse side of
// that face carries the mean of its four fine faces' fluxes, as the flux correction
// gives it.
#include "ak_internal.cuh"
#include "hydro_ops.cuh"
#include "stage_common.cuh"

namespace ak {

namespace {

constexpr int kFofcThreads = 256;

__device__ __forceinline__ long long cell_id(const ak_meshdev& md, int4 c) {
  const ak_block& B = md.blocks[c.x];
  return md.cell_off[c.x] + ((long long)c.w * B.nx2 + c.z) * B.nx1 + c.y;
}

// leaf of level l holding the level-l cell (q0, q1, q2) (periodic), or -1
__device__ __forceinline__ int leaf_at(const ak_meshdev& md, int l, int q0, int q1, int q2) {
  if (l < 0 || l >= md.nlev) return -1;
  const ak_level& L = md.levels[l];
  if (L.bs1 == 0) return -1;
  q0 = q0 < 0 ? q0 + L.n1 : (q0 >= L.n1 ? q0 - L.n1 : q0);
  q1 = q1 < 0 ? q1 + L.n2 : (q1 >= L.n2 ? q1 - L.n2 : q1);
  q2 = q2 < 0 ? q2 + L.n3 : (q2 >= L.n3 ? q2 - L.n3 : q2);
  return md.map[L.map_off + ((q2 / L.bs3) * L.md2 + q1 / L.bs2) * L.md1 + q0 / L.bs1];
}

// interior cell of leaf `blk` at the level-l cell q (periodic)
__device__ __forceinline__ int4 local_cell(const ak_meshdev& md, int blk, int q0, int q1, int q2) {
  const ak_block& B = md.blocks[blk];
  const ak_level& L = md.levels[B.level];
  int r0 = q0 - B.lx1, r1 = q1 - B.lx2, r2 = q2 - B.lx3;
  r0 = r0 < 0 ? r0 + L.n1 : (r0 >= L.n1 ? r0 - L.n1 : r0);
  r1 = r1 < 0 ? r1 + L.n2 : (r1 >= L.n2 ? r1 - L.n2 : r1);
  r2 = r2 < 0 ? r2 + L.n3 : (r2 >= L.n3 ? r2 - L.n3 : r2);
  return make_int4(blk, r0, r1, r2);
}

// The cells across one face of interior cell c (direction d, dir = -1 / +1): one cell of
// the same level (kind 0) or of the coarser level (kind 1), or the four cells of the
// finer level that share the face (kind 2).
struct Across {
  int kind, n;
  int4 c[4];
};
__device__ __noinline__ Across across(const ak_meshdev& md, int4 c, int d, int dir) {
  const ak_block& B = md.blocks[c.x];
  const int l = B.level;
  const ak_level& L = md.levels[l];
  const int n[3] = {L.n1, L.n2, L.n3};
  int q[3] = {B.lx1 + c.y, B.lx2 + c.z, B.lx3 + c.w};
  q[d] += dir;
  q[d] = q[d] < 0 ? q[d] + n[d] : (q[d] >= n[d] ? q[d] - n[d] : q[d]);
  Across a;
  int b = leaf_at(md, l, q[0], q[1], q[2]);
  if (b >= 0) {
    a.kind = 0;
    a.n = 1;
    a.c[0] = local_cell(md, b, q[0], q[1], q[2]);
    return a;
  }
  b = leaf_at(md, l - 1, q[0] >> 1, q[1] >> 1, q[2] >> 1);
  if (b >= 0) {
    a.kind = 1;
    a.n = 1;
    a.c[0] = local_cell(md, b, q[0] >> 1, q[1] >> 1, q[2] >> 1);
    return a;
  }
  a.kind = 2;
  a.n = 0;
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  for (int u = 0; u < 4; ++u) {
    int Q[3];
    Q[d] = 2 * q[d] + (dir > 0 ? 0 : 1);  // the fine layer next to the face
    Q[t1] = 2 * q[t1] + (u & 1);
    Q[t2] = 2 * q[t2] + (u >> 1);
    const int f = leaf_at(md, l + 1, Q[0], Q[1], Q[2]);
    if (f >= 0) a.c[a.n++] = local_cell(md, f, Q[0], Q[1], Q[2]);
  }
  return a;
}

__device__ __forceinline__ bool flagged(const ak_meshdev& md, int4 c) {
  return md.fflag[cell_id(md, c)] != 0;
}

// Flux through the face of cell c on side `side` (0: lower, 1: upper) of direction d,
// from the stage input (ghost cells filled): the LLF flux of the two cells' own states
// (first order) or the reconstructed flux, in the stage kernels' precision.
template <int NG, bool MIXED>
__device__ void face_flux(const double* uin, const ak_meshdev& md, const Bg& bg,
                          const Counters& cn, int4 c, int d, int side, bool first_order,
                          typename std::conditional<MIXED, float, double>::type* f) {
  using R = typename std::conditional<MIXED, float, double>::type;
  const ak_block& B = md.blocks[c.x];
  int p[3] = {c.y + NG, c.z + NG, c.w + NG};  // padded indices of c
  const long long st[3] = {1, B.s1, (long long)B.s1 * B.p2};
  // padded position along d of the face's left cell
  const int pl = p[d] - 1 + side;
  p[d] = 0;
  const double* base = uin + B.off + ((long long)p[2] * B.p2 + p[1]) * B.s1 + p[0];
  R W[2 * NG][5];  // cells pl-NG+1 .. pl+NG along d
#pragma unroll
  for (int m = 0; m < 2 * NG; ++m) {
    const double* e = base + (long long)(pl - NG + 1 + m) * st[d];
    double u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = e[v * B.var_stride];
    if (bg.recon == AK_WENOZ || bg.recon == AK_PPMX)
      c2p_t<true>(u, W[m], bg, cn);
    else
      c2p_t<false>(u, W[m], bg, cn);
  }
  if (first_order) {
    Bg bl = bg;
    bl.rsolver = AK_LLF;
    solve(d, W[NG - 1], W[NG], bl, f);
    return;
  }
  R lo_a[5], hi_a[5], lo_b[5], hi_b[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    R qa[2 * NG - 1], qb[2 * NG - 1];
#pragma unroll
    for (int m = 0; m < 2 * NG - 1; ++m) {
      qa[m] = W[m][v];
      qb[m] = W[m + 1][v];
    }
    edges<NG>(qa, lo_a[v], hi_a[v], bg.recon);
    edges<NG>(qb, lo_b[v], hi_b[v], bg.recon);
  }
  if (bg.recon == AK_WENOZ || bg.recon == AK_PPMX)
    solve<true>(d, hi_a, lo_b, bg, f);
  else
    solve<false>(d, hi_a, lo_b, bg, f);
}

// F_LLF - F_high through that face, in FP64
template <int NG, bool MIXED>
__device__ void face_change(const double* uin, const ak_meshdev& md, const Bg& bg,
                            const Counters& cn, int4 c, int d, int side, double* df) {
  using R = typename std::conditional<MIXED, float, double>::type;
  R fl[5], fh[5];
  face_flux<NG, MIXED>(uin, md, bg, cn, c, d, side, true, fl);
  face_flux<NG, MIXED>(uin, md, bg, cn, c, d, side, false, fh);
#pragma unroll
  for (int v = 0; v < 5; ++v) df[v] = (double)fl[v] - (double)fh[v];
}

// CFL ratio dx / (|v| + c_s), min over directions, of a corrected state (Eq. (3))
__device__ __forceinline__ double cfl_ratio(const double* un, const ak_block& B, const Bg& bg) {
  const double rho = un[0] > AK_RHO_FLOOR ? un[0] : AK_RHO_FLOOR;
  double ug = un[4] - 0.5 * (un[1] * un[1] + un[2] * un[2] + un[3] * un[3]) / rho;
  ug = ug > AK_UG_FLOOR ? ug : AK_UG_FLOOR;
  const double cs = sqrt(bg.gamma * bg.gm1 * ug / rho);
  double t = B.dx1 / (fabs(un[1] / rho) + cs);
  t = fmin(t, B.dx2 / (fabs(un[2] / rho) + cs));
  return fmin(t, B.dx3 / (fabs(un[3] / rho) + cs));
}

template <int NG, bool MIXED>
__global__ void __launch_bounds__(kFofcThreads)
    fofc_kernel(const double* __restrict__ uin, const double* __restrict__ u0, double* uout,
                ak_meshdev md, Bg bg, ak_dev_scalars* sc, double a, double b, int form,
                int last_stage) {
  using R = typename std::conditional<MIXED, float, double>::type;
  const unsigned nflag = sc->fofc_n;
  const unsigned n = nflag < (unsigned)md.fcap ? nflag : (unsigned)md.fcap;
  const double dt = sc->dt;
  // the stage already counted any floor of these cells: recounts go to a sink
  const Counters cn{&sc->sink[0], &sc->sink[1]};
  double dtmin = __longlong_as_double(0x7ff0000000000000ll);
  for (unsigned idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int4 f = md.flist[idx];
    const long long gf = cell_id(md, f);
    // (a) the flagged cell itself: every face first order; its stage update redone from
    //     the stage input, U0 as the stage kernel saved it, and L of the LLF fluxes, in
    //     the stage kernels' order of operations (its stored output may not be a number)
    {
      const ak_block& B = md.blocks[f.x];
      R fl[3][5], fu[3][5];  // fluxes through the lower and upper face in each direction
      for (int q = 0; q < 6; ++q) {
        const int d = q >> 1, side = q & 1;
        R* fq = side ? fu[d] : fl[d];
        const Across a = across(md, f, d, side ? 1 : -1);
        if (a.kind != 2) {
          face_flux<NG, MIXED>(uin, md, bg, cn, f, d, side, true, fq);
        } else {  // coarse side of a level boundary: the mean of the four fine faces
          R sum[5] = {R(0), R(0), R(0), R(0), R(0)};
          for (int u = 0; u < a.n; ++u) {
            R fj[5];
            face_flux<NG, MIXED>(uin, md, bg, cn, a.c[u], d, 1 - side, true, fj);
#pragma unroll
            for (int v = 0; v < 5; ++v) sum[v] += fj[v];
          }
#pragma unroll
          for (int v = 0; v < 5; ++v) fq[v] = R(0.25) * sum[v];
        }
      }
      const long long e = B.off + ((long long)(f.w + NG) * B.p2 + (f.z + NG)) * B.s1 + f.y + NG;
      const double idx1 = 1.0 / B.dx1, idx2 = 1.0 / B.dx2, idx3 = 1.0 / B.dx3;
      double un[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const R d1 = fu[0][v] - fl[0][v], d2 = fu[1][v] - fl[1][v], d3 = fu[2][v] - fl[2][v];
        const double ui = uin[e + v * B.var_stride];
        const double u0i = form != 0 ? md.fu0[(long long)idx * 5 + v] : 0.0;
        double r;
        if constexpr (MIXED) {
          const float L = -fmaf(d1, (float)idx1, fmaf(d2, (float)idx2, d3 * (float)idx3));
          r = rk_update_mixed(form, a, b, dt, L, ui, u0i);
        } else {
          const double cdt[3] = {dt * idx1, dt * idx2, dt * idx3};
          r = rk_update_fp64(form, a, b, cdt, d1, d2, d3, ui, u0i);
        }
        un[v] = r;
        uout[e + v * B.var_stride] = r;
      }
      if (last_stage) dtmin = fmin(dtmin, cfl_ratio(un, B, bg));
    }
    // (b) the unflagged cells across f's faces (each once): their stored output changes
    //     by b dt times the change of L from their faces next to flagged cells
    int4 cand[6 * 4];
    long long cid[6 * 4];
    int nc = 0;
    for (int q = 0; q < 6; ++q) {
      const Across a = across(md, f, q >> 1, (q & 1) ? 1 : -1);
      for (int u = 0; u < a.n; ++u) {
        if (flagged(md, a.c[u])) continue;
        const long long g = cell_id(md, a.c[u]);
        bool seen = false;
        for (int t = 0; t < nc; ++t) seen |= cid[t] == g;
        if (!seen) {
          cand[nc] = a.c[u];
          cid[nc++] = g;
        }
      }
    }
    for (int ci = 0; ci < nc; ++ci) {
      const int4 c = cand[ci];
      // owner of c: the lowest-numbered flagged cell across its faces
      long long owner = 0x7fffffffffffffffll;
      for (int q = 0; q < 6; ++q) {
        const Across a = across(md, c, q >> 1, (q & 1) ? 1 : -1);
        for (int u = 0; u < a.n; ++u)
          if (flagged(md, a.c[u])) {
            const long long g = cell_id(md, a.c[u]);
            owner = g < owner ? g : owner;
          }
      }
      if (owner != gf) continue;
      const ak_block& B = md.blocks[c.x];
      const double idx_d[3] = {1.0 / B.dx1, 1.0 / B.dx2, 1.0 / B.dx3};
      double dl[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      for (int q = 0; q < 6; ++q) {  // face q: direction q/2, lower (q even) or upper
        const int d = q >> 1, side = q & 1;
        const Across a = across(md, c, d, side ? 1 : -1);
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        bool any = false;
        if (a.kind != 2) {
          // a face of c's own block (same level, or fine side of a level boundary)
          if (flagged(md, a.c[0])) {
            face_change<NG, MIXED>(uin, md, bg, cn, c, d, side, acc);
            any = true;
          }
        } else {
          // coarse side of a level boundary: the mean of the four fine faces' changes
          for (int u = 0; u < a.n; ++u) {
            if (!flagged(md, a.c[u])) continue;
            double df[5];
            face_change<NG, MIXED>(uin, md, bg, cn, a.c[u], d, 1 - side, df);
#pragma unroll
            for (int v = 0; v < 5; ++v) acc[v] += df[v];
            any = true;
          }
#pragma unroll
          for (int v = 0; v < 5; ++v) acc[v] *= 0.25;
        }
        if (!any) continue;
        // L = -(F_upper - F_lower) / dx: a lower face adds, an upper face subtracts
#pragma unroll
        for (int v = 0; v < 5; ++v) dl[v] += (side ? -acc[v] : acc[v]) * idx_d[d];
      }
      const long long e = B.off + ((long long)(c.w + NG) * B.p2 + (c.z + NG)) * B.s1 + c.y + NG;
      double un[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        un[v] = fma(b * dt, dl[v], uout[e + v * B.var_stride]);
        uout[e + v * B.var_stride] = un[v];
      }
      if (last_stage) dtmin = fmin(dtmin, cfl_ratio(un, B, bg));
    }
  }
  if (last_stage && dtmin < __longlong_as_double(0x7ff0000000000000ll))
    atomicMin(&sc->dtmin_bits, (unsigned long long)__double_as_longlong(dtmin));
  __syncthreads();  // every flag is read before any is cleared
  for (unsigned idx = threadIdx.x; idx < n; idx += blockDim.x)
    md.fflag[cell_id(md, md.flist[idx])] = 0;
  if (threadIdx.x == 0) {
    sc->counters[3] += n;
    sc->fofc_n = 0;
  }
}

}  // namespace

}  // namespace ak

cudaError_t ak_launch_fofc(const ak_mesh* m, int stage, const double* u_in, double* u_out,
                           int last_stage) {
  using namespace ak;
  static const double a2[2] = {0.0, 0.5}, b2[2] = {1.0, 0.5};
  static const double a3[3] = {0.0, 0.75, 1.0 / 3.0}, b3[3] = {1.0, 0.25, 2.0 / 3.0};
  const bool rk3 = m->desc.rk == 3;
  const double a = rk3 ? a3[stage - 1] : a2[stage - 1];
  const double b = rk3 ? b3[stage - 1] : b2[stage - 1];
  // the stage kernels' forms: 0 = U + dt L, 1 = RK2 final (U0 + U + dt L) / 2, 2 = general
  const int form = (!rk3 && stage == 2) ? 1 : (a == 0.0 ? 0 : 2);
  const double* u0 = m->reg[0];
  const Bg bg = stage_bg(m);
  const bool mixed = m->desc.precision == AK_MIXED;
  if (m->desc.recon == AK_PLM) {
    if (mixed)
      fofc_kernel<2, true><<<1, kFofcThreads, 0, m->stream>>>(u_in, u0, u_out, m->md, bg, m->d_sc, a, b, form, last_stage);
    else
      fofc_kernel<2, false><<<1, kFofcThreads, 0, m->stream>>>(u_in, u0, u_out, m->md, bg, m->d_sc, a, b, form, last_stage);
  } else {
    if (mixed)
      fofc_kernel<3, true><<<1, kFofcThreads, 0, m->stream>>>(u_in, u0, u_out, m->md, bg, m->d_sc, a, b, form, last_stage);
    else
      fofc_kernel<3, false><<<1, kFofcThreads, 0, m->stream>>>(u_in, u0, u_out, m->md, bg, m->d_sc, a, b, form, last_stage);
  }
  return cudaGetLastError();
}
