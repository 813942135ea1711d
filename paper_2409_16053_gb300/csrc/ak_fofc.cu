// First-order flux correction (FOFC, Section 3): after a stage, a cell whose density or
// internal energy would not be positive gets, on all its faces, the LLF flux of the
// piecewise-constant states of the two cells instead of the reconstructed flux.
//
// The stage kernels flag such cells (fofc_flag) while they write the stage's output.
// This kernel then corrects that output: every cell with a flagged cell among itself
// and its six face neighbours changes by b dt (the stage's weight of dt L) times the
// change of L(U) from its corrected faces, dL = sum_faces -+ (F_LLF - F_high) / dx_d.
// F_high is recomputed from the stage's input with the stage kernels' own device code,
// so it equals the flux the stage used.  Each affected cell is corrected by exactly
// one thread -- the one holding the lowest-numbered flagged cell next to it -- so the
// result does not depend on thread order.  One CTA runs it; flagged cells are rare.
// Uniform meshes only (faces of one level, no level flux correction).
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

// face neighbour of interior cell c = (block, i, j, k) across direction d, dir = -1 / +1
// (periodic; the level's leaf map gives the neighbour block)
__device__ __forceinline__ int4 neighbour(const ak_meshdev& md, int4 c, int d, int dir) {
  const ak_block& B = md.blocks[c.x];
  const ak_level& L = md.levels[B.level];
  int q[3] = {B.lx1 + c.y, B.lx2 + c.z, B.lx3 + c.w};
  const int n[3] = {L.n1, L.n2, L.n3}, bs[3] = {L.bs1, L.bs2, L.bs3};
  q[d] += dir;
  q[d] = q[d] < 0 ? q[d] + n[d] : (q[d] >= n[d] ? q[d] - n[d] : q[d]);
  const int b0 = q[0] / bs[0], b1 = q[1] / bs[1], b2 = q[2] / bs[2];
  const int blk = md.map[L.map_off + (b2 * L.md2 + b1) * L.md1 + b0];
  return make_int4(blk, q[0] - b0 * bs[0], q[1] - b1 * bs[1], q[2] - b2 * bs[2]);
}

__device__ __forceinline__ bool flagged(const ak_meshdev& md, int4 c) {
  return md.fflag[cell_id(md, c)] != 0;
}

// Flux change F_LLF - F_high through the face of cell c on side `side` (0: lower,
// 1: upper) of direction d, from the stage input (ghost cells filled).
template <int NG, bool MIXED>
__device__ void face_change(const double* uin, const ak_meshdev& md, const Bg& bg,
                            const Counters& cn, int4 c, int d, int side, double* df) {
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
    c2p(u, W[m], bg, cn);
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
    edges<NG>(qa, lo_a[v], hi_a[v], bg.wenoz);
    edges<NG>(qb, lo_b[v], hi_b[v], bg.wenoz);
  }
  R fh[5], fl[5];
  solve(d, hi_a, lo_b, bg, fh);
  Bg bl = bg;
  bl.rsolver = AK_LLF;
  solve(d, W[NG - 1], W[NG], bl, fl);
#pragma unroll
  for (int v = 0; v < 5; ++v) df[v] = (double)fl[v] - (double)fh[v];
}

template <int NG, bool MIXED>
__global__ void __launch_bounds__(kFofcThreads)
    fofc_kernel(const double* __restrict__ uin, double* uout, ak_meshdev md, Bg bg,
                ak_dev_scalars* sc, double b, int last_stage) {
  const unsigned nflag = sc->fofc_n;
  const unsigned n = nflag < (unsigned)md.fcap ? nflag : (unsigned)md.fcap;
  const double dt = sc->dt;
  // the stage already counted any floor of these cells: recounts go to a sink
  const Counters cn{&sc->sink[0], &sc->sink[1]};
  double dtmin = __longlong_as_double(0x7ff0000000000000ll);
  for (unsigned idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int4 f = md.flist[idx];
    const long long gf = cell_id(md, f);
    for (int c7 = 0; c7 < 7; ++c7) {
      const int4 c = c7 == 0 ? f : neighbour(md, f, (c7 - 1) >> 1, (c7 & 1) ? -1 : 1);
      // owner of c: the lowest-numbered flagged cell among c and its neighbours
      long long owner = flagged(md, c) ? cell_id(md, c) : 0x7fffffffffffffffll;
      bool nb_flag[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const int4 nq = neighbour(md, c, q >> 1, (q & 1) ? 1 : -1);
        nb_flag[q] = flagged(md, nq);
        const long long gq = cell_id(md, nq);
        if (nb_flag[q] && gq < owner) owner = gq;
      }
      if (owner != gf) continue;
      const bool cf = flagged(md, c);
      const ak_block& B = md.blocks[c.x];
      const double idx_d[3] = {1.0 / B.dx1, 1.0 / B.dx2, 1.0 / B.dx3};
      double dl[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      for (int q = 0; q < 6; ++q) {  // face q: direction q/2, lower (q even) or upper
        if (!cf && !nb_flag[q]) continue;
        const int d = q >> 1, side = q & 1;
        double df[5];
        face_change<NG, MIXED>(uin, md, bg, cn, c, d, side, df);
        // L = -(F_upper - F_lower) / dx: a lower face adds, an upper face subtracts
#pragma unroll
        for (int v = 0; v < 5; ++v) dl[v] += (side ? -df[v] : df[v]) * idx_d[d];
      }
      const long long e = B.off + ((long long)(c.w + NG) * B.p2 + (c.z + NG)) * B.s1 + c.y + NG;
      double un[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        un[v] = fma(b * dt, dl[v], uout[e + v * B.var_stride]);
        uout[e + v * B.var_stride] = un[v];
      }
      if (last_stage) {  // CFL ratio of the corrected cell (Eq. (3))
        const double rho = un[0] > AK_RHO_FLOOR ? un[0] : AK_RHO_FLOOR;
        double ug = un[4] - 0.5 * (un[1] * un[1] + un[2] * un[2] + un[3] * un[3]) / rho;
        ug = ug > AK_UG_FLOOR ? ug : AK_UG_FLOOR;
        const double cs = sqrt(bg.gamma * bg.gm1 * ug / rho);
        double t = B.dx1 / (fabs(un[1] / rho) + cs);
        t = fmin(t, B.dx2 / (fabs(un[2] / rho) + cs));
        t = fmin(t, B.dx3 / (fabs(un[3] / rho) + cs));
        dtmin = fmin(dtmin, t);
      }
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
  static const double b2[2] = {1.0, 0.5};
  static const double b3[3] = {1.0, 0.25, 2.0 / 3.0};
  const double b = m->desc.rk == 3 ? b3[stage - 1] : b2[stage - 1];
  const Bg bg = stage_bg(m);
  const bool mixed = m->desc.precision == AK_MIXED;
  if (m->desc.recon == AK_PLM) {
    if (mixed)
      fofc_kernel<2, true><<<1, kFofcThreads, 0, m->stream>>>(u_in, u_out, m->md, bg, m->d_sc, b, last_stage);
    else
      fofc_kernel<2, false><<<1, kFofcThreads, 0, m->stream>>>(u_in, u_out, m->md, bg, m->d_sc, b, last_stage);
  } else {
    if (mixed)
      fofc_kernel<3, true><<<1, kFofcThreads, 0, m->stream>>>(u_in, u_out, m->md, bg, m->d_sc, b, last_stage);
    else
      fofc_kernel<3, false><<<1, kFofcThreads, 0, m->stream>>>(u_in, u_out, m->md, bg, m->d_sc, b, last_stage);
  }
  return cudaGetLastError();
}
