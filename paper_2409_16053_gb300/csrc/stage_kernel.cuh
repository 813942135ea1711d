// The fused hydro stage kernel: primitive recovery, reconstruction in x1/x2/x3, HLLC
// at every face, flux divergence and the RK stage update of AthenaK's Godunov scheme
// (arXiv 2409.16053, Section 3 Eq. (1), Section 3.1 Eq. (4)), plus the CFL minimum of
// Section 3 Eq. (3) on the last stage.
//
// Work decomposition (one launch covers every MeshBlock, as Section 2's MeshBlockPack
// does): a CTA owns a TX x TY column tile of one block and marches along x3 over a
// segment of planes.  A ring of 2*NG planes of primitives (tile plus NG halo cells in
// x1 and x2) lives in shared memory; each plane is loaded from HBM and converted once.
// Per plane:
//   A. reconstruction: the x1 and x2 face values (lower and upper edge) of every cell
//      the tile's faces touch go to shared memory; each thread also reconstructs its
//      own column's next cell along x3 and keeps the upper edge in registers;
//   B. HLLC on every x1 and x2 face of the plane (fluxes to shared memory) and on the
//      x3 face above each column (flux in registers, carried to the next plane);
//   C. flux divergence and the RK update of the column's cell.
// Every cell is reconstructed once per direction and every face of a tile is solved
// once; faces on tile edges are solved by both tiles from identical inputs, so they
// agree bit for bit and the update stays conservative.
//
// The reconstruction is a template argument (RC: AK_PLM, AK_PPM4, AK_WENOZ or AK_PPMX),
// as the paper does for algorithmic options to spare registers; each reconstruction's
// kernels are instantiated in a translation unit of their own (ak_stage_<recon>.cu).
#pragma once

#include <type_traits>

#include "ak_internal.cuh"
#include "hydro_ops.cuh"
#include "stage_common.cuh"

namespace ak {

template <int NG, int RC, bool MIXED, int TX, int TY>
struct StageCfg {
  using R = typename std::conditional<MIXED, float, double>::type;
  // FP64 PPM4 carries its x3 slopes and interface values from cell to cell, so no plane
  // below the current one is read again: the ring holds the current plane, the three
  // above it and the one being replaced (5 slots instead of 2 NG).
  static constexpr bool CARRY = !MIXED && RC == AK_PPM4;
  // FP64 PLM: x1 and x2 sweeps one after the other through one edge buffer, so that two
  // CTAs fit in an SM's shared memory (FP64 PPM4 runs one CTA per SM and does both at
  // once).  Mixed: both sweeps at once, and the next plane of the state is prefetched
  // into registers while the current one is computed.
  static constexpr bool SPLIT = !MIXED && !CARRY;
  static constexpr bool PREFETCH = MIXED;
  static constexpr int WX = TX + 2 * NG, WY = TY + 2 * NG, NPL = WX * WY;
  static constexpr int NR = CARRY ? 5 : 2 * NG;
  // cells of a plane that are converted: the tile and its x1 / x2 halos (no corners)
  static constexpr int NCROSS = TX * TY + 2 * NG * (TX + TY);
  static constexpr int NT = TX * TY;
  static constexpr int NPT = (NCROSS + NT - 1) / NT;  // cells per thread
  static constexpr int E1 = 5 * TY * (TX + 2);  // x1 edges of cells i0-1 .. i0+TX
  static constexpr int E2 = 5 * (TY + 2) * TX;  // x2 edges of cells j0-1 .. j0+TY
  static constexpr int EB = SPLIT ? (E1 > E2 ? E1 : E2) : E1 + E2;
  static constexpr int F1 = 5 * TY * (TX + 1);
  static constexpr int F2 = 5 * (TY + 1) * TX;
  static constexpr size_t bytes = sizeof(R) * (size_t)(NR * 5 * NPL + 2 * EB + F1 + F2);
};

// FP64 PPM4 computes each plane's x1 and x2 limited half slopes once per cell, into
// shared memory behind the StageCfg buffers, for the edge items that share them.
template <int NG, int RC, bool MIXED>
constexpr bool shared_slopes() {
  return !MIXED && NG == 3 && RC == AK_PPM4;
}
template <int NG, int RC, bool MIXED, int TX, int TY>
constexpr size_t stage_smem() {
  // half slopes [5][TY][TX+4] and [5][TY+4][TX], interface values [5][TY][TX+3] and
  // [5][TY+3][TX]
  return StageCfg<NG, RC, MIXED, TX, TY>::bytes +
         (shared_slopes<NG, RC, MIXED>()
              ? sizeof(double) * 5 *
                    (size_t)(TY * (TX + 4) + (TY + 4) * TX + TY * (TX + 3) + (TY + 3) * TX)
              : 0);
}

// PERSIST: the persistent fused form for meshes that need a ghost fill (static
// refinement, FOFC): a cooperative launch of at most one resident wave of CTAs first runs
// the fill and the flux correction (fused_prologue), then loops over the work list.
// FORM >= 0, LAST >= 0: the RK form and the last-stage flag fixed at compile time (else
// the run-time arguments).  FAST: a uniform mesh read through direct halo reads, HLLC,
// no FOFC and no corrected faces -- the tests of those options compile away (a smaller
// plane loop, which stays in the instruction cache).
template <int NG, int RC, bool MIXED, int TX, int TY, bool PERSIST, int FORM = -1,
          int LAST = -1, bool FAST = false>
__global__ void __launch_bounds__(TX* TY, (MIXED || NG == 2) ? 2 : 1)
    stage_kernel(const double* __restrict__ uin_arg, const double* u0, double* uout,
                 ak_meshdev md, const ak_work* __restrict__ work, Bg bg, double a, double b,
                 int form, ak_dev_scalars* sc, int last_stage, int nwork) {
  // form: 0 = first stage U + dt L; 1 = RK2 final (U0 + U + dt L) / 2;
  //       2 = a U0 + b (U + dt L)
  static_assert(!(FAST && PERSIST), "the persistent form serves meshes with a ghost fill");
  if constexpr (FORM >= 0) form = FORM;
  if constexpr (LAST >= 0) last_stage = LAST;
  const bool direct = FAST || md.direct;
  const bool fofc = !FAST && md.fofc;
  using C = StageCfg<NG, RC, MIXED, TX, TY>;
  using R = typename C::R;
  // reconstructions that can overshoot: a face without a sound speed gives a NaN flux
  constexpr bool NANCHK = RC == AK_WENOZ || RC == AK_PPMX;
  constexpr int NT = C::NT, WX = C::WX, NPL = C::NPL, NR = C::NR, NPT = C::NPT;
  constexpr int C1 = TX + 2;  // x1 edge row length
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  R* ring = reinterpret_cast<R*>(smem_raw);  // [NR][5][WY][WX]
  R* e1lo = ring + NR * 5 * NPL;             // [5][TY][TX+2]
  R* e1hi = e1lo + C::EB;
  R* e2lo = C::SPLIT ? e1lo : e1lo + C::E1;  // [5][TY+2][TX]
  R* e2hi = C::SPLIT ? e1hi : e1hi + C::E1;
  R* f1 = e1hi + C::EB;                      // [5][TY][TX+1]
  R* f2 = f1 + C::F1;                        // [5][TY+1][TX]
  // FP64 PPM4: half slopes of the cells i0-2 .. i0+TX+1 of the tile rows ([5][TY][TX+4])
  // and of the cells j0-2 .. j0+TY+1 of the tile columns ([5][TY+4][TX])
  constexpr bool HSLOPE = shared_slopes<NG, RC, MIXED>();
  double* hs1 = reinterpret_cast<double*>(smem_raw + C::bytes);
  double* hs2 = hs1 + 5 * TY * (TX + 4);
  // and the interface values between them: x1 faces between padded x f+1 and f+2
  // ([5][TY][TX+3]), x2 faces between padded y f+1 and f+2 ([5][TY+3][TX])
  double* ia1 = hs2 + 5 * (TY + 4) * TX;
  double* ia2 = ia1 + 5 * TY * (TX + 3);
  __shared__ double red[NT / 32];
  __shared__ long long nbr[27];  // direct halo reads: the neighbour blocks

  if constexpr (PERSIST) {
    constexpr int KB = C::bytes / (NT * 80) < 8 ? (int)(C::bytes / (NT * 80)) : 8;
    static_assert(KB >= 1, "no room to stage the fill");
    fused_prologue<NG, MIXED, KB>(launder(const_cast<double*>(uin_arg)), md, bg, sc, smem_raw);
  }
  // one tile per CTA, or (persistent) tiles taken from the list until it runs out
  __shared__ int wslot;
  for (int it = 0; it < (PERSIST ? 0x7fffffff : 1); ++it) {
  const int wi = PERSIST ? next_tile(sc, &wslot) : (int)blockIdx.x;
  if (PERSIST && wi >= nwork) break;
  const double* __restrict__ uin = PERSIST ? launder(uin_arg) : uin_arg;
  const int tid = threadIdx.x;
  // this CTA's column tile of one MeshBlock, and that block's geometry
  const ak_work w = work[wi];
  const ak_block g = md.blocks[w.block];
  if (direct) neighbour_table(md, w.block, nbr);
  __syncthreads();
  const int blk = w.block;
  const int i0 = w.i0, j0 = w.j0, k0 = w.k0, k1 = w.k1;
  int kcur = k0;  // the plane whose x1/x2 faces are being solved

  const long long boff = g.off;
  const double* ub = uin + boff;
  const Counters cn{&sc->counters[0], &sc->counters[1]};
  const double dt = sc->dt;
  const double idx1 = 1.0 / g.dx1, idx2 = 1.0 / g.dx2, idx3 = 1.0 / g.dx3;
  const double cdt[3] = {dt * idx1, dt * idx2, dt * idx3};  // FP64 update: dt / dx_d
  const double g2 = bg.gamma * bg.gm1;
  const float g2h = f64_to_f32(g2), g2l = f64_to_f32(g2 - f32_to_f64(g2h));  // g2 = g2h + g2l
  const bool cubic = idx1 == idx2 && idx2 == idx3;
  const bool need_u0 = form != 0;

  auto slot = [](int k) { return (k + 4 * NR) % NR; };
  // ring position of the c-th converted cell: halo rows above, full rows, halo rows below
  auto cross_xy = [](int c, int& x, int& y) {
    constexpr int TOP = NG * TX, MID = TY * (TX + 2 * NG);
    if (c < TOP) {
      y = c / TX;
      x = NG + c % TX;
    } else if (c < TOP + MID) {
      const int d = c - TOP;
      y = NG + d / (TX + 2 * NG);
      x = d % (TX + 2 * NG);
    } else {
      const int d = c - TOP - MID;
      y = NG + TY + d / TX;
      x = NG + d % TX;
    }
  };
  // global loads of this thread's cells of plane kp (interior index; ghost planes ok)
  auto fetch = [&](int kp, double (&u)[NPT][5], int (&pos)[NPT]) {
#pragma unroll
    for (int m = 0; m < NPT; ++m) {
      const int c = tid + m * NT;
      pos[m] = -1;
      if (c < C::NCROSS) {
        int x, y;
        cross_xy(c, x, y);
        const int ip = i0 + x, jp = j0 + y;  // padded indices (halo starts at i0 - NG)
        if (ip < g.p1 && jp < g.p2) {
          const bool halo = ip < NG || ip >= NG + g.nx1 || jp < NG || jp >= NG + g.nx2 ||
                            kp < 0 || kp >= g.nx3;
          const double* src = (direct && halo)
                                  ? uin + halo_elem(g, nbr, NG, ip, jp, kp)
                                  : ub + ((long long)(kp + NG) * g.p2 + jp) * g.s1 + ip;
#pragma unroll
          for (int v = 0; v < 5; ++v) u[m][v] = src[v * g.var_stride];
          pos[m] = y * WX + x;
        }
      }
    }
  };
  // primitive recovery of fetched cells into the ring slot of plane kp
  auto store = [&](int kp, const double (&u)[NPT][5], const int (&pos)[NPT]) {
    R* dst = ring + slot(kp) * 5 * NPL;
#pragma unroll
    for (int m = 0; m < NPT; ++m) {
      if (pos[m] >= 0) {
        R w[5];
        c2p_t<NANCHK>(u[m], w, bg, cn);
#pragma unroll
        for (int v = 0; v < 5; ++v) dst[v * NPL + pos[m]] = w[v];
      }
    }
  };
  auto load_plane = [&](int kp) {
    double u[NPT][5];
    int pos[NPT];
    fetch(kp, u, pos);
    store(kp, u, pos);
  };

  // own column of this thread
  const int tx = tid % TX, ty = tid / TX;
  const int ci = i0 + tx, cj = j0 + ty;
  const bool own = (ci < g.nx1) && (cj < g.nx2);
  const int oc = (ty + NG) * WX + (tx + NG);
  const long long ecol = boff + ((long long)NG * g.p2 + (cj + NG)) * g.s1 + (ci + NG);
  const long long plane_stride = (long long)g.p2 * g.s1;

  // x3 edges of the own column's cell kc (stencil planes kc-NG+1 .. kc+NG-1)
  auto x3_edges = [&](int kc, R* lo, R* hi) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R q[2 * NG - 1];
#pragma unroll
      for (int m = 0; m < 2 * NG - 1; ++m) q[m] = ring[slot(kc - NG + 1 + m) * 5 * NPL + v * NPL + oc];
      edges_t<NG, RC>(q, lo[v], hi[v]);
    }
  };
  // FP64 PPM4: the column carries, from cell to cell along x3, the half slope of the next
  // cell (xh) and its lower interface value (xa), both computed for the cell below with
  // the same operations on the same operands (the same bits): per cell one new slope and
  // one new interface value instead of three and two
  constexpr bool CARRY = C::CARRY;
  double xh[5], xa[5];
  auto x3_edges_carry = [&](int kc, R* lo, R* hi) {
    if constexpr (CARRY) {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double qc = ring[slot(kc) * 5 * NPL + v * NPL + oc];
        const double qn = ring[slot(kc + 1) * 5 * NPL + v * NPL + oc];
        const double hn =
            ppm_half_slope_fp64(qc, qn, ring[slot(kc + 2) * 5 * NPL + v * NPL + oc]);
        const double ahi = ppm_interface_fp64(qc, qn, xh[v], hn);
        ppm_monotonize_fp64(xa[v], ahi, qc, lo[v], hi[v]);
        xh[v] = hn;
        xa[v] = ahi;
      }
    }
  };
  // FP64 PPM4: the plane's half slopes, each computed once (x1: padded x 1 .. TX+4 of the
  // tile rows; x2: padded y 1 .. TY+4 of the tile columns); cells outside the block's
  // padded extent are skipped, as the edge items that would read them are
  auto half_slopes = [&](const R* pl) {
    if constexpr (HSLOPE) {
      constexpr int N1 = TY * (TX + 4), N2 = (TY + 4) * TX;
      for (int it = tid; it < 5 * (N1 + N2); it += NT) {
        if (it < 5 * N1) {
          const int v = it / N1, e = it % N1, r = e / (TX + 4), c = e % (TX + 4);
          if (i0 + c + 2 < g.p1 && j0 + r < g.nx2) {
            const double* q = pl + v * NPL + (r + NG) * WX + c;  // padded x = c + 1 centre
            hs1[it] = ppm_half_slope_fp64(q[0], q[1], q[2]);
          }
        } else {
          const int e2 = it - 5 * N1, v = e2 / N2, e = e2 % N2, r = e / TX, c = e % TX;
          if (i0 + c < g.nx1 && j0 + r + 2 < g.p2) {
            const double* q = pl + v * NPL + r * WX + c + NG;  // padded y = r + 1 centre
            hs2[e2] = ppm_half_slope_fp64(q[0], q[WX], q[2 * WX]);
          }
        }
      }
    }
  };
  auto interfaces = [&](const R* pl) {
    if constexpr (HSLOPE) {
      constexpr int N1 = TY * (TX + 3), N2 = (TY + 3) * TX;
      for (int it = tid; it < 5 * (N1 + N2); it += NT) {
        if (it < 5 * N1) {
          const int v = it / N1, e = it % N1, r = e / (TX + 3), f = e % (TX + 3);
          if (i0 + f + 3 < g.p1 && j0 + r < g.nx2) {
            const double* q = pl + v * NPL + (r + NG) * WX + f;
            const double* h = hs1 + (v * TY + r) * (TX + 4) + f;
            ia1[it] = ppm_interface_fp64(q[1], q[2], h[0], h[1]);
          }
        } else {
          const int e2 = it - 5 * N1, v = e2 / N2, e = e2 % N2, r = e / TX, c = e % TX;
          if (i0 + c < g.nx1 && j0 + r + 3 < g.p2) {
            const double* q = pl + v * NPL + r * WX + c + NG;
            const double* h = hs2 + (v * (TY + 4) + r) * TX + c;
            ia2[e2] = ppm_interface_fp64(q[WX], q[2 * WX], h[0], h[TX]);
          }
        }
      }
    }
  };
  // FP64 PLM: x1 and x2 edges of two neighbouring cells per item, which share the
  // difference between them (the same operation on the same operands, so the same bits)
  constexpr bool PAIR = !MIXED && RC == AK_PLM;
  static_assert(!PAIR || (C1 % 2 == 0 && TY % 2 == 0), "cell pairs need even rows");
  auto x1_edges = [&](const R* pl) {  // cells i0-1 .. i0+TX of the tile's rows
    if constexpr (PAIR) {
      for (int it = tid; it < (C1 / 2) * TY; it += NT) {
        const int c = 2 * (it % (C1 / 2)), r = it / (C1 / 2);
        // cell c+1 only exists where cell c does; its stencil (x up to c + 3 <= TX + 3)
        // stays inside the ring row even where the cell itself is skipped
        if (i0 - 1 + c <= g.nx1 && j0 + r < g.nx2) {
          const bool second = i0 + c <= g.nx1;
          const int base = (r + NG) * WX + c;
#pragma unroll 1
          for (int v = 0; v < 5; ++v) {
            const double* q = pl + v * NPL + base;
            const double d1 = q[2] - q[1];
            const int o = (v * TY + r) * C1 + c;
            plm_edges_fp64(q[1] - q[0], d1, q[1], e1lo[o], e1hi[o]);
            if (second) plm_edges_fp64(d1, q[3] - q[2], q[2], e1lo[o + 1], e1hi[o + 1]);
          }
        }
      }
      return;
    }
    for (int it = tid; it < C::E1 / 5; it += NT) {
      const int c = it % C1, r = it / C1;
      if (i0 - 1 + c <= g.nx1 && j0 + r < g.nx2) {
        const int base = (r + NG) * WX + c;  // stencil x = c .. c + 2NG - 2
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          if constexpr (HSLOPE) {  // interface values of faces c, c+1 (shared)
            const double* ia = ia1 + (v * TY + r) * (TX + 3) + c;
            ppm_monotonize_fp64(ia[0], ia[1], pl[v * NPL + base + 2],
                                e1lo[(v * TY + r) * C1 + c], e1hi[(v * TY + r) * C1 + c]);
          } else {
            R q[2 * NG - 1];
#pragma unroll
            for (int m = 0; m < 2 * NG - 1; ++m) q[m] = pl[v * NPL + base + m];
            edges_t<NG, RC>(q, e1lo[(v * TY + r) * C1 + c], e1hi[(v * TY + r) * C1 + c]);
          }
        }
      }
    }
  };
  auto x2_edges = [&](const R* pl) {  // cells j0-1 .. j0+TY of the tile's columns
    if constexpr (PAIR) {
      for (int it = tid; it < TX * ((TY + 2) / 2); it += NT) {
        const int c = it % TX, r = 2 * (it / TX);
        // rows r .. r + 3 <= TY + 3 of the ring, as for x1
        if (i0 + c < g.nx1 && j0 - 1 + r <= g.nx2) {
          const bool second = j0 + r <= g.nx2;
          const int base = r * WX + c + NG;
#pragma unroll 1
          for (int v = 0; v < 5; ++v) {
            const double* q = pl + v * NPL + base;
            const double d1 = q[2 * WX] - q[WX];
            const int o = (v * (TY + 2) + r) * TX + c;
            plm_edges_fp64(q[WX] - q[0], d1, q[WX], e2lo[o], e2hi[o]);
            if (second) plm_edges_fp64(d1, q[3 * WX] - q[2 * WX], q[2 * WX], e2lo[o + TX], e2hi[o + TX]);
          }
        }
      }
      return;
    }
    for (int it = tid; it < C::E2 / 5; it += NT) {
      const int c = it % TX, r = it / TX;
      if (i0 + c < g.nx1 && j0 - 1 + r <= g.nx2) {
        const int base = r * WX + c + NG;  // stencil y = r .. r + 2NG - 2
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          if constexpr (HSLOPE) {
            const double* ia = ia2 + (v * (TY + 3) + r) * TX + c;
            ppm_monotonize_fp64(ia[0], ia[TX], pl[v * NPL + base + 2 * WX],
                                e2lo[(v * (TY + 2) + r) * TX + c],
                                e2hi[(v * (TY + 2) + r) * TX + c]);
          } else {
            R q[2 * NG - 1];
#pragma unroll
            for (int m = 0; m < 2 * NG - 1; ++m) q[m] = pl[v * NPL + base + m * WX];
            edges_t<NG, RC>(q, e2lo[(v * (TY + 2) + r) * TX + c], e2hi[(v * (TY + 2) + r) * TX + c]);
          }
        }
      }
    }
  };
  auto x1_faces = [&]() {
    for (int it = tid; it < C::F1 / 5; it += NT) {
      const int fx = it % (TX + 1), fy = it / (TX + 1);
      if (i0 + fx <= g.nx1 && j0 + fy < g.nx2) {
        R l[5], r[5], f[5];
        const int fi = i0 + fx;
        const int ov = FAST ? -1 : (fi == 0 ? g.ovr[0] : (fi == g.nx1 ? g.ovr[1] : -1));
        if (ov >= 0) {  // coarse face next to a refined region: the fine-flux mean
          corrected_flux(md.fcbuf, ov + kcur * g.nx2 + j0 + fy, f);
        } else {
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            l[v] = e1hi[(v * TY + fy) * C1 + fx];       // cell i-1: column fx
            r[v] = e1lo[(v * TY + fy) * C1 + fx + 1];   // cell i:   column fx+1
          }
          solve<NANCHK, FAST>(0, l, r, bg, f);
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) f1[(v * TY + fy) * (TX + 1) + fx] = f[v];
      }
    }
  };
  auto x2_faces = [&]() {
    for (int it = tid; it < C::F2 / 5; it += NT) {
      const int fx = it % TX, fy = it / TX;
      if (i0 + fx < g.nx1 && j0 + fy <= g.nx2) {
        R l[5], r[5], f[5];
        const int fj = j0 + fy;
        const int ov = FAST ? -1 : (fj == 0 ? g.ovr[2] : (fj == g.nx2 ? g.ovr[3] : -1));
        if (ov >= 0) {
          corrected_flux(md.fcbuf, ov + kcur * g.nx1 + i0 + fx, f);
        } else {
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            l[v] = e2hi[(v * (TY + 2) + fy) * TX + fx];      // cell j-1: row fy
            r[v] = e2lo[(v * (TY + 2) + fy + 1) * TX + fx];  // cell j:   row fy+1
          }
          solve<NANCHK, FAST>(1, l, r, bg, f);
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) f2[(v * (TY + 1) + fy) * TX + fx] = f[v];
      }
    }
  };

  // prologue: planes k0-NG .. k0+NG-1, the flux through the face below k0, then plane
  // k0+NG (its slot held plane k0-NG, used by that flux).  The 5-slot ring first holds
  // planes k0-3 .. k0+1 for the edge values of cell k0-1, then takes plane k0+2 in the
  // slot of plane k0-3.
  R hi3[5], f3m[5], f3p[5];
  R lo_a[5], hi_a[5];
  if constexpr (NR < 2 * NG) {
    for (int kp = k0 - NG; kp < k0 + NG - 1; ++kp) load_plane(kp);
    __syncthreads();
    if (own) x3_edges(k0 - 1, lo_a, hi_a);
    __syncthreads();
    load_plane(k0 + NG - 1);
  } else {
    for (int kp = k0 - NG; kp < k0 + NG; ++kp) load_plane(kp);
  }
  __syncthreads();
  if (own) {
    R lo_b[5];
    if constexpr (NR >= 2 * NG) x3_edges(k0 - 1, lo_a, hi_a);
    x3_edges(k0, lo_b, hi3);
    if constexpr (CARRY) {  // the carry for cell k0 + 1
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double qm = ring[slot(k0 - 1) * 5 * NPL + v * NPL + oc];
        const double q0 = ring[slot(k0) * 5 * NPL + v * NPL + oc];
        const double q1 = ring[slot(k0 + 1) * 5 * NPL + v * NPL + oc];
        const double q2 = ring[slot(k0 + 2) * 5 * NPL + v * NPL + oc];
        const double h0 = ppm_half_slope_fp64(qm, q0, q1);
        xh[v] = ppm_half_slope_fp64(q0, q1, q2);
        xa[v] = ppm_interface_fp64(q0, q1, h0, xh[v]);
      }
    }
    if (!FAST && k0 == 0 && g.ovr[4] >= 0)
      corrected_flux(md.fcbuf, g.ovr[4] + cj * g.nx1 + ci, f3m);
    else
      solve<NANCHK, FAST>(2, hi_a, lo_b, bg, f3m);
  }
  __syncthreads();
  load_plane(k0 + NG);

  float dtmin_f = __int_as_float(0x7f800000);
  double dtmin = __longlong_as_double(0x7ff0000000000000ll);
  double lam_max = 0.0;
  double pf[NPT][5];
  int pfpos[NPT];
  for (int k = k0; k < k1; ++k) {
    // the ring holds planes k-NG+1 .. k+NG (5-slot ring: k-1 .. k+3) once this barrier
    // is passed
    const bool more = k + 1 < k1;
    if constexpr (C::PREFETCH) {
      if (more) fetch(k + NG + 1, pf, pfpos);
    }
    double uik[5], u0k[5];
    if constexpr (MIXED) {
      if (own) {
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          uik[v] = uin[ecol + k * plane_stride + v * g.var_stride];
          u0k[v] = need_u0 ? u0[ecol + k * plane_stride + v * g.var_stride] : 0.0;
        }
      }
    }
    __syncthreads();
    const R* pl = ring + slot(k) * 5 * NPL;
    kcur = k;
    R lo3[5], hi3n[5];
    if constexpr (HSLOPE) {
      half_slopes(pl);
      __syncthreads();
      interfaces(pl);
      __syncthreads();
    }

    if constexpr (C::SPLIT) {
      x1_edges(pl);
      if (own) {
        if constexpr (CARRY)
          x3_edges_carry(k + 1, lo3, hi3n);
        else
          x3_edges(k + 1, lo3, hi3n);
      }
      __syncthreads();
      x1_faces();
      __syncthreads();
      x2_edges(pl);
      __syncthreads();
      x2_faces();
    } else {
      x1_edges(pl);
      x2_edges(pl);
      if (own) {
        if constexpr (CARRY)
          x3_edges_carry(k + 1, lo3, hi3n);
        else
          x3_edges(k + 1, lo3, hi3n);
      }
      __syncthreads();
      x1_faces();
      x2_faces();
    }
    if (own) {
      if (!FAST && k + 1 == g.nx3 && g.ovr[5] >= 0)
        corrected_flux(md.fcbuf, g.ovr[5] + cj * g.nx1 + ci, f3p);
      else
        solve<NANCHK, FAST>(2, hi3, lo3, bg, f3p);
#pragma unroll
      for (int v = 0; v < 5; ++v) hi3[v] = hi3n[v];
    }
    __syncthreads();

    // ---- divergence and RK update ---------------------------------------------
    if (own) {
      const long long e = ecol + k * plane_stride;
      double un[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const R d1 = f1[(v * TY + ty) * (TX + 1) + tx + 1] - f1[(v * TY + ty) * (TX + 1) + tx];
        const R d2 = f2[(v * (TY + 1) + ty + 1) * TX + tx] - f2[(v * (TY + 1) + ty) * TX + tx];
        const R d3 = f3p[v] - f3m[v];
        double r;
        if constexpr (MIXED) {
          const float L = -fmaf(d1, (float)idx1, fmaf(d2, (float)idx2, d3 * (float)idx3));
          r = rk_update_mixed(form, a, b, dt, L, uik[v], u0k[v]);
        } else {
          r = rk_update_fp64(form, a, b, cdt, d1, d2, d3, uin[e + v * g.var_stride],
                             form != 0 ? u0[e + v * g.var_stride] : 0.0);
        }
        un[v] = r;
        f3m[v] = f3p[v];
      }
      if (fofc) {
        // a flagged cell's U0, saved before the output (which may overwrite U0) is stored
        const int fi = fofc_flag(un, md, sc, blk, g, ci, cj, k);
        if (fi >= 0 && form != 0) {
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            if constexpr (MIXED)
              md.fu0[(long long)fi * 5 + v] = u0k[v];
            else
              md.fu0[(long long)fi * 5 + v] = u0[e + v * g.var_stride];
          }
        }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) uout[e + v * g.var_stride] = un[v];
      if (last_stage) {
        if constexpr (MIXED) {
          // CFL ratio in FP32: it only sets the next step's dt
          const float rho = fmaxf(f64_to_f32(un[0]), (float)AK_RHO_FLOOR);
          const float ir = rcp_approx_f32(rho);
          const float m1 = f64_to_f32(un[1]), m2 = f64_to_f32(un[2]), m3 = f64_to_f32(un[3]);
          const float ug = fmaxf(fmaf(-0.5f * ir, fmaf(m1, m1, fmaf(m2, m2, m3 * m3)),
                                      f64_to_f32(un[4])), (float)AK_UG_FLOOR);
          const float cs = sqrt_fast(bg.gamma_f * (bg.gamma_f - 1.0f) * ug * ir);
          float lam = fmaf(fabsf(m1), ir, cs) * (float)idx1;
          lam = fmaxf(lam, fmaf(fabsf(m2), ir, cs) * (float)idx2);
          lam = fmaxf(lam, fmaf(fabsf(m3), ir, cs) * (float)idx3);
          dtmin_f = fminf(dtmin_f, rcp_approx_f32(lam));
        } else {
          // CFL in FP64 (the FP64 form reproduces the oracle's dt to ~1e-13): the
          // largest (|v_d| + c_s) / dx_d of the column; dt = 1 / max at the end
          double rho = un[0];
          rho = at_least(rho, AK_RHO_FLOOR) ? rho : AK_RHO_FLOOR;
          const double r = rcp64(rho);
          const double m2 = fma(un[1], un[1], fma(un[2], un[2], un[3] * un[3]));
          double ug = fma(-m2, dscale(r, -1), un[4]);
          ug = at_least(ug, AK_UG_FLOOR) ? ug : AK_UG_FLOOR;
          // sqrt(gamma (gamma - 1) u_g / rho)
          const double cs = sqrt_gratio64(ug, rho, g2, g2h, g2l);
          const double a1 = fabs(un[1]), a2 = fabs(un[2]), a3 = fabs(un[3]);
          double lam;
          if (cubic) {
            // equal widths: (a r + c_s) / dx rises with a, so the largest |v_d| gives the
            // largest rate (the same value as the maximum over the three)
            double am = dgt_pos(a2, a1) ? a2 : a1;
            am = dgt_pos(a3, am) ? a3 : am;
            lam = fma(am, r, cs) * idx1;
          } else {
            const double l1 = fma(a1, r, cs) * idx1, l2 = fma(a2, r, cs) * idx2,
                         l3 = fma(a3, r, cs) * idx3;
            lam = dgt_pos(l2, l1) ? l2 : l1;
            lam = dgt_pos(l3, lam) ? l3 : lam;
          }
          lam_max = dgt_pos(lam, lam_max) ? lam : lam_max;
        }
      }
    }
    // next plane into the slot of plane k-NG+1 (5-slot ring: k-1), whose last reader
    // was this iteration's reconstruction or an earlier one (finished before the
    // barrier above)
    if (more) {
      if constexpr (C::PREFETCH)
        store(k + NG + 1, pf, pfpos);
      else
        load_plane(k + NG + 1);
    }
  }

  if (last_stage) {
    if constexpr (MIXED)
      dtmin = f32_to_f64(dtmin_f);
    else
      dtmin = dpos(lam_max) ? 1.0 / lam_max : dtmin;
    // CTA min of the CFL ratio -> one atomic per CTA (non-negative doubles order as
    // their bit patterns)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dtmin = fmin(dtmin, __shfl_xor_sync(0xffffffffu, dtmin, o));
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = dtmin;
    __syncthreads();
    if (tid < 32) {
      double v = tid < NT / 32 ? red[tid] : __longlong_as_double(0x7ff0000000000000ll);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (tid == 0)
        atomicMin(&sc->dtmin_bits, (unsigned long long)__double_as_longlong(v));
    }
  }
  if constexpr (PERSIST) __syncthreads();  // the next tile reuses the shared memory
  }
}

Bg make_bg(const ak_mesh* m);

// Launch (or, prepare_only, raise the shared-memory limit of) the stage kernel of one
// configuration over the mesh's work list; m->fused selects the persistent variant.
using stage_kern_t = void (*)(const double*, const double*, double*, ak_meshdev, const ak_work*,
                             Bg, double, double, int, ak_dev_scalars*, int, int);

// WITH_FAST: the compile-time instances for uniform HLLC meshes without FOFC (FAST, with
// each RK form and last-stage flag) exist and are launched where they apply.
template <int NG, int RC, bool MIXED, int TX, int TY, bool WITH_FAST = false>
inline cudaError_t launch(const ak_mesh* m, const double* uin, const double* u0, double* uout,
                          double a, double b, int rk2_final, int last_stage, bool prepare_only) {
  const size_t smem = stage_smem<NG, RC, MIXED, TX, TY>();
  auto kern = stage_kernel<NG, RC, MIXED, TX, TY, false>;
  auto pk = stage_kernel<NG, RC, MIXED, TX, TY, true>;
  stage_kern_t fast[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if constexpr (WITH_FAST) {
    fast[0] = stage_kernel<NG, RC, MIXED, TX, TY, false, 0, 0, true>;
    fast[1] = stage_kernel<NG, RC, MIXED, TX, TY, false, 1, 0, true>;
    fast[2] = stage_kernel<NG, RC, MIXED, TX, TY, false, 2, 0, true>;
    fast[3] = stage_kernel<NG, RC, MIXED, TX, TY, false, 0, 1, true>;
    fast[4] = stage_kernel<NG, RC, MIXED, TX, TY, false, 1, 1, true>;
    fast[5] = stage_kernel<NG, RC, MIXED, TX, TY, false, 2, 1, true>;
  }
  if (prepare_only) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int i = 0; i < 6 && e == cudaSuccess && fast[i]; ++i)
      e = cudaFuncSetAttribute(fast[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
  }
  const Bg bg = make_bg(m);
  const int form = rk2_final ? 1 : (a == 0.0 ? 0 : 2);
  if (m->fused)
    return launch_persistent(m, pk, TX * TY, smem, uin, u0, uout, m->md, m->d_work, bg, a, b,
                             form, m->d_sc, last_stage, m->nwork);
  if (WITH_FAST && m->md.direct && !m->md.fofc && bg.rsolver == AK_HLLC && m->nfc == 0) {
    const stage_kern_t k = fast[form + 3 * (last_stage ? 1 : 0)];
    k<<<(unsigned)m->nwork, TX * TY, smem, m->stream>>>(uin, u0, uout, m->md, m->d_work, bg, a,
                                                         b, form, m->d_sc, last_stage, m->nwork);
    return cudaGetLastError();
  }
  kern<<<(unsigned)m->nwork, TX * TY, smem, m->stream>>>(uin, u0, uout, m->md, m->d_work, bg, a,
                                                          b, form, m->d_sc, last_stage, m->nwork);
  return cudaGetLastError();
}

// Per-reconstruction launchers (one translation unit each): the stage of this mesh with
// the given RK weights; prepare: raise the kernels' shared-memory limits instead.
cudaError_t launch_stage_plm(const ak_mesh* m, const double* uin, const double* u0,
                             double* uout, double a, double b, int rk2_final,
                             int last_stage, bool prepare);
cudaError_t launch_stage_ppm4(const ak_mesh* m, const double* uin, const double* u0,
                              double* uout, double a, double b, int rk2_final,
                              int last_stage, bool prepare);
cudaError_t launch_stage_wenoz(const ak_mesh* m, const double* uin, const double* u0,
                               double* uout, double a, double b, int rk2_final,
                               int last_stage, bool prepare);
cudaError_t launch_stage_ppmx(const ak_mesh* m, const double* uin, const double* u0,
                              double* uout, double a, double b, int rk2_final,
                              int last_stage, bool prepare);

}  // namespace ak
