// Mixed-form stage kernel with paired x1/x2 work: the same stage as the mixed instance
// of stage_kernel (primitive recovery, reconstruction, Riemann solver, divergence, RK
// update and CFL of Section 3, Eqs. (1), (3), (4)), organised for GB300's issue rate,
// for PLM (NG = 2) and for the three-ghost-cell reconstructions (NG = 3: PPM4, WENO-Z,
// PPMX).
//
// A CTA owns a T x T column tile of one MeshBlock and marches along x3, with
// T (T + 2) threads: thread t owns x1 edge item t and x2 edge item t (the tile's rows
// with one extra cell on each side, and its columns likewise), the x1 face to the right
// of its x1 item and the x2 face above its x2 item.  The two items of a thread, and its
// two faces, are computed together in the two lanes of packed FP32x2 arithmetic
// (lanes.cuh), which gives the same bits as solving each alone.  The upper edge values
// of a thread's items stay in its registers for its faces; only the lower ones go
// through shared memory.  The first T^2 threads also own one column: its x3
// reconstruction, x3 face and update.
//
// Per plane k, between two barriers:
//   P1  primitive recovery of plane k+NG (first, so that its dependent FP64 operations
//       overlap the FP32 work below; every column thread converts one cell of the cross,
//       the first ones a second); x1/x2 edges of plane k (paired); the column's x3
//       edge of cell k, the x3 face below it, and the divergence, RK update and CFL of
//       cell k-1 (whose x1/x2 fluxes the previous P2 left in shared memory);
//   P2  x1/x2 faces of plane k (paired).
// The conserved state of plane k+NG+1 and the columns' U_in / U0 of plane k arrive in
// shared memory by cp.async issued at the start of P2, so no register holds data in
// flight across the phases.
//
// Primitives live in NG + 1 cross-shaped plane slots (the tile with NG halo cells in x1
// and x2: planes k .. k+NG) and NG - 1 column slots (the tile's cells only: planes
// k-NG+1 .. k-1, the lower part of the x3 stencil, which needs no halo).  A column
// thread moves its own cell of plane k from the cross slot to a column slot once its
// x3 edge is done, so the cross slot can take plane k+NG+1.
#pragma once

#include "ak_internal.cuh"
#include "hydro_ops.cuh"
#include "stage_common.cuh"

namespace ak {
namespace mx {

// 16-byte copy global -> shared through L2 only
static __device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
static __device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// waits until at most N of this thread's committed copy groups are still in flight
template <int N>
static __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int NG, int T>
struct MxCfg {
  static constexpr int TX = T, TY = T;
  static constexpr int C1 = TX + 2;                 // x1 edge items per tile row
  static constexpr int NE = TY * C1;                // x1 edge items (= x2 edge items)
  static constexpr int NF = TY * (TX + 1);          // x1 faces (= x2 faces)
  static constexpr int NTH = (NE + 31) / 32 * 32;
  static constexpr int NOWN = TX * TY;              // threads with a column
  static constexpr int WX = TX + 2 * NG, WY = TY + 2 * NG, NPL = WX * WY;
  static constexpr int NXS = NG + 1;                // cross-shaped plane slots
  static constexpr int NCS = NG - 1;                // column plane slots
  static constexpr int NCROSS = TX * TY + 2 * NG * (TX + TY);  // converted cells per plane
  static constexpr int NSPARE = NTH - NOWN;         // threads without a column
  // staged rows: 16-byte chunks start at padded x = NG mod 2 (a row's interior is 32-byte
  // aligned), so for odd NG a tile row is staged one cell wider on each side
  static constexpr int ODD = NG & 1;
  static constexpr int WSX = TX + 2 * NG + 2 * ODD;   // staged cells of a tile row
  static constexpr int NSTG = 2 * NG * TX + TY * WSX;  // staged cells per plane
  static_assert(NE == (TY + 2) * TX && NF == (TY + 1) * TX, "square tiles");
  static_assert(NSPARE > 0, "more edge items than columns");
  static constexpr size_t bytes =
      sizeof(double) * (5 * NSTG + 2 * 5 * NOWN) +
      sizeof(float) * (NXS * 5 * NPL + NCS * 5 * NOWN + 2 * 5 * NE + 2 * 5 * NF);
};

// PERSIST: the persistent fused form (see stage_kernel): ghost fill and flux correction
// in a cooperative prologue, then a loop over the work list.
// FORM >= 0, LAST >= 0: the RK form and the last-stage flag fixed at compile time (else
// the run-time arguments).  FAST: a uniform mesh read through direct halo reads, HLLC,
// no FOFC and no corrected faces -- the tests of those options compile away, which
// shortens the plane loop and keeps its code in the instruction cache.
// RC: the reconstruction (AK_PLM with NG = 2; AK_PPM4, AK_WENOZ or AK_PPMX with NG = 3).
template <int NG, int RC, int T, bool PERSIST = false, int FORM = -1, int LAST = -1,
          bool FAST = false>
__global__ void __launch_bounds__(MxCfg<NG, T>::NTH, 2)
    stage_mx_kernel(const double* __restrict__ uin_arg, const double* u0, double* uout,
                    ak_meshdev md, const ak_work* __restrict__ work, Bg bg, double a, double b,
                    int form, ak_dev_scalars* sc, int last_stage, int nwork) {
  // form: 0 = first stage U + dt L; 1 = RK2 final (U0 + U + dt L) / 2;
  //       2 = a U0 + b (U + dt L)
  static_assert(!(FAST && PERSIST), "the persistent form serves meshes with a ghost fill");
  static_assert((NG == 2) == (RC == AK_PLM), "PLM uses two ghost cells, the others three");
  if constexpr (FORM >= 0) form = FORM;
  if constexpr (LAST >= 0) last_stage = LAST;
  const bool direct = FAST || md.direct;
  const bool fofc = !FAST && md.fofc;
  const bool hllc = FAST || bg.rsolver == AK_HLLC;
  using C = MxCfg<NG, T>;
  constexpr int TX = C::TX, WX = C::WX, NPL = C::NPL, NE = C::NE, NF = C::NF;
  constexpr int C1 = C::C1, NOWN = C::NOWN, NCROSS = C::NCROSS, NXS = C::NXS;
  constexpr int ODD = C::ODD, WSX = C::WSX, NSTG = C::NSTG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* stg = reinterpret_cast<double*>(smem_raw);          // [5][NSTG] next plane
  double* ucol = stg + 5 * NSTG;                                // [2][5][NOWN] U_in, U0
  float* ring = reinterpret_cast<float*>(ucol + 10 * NOWN);      // [NXS][5][NPL] W'
  float* cring = ring + NXS * 5 * NPL;                          // [NCS][5][NOWN] W'
  float* e1lo = cring + C::NCS * 5 * NOWN;                      // [5][NE]
  float* e2lo = e1lo + 5 * NE;
  float* f1 = e2lo + 5 * NE;                                    // [5][NF]
  float* f2 = f1 + 5 * NF;
  __shared__ double red[C::NTH / 32];
  __shared__ long long nbr[27];  // direct halo reads: the neighbour blocks

  if constexpr (PERSIST) {
    constexpr int KB = C::bytes / (C::NTH * 80) < 8 ? (int)(C::bytes / (C::NTH * 80)) : 8;
    static_assert(KB >= 1, "no room to stage the fill");
    fused_prologue<NG, true, KB>(launder(const_cast<double*>(uin_arg)), md, bg, sc, smem_raw);
  }
  // one tile per CTA, or (persistent) tiles taken from the list until it runs out
  __shared__ int wslot;
  for (int it = 0; it < (PERSIST ? 0x7fffffff : 1); ++it) {
  const int wi = PERSIST ? next_tile(sc, &wslot) : (int)blockIdx.x;
  if (PERSIST && wi >= nwork) break;
  const double* __restrict__ uin = PERSIST ? launder(uin_arg) : uin_arg;
  const int tid = threadIdx.x;
  const ak_work w = work[wi];
  const ak_block g = md.blocks[w.block];
  if (direct) neighbour_table(md, w.block, nbr);
  const int i0 = w.i0, j0 = w.j0, k0 = w.k0, k1 = w.k1;
  const double* ub = uin + g.off;
  const Counters cn{&sc->counters[0], &sc->counters[1]};
  const double dt = sc->dt;
  const double idx1 = 1.0 / g.dx1, idx2 = 1.0 / g.dx2, idx3 = 1.0 / g.dx3;
  const float idx1f = (float)idx1, idx2f = (float)idx2, idx3f = (float)idx3;
  const bool need_u0 = form != 0;
  const long long pst = (long long)g.p2 * g.s1;  // plane stride
  const long long vst = g.var_stride;

  // cross slot and column slot of plane k (k >= -NG)
  auto xslot = [](int k) { return (k + 4 * NXS) % NXS; };
  auto cslot = [](int k) { return NG == 2 ? 0 : (k + 4) & 1; };

  // ---- cells of the cross-shaped plane this thread converts ------------------------------
  // cell c: halo rows above, tile rows with their x1 halo, halo rows below (no corners)
  auto cross_xy = [](int c, int& x, int& y) {
    constexpr int TOP = NG * TX, MID = C::TY * (TX + 2 * NG);
    if (c < TOP) {
      y = c / TX;
      x = NG + c % TX;
    } else if (c < TOP + MID) {
      const int d = c - TOP;
      y = NG + d / (TX + 2 * NG);
      x = d % (TX + 2 * NG);
    } else {
      const int d = c - TOP - MID;
      y = NG + C::TY + d / TX;
      x = NG + d % TX;
    }
  };
  // staged element of cross cell c (tile rows are staged WSX wide, from padded x = -ODD)
  auto stg_of = [](int c) {
    constexpr int TOP = NG * TX, MID = C::TY * (TX + 2 * NG);
    if (c < TOP) return c;
    if (c < TOP + MID) {
      const int d = c - TOP;
      return TOP + (d / (TX + 2 * NG)) * WSX + d % (TX + 2 * NG) + ODD;
    }
    return c - MID + C::TY * WSX;
  };
  // Column thread t converts cross cell t, and the first NLOW of them also cell NOWN + t:
  // whole warps, one extra cell each.  A warp that converted several cells in a row
  // would sit on the dependent FP64 operations of each and hold the plane's barrier;
  // spread over the column warps, that latency overlaps their FP32 work.  The spare
  // threads convert none.
  constexpr int NLOW = NCROSS - NOWN;
  static_assert(NLOW % 32 == 0 && NLOW <= NOWN, "whole warps of second cells");
  constexpr int NMY = 2;  // slot 0: cross cell t; slot 1: cross cell NOWN + t
  auto cell_of = [&](int m) {
    if (tid >= NOWN) return NCROSS;
    return m == 0 ? tid : (tid < NLOW ? NOWN + tid : NCROSS);
  };
  int mypos[NMY];  // ring position of the slot's cell, or -1 (none, or outside the block)
  int mystg[NMY];  // its staged element
#pragma unroll
  for (int m = 0; m < NMY; ++m) {
    const int c = cell_of(m);
    mypos[m] = -1;
    mystg[m] = 0;
    if (c < NCROSS) {
      int x, y;
      cross_xy(c, x, y);
      if (i0 + x < g.p1 && j0 + y < g.p2) {
        mypos[m] = y * WX + x;
        mystg[m] = stg_of(c);
      }
    }
  }
  // ---- 16-byte copy chunks of this thread ----------------------------------------------
  // The next plane's cross, two cells per chunk.  Chunks start at padded x = NG mod 2
  // (plus even offsets): there the element index in the register is even (the interior of
  // a row is 32-byte aligned, tiles start at multiples of 16), and block boundaries
  // (padded x = NG and NG + nx1, with nx1 even) fall between chunks, so a chunk is inside
  // one block when its first cell is.
  constexpr int FULLC = WSX / 2;                      // chunks of a row with its x1 halo
  constexpr int HALOC = TX / 2;                       // chunks of an x2 halo row
  constexpr int CPV = C::TY * FULLC + 2 * NG * HALOC;  // chunks per variable
  constexpr int NSC = (5 * CPV + C::NTH - 1) / C::NTH;
  // shared element index (-1: none) with, for direct halo reads, the x/y direction
  // (dx + 1) + 3 (dy + 1) of its halo region in bits 16..19; element offset of the chunk
  // at plane 0 from the base of that region (see halo_elem)
  int sc_s[NSC], sc_g[NSC];
#pragma unroll
  for (int m = 0; m < NSC; ++m) {
    const int q = tid + C::NTH * m;
    sc_s[m] = -1;
    sc_g[m] = 0;
    if (q < 5 * CPV) {
      const int v = q / CPV;
      int r = q % CPV, x, y, s;
      if (r < C::TY * FULLC) {
        y = NG + r / FULLC;
        x = 2 * (r % FULLC) - ODD;
        s = NG * TX + (y - NG) * WSX + x + ODD;
      } else {
        r -= C::TY * FULLC;
        const int hr = r / HALOC;
        x = NG + 2 * (r % HALOC);
        y = hr < NG ? hr : hr + C::TY;
        s = y < NG ? y * TX + (x - NG) : NG * TX + C::TY * WSX + (y - NG - C::TY) * TX + (x - NG);
      }
      const int ip = i0 + x, jp = j0 + y;
      if (ip < g.p1 && jp < g.p2) {
        const int dx = ip < NG ? -1 : (ip >= NG + g.nx1 ? 1 : 0);
        const int dy = jp < NG ? -1 : (jp >= NG + g.nx2 ? 1 : 0);
        sc_s[m] = (v * NSTG + s) | (((dx + 1) + 3 * (dy + 1)) << 16);
        sc_g[m] = v * (int)vst + (NG * g.p2 + jp) * g.s1 + ip;
      }
    }
  }
  auto stage_plane = [&](int kp) {
    // direct halo reads: each chunk from the base of its halo region (x, y and the plane's
    // x3 direction)
    const int dz = kp < 0 ? -1 : (kp >= g.nx3 ? 1 : 0);
    const long long po = (long long)kp * pst;
#pragma unroll
    for (int m = 0; m < NSC; ++m) {
      if (sc_s[m] >= 0) {
        const long long base = direct ? nbr[(sc_s[m] >> 16) + 9 * (dz + 1)] : g.off;
        cp_async16(&stg[sc_s[m] & 0xffff], uin + (base + sc_g[m] + po));
      }
    }
  };
  // The columns' U_in and U0: NOWN / 2 chunks (two cells of a tile row) per variable.
  static_assert(NOWN % 2 == 0 && (NOWN / 2) % 32 == 0, "chunk rows per warp");
  const int ocy = (tid % (NOWN / 2)) / (TX / 2), ocx = 2 * (tid % (TX / 2));
  const int ocell = ocy * TX + ocx;
  const bool ochunk = tid < NOWN && i0 + ocx < g.nx1 && j0 + ocy < g.nx2;
  const int ooff = (NG * g.p2 + j0 + ocy + NG) * g.s1 + i0 + ocx + NG;  // from the block start
  // primitive recovery of the staged cells of this thread into the cross slot of plane kp
  auto convert_staged = [&](int kp) {
    float* dst = ring + xslot(kp) * 5 * NPL;
#pragma unroll
    for (int m = 0; m < NMY; ++m) {
      if (mypos[m] >= 0) {
        double u[5];
        float wv[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = stg[v * NSTG + mystg[m]];
        c2p(u, wv, bg, cn);
#pragma unroll
        for (int v = 0; v < 5; ++v) dst[v * NPL + mypos[m]] = wv[v];
      }
    }
  };
  const int tx = tid % TX, ty = tid / TX;
  const int ci = i0 + tx, cj = j0 + ty;
  const bool column = tid < NOWN;
  const bool own = column && ci < g.nx1 && cj < g.nx2;
  const int oc = (ty + NG) * WX + (tx + NG);
  const long long ecol = g.off + ((long long)NG * g.p2 + (cj + NG)) * g.s1 + (ci + NG);
  // direct load and conversion of plane kp (prologue) into its cross slot
  auto load_plane = [&](int kp) {
#pragma unroll
    for (int m = 0; m < NMY; ++m) {
      if (mypos[m] >= 0) {
        const int x = mypos[m] % WX, y = mypos[m] / WX;  // padded (i0 + x, j0 + y)
        const int ip = i0 + x, jp = j0 + y;
        const bool halo = ip < NG || ip >= NG + g.nx1 || jp < NG || jp >= NG + g.nx2 || kp < 0 ||
                          kp >= g.nx3;
        const double* src = (direct && halo)
                                ? uin + halo_elem(g, nbr, NG, ip, jp, kp)
                                : ub + ((long long)(kp + NG) * g.p2 + jp) * g.s1 + ip;
        double u[5];
        float wv[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = src[v * vst];
        c2p(u, wv, bg, cn);
        float* dst = ring + xslot(kp) * 5 * NPL;
#pragma unroll
        for (int v = 0; v < 5; ++v) dst[v * NPL + mypos[m]] = wv[v];
      }
    }
  };
  // the same for this column's own cell of plane kp into its column slot (prologue, the
  // planes below k0 - 1)
  auto load_column = [&](int kp) {
    if (column && ci < g.nx1 && cj < g.nx2) {
      const double* src = (direct && (kp < 0 || kp >= g.nx3))
                              ? uin + halo_elem(g, nbr, NG, ci + NG, cj + NG, kp)
                              : ub + ((long long)(kp + NG) * g.p2 + cj + NG) * g.s1 + ci + NG;
      double u[5];
      float wv[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) u[v] = src[v * vst];
      c2p(u, wv, bg, cn);
      float* dst = cring + cslot(kp) * 5 * NOWN;
#pragma unroll
      for (int v = 0; v < 5; ++v) dst[v * NOWN + tid] = wv[v];
    }
  };

  // ---- this thread's edge items, faces and column ---------------------------------------
  const int r1 = tid / C1, c1 = tid % C1;            // x1 item: cell (i0 - 1 + c1, j0 + r1)
  const int r2 = tid / TX, c2 = tid % TX;            // x2 item: cell (i0 + c2, j0 - 1 + r2)
  const int base1 = (r1 + NG) * WX + c1;             // stencil start in a ring plane (x)
  const int base2 = r2 * WX + c2 + NG;               // (y, stride WX)
  // x1 face to the right of x1 item t: i = i0 + c1 (between cells i0-1+c1 and i0+c1), row
  // j0 + r1; x2 face above x2 item t: j = j0 + r2, column i0 + c2
  const bool face1 = tid < NE && c1 < TX + 1 && i0 + c1 <= g.nx1 && j0 + r1 < g.nx2;
  const bool face2 = tid < NF && i0 + c2 < g.nx1 && j0 + r2 <= g.nx2;
  const int fl1 = r1 * (TX + 1) + c1;                // flux index of the x1 face
  const int ov1 = (FAST || !face1) ? -1
                                   : (i0 + c1 == 0 ? g.ovr[0] : (i0 + c1 == g.nx1 ? g.ovr[1] : -1));
  const int ov2 = (FAST || !face2) ? -1
                                   : (j0 + r2 == 0 ? g.ovr[2] : (j0 + r2 == g.nx2 ? g.ovr[3] : -1));

  // x3 edges of this column's cell kc: planes kc-NG+1 .. kc-1 from the column slots,
  // kc .. kc+NG-1 from the cross slots; then cell kc moves to its column slot
  auto x3_edges = [&](int kc, float* lo, float* hi) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      float q[2 * NG - 1];
#pragma unroll
      for (int m = 0; m < 2 * NG - 1; ++m) {
        const int kp = kc - NG + 1 + m;
        q[m] = m < NG - 1 ? cring[cslot(kp) * 5 * NOWN + v * NOWN + tid]
                          : ring[xslot(kp) * 5 * NPL + v * NPL + oc];
      }
      edges_t<NG, RC>(q, lo[v], hi[v]);
      cring[cslot(kc) * 5 * NOWN + v * NOWN + tid] = q[NG - 1];
    }
  };
  // PPM4 carries, from cell to cell of the column, the limited slope of cell kc (column
  // slot 0) and its lower interface value (slot 1), both computed for cell kc-1 already:
  // per cell one new slope and one new interface value instead of three and two, with
  // the same operations on the same operands (the same bits)
  constexpr bool CARRY = RC == AK_PPM4;
  auto x3_edges_carry = [&](int kc, float* lo, float* hi) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const float qc = ring[xslot(kc) * 5 * NPL + v * NPL + oc];
      const float qn = ring[xslot(kc + 1) * 5 * NPL + v * NPL + oc];
      const float sp = ppm_slope_v(qc, qn, ring[xslot(kc + 2) * 5 * NPL + v * NPL + oc]);
      float* cs = cring + v * NOWN + tid;
      float* ca = cring + 5 * NOWN + v * NOWN + tid;
      const float ahi = ppm_interface_v(qc, qn, *cs, sp);
      ppm_monotonize_v(*ca, ahi, qc, lo[v], hi[v]);
      *cs = sp;
      *ca = ahi;
    }
  };

  // ---- prologue: plane k0+NG staged; planes k0-NG .. k0+NG-1 loaded and converted (the
  //      lowest NG-1 into column slots), the upper x3 edge of cell k0-1 -----------------
  __syncthreads();  // the neighbour table
  stage_plane(k0 + NG);
  cp_async_commit();
  for (int kp = k0 - NG; kp < k0 - 1; ++kp) load_column(kp);
  for (int kp = k0 - 1; kp < k0 + NG; ++kp) load_plane(kp);
  __syncthreads();
  float hi3[5], f3lo[5];  // upper x3 edge of cell k-1; flux through the face below cell k-1
  if (column) {
    float lo_a[5];
    x3_edges(k0 - 1, lo_a, hi3);
    if constexpr (CARRY) {  // column slots from planes to the carried slope and interface
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const float qm2 = cring[cslot(k0 - 2) * 5 * NOWN + v * NOWN + tid];
        const float qm1 = ring[xslot(k0 - 1) * 5 * NPL + v * NPL + oc];
        const float q0 = ring[xslot(k0) * 5 * NPL + v * NPL + oc];
        const float q1 = ring[xslot(k0 + 1) * 5 * NPL + v * NPL + oc];
        const float sm = ppm_slope_v(qm2, qm1, q0), s0 = ppm_slope_v(qm1, q0, q1);
        cring[v * NOWN + tid] = s0;
        cring[5 * NOWN + v * NOWN + tid] = ppm_interface_v(qm1, q0, sm, s0);
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();

  float dtmin_f = __int_as_float(0x7f800000);
  for (int k = k0;; ++k) {
    const bool plane = k < k1;  // plane k is in this CTA's segment
    if (plane) convert_staged(k + NG);  // staged during the previous P2 (or the prologue)
    // ---- P1: x1/x2 edges of plane k (paired); x3 edge of cell k and the face below it;
    //      update of plane k-1 ---------------------------------------------------------
    float2 hi12[5];  // upper edges of this thread's x1 and x2 items, for its faces in P2
    if (plane && tid < NE) {
      const float* pl = ring + xslot(k) * 5 * NPL;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        float2 q[2 * NG - 1];
#pragma unroll
        for (int m = 0; m < 2 * NG - 1; ++m)
          q[m] = make_float2(pl[v * NPL + base1 + m], pl[v * NPL + base2 + m * WX]);
        float2 lo;
        if constexpr (RC == AK_PLM) {
          plm_edges_v(q[0], q[1], q[2], lo, hi12[v]);
        } else if constexpr (RC == AK_PPM4) {
          ppm_edges_v(q[0], q[1], q[2], q[3], q[4], lo, hi12[v]);
        } else {
          // WENO-Z and PPMX: one item at a time (their limiters branch per value)
          float qa[2 * NG - 1], qb[2 * NG - 1];
#pragma unroll
          for (int m = 0; m < 2 * NG - 1; ++m) {
            qa[m] = q[m].x;
            qb[m] = q[m].y;
          }
          edges_t<NG, RC>(qa, lo.x, hi12[v].x);
          edges_t<NG, RC>(qb, lo.y, hi12[v].y);
        }
        e1lo[v * NE + tid] = lo.x;
        e2lo[v * NE + tid] = lo.y;
      }
    }
    if (column) {
      float lo3[5], hi3k[5], f3hi[5];  // f3hi: the face between cells k-1 and k
      if constexpr (CARRY)
        x3_edges_carry(k, lo3, hi3k);
      else
        x3_edges(k, lo3, hi3k);
      if (!FAST && k == 0 && g.ovr[4] >= 0)
        corrected_flux(md.fcbuf, g.ovr[4] + cj * g.nx1 + ci, f3hi);
      else if (!FAST && k == g.nx3 && g.ovr[5] >= 0)
        corrected_flux(md.fcbuf, g.ovr[5] + cj * g.nx1 + ci, f3hi);
      else if (FAST) {
        // x3 face: (rho, v3; v1, v2, u_g)
        const float wl3[5] = {hi3[0], hi3[3], hi3[1], hi3[2], hi3[4]};
        const float wr3[5] = {lo3[0], lo3[3], lo3[1], lo3[2], lo3[4]};
        float fn3[5];
        hllc_mixed(wl3, wr3, bg, fn3);
        f3hi[0] = fn3[0];
        f3hi[3] = fn3[1];
        f3hi[1] = fn3[2];
        f3hi[2] = fn3[3];
        f3hi[4] = fn3[4];
      } else
        solve(2, hi3, lo3, bg, f3hi);
#pragma unroll
      for (int v = 0; v < 5; ++v) hi3[v] = hi3k[v];
      // ---- divergence, RK update and CFL of cell k-1 (fluxes of the previous P2) -----
      if (own && k > k0) {
        const int kc = k - 1;
        const long long e = ecol + kc * pst;
        double un[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const float d1 = f1[v * NF + ty * (TX + 1) + tx + 1] - f1[v * NF + ty * (TX + 1) + tx];
          const float d2 = f2[v * NF + (ty + 1) * TX + tx] - f2[v * NF + ty * TX + tx];
          const float d3 = f3hi[v] - f3lo[v];
          const float L = -fmaf(d1, idx1f, fmaf(d2, idx2f, d3 * idx3f));
          const double r =
              rk_update_mixed(form, a, b, dt, L, ucol[v * NOWN + tid], ucol[(5 + v) * NOWN + tid]);
          un[v] = r;
          uout[e + v * vst] = r;
        }
        if (fofc) {
          const int fi = fofc_flag(un, md, sc, w.block, g, ci, cj, kc);
          if (fi >= 0 && form != 0) {
#pragma unroll
            for (int v = 0; v < 5; ++v) md.fu0[(long long)fi * 5 + v] = ucol[(5 + v) * NOWN + tid];
          }
        }
        if (last_stage) {
          // CFL ratio in FP32: it only sets the next step's dt
          const float rho = fmaxf(f64_to_f32(un[0]), (float)AK_RHO_FLOOR);
          const float ir = rcp_approx_f32(rho);
          const float m1 = f64_to_f32(un[1]), m2 = f64_to_f32(un[2]), m3 = f64_to_f32(un[3]);
          const float ug = fmaxf(fmaf(-0.5f * ir, fmaf(m1, m1, fmaf(m2, m2, m3 * m3)),
                                      f64_to_f32(un[4])), (float)AK_UG_FLOOR);
          const float cs = sqrt_fast(bg.gamma_f * (bg.gamma_f - 1.0f) * ug * ir);
          float lam = fmaf(fabsf(m1), ir, cs) * idx1f;
          lam = fmaxf(lam, fmaf(fabsf(m2), ir, cs) * idx2f);
          lam = fmaxf(lam, fmaf(fabsf(m3), ir, cs) * idx3f);
          dtmin_f = fminf(dtmin_f, rcp_approx_f32(lam));
        }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) f3lo[v] = f3hi[v];
    }
    if (!plane) break;
    __syncthreads();  // Y: lower edges, plane k+NG; the update's reads of fluxes and U_in / U0

    if (k + 1 < k1) stage_plane(k + NG + 1);
    cp_async_commit();
    if (ochunk) {
      // column thread t copies, for the row chunk (ocy, ocx), the arrays/variables
      // vv = t / 128 + 2 m (U_in for vv < 5, U0 above): 5 x 2 x 128 chunks in all
      const long long po = g.off + ooff + k * pst;
#pragma unroll
      for (int m = 0; m < 10 * NOWN / 2 / NOWN; ++m) {
        const int vv = tid / (NOWN / 2) + 2 * m;
        if (vv < 5)
          cp_async16(&ucol[vv * NOWN + ocell], uin + po + vv * vst);
        else if (need_u0)
          cp_async16(&ucol[vv * NOWN + ocell], u0 + po + (vv - 5) * vst);
      }
    }
    cp_async_commit();

    // ---- P2: the x1 face right of this thread's x1 item and the x2 face above its x2
    //      item, paired: upper edges from registers, lower ones of the neighbour items -----
    if (tid < NE) {
      // x1 face: (rho, v1; v2, v3, u_g); x2 face: (rho, v2; v3, v1, u_g)
      constexpr int P2[5] = {0, 2, 3, 1, 4};
      // neighbour items (clamped for the threads without that face; their lane is unused)
      const int n1 = c1 < TX + 1 ? tid + 1 : tid;
      const int n2 = tid < NF ? tid + TX : tid;
      float2 wl[5], wr[5], fn[5];
#pragma unroll
      for (int n = 0; n < 5; ++n) {
        wl[n] = make_float2(hi12[n].x, hi12[P2[n]].y);
        wr[n] = make_float2(e1lo[n * NE + n1], e2lo[P2[n] * NE + n2]);
      }
      if (hllc) {
        hllc_mixed(wl, wr, bg, fn);  // both faces in the two lanes
      } else {
        // HLLE / LLF: one face at a time (their packed form did not reproduce the
        // scalar bits of the flux-correction and unpaired kernels)
        float la[5], ra[5], lb[5], rb[5], ga[5], gb[5];
#pragma unroll
        for (int n = 0; n < 5; ++n) {
          la[n] = wl[n].x;
          ra[n] = wr[n].x;
          lb[n] = wl[n].y;
          rb[n] = wr[n].y;
        }
        riemann(la, ra, bg, ga);
        riemann(lb, rb, bg, gb);
#pragma unroll
        for (int n = 0; n < 5; ++n) fn[n] = make_float2(ga[n], gb[n]);
      }
      float fa[5], fb[5];
#pragma unroll
      for (int n = 0; n < 5; ++n) {
        fa[n] = fn[n].x;
        fb[P2[n]] = fn[n].y;
      }
      if (ov1 >= 0) corrected_flux(md.fcbuf, ov1 + k * g.nx2 + j0 + r1, fa);
      if (ov2 >= 0) corrected_flux(md.fcbuf, ov2 + k * g.nx1 + i0 + c2, fb);
      if (c1 < TX + 1) {
#pragma unroll
        for (int v = 0; v < 5; ++v) f1[v * NF + fl1] = fa[v];
      }
      if (tid < NF) {
#pragma unroll
        for (int v = 0; v < 5; ++v) f2[v * NF + tid] = fb[v];
      }
    }
    cp_async_wait<0>();
    __syncthreads();  // X: fluxes, the staged plane and the columns' U_in / U0
  }

  if (last_stage) {
    double dtmin = f32_to_f64(dtmin_f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dtmin = fmin(dtmin, __shfl_xor_sync(0xffffffffu, dtmin, o));
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = dtmin;
    __syncthreads();
    if (tid < 32) {
      double v = tid < C::NTH / 32 ? red[tid] : __longlong_as_double(0x7ff0000000000000ll);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (tid == 0) atomicMin(&sc->dtmin_bits, (unsigned long long)__double_as_longlong(v));
    }
  }
  if constexpr (PERSIST) __syncthreads();  // the next tile reuses the shared memory
  }
}

using mx_kern_t = void (*)(const double*, const double*, double*, ak_meshdev, const ak_work*, Bg,
                           double, double, int, ak_dev_scalars*, int, int);

template <int NG, int RC, int FORM, int LAST>
void launch_fast(const ak_mesh* m, size_t smem, const double* uin, const double* u0,
                 double* uout, const Bg& bg, double a, double b, int form, int last_stage) {
  stage_mx_kernel<NG, RC, 16, false, FORM, LAST, true>
      <<<(unsigned)m->nwork, MxCfg<NG, 16>::NTH, smem, m->stream>>>(
          uin, u0, uout, m->md, m->d_work, bg, a, b, form, m->d_sc, last_stage, m->nwork);
}

template <int NG, int RC>
cudaError_t launch_paired(const ak_mesh* m, const double* uin, const double* u0, double* uout,
                          const Bg& bg, double a, double b, int form, int last_stage,
                          bool prepare_only) {
  using C = MxCfg<NG, 16>;
  const mx_kern_t kern = stage_mx_kernel<NG, RC, 16>;
  const mx_kern_t pk = stage_mx_kernel<NG, RC, 16, true>;
  if (prepare_only) {
    const mx_kern_t fast[6] = {
        stage_mx_kernel<NG, RC, 16, false, 0, 0, true>, stage_mx_kernel<NG, RC, 16, false, 1, 0, true>,
        stage_mx_kernel<NG, RC, 16, false, 2, 0, true>, stage_mx_kernel<NG, RC, 16, false, 0, 1, true>,
        stage_mx_kernel<NG, RC, 16, false, 1, 1, true>, stage_mx_kernel<NG, RC, 16, false, 2, 1, true>};
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::bytes);
    for (int i = 0; i < 6 && e == cudaSuccess; ++i)
      e = cudaFuncSetAttribute(fast[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::bytes);
    return e;
  }
  if (m->fused)
    return launch_persistent(m, pk, C::NTH, C::bytes, uin, u0, uout, m->md, m->d_work, bg, a, b,
                             form, m->d_sc, last_stage, m->nwork);
  // the common case: one level read through direct halo reads, HLLC, no FOFC
  if (m->md.direct && !m->md.fofc && bg.rsolver == AK_HLLC && m->nfc == 0) {
    const int key = form + 3 * (last_stage ? 1 : 0);
    switch (key) {
      case 0: launch_fast<NG, RC, 0, 0>(m, C::bytes, uin, u0, uout, bg, a, b, form, last_stage); break;
      case 1: launch_fast<NG, RC, 1, 0>(m, C::bytes, uin, u0, uout, bg, a, b, form, last_stage); break;
      case 2: launch_fast<NG, RC, 2, 0>(m, C::bytes, uin, u0, uout, bg, a, b, form, last_stage); break;
      case 3: launch_fast<NG, RC, 0, 1>(m, C::bytes, uin, u0, uout, bg, a, b, form, last_stage); break;
      case 4: launch_fast<NG, RC, 1, 1>(m, C::bytes, uin, u0, uout, bg, a, b, form, last_stage); break;
      default: launch_fast<NG, RC, 2, 1>(m, C::bytes, uin, u0, uout, bg, a, b, form, last_stage); break;
    }
    return cudaGetLastError();
  }
  kern<<<(unsigned)m->nwork, C::NTH, C::bytes, m->stream>>>(uin, u0, uout, m->md, m->d_work, bg,
                                                            a, b, form, m->d_sc, last_stage,
                                                            m->nwork);
  return cudaGetLastError();
}

}  // namespace mx
}  // namespace ak
