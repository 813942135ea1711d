// The fused hydro stage kernel: primitive recovery, reconstruction in x1/x2/x3, HLLC
// at every face, flux divergence and the RK stage update of AthenaK's Godunov scheme
// (arXiv 2409.16053, Section 3 Eq. (1), Section 3.1 Eq. (4)), plus the CFL minimum of
// Section 3 Eq. (3) on the last stage.
//
// Work decomposition (one launch covers every MeshBlock, as Section 2's MeshBlockPack
// does): a CTA owns a TX x TY column tile of one block and marches along x3 over a
// segment of planes.  A ring of 2*NG planes of primitives (tile plus NG halo cells in
// x1 and x2) lives in shared memory; each plane is loaded from HBM and converted once.
// x1 and x2 faces of the current plane are solved from the ring and their fluxes kept
// in shared memory; the x3 face above each column is solved by the column's thread,
// which carries the flux of the face below from the previous plane.  Every face of a
// tile is solved once; faces on tile edges are solved by both tiles with identical
// inputs, so they agree bit for bit and the update stays conservative.
#include <type_traits>

#include "ak_internal.cuh"
#include "hydro_ops.cuh"

namespace ak {

struct Counters {
  unsigned long long* floors;
  unsigned long long* nonfinite;
};

__device__ __forceinline__ void count(unsigned long long* c) { atomicAdd(c, 1ull); }

// Conserved -> primitive (Section 3.1 Eq. (4)), FP64 form.
__device__ __forceinline__ void c2p(const double* u, double* w, const Bg&, Counters cn) {
  double rho = u[0];
  if (!(rho == rho) || !(u[4] == u[4])) count(cn.nonfinite);
  if (!(rho >= AK_RHO_FLOOR)) {
    rho = AK_RHO_FLOOR;
    count(cn.floors);
  }
  const double v1 = u[1] / rho, v2 = u[2] / rho, v3 = u[3] / rho;
  double ug = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / rho;
  if (!(ug >= AK_UG_FLOOR)) {
    ug = AK_UG_FLOOR;
    count(cn.floors);
  }
  w[0] = rho;
  w[1] = v1;
  w[2] = v2;
  w[3] = v3;
  w[4] = ug;
}

// Conserved -> primitive, mixed form: the internal-energy recovery
// u_g = E - |M|^2 / (2 rho) and the background subtraction run in FP64; the
// deviations W' are rounded to FP32.
__device__ __forceinline__ void c2p(const double* u, float* w, const Bg& bg, Counters cn) {
  double rho = u[0];
  if (!(rho == rho) || !(u[4] == u[4])) count(cn.nonfinite);
  if (!(rho >= AK_RHO_FLOOR)) {
    rho = AK_RHO_FLOOR;
    count(cn.floors);
  }
  const double r = 1.0 / rho;
  double ug = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * r;
  if (!(ug >= AK_UG_FLOOR)) {
    ug = AK_UG_FLOOR;
    count(cn.floors);
  }
  w[0] = (float)(rho - bg.rho);
  w[1] = (float)(u[1] * r);
  w[2] = (float)(u[2] * r);
  w[3] = (float)(u[3] * r);
  w[4] = (float)(ug - bg.ug);
}

__device__ __forceinline__ void riemann(const double* wl, const double* wr, const Bg& bg,
                                        double* f) {
  hllc_fp64(wl, wr, bg.gamma, f);
}
__device__ __forceinline__ void riemann(const float* wl, const float* wr, const Bg& bg,
                                        float* f) {
  hllc_mixed(wl, wr, bg, f);
}

// Left/right states at the face between q[NG-1] and q[NG] of a stencil of 2*NG cells.
template <int NG, typename R>
__device__ __forceinline__ void face_states(const R* q, R& left, R& right) {
  if constexpr (NG == 2) {
    left = q[1] + R(0.5) * plm_slope(q[0], q[1], q[2]);
    right = q[2] - R(0.5) * plm_slope(q[1], q[2], q[3]);
  } else {
    R lo, hi, lo2, hi2;
    ppm_edges(q[0], q[1], q[2], q[3], q[4], lo, hi);
    ppm_edges(q[1], q[2], q[3], q[4], q[5], lo2, hi2);
    left = hi;
    right = lo2;
  }
}

// Solves one face of direction d.  `cellv(v, m)` returns variable v of the m-th cell
// of the stencil (m = 0 .. 2NG-1; the face lies between m = NG-1 and m = NG).
template <int NG, typename R, typename Get>
__device__ __forceinline__ void solve_face(int d, const Bg& bg, Get cellv, R* f) {
  const int perm[5] = {0, 1 + d, 1 + (d + 1) % 3, 1 + (d + 2) % 3, 4};
  R wl[5], wr[5];
#pragma unroll
  for (int n = 0; n < 5; ++n) {
    R q[2 * NG];
#pragma unroll
    for (int m = 0; m < 2 * NG; ++m) q[m] = cellv(perm[n], m);
    face_states<NG>(q, wl[n], wr[n]);
  }
  R fn[5];
  riemann(wl, wr, bg, fn);
#pragma unroll
  for (int n = 0; n < 5; ++n) f[perm[n]] = fn[n];
}

template <int NG, bool MIXED, int TX, int TY>
__global__ void __launch_bounds__(TX* TY)
    stage_kernel(const double* __restrict__ uin, const double* u0, double* uout, ak_geom g,
                 Bg bg, double a, double b, ak_dev_scalars* sc, int nseg, int last_stage) {
  using R = typename std::conditional<MIXED, float, double>::type;
  constexpr int NT = TX * TY;
  constexpr int WX = TX + 2 * NG, WY = TY + 2 * NG, NPL = WX * WY;
  constexpr int NR = 2 * NG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* ring = reinterpret_cast<R*>(smem_raw);  // [NR][5][WY][WX]
  R* f1 = ring + NR * 5 * NPL;               // [5][TY][TX+1]
  R* f2 = f1 + 5 * TY * (TX + 1);            // [5][TY+1][TX]
  __shared__ double red[NT / 32];

  const int tid = threadIdx.x;
  const int ntx = (g.nx1 + TX - 1) / TX, nty = (g.nx2 + TY - 1) / TY;
  int bid = blockIdx.x;
  const int tile_x = bid % ntx;
  bid /= ntx;
  const int tile_y = bid % nty;
  bid /= nty;
  const int seg = bid % nseg;
  const int blk = bid / nseg;
  const int i0 = tile_x * TX, j0 = tile_y * TY;
  const int kseg = (g.nx3 + nseg - 1) / nseg;
  const int k0 = seg * kseg;
  const int k1 = min(g.nx3, k0 + kseg);
  if (k0 >= k1) return;

  const long long boff = (long long)blk * g.block_stride;
  const double* ub = uin + boff;
  const Counters cn{&sc->counters[0], &sc->counters[1]};
  const double dt = sc->dt;
  const double idx1 = 1.0 / g.dx1, idx2 = 1.0 / g.dx2, idx3 = 1.0 / g.dx3;

  auto plane_slot = [](int k) { return (k + 4 * NR) % NR; };
  // Load plane kp (interior index, may be a ghost plane) of the halo'd tile, convert to
  // primitives and store in its ring slot.
  auto load_plane = [&](int kp) {
    R* dst = ring + plane_slot(kp) * 5 * NPL;
    for (int c = tid; c < NPL; c += NT) {
      const int x = c % WX, y = c / WX;
      const int ip = i0 + x, jp = j0 + y;  // padded indices (halo starts at i0 - NG)
      if (ip < g.p1 && jp < g.p2) {
        const long long e = ((long long)(kp + NG) * g.p2 + jp) * g.p1 + ip;
        double u[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = ub[e + v * g.var_stride];
        R w[5];
        c2p(u, w, bg, cn);
#pragma unroll
        for (int v = 0; v < 5; ++v) dst[v * NPL + c] = w[v];
      }
    }
  };

  // own column of this thread
  const int tx = tid % TX, ty = tid / TX;
  const int ci = i0 + tx, cj = j0 + ty;
  const bool own = (ci < g.nx1) && (cj < g.nx2);
  const int oc = (ty + NG) * WX + (tx + NG);  // own cell inside a ring plane

  // x3 face below plane k (between k-1 and k): stencil planes k-NG .. k+NG-1
  auto x3_face = [&](int k, R* f) {
    solve_face<NG, R>(2, bg,
                      [&](int v, int m) {
                        return ring[plane_slot(k - NG + m) * 5 * NPL + v * NPL + oc];
                      },
                      f);
  };

  // prologue: planes k0-NG .. k0+NG-1, and the flux through the face below k0
  for (int kp = k0 - NG; kp < k0 + NG; ++kp) load_plane(kp);
  __syncthreads();
  R f3m[5], f3p[5];
  if (own) x3_face(k0, f3m);

  double dtmin = __longlong_as_double(0x7ff0000000000000ll);  // +inf
  for (int k = k0; k < k1; ++k) {
    // the ring now holds planes k-NG .. k+NG-1; bring in k+NG (replaces k-NG)
    __syncthreads();
    load_plane(k + NG);
    __syncthreads();
    const R* pl = ring + plane_slot(k) * 5 * NPL;
    // x1 faces of plane k: (TX+1) x TY
    for (int f = tid; f < (TX + 1) * TY; f += NT) {
      const int fx = f % (TX + 1), fy = f / (TX + 1);
      if (i0 + fx <= g.nx1 && j0 + fy < g.nx2) {
        R fl[5];
        const int base = (fy + NG) * WX + fx;  // stencil cell m at x = fx + m
        solve_face<NG, R>(0, bg, [&](int v, int m) { return pl[v * NPL + base + m]; }, fl);
#pragma unroll
        for (int v = 0; v < 5; ++v) f1[(v * TY + fy) * (TX + 1) + fx] = fl[v];
      }
    }
    // x2 faces of plane k: TX x (TY+1)
    for (int f = tid; f < TX * (TY + 1); f += NT) {
      const int fx = f % TX, fy = f / TX;
      if (i0 + fx < g.nx1 && j0 + fy <= g.nx2) {
        R fl[5];
        const int base = fy * WX + fx + NG;  // stencil cell m at y = fy + m
        solve_face<NG, R>(1, bg, [&](int v, int m) { return pl[v * NPL + base + m * WX]; },
                          fl);
#pragma unroll
        for (int v = 0; v < 5; ++v) f2[(v * (TY + 1) + fy) * TX + fx] = fl[v];
      }
    }
    // x3 face above plane k
    if (own) x3_face(k + 1, f3p);
    __syncthreads();

    if (own) {
      const long long e = boff + ((long long)(k + NG) * g.p2 + (cj + NG)) * g.p1 + (ci + NG);
      double un[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const R d1 = f1[(v * TY + ty) * (TX + 1) + tx + 1] - f1[(v * TY + ty) * (TX + 1) + tx];
        const R d2 = f2[(v * (TY + 1) + ty + 1) * TX + tx] - f2[(v * (TY + 1) + ty) * TX + tx];
        const R d3 = f3p[v] - f3m[v];
        double L;
        if constexpr (MIXED) {
          L = (double)(-(d1 * (float)idx1 + d2 * (float)idx2 + d3 * (float)idx3));
        } else {
          L = -(d1 * idx1 + d2 * idx2 + d3 * idx3);
        }
        const double ui = uin[e + v * g.var_stride];
        double r = ui + dt * L;
        if (a != 0.0) r = a * u0[e + v * g.var_stride] + b * r;
        un[v] = r;
        uout[e + v * g.var_stride] = r;
        f3m[v] = f3p[v];
      }
      if (last_stage) {
        // CFL ratio of the new state (Eq. (3)); floors applied silently here
        double rho = un[0];
        rho = rho >= AK_RHO_FLOOR ? rho : AK_RHO_FLOOR;
        const double v1 = un[1] / rho, v2 = un[2] / rho, v3 = un[3] / rho;
        double ug = un[4] - 0.5 * (un[1] * un[1] + un[2] * un[2] + un[3] * un[3]) / rho;
        ug = ug >= AK_UG_FLOOR ? ug : AK_UG_FLOOR;
        const double cs = sqrt(g.gamma * (g.gamma - 1.0) * ug / rho);
        double t = g.dx1 / (fabs(v1) + cs);
        t = fmin(t, g.dx2 / (fabs(v2) + cs));
        t = fmin(t, g.dx3 / (fabs(v3) + cs));
        dtmin = fmin(dtmin, t);
      }
    }
  }

  if (last_stage) {
    // CTA min of the CFL ratio -> one atomic per CTA (positive doubles order as their
    // bit patterns)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dtmin = fmin(dtmin, __shfl_xor_sync(0xffffffffu, dtmin, o));
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
}

template <int NG, bool MIXED, int TX, int TY>
static cudaError_t launch(const ak_mesh* m, const double* uin, const double* u0, double* uout,
                          double a, double b, int last_stage, bool prepare_only = false) {
  using R = typename std::conditional<MIXED, float, double>::type;
  constexpr int NPL = (TX + 2 * NG) * (TY + 2 * NG);
  const size_t smem = sizeof(R) * (2 * NG * 5 * NPL + 5 * TY * (TX + 1) + 5 * (TY + 1) * TX);
  auto kern = stage_kernel<NG, MIXED, TX, TY>;
  if (prepare_only)
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const ak_geom& g = m->geom;
  const int ntx = (g.nx1 + TX - 1) / TX, nty = (g.nx2 + TY - 1) / TY;
  const long long nblk = (long long)g.nblocks * ntx * nty * m->seg3;
  Bg bg;
  bg.gamma = g.gamma;
  bg.gamma_f = (float)g.gamma;
  bg.rho = m->desc.ref_rho;
  bg.ug = m->desc.ref_p / (g.gamma - 1.0);
  bg.rho_f = (float)bg.rho;
  bg.ug_f = (float)bg.ug;
  kern<<<(unsigned)nblk, TX * TY, smem, m->stream>>>(uin, u0, uout, g, bg, a, b, m->d_sc,
                                                      m->seg3, last_stage);
  return cudaGetLastError();
}

}  // namespace ak

cudaError_t ak_launch_stage(const ak_mesh* m, int stage, const double* u_in, const double* u0,
                            double* u_out, int last_stage) {
  static const double a2[2] = {0.0, 0.5}, b2[2] = {1.0, 0.5};
  static const double a3[3] = {0.0, 0.75, 1.0 / 3.0}, b3[3] = {1.0, 0.25, 2.0 / 3.0};
  const bool rk3 = m->desc.rk == 3;
  const double a = rk3 ? a3[stage - 1] : a2[stage - 1];
  const double b = rk3 ? b3[stage - 1] : b2[stage - 1];
  const bool mixed = m->desc.precision == AK_MIXED;
  if (m->desc.recon == AK_PLM) {
    return mixed ? ak::launch<2, true, 16, 16>(m, u_in, u0, u_out, a, b, last_stage)
                 : ak::launch<2, false, 16, 16>(m, u_in, u0, u_out, a, b, last_stage);
  }
  return mixed ? ak::launch<3, true, 16, 16>(m, u_in, u0, u_out, a, b, last_stage)
               : ak::launch<3, false, 16, 16>(m, u_in, u0, u_out, a, b, last_stage);
}

// Raises the dynamic shared-memory limit of the stage kernel this mesh uses (called once
// at mesh creation, outside any stream capture).
cudaError_t ak_stage_prepare(const ak_mesh* m) {
  const bool mixed = m->desc.precision == AK_MIXED;
  if (m->desc.recon == AK_PLM)
    return mixed ? ak::launch<2, true, 16, 16>(m, 0, 0, 0, 0, 0, 0, true)
                 : ak::launch<2, false, 16, 16>(m, 0, 0, 0, 0, 0, 0, true);
  return mixed ? ak::launch<3, true, 16, 16>(m, 0, 0, 0, 0, 0, 0, true)
               : ak::launch<3, false, 16, 16>(m, 0, 0, 0, 0, 0, 0, true);
}
