// Device building blocks shared by the stage kernels and the flux-correction kernel:
// primitive recovery (Section 3.1, Eq. (4)), reconstruction edges, the direction
// permutation around the Riemann solver, and the corrected coarse-face fluxes of
// static refinement.
#pragma once

#include <type_traits>
#include <utility>

#include "ak_internal.cuh"
#include "hydro_ops.cuh"
#include "exchange.cuh"

namespace ak {

struct Counters {
  unsigned long long* floors;
  unsigned long long* nonfinite;
};

__device__ __forceinline__ void count(unsigned long long* c) { atomicAdd(c, 1ull); }

// Bit-level tests that keep comparisons of doubles off the FP64 pipe.
__device__ __forceinline__ bool not_finite(double x) {
  return ((unsigned)__double2hiint(x) & 0x7ff00000u) == 0x7ff00000u;
}
// x >= floor for a positive, finite `floor` (false for negative x and NaN-free x < floor)
__device__ __forceinline__ bool at_least(double x, double floor) {
  return __double_as_longlong(x) >= __double_as_longlong(floor);
}

// Conserved -> primitive (Section 3.1 Eq. (4)), FP64 form.
__device__ __forceinline__ void c2p(const double* u, double* w, const Bg&, Counters cn) {
  double rho = u[0];
  if (not_finite(rho) || not_finite(u[4])) count(cn.nonfinite);
  if (!at_least(rho, AK_RHO_FLOOR)) {
    rho = AK_RHO_FLOOR;
    count(cn.floors);
  }
  const double r = rcp64(rho);
  const double v1 = u[1] * r, v2 = u[2] * r, v3 = u[3] * r;
  double ug = fma(-0.5, fma(u[1], v1, fma(u[2], v2, u[3] * v3)), u[4]);
  if (!at_least(ug, AK_UG_FLOOR)) {
    ug = AK_UG_FLOOR;
    count(cn.floors);
  }
  w[0] = rho;
  w[1] = v1;
  w[2] = v2;
  w[3] = v3;
  w[4] = ug;
}

// Conserved -> primitive, mixed form (floors: bg.rho_min and bg.ug_floor_f, the
// absolute floors raised to 2^-20 of the background).  The internal-energy recovery runs in FP64 with
// the cancellation done before any division: 2 rho (u_g - u_g,b) = 2 rho (E - u_g,b) -
// |M|^2 is formed in FP64, rounded to FP32 and only then divided by 2 rho (FP32
// reciprocal), so u_g - u_g,b keeps FP32 relative precision whatever the Mach number,
// without an FP64 reciprocal.  rho - rho_b is an FP64 difference; velocities come from
// FP32 arithmetic; the deviations W' are rounded to FP32 on the integer pipe.
__device__ __forceinline__ void c2p(const double* u, float* w, const Bg& bg, Counters cn) {
  double rho = u[0];
  if (not_finite(rho) || not_finite(u[4])) count(cn.nonfinite);
  if (!at_least(rho, bg.rho_min)) {
    rho = bg.rho_min;
    count(cn.floors);
  }
  const float rhof = f64_to_f32(rho);
  float rf = rcp_approx_f32(rhof);
  rf = fmaf(rf, fmaf(-rhof, rf, 1.0f), rf);
  const double m2 = fma(u[1], u[1], fma(u[2], u[2], u[3] * u[3]));
  // 2 rho (u_g - u_g,b); rho >= its floor is normal, so 2 rho is an exponent increment
  const double num2 = fma(u[4] - bg.ug, dscale(rho, 1), -m2);
  float dugf = f64_to_f32(num2) * (0.5f * rf);
  if (!(dugf >= bg.ug_floor_f)) {           // u_g below its floor (FP32 resolution)
    dugf = bg.ug_floor_f;
    count(cn.floors);
  }
  w[0] = f64_to_f32(rho - bg.rho);
  w[1] = f64_to_f32(u[1]) * rf;
  w[2] = f64_to_f32(u[2]) * rf;
  w[3] = f64_to_f32(u[3]) * rf;
  w[4] = dugf;
}

// FP64 primitive recovery with IEEE division in the plain order of Eq. (4), for the
// reconstructions that can overshoot (WENO-Z, PPMX): there the sign of a reconstructed
// face pressure near zero decides which faces FOFC corrects, so their primitives carry
// the bits of the definition rather than those of the Newton reciprocal.
__device__ __forceinline__ void c2p_exact(const double* u, double* w, const Bg&, Counters cn) {
  double rho = u[0];
  if (not_finite(rho) || not_finite(u[4])) count(cn.nonfinite);
  if (!(rho >= AK_RHO_FLOOR)) {
    rho = AK_RHO_FLOOR;
    count(cn.floors);
  }
  w[1] = u[1] / rho;
  w[2] = u[2] / rho;
  w[3] = u[3] / rho;
  double ug = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / rho;
  if (!(ug >= AK_UG_FLOOR)) {
    ug = AK_UG_FLOOR;
    count(cn.floors);
  }
  w[0] = rho;
  w[4] = ug;
}
// primitive recovery of the stage kernels: EXACT selects c2p_exact in the FP64 form
template <bool EXACT>
__device__ __forceinline__ void c2p_t(const double* u, double* w, const Bg& bg, Counters cn) {
  if constexpr (EXACT)
    c2p_exact(u, w, bg, cn);
  else
    c2p(u, w, bg, cn);
}
template <bool EXACT>
__device__ __forceinline__ void c2p_t(const double* u, float* w, const Bg& bg, Counters cn) {
  c2p(u, w, bg, cn);
}

// The Riemann solver of the mesh (one choice per launch, a uniform branch); NANCHK:
// NaN flux for a face state without a sound speed (FP64 form)
template <bool NANCHK = false>
__device__ __forceinline__ void riemann(const double* wl, const double* wr, const Bg& bg,
                                        double* f) {
  if (bg.rsolver == AK_HLLE)
    hlle_fp64<NANCHK>(wl, wr, bg, f);
  else if (bg.rsolver == AK_LLF)
    llf_fp64<NANCHK>(wl, wr, bg, f);
  else
    hllc_fp64<NANCHK>(wl, wr, bg, f);
}
template <bool NANCHK = false, typename V>
__device__ __forceinline__ void riemann(const V* wl, const V* wr, const Bg& bg, V* f) {
  if (bg.rsolver == AK_HLLE)
    hlle_mixed(wl, wr, bg, f);
  else if (bg.rsolver == AK_LLF)
    llf_mixed(wl, wr, bg, f);
  else
    hllc_mixed(wl, wr, bg, f);
}

// Lower and upper edge values of the middle cell of q[0 .. 2NG-2] for the
// reconstruction RC (NG = 2: PLM; NG = 3: AK_PPM4, AK_WENOZ or AK_PPMX).
template <int NG, int RC, typename R>
__device__ __forceinline__ void edges_t(const R* q, R& lo, R& hi) {
  if constexpr (NG == 3 && RC == AK_WENOZ) {
    if constexpr (std::is_same<R, double>::value) {
      hi = wenoz_value_fp64(q[0], q[1], q[2], q[3], q[4]);
      lo = wenoz_value_fp64(q[4], q[3], q[2], q[1], q[0]);
    } else {
      wenoz_edges(q[0], q[1], q[2], q[3], q[4], lo, hi);
    }
  } else if constexpr (NG == 3 && RC == AK_PPMX) {
    ppmx_edges(q[0], q[1], q[2], q[3], q[4], lo, hi);
  } else if constexpr (std::is_same<R, float>::value) {
    if constexpr (NG == 2)
      plm_edges_v(q[0], q[1], q[2], lo, hi);
    else
      ppm_edges_v(q[0], q[1], q[2], q[3], q[4], lo, hi);
  } else if constexpr (NG == 2) {
    plm_edges_fp64(q[1] - q[0], q[2] - q[1], q[1], lo, hi);
  } else {
    ppm_edges_fp64(q[0], q[1], q[2], q[3], q[4], lo, hi);
  }
}

// The same with the reconstruction chosen at run time (the flux-correction and FOFC
// kernels, which serve every reconstruction).
template <int NG, typename R>
__device__ __forceinline__ void edges(const R* q, R& lo, R& hi, int recon) {
  if constexpr (NG == 3) {
    if (recon == AK_WENOZ)
      edges_t<3, AK_WENOZ>(q, lo, hi);
    else if (recon == AK_PPMX)
      edges_t<3, AK_PPMX>(q, lo, hi);
    else
      edges_t<3, AK_PPM4>(q, lo, hi);
  } else {
    edges_t<2, AK_PLM>(q, lo, hi);
  }
}

// The mesh's Riemann solver (HLLC_ONLY: HLLC without the run-time choice) on one face of
// direction d from edge values in natural variable order; the flux comes back in natural
// order (rho, M1, M2, M3, E).
template <bool NANCHK = false, bool HLLC_ONLY = false, typename R>
__device__ __forceinline__ void solve(int d, const R* l, const R* r, const Bg& bg, R* f) {
  const int perm[5] = {0, 1 + d, 1 + (d + 1) % 3, 1 + (d + 2) % 3, 4};
  R wl[5], wr[5], fn[5];
#pragma unroll
  for (int n = 0; n < 5; ++n) {
    wl[n] = l[perm[n]];
    wr[n] = r[perm[n]];
  }
  if constexpr (HLLC_ONLY && std::is_same<R, double>::value)
    hllc_fp64<NANCHK>(wl, wr, bg, fn);
  else if constexpr (HLLC_ONLY)
    hllc_mixed(wl, wr, bg, fn);
  else if constexpr (std::is_same<R, double>::value)
    riemann<NANCHK>(wl, wr, bg, fn);
  else
    riemann(wl, wr, bg, fn);
#pragma unroll
  for (int n = 0; n < 5; ++n) f[perm[n]] = fn[n];
}

// 0.5 * x on the integer pipe: exact for normal results; a result below the normal
// range (|x| < 2^-1021) becomes a signed zero, inf and NaN stay
__device__ __forceinline__ double half(double x) {
  const int hi = __double2hiint(x);
  const int sub = (hi & 0x7fe00000) == 0;
  const int special = (hi & 0x7ff00000) == 0x7ff00000;
  const int h = special ? hi : (sub ? (hi & (int)0x80000000) : hi - 0x00100000);
  const int l = (special || !sub) ? __double2loint(x) : 0;
  return __hiloint2double(h, l);
}

// The corrected (fine-mean) flux of one coarse face cell from the correction buffer.
__device__ __forceinline__ void corrected_flux(const double* buf, int cell, double* f) {
#pragma unroll
  for (int v = 0; v < 5; ++v) f[v] = __ldcg(buf + (long long)cell * 5 + v);
}
__device__ __forceinline__ void corrected_flux(const double* buf, int cell, float* f) {
#pragma unroll
  for (int v = 0; v < 5; ++v) f[v] = f64_to_f32(__ldcg(buf + (long long)cell * 5 + v));
}

// Flux correction at level boundaries (Section 2): for every coarse face cell next to a
// refined region, the mean of the 2x2 fine fluxes through it, computed from the fine
// block's cells (interior and prolonged ghosts) with the same reconstruction and HLLC
// code the stage kernel runs (register reads through L2 only, as the fused stage kernel
// needs), so the fine block's own update sees the same fluxes.
template <int NG, bool MIXED>
__device__ __forceinline__ void flux_correction_cell(const double* reg, const ak_meshdev& md,
                                                     const Bg& bg, ak_dev_scalars* sc,
                                                     long long t) {
  using R = typename std::conditional<MIXED, float, double>::type;
  int lo = 0, hi = md.nfc - 1;  // face entry holding cell t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (md.fc[mid].z <= t) lo = mid; else hi = mid - 1;
  }
  const int4 F = md.fc[lo];
  const int cell = (int)(t - F.z);
  const ak_block B = md.blocks[F.x];
  const int d = F.y >> 1, side = F.y & 1;
  const int n[3] = {B.nx1, B.nx2, B.nx3};
  const int org[3] = {B.lx1, B.lx2, B.lx3};
  const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
  int loc[3];
  loc[d] = side ? n[d] - 1 : 0;
  loc[a1] = cell % n[a1];
  loc[a2] = cell / n[a1];
  const ak_level LV = md.levels[B.level];
  const int nl[3] = {LV.n1, LV.n2, LV.n3};
  int N[3];
  for (int q = 0; q < 3; ++q) {
    int v = org[q] + loc[q] + (q == d ? (side ? 1 : -1) : 0);
    N[q] = v < 0 ? v + nl[q] : (v >= nl[q] ? v - nl[q] : v);
  }
  const ak_level LF = md.levels[B.level + 1];
  const int fine = md.map[LF.map_off + ((2 * N[2] / LF.bs3) * LF.md2 + 2 * N[1] / LF.bs2) * LF.md1 +
                          2 * N[0] / LF.bs1];
  const ak_block Fb = md.blocks[fine];
  const int forg[3] = {Fb.lx1, Fb.lx2, Fb.lx3};
  const Counters cn{&sc->counters[0], &sc->counters[1]};
  R sum[5] = {R(0), R(0), R(0), R(0), R(0)};
  for (int u2 = 0; u2 < 2; ++u2)
    for (int u1 = 0; u1 < 2; ++u1) {
      int q[3];
      q[d] = (side ? 2 * N[d] : 2 * N[d] + 1) - forg[d];
      q[a1] = 2 * N[a1] + u1 - forg[a1];
      q[a2] = 2 * N[a2] + u2 - forg[a2];
      const int fi = q[d] + (side ? 0 : 1);  // the face between fine cells fi-1 and fi
      R W[2 * NG][5];
#pragma unroll
      for (int mm = 0; mm < 2 * NG; ++mm) {
        int c[3] = {q[0], q[1], q[2]};
        c[d] = fi - NG + mm;
        const long long e = Fb.off + ((long long)(c[2] + NG) * Fb.p2 + (c[1] + NG)) * Fb.s1 +
                            (c[0] + NG);
        double u[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = __ldcg(reg + e + v * Fb.var_stride);
        if (bg.recon == AK_WENOZ || bg.recon == AK_PPMX)
          c2p_t<true>(u, W[mm], bg, cn);
        else
          c2p_t<false>(u, W[mm], bg, cn);
      }
      R lo_a[5], hi_a[5], lo_b[5], hi_b[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        R qa[2 * NG - 1], qb[2 * NG - 1];
#pragma unroll
        for (int mm = 0; mm < 2 * NG - 1; ++mm) {
          qa[mm] = W[mm][v];
          qb[mm] = W[mm + 1][v];
        }
        edges<NG>(qa, lo_a[v], hi_a[v], bg.recon);
        edges<NG>(qb, lo_b[v], hi_b[v], bg.recon);
      }
      R f[5];
      if (bg.recon == AK_WENOZ || bg.recon == AK_PPMX)
        solve<true>(d, hi_a, lo_b, bg, f);
      else
        solve<false>(d, hi_a, lo_b, bg, f);
#pragma unroll
      for (int v = 0; v < 5; ++v) sum[v] += f[v];
    }
  double* out = md.fcbuf + (long long)(B.ovr[F.y] + cell) * 5;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    if constexpr (MIXED)
      out[v] = f32_to_f64(R(0.25) * sum[v]);
    else
      out[v] = R(0.25) * sum[v];
  }
}

// A pointer the compiler cannot relate to any other (so no restrict promise of a kernel
// parameter carries over to the accesses made through it).
template <typename T>
__device__ __forceinline__ T* launder(T* p) {
  T* q;
  asm volatile("mov.b64 %0, %1;" : "=l"(q) : "l"(p) : "memory");
  return q;
}

// Prologue of the persistent fused stage kernel (static refinement, Section 2): the
// ghost fill of the stage's input register (pass 1, then pass 2) and the flux
// correction, each spread over all threads of the cooperative grid and separated by
// grid barriers; a last barrier makes everything visible to the stage tiles.
// smem: the kernel's dynamic shared memory, idle until the stage tiles start; KB
// 16-byte-pair slots per thread of it (5 x 16 B each) stage the pass-1 copies.
template <int NG, bool MIXED, int KB>
__device__ __forceinline__ void fused_prologue(double* reg, const ak_meshdev& md, const Bg& bg,
                                               ak_dev_scalars* sc, unsigned char* smem) {
  __shared__ long long vstride[AK_MAX_LEVELS];
  __shared__ int srow[AK_MAX_LEVELS], splane[AK_MAX_LEVELS];
  if (threadIdx.x < md.nlev) {
    vstride[threadIdx.x] = md.levels[threadIdx.x].var_stride;
    srow[threadIdx.x] = md.levels[threadIdx.x].row;
    splane[threadIdx.x] = md.levels[threadIdx.x].plane;
  }
  __syncthreads();
  const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  double2* buf = reinterpret_cast<double2*>(smem) + (long long)threadIdx.x * KB * AK_NVAR;
  for (long long p = gt; p < (md.nxa + 1) / 2; p += KB * gs)
    xfer_pass1_staged<KB>(reg, md, p, gs, buf, vstride, srow, splane);
  // the prolongations and the face cells of the flux correction are few: spread them
  // across the CTAs (item t to CTA t mod grid), not over the first CTAs' threads
  const long long gi = (long long)threadIdx.x * gridDim.x + blockIdx.x;
  if (md.nxb) {
    grid_barrier(sc);
    for (long long t = gi; t < md.nxb; t += gs) xfer_prolong(reg, md, t);
  }
  if (md.nfc) {
    grid_barrier(sc);
    for (long long t = gi; t < md.fc_cells; t += gs) flux_correction_cell<NG, MIXED>(reg, md, bg, sc, t);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->work_next = 0u;  // tiles are handed out next
  grid_barrier(sc);
}

// Cooperative launch of a persistent stage kernel over the mesh's work list: at most
// one resident wave of CTAs (the occupancy of `kern` times the SM count), so that the
// grid barriers of its prologue are met by every CTA.
template <typename... P, typename... A>
inline cudaError_t launch_persistent(const ak_mesh* m, void (*kern)(P...), int threads,
                                     size_t smem, A&&... args) {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  const long long cap = (long long)per_sm * nsm;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(m->nwork < cap ? m->nwork : cap));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = m->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

// Index of the next stage tile of a persistent kernel: handed out one by one from a
// device counter (reset by the prologue), so CTAs that finish early take more tiles.
__device__ __forceinline__ int next_tile(ak_dev_scalars* sc, int* slot) {
  if (threadIdx.x == 0) *slot = (int)atomicAdd(&sc->work_next, 1u);
  __syncthreads();
  return *slot;
}

// RK stage update of one conserved value in the mixed form (Section 3), in FP64 from
// the FP32 L:  form 0: u + dt L;  form 1: (u0 + u + dt L) / 2;  form 2: a u0 + b (u + dt L)
__device__ __forceinline__ double rk_update_mixed(int form, double a, double b, double dt,
                                                  float L, double u, double u0) {
  const double Ld = f32_to_f64(L);
  if (form == 0) return fma(dt, Ld, u);
  if (form == 1) return half(u0 + fma(dt, Ld, u));
  return fma(b, fma(dt, Ld, u), a * u0);
}

// RK stage update of one conserved value in the FP64 form (Section 3) from the flux
// differences d_d = F_{d,+} - F_{d,-} and cdt_d = dt / dx_d:  U + dt L = U - sum_d cdt_d d_d
// as one chain of fused multiply-adds;  form 0: U + dt L;  form 1: (U0 + U + dt L) / 2;
// form 2: a U0 + b (U + dt L)
__device__ __forceinline__ double rk_update_fp64(int form, double a, double b,
                                                 const double* cdt, double d1, double d2,
                                                 double d3, double u, double u0) {
  double r = fma(-d1, cdt[0], fma(-d2, cdt[1], fma(-d3, cdt[2], u)));
  if (form == 1)
    r = half(u0 + r);
  else if (form == 2)
    r = fma(a, u0, b * r);
  return r;
}

// x > 0 and not NaN (as the comparison x > 0 is), on the integer pipe
__device__ __forceinline__ bool dpos_num(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b <= 0x7ff0000000000000ll;
}

// FOFC flag of an updated cell (Section 3): density or internal energy not positive,
// i.e. not (rho > 0 and rho (2E) - |M|^2 > 0) -- a NaN state, which a high-order flux
// through a face with negative reconstructed pressure leaves, is flagged as well.
// Flagged cells go to the mesh's list and flag array for the correction kernel; the
// list entry is returned (the caller saves the cell's U0 there), or -1 (not flagged, or
// beyond the list's capacity: counted and left to the floors).
__device__ __forceinline__ int fofc_flag(const double* un, const ak_meshdev& md,
                                         ak_dev_scalars* sc, int blk, const ak_block& g,
                                         int i, int j, int k) {
  const double m2 = fma(un[1], un[1], fma(un[2], un[2], un[3] * un[3]));
  if (dpos_num(un[0]) && dpos_num(fma(un[0], un[4] + un[4], -m2))) return -1;
  const unsigned idx = atomicAdd(&sc->fofc_n, 1u);
  if (idx < (unsigned)md.fcap) {
    md.flist[idx] = make_int4(blk, i, j, k);
    md.fflag[md.cell_off[blk] + ((long long)k * g.nx2 + j) * g.nx1 + i] = 1;
    return (int)idx;
  }
  atomicAdd(&sc->fofc_dropped, 1u);
  return -1;
}

// Direct halo reads (meshes without FOFC): threads 0..26 of the CTA copy block `blk`'s
// 27 element bases, entry (dx + 1) + 3 (dy + 1) + 9 (dz + 1) for the halo region in
// direction (dx, dy, dz): a same-level neighbour's offset shifted back by the block
// extents, or the block's own offset where that region is at another level (its ghost
// cells, filled by restriction or prolongation) -- see halo_elem.
__device__ __forceinline__ void neighbour_table(const ak_meshdev& md, int blk, long long* nb) {
  const int t = threadIdx.x;
  if (t < 27) nb[t] = md.nbase[27 * (long long)blk + t];
}

// Element of the cell at padded indices (ip, jp) and interior plane kp of block g, read
// where the stage finds it: in the same-level neighbour block that holds it (blocks of a
// level share g's geometry and are at least NG cells wide, so a halo cell is at most one
// block away), or in g's own ghost cells.
__device__ __forceinline__ long long halo_elem(const ak_block& g, const long long* nb, int ng,
                                               int ip, int jp, int kp) {
  const int dx = ip < ng ? -1 : (ip >= ng + g.nx1 ? 1 : 0);
  const int dy = jp < ng ? -1 : (jp >= ng + g.nx2 ? 1 : 0);
  const int dz = kp < 0 ? -1 : (kp >= g.nx3 ? 1 : 0);
  return nb[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] +
         ((long long)(kp + ng) * g.p2 + jp) * g.s1 + ip;
}

// The stage kernels' background state and EOS constants of a mesh (ak_stage.cu).
Bg stage_bg(const ak_mesh* m);

// Mixed-form PLM stage with paired x1/x2 work (ak_stage_mx.cu); prepare_only sets the
// kernel's shared-memory attribute.
cudaError_t launch_stage_mx(const ak_mesh* m, const double* uin, const double* u0, double* uout,
                            const Bg& bg, double a, double b, int form, int last_stage,
                            bool prepare_only);

}  // namespace ak
