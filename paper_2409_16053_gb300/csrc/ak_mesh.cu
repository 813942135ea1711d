// Mesh-level kernels over every leaf MeshBlock of a (possibly refined) mesh:
//   - ghost-zone fill (Section 2, Boundary conditions) by a precomputed exchange plan:
//     same-level copies and restrictions (fine -> coarse) in a first pass, prolongations
//     (coarse -> fine) in a second one, so that every coarse value a prolongation reads
//     is final;
//   - the CFL minimum of Section 3 Eq. (3) over all leaves (uniform dt across levels);
//   - interior pack/unpack for host transfers; the device-resident dt scalars.
// Readings: restriction is the mean of the 2x2x2 fine cells; prolongation adds
// minmod-limited slopes of the conserved variables, U_f = U_c + sum_d (+-1/4) s_d, so the
// eight fine cells average back to U_c.
#include "ak_internal.cuh"
#include "exchange.cuh"
#include "fastmath.cuh"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ long long elem(const ak_block& B, int ng, int v, int i, int j, int k) {
  return B.off + v * B.var_stride + ((long long)(k + ng) * B.p2 + (j + ng)) * B.s1 + (i + ng);
}

// Ghost fill, pass 1 of the exchange plan: one thread per pair of plan entries.
__global__ void fill_copy_restrict_kernel(double* reg, ak_meshdev md) {
  __shared__ long long vstride[AK_MAX_LEVELS];
  __shared__ int srow[AK_MAX_LEVELS], splane[AK_MAX_LEVELS];
  if (threadIdx.x < md.nlev) {
    vstride[threadIdx.x] = md.levels[threadIdx.x].var_stride;
    srow[threadIdx.x] = md.levels[threadIdx.x].row;
    splane[threadIdx.x] = md.levels[threadIdx.x].plane;
  }
  __syncthreads();
  ak::xfer_pass1_pair(reg, md, blockIdx.x * (long long)blockDim.x + threadIdx.x, vstride, srow,
                      splane);
}

// Ghost fill, pass 2 of the exchange plan: prolongation, after pass 1 has made every
// coarse value it reads final (proper nesting).  One thread per coarse cell.
__global__ void fill_prolong_kernel(double* reg, ak_meshdev md) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < md.nxb) ak::xfer_prolong(reg, md, t);
}

// packed[pack_off[b]*5 + (v*nx3 + k)*nx2*nx1 + j*nx1 + i] <-> register layout
template <bool TO_PACKED>
__global__ void pack_kernel(double* reg, double* packed, ak_meshdev md, const long long* pack_off,
                            int parts) {
  const int b = blockIdx.x % md.nblocks;
  const int part = blockIdx.x / md.nblocks;
  const ak_block B = md.blocks[b];
  const long long per_var = (long long)B.nx1 * B.nx2 * B.nx3;
  const long long n = AK_NVAR * per_var;
  const long long span = (n + parts - 1) / parts;
  const long long c0 = (long long)part * span;
  const long long c1 = c0 + span < n ? c0 + span : n;
  double* pb = packed + AK_NVAR * pack_off[b];
  for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const int v = (int)(c / per_var);
    const long long r = c - v * per_var;
    const int i = (int)(r % B.nx1);
    const int j = (int)((r / B.nx1) % B.nx2);
    const int k = (int)(r / ((long long)B.nx1 * B.nx2));
    const long long e = elem(B, md.ng, v, i, j, k);
    if (TO_PACKED)
      pb[c] = reg[e];
    else
      reg[e] = pb[c];
  }
}

// CFL minimum over interior cells of every leaf (Eq. (3)), into sc->dtmin_bits, as
// 1 / max over cells and d of (|v_d| + c_s) / dx_d: a CTA takes the largest signal rate of
// its cells and stores one reciprocal.  1 / rho and c_s come from single-precision seeds
// (rcp64, rsqrt64) refined by one Newton step in FP64, so a cell costs about 17 FP64
// operations instead of eight IEEE divisions and a square root, and the dt stays within
// a few units in the last place of the definition.  A cell whose rate is not finite is
// skipped, as fmin skips a NaN candidate.
__global__ void cfl_kernel(const double* __restrict__ reg, ak_meshdev md, ak_dev_scalars* sc,
                           int parts) {
  __shared__ double red[kThreads / 32];
  const int b = blockIdx.x % md.nblocks;
  const int part = blockIdx.x / md.nblocks;
  const ak_block B = md.blocks[b];
  const long long n = (long long)B.nx1 * B.nx2 * B.nx3;
  const long long span = (n + parts - 1) / parts;
  const long long c0 = (long long)part * span;
  const long long c1 = c0 + span < n ? c0 + span : n;
  const double g2 = md.gamma * (md.gamma - 1.0);
  const double idx1 = 1.0 / B.dx1, idx2 = 1.0 / B.dx2, idx3 = 1.0 / B.dx3;
  double lam = 0.0;
  for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const int i = (int)(c % B.nx1);
    const long long r = c / B.nx1;
    const int j = (int)(r % B.nx2);
    const int k = (int)(r / B.nx2);
    const long long e = elem(B, md.ng, 0, i, j, k);
    double u[AK_NVAR];
#pragma unroll
    for (int v = 0; v < AK_NVAR; ++v) u[v] = reg[e + v * B.var_stride];
    const double rho = u[0] >= AK_RHO_FLOOR ? u[0] : AK_RHO_FLOOR;
    double ir = ak::rcp64(rho);
    ir = fma(ir, fma(-rho, ir, 1.0), ir);  // Newton: 1 / rho to about an ulp
    const double m2 = fma(u[1], u[1], fma(u[2], u[2], u[3] * u[3]));
    double ug = fma(-m2, ak::dscale(ir, -1), u[4]);
    ug = ug >= AK_UG_FLOOR ? ug : AK_UG_FLOOR;
    const double cs2 = (g2 * ug) * ir;
    // c_s = sqrt(cs2): s = cs2 y with y ~ 1/sqrt(cs2), then s + (y/2)(cs2 - s^2)
    const double y = ak::rsqrt64(cs2);
    const double s0 = cs2 * y;
    const double cs = fma(ak::dscale(y, -1), fma(-s0, s0, cs2), s0);
    const double l1 = fma(fabs(u[1]), ir, cs) * idx1;
    const double l2 = fma(fabs(u[2]), ir, cs) * idx2;
    const double l3 = fma(fabs(u[3]), ir, cs) * idx3;
    // rates are >= 0: compare bit patterns on the integer pipe, skipping inf / NaN
    const long long inf = 0x7ff0000000000000ll;
    const long long b1 = __double_as_longlong(l1), b2 = __double_as_longlong(l2),
                    b3 = __double_as_longlong(l3);
    long long bl = __double_as_longlong(lam);
    bl = (b1 > bl && b1 < inf) ? b1 : bl;
    bl = (b2 > bl && b2 < inf) ? b2 : bl;
    bl = (b3 > bl && b3 < inf) ? b3 : bl;
    lam = __longlong_as_double(bl);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lam;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) {
      const double t = 1.0 / v;  // +inf for a CTA of cells at rest with c_s = 0
      atomicMin(&sc->dtmin_bits, (unsigned long long)__double_as_longlong(t));
    }
  }
}

// dt_next = cfl * min; the device-resident dt becomes dt_next; the min is reset.
__global__ void finalize_dt_kernel(ak_dev_scalars* sc, double cfl) {
  const double m = __longlong_as_double((long long)sc->dtmin_bits);
  sc->dt_next = cfl * m;
  sc->dt = sc->dt_next;
  sc->dtmin_bits = 0x7ff0000000000000ull;
}

__global__ void set_dt_kernel(ak_dev_scalars* sc, double dt) { sc->dt = dt; }

// CTAs per block so that a launch has at least ~2048 CTAs of work
inline int parts_for(const ak_mesh* m) {
  int p = (2048 + m->nblocks - 1) / m->nblocks;
  return p < 1 ? 1 : p;
}

}  // namespace

cudaError_t ak_launch_fill_ghosts(const ak_mesh* m, double* reg, bool full) {
  ak_meshdev md = m->md;
  if (full) {  // the whole plan, not only what a stage with direct halo reads needs
    md.xa = m->d_xa;
    md.nxa = m->nxa_full;
  }
  if (md.nxa)
    fill_copy_restrict_kernel<<<(unsigned)(((md.nxa + 1) / 2 + kThreads - 1) / kThreads),
                                kThreads, 0, m->stream>>>(reg, md);
  if (md.nxb)
    fill_prolong_kernel<<<(unsigned)((md.nxb + kThreads - 1) / kThreads), kThreads, 0,
                          m->stream>>>(reg, md);
  return cudaGetLastError();
}

cudaError_t ak_launch_pack(const ak_mesh* m, const double* reg, double* packed) {
  const int parts = parts_for(m);
  pack_kernel<true><<<(unsigned)(m->nblocks * parts), kThreads, 0, m->stream>>>(
      const_cast<double*>(reg), packed, m->md, m->d_pack_off, parts);
  return cudaGetLastError();
}

cudaError_t ak_launch_unpack(const ak_mesh* m, const double* packed, double* reg) {
  const int parts = parts_for(m);
  pack_kernel<false><<<(unsigned)(m->nblocks * parts), kThreads, 0, m->stream>>>(
      reg, const_cast<double*>(packed), m->md, m->d_pack_off, parts);
  return cudaGetLastError();
}

cudaError_t ak_launch_cfl(const ak_mesh* m, const double* reg) {
  const int parts = parts_for(m);
  cfl_kernel<<<(unsigned)(m->nblocks * parts), kThreads, 0, m->stream>>>(reg, m->md, m->d_sc,
                                                                         parts);
  return cudaGetLastError();
}

cudaError_t ak_launch_finalize_dt(const ak_mesh* m, int) {
  finalize_dt_kernel<<<1, 1, 0, m->stream>>>(m->d_sc, m->desc.cfl);
  return cudaGetLastError();
}

cudaError_t ak_launch_set_dt(const ak_mesh* m, double dt) {
  set_dt_kernel<<<1, 1, 0, m->stream>>>(m->d_sc, dt);
  return cudaGetLastError();
}

// Self-test of the bounded barrier wait: all CTAs meet at grid_barrier, except CTA 1
// when `absent` is set, so that the others' wait runs out.
namespace {
__global__ void barrier_selftest_kernel(ak_dev_scalars* sc, int absent) {
  if (absent && blockIdx.x == 1) return;
  ak::grid_barrier(sc);
}
}  // namespace

cudaError_t ak_launch_barrier_selftest(const ak_mesh* m, int absent) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2);
  cfg.blockDim = dim3(32);
  cfg.stream = m->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, barrier_selftest_kernel, m->d_sc, absent);
}
