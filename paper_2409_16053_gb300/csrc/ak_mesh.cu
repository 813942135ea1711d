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

// CFL minimum over interior cells of every leaf (Eq. (3)), into sc->dtmin_bits.
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
  const double gamma = md.gamma;
  double m = __longlong_as_double(0x7ff0000000000000ll);
  for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const int i = (int)(c % B.nx1);
    const int j = (int)((c / B.nx1) % B.nx2);
    const int k = (int)(c / ((long long)B.nx1 * B.nx2));
    const long long e = elem(B, md.ng, 0, i, j, k);
    double u[AK_NVAR];
#pragma unroll
    for (int v = 0; v < AK_NVAR; ++v) u[v] = reg[e + v * B.var_stride];
    double rho = u[0] >= AK_RHO_FLOOR ? u[0] : AK_RHO_FLOOR;
    const double v1 = u[1] / rho, v2 = u[2] / rho, v3 = u[3] / rho;
    double ug = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / rho;
    ug = ug >= AK_UG_FLOOR ? ug : AK_UG_FLOOR;
    const double cs = sqrt(gamma * (gamma - 1.0) * ug / rho);
    double t = B.dx1 / (fabs(v1) + cs);
    t = fmin(t, B.dx2 / (fabs(v2) + cs));
    t = fmin(t, B.dx3 / (fabs(v3) + cs));
    m = fmin(m, t);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kThreads / 32 ? red[threadIdx.x]
                                           : __longlong_as_double(0x7ff0000000000000ll);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) atomicMin(&sc->dtmin_bits, (unsigned long long)__double_as_longlong(v));
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
