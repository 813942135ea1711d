// Mesh-level kernels: ghost-zone fill between MeshBlocks on one device (Section 2,
// Boundary conditions), interior pack/unpack for host transfers, the CFL minimum of
// Section 3 Eq. (3), and the device-resident dt scalars.
#include "ak_internal.cuh"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Every ghost cell of every block takes the interior cell that the periodic domain
// maps it to.  One thread per padded cell; interior cells return at once.
__global__ void fill_ghosts_kernel(double* reg, ak_geom g, const int32_t* __restrict__ loc,
                                   const int32_t* __restrict__ map) {
  const long long total = (long long)g.nblocks * g.var_stride;
  const int n1 = g.nbx1 * g.nx1, n2 = g.nbx2 * g.nx2, n3 = g.nbx3 * g.nx3;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(idx / g.var_stride);
    const long long rem = idx - (long long)b * g.var_stride;
    const int ip = (int)(rem % g.s1);
    const int jp = (int)((rem / g.s1) % g.p2);
    const int kp = (int)(rem / ((long long)g.s1 * g.p2));
    const int i = ip - g.ng, j = jp - g.ng, k = kp - g.ng;
    if (ip >= g.p1) continue;  // row padding
    if (i >= 0 && i < g.nx1 && j >= 0 && j < g.nx2 && k >= 0 && k < g.nx3) continue;
    const int gi = wrapi(loc[3 * b + 0] * g.nx1 + i, n1);
    const int gj = wrapi(loc[3 * b + 1] * g.nx2 + j, n2);
    const int gk = wrapi(loc[3 * b + 2] * g.nx3 + k, n3);
    const int sbx = gi / g.nx1, sby = gj / g.nx2, sbz = gk / g.nx3;
    const int sb = map[(sbz * g.nbx2 + sby) * g.nbx1 + sbx];
    const long long src = (long long)sb * g.block_stride + g.front +
                          ((long long)(gk - sbz * g.nx3 + g.ng) * g.p2 + (gj - sby * g.nx2 + g.ng)) *
                              g.s1 +
                          (gi - sbx * g.nx1 + g.ng);
    const long long dst = (long long)b * g.block_stride + g.front + rem;
#pragma unroll
    for (int v = 0; v < AK_NVAR; ++v) reg[dst + v * g.var_stride] = reg[src + v * g.var_stride];
  }
}

// packed[b][v][k][j][i] (interior only) <-> register layout
template <bool TO_PACKED>
__global__ void pack_kernel(double* reg, double* packed, ak_geom g) {
  const long long per_var = (long long)g.nx1 * g.nx2 * g.nx3;
  const long long total = (long long)g.nblocks * AK_NVAR * per_var;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long bv = idx / per_var;
    const long long rem = idx - bv * per_var;
    const int b = (int)(bv / AK_NVAR), v = (int)(bv % AK_NVAR);
    const int i = (int)(rem % g.nx1);
    const int j = (int)((rem / g.nx1) % g.nx2);
    const int k = (int)(rem / ((long long)g.nx1 * g.nx2));
    const long long e = (long long)b * g.block_stride + g.front + v * g.var_stride +
                        ((long long)(k + g.ng) * g.p2 + (j + g.ng)) * g.s1 + (i + g.ng);
    if (TO_PACKED)
      packed[idx] = reg[e];
    else
      reg[e] = packed[idx];
  }
}

// CFL minimum over interior cells (Eq. (3)), accumulated into sc->dtmin_bits.
__global__ void cfl_kernel(const double* __restrict__ reg, ak_geom g, ak_dev_scalars* sc) {
  __shared__ double red[kThreads / 32];
  const long long per_blk = (long long)g.nx1 * g.nx2 * g.nx3;
  const long long total = (long long)g.nblocks * per_blk;
  double m = __longlong_as_double(0x7ff0000000000000ll);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(idx / per_blk);
    const long long rem = idx - (long long)b * per_blk;
    const int i = (int)(rem % g.nx1);
    const int j = (int)((rem / g.nx1) % g.nx2);
    const int k = (int)(rem / ((long long)g.nx1 * g.nx2));
    const long long e = (long long)b * g.block_stride + g.front +
                        ((long long)(k + g.ng) * g.p2 + (j + g.ng)) * g.s1 + (i + g.ng);
    double u[AK_NVAR];
#pragma unroll
    for (int v = 0; v < AK_NVAR; ++v) u[v] = reg[e + v * g.var_stride];
    double rho = u[0] >= AK_RHO_FLOOR ? u[0] : AK_RHO_FLOOR;
    const double v1 = u[1] / rho, v2 = u[2] / rho, v3 = u[3] / rho;
    double ug = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / rho;
    ug = ug >= AK_UG_FLOOR ? ug : AK_UG_FLOOR;
    const double cs = sqrt(g.gamma * (g.gamma - 1.0) * ug / rho);
    double t = g.dx1 / (fabs(v1) + cs);
    t = fmin(t, g.dx2 / (fabs(v2) + cs));
    t = fmin(t, g.dx3 / (fabs(v3) + cs));
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

inline unsigned grid_for(long long n) {
  long long g = (n + kThreads - 1) / kThreads;
  if (g > 152 * 64) g = 152 * 64;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t ak_launch_fill_ghosts(const ak_mesh* m, double* reg) {
  const long long n = (long long)m->geom.nblocks * m->geom.var_stride;
  fill_ghosts_kernel<<<grid_for(n), kThreads, 0, m->stream>>>(reg, m->geom, m->d_block_loc,
                                                              m->d_block_map);
  return cudaGetLastError();
}

cudaError_t ak_launch_pack(const ak_mesh* m, const double* reg, double* packed) {
  const long long n = (long long)m->geom.nblocks * AK_NVAR * m->geom.nx1 * m->geom.nx2 * m->geom.nx3;
  pack_kernel<true><<<grid_for(n), kThreads, 0, m->stream>>>(const_cast<double*>(reg), packed,
                                                             m->geom);
  return cudaGetLastError();
}

cudaError_t ak_launch_unpack(const ak_mesh* m, const double* packed, double* reg) {
  const long long n = (long long)m->geom.nblocks * AK_NVAR * m->geom.nx1 * m->geom.nx2 * m->geom.nx3;
  pack_kernel<false><<<grid_for(n), kThreads, 0, m->stream>>>(reg, const_cast<double*>(packed),
                                                              m->geom);
  return cudaGetLastError();
}

cudaError_t ak_launch_cfl(const ak_mesh* m, const double* reg) {
  const long long n = (long long)m->geom.nblocks * m->geom.nx1 * m->geom.nx2 * m->geom.nx3;
  cfl_kernel<<<grid_for(n), kThreads, 0, m->stream>>>(reg, m->geom, m->d_sc);
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
