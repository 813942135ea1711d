// Mesh-level kernels over every leaf MeshBlock of a (possibly refined) mesh:
//   - ghost-zone fill (Section 2, Boundary conditions): same-level copies and
//     restrictions (fine -> coarse) in a first pass, prolongations (coarse -> fine) in a
//     second one, so that every coarse value a prolongation reads is final;
//   - the CFL minimum of Section 3 Eq. (3) over all leaves (uniform dt across levels);
//   - interior pack/unpack for host transfers; the device-resident dt scalars.
// Readings: restriction is the mean of the 2x2x2 fine cells; prolongation adds
// minmod-limited slopes of the conserved variables, U_f = U_c + sum_d (+-1/4) s_d, so the
// eight fine cells average back to U_c.
#include "ak_internal.cuh"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// leaf containing cell (x, y, z) of level l (coordinates already wrapped), or -1
__device__ __forceinline__ int leaf_at(const ak_meshdev& md, int l, int x, int y, int z) {
  if (l < 0 || l >= md.nlev) return -1;
  const ak_level L = md.levels[l];
  if (L.bs1 == 0) return -1;
  return md.map[L.map_off + ((z / L.bs3) * L.md2 + y / L.bs2) * L.md1 + x / L.bs1];
}

__device__ __forceinline__ long long elem(const ak_block& B, int ng, int v, int i, int j, int k) {
  return B.off + v * B.var_stride + ((long long)(k + ng) * B.p2 + (j + ng)) * B.s1 + (i + ng);
}

__device__ __forceinline__ double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return fabs(a) < fabs(b) ? a : b;
}

// One pass of the ghost fill.  The grid is nblocks x parts CTAs; CTA (b, part) walks a
// contiguous share of block b's padded cells (interior cells and row padding skipped).
template <int PASS>
__global__ void fill_pass_kernel(double* reg, ak_meshdev md, int parts) {
  const int b = blockIdx.x % md.nblocks;
  const int part = blockIdx.x / md.nblocks;
  const ak_block B = md.blocks[b];
  const int ng = md.ng;
  const ak_level LV = md.levels[B.level];
  const long long n = B.var_stride;
  const long long span = (n + parts - 1) / parts;
  const long long c0 = (long long)part * span;
  const long long c1 = c0 + span < n ? c0 + span : n;
  for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const int ip = (int)(c % B.s1);
    const int jp = (int)((c / B.s1) % B.p2);
    const int kp = (int)(c / ((long long)B.s1 * B.p2));
    if (ip >= B.p1) continue;  // row padding
    const int i = ip - ng, j = jp - ng, k = kp - ng;
    if (i >= 0 && i < B.nx1 && j >= 0 && j < B.nx2 && k >= 0 && k < B.nx3) continue;
    const int gx = wrapi(B.lx1 + i, LV.n1), gy = wrapi(B.lx2 + j, LV.n2),
              gz = wrapi(B.lx3 + k, LV.n3);
    const long long dst = B.off + c;
    const int same = leaf_at(md, B.level, gx, gy, gz);
    if (PASS == 1) {
      if (same >= 0) {
        const ak_block S = md.blocks[same];
        const long long src = elem(S, ng, 0, gx - S.lx1, gy - S.lx2, gz - S.lx3);
#pragma unroll
        for (int v = 0; v < AK_NVAR; ++v) reg[dst + v * B.var_stride] = reg[src + v * S.var_stride];
        continue;
      }
      const int fine = leaf_at(md, B.level + 1, 2 * gx, 2 * gy, 2 * gz);
      if (fine >= 0) {  // restriction: mean of the 2x2x2 fine cells
        const ak_block F = md.blocks[fine];
        const int fi = 2 * gx - F.lx1, fj = 2 * gy - F.lx2, fk = 2 * gz - F.lx3;
#pragma unroll
        for (int v = 0; v < AK_NVAR; ++v) {
          double s = 0.0;
          for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
              for (int dx = 0; dx < 2; ++dx) s += reg[elem(F, ng, v, fi + dx, fj + dy, fk + dz)];
          reg[dst + v * B.var_stride] = s / 8.0;
        }
      }
    } else {
      if (same >= 0) continue;
      if (leaf_at(md, B.level + 1, 2 * gx, 2 * gy, 2 * gz) >= 0) continue;
      const int cx = gx >> 1, cy = gy >> 1, cz = gz >> 1;
      const int coarse = leaf_at(md, B.level - 1, cx, cy, cz);
      if (coarse < 0) continue;
      const ak_block C = md.blocks[coarse];
      const int li = cx - C.lx1, lj = cy - C.lx2, lk = cz - C.lx3;
      const int h1 = gx & 1, h2 = gy & 1, h3 = gz & 1;
#pragma unroll
      for (int v = 0; v < AK_NVAR; ++v) {
        const double uc = reg[elem(C, ng, v, li, lj, lk)];
        double u = uc;
        {
          const double s = minmod(reg[elem(C, ng, v, li + 1, lj, lk)] - uc,
                                  uc - reg[elem(C, ng, v, li - 1, lj, lk)]);
          u += (h1 ? 0.25 : -0.25) * s;
        }
        {
          const double s = minmod(reg[elem(C, ng, v, li, lj + 1, lk)] - uc,
                                  uc - reg[elem(C, ng, v, li, lj - 1, lk)]);
          u += (h2 ? 0.25 : -0.25) * s;
        }
        {
          const double s = minmod(reg[elem(C, ng, v, li, lj, lk + 1)] - uc,
                                  uc - reg[elem(C, ng, v, li, lj, lk - 1)]);
          u += (h3 ? 0.25 : -0.25) * s;
        }
        reg[dst + v * B.var_stride] = u;
      }
    }
  }
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

cudaError_t ak_launch_fill_ghosts(const ak_mesh* m, double* reg) {
  const int parts = parts_for(m);
  fill_pass_kernel<1><<<(unsigned)(m->nblocks * parts), kThreads, 0, m->stream>>>(reg, m->md,
                                                                                 parts);
  if (m->multilevel)
    fill_pass_kernel<2><<<(unsigned)(m->nblocks * parts), kThreads, 0, m->stream>>>(reg, m->md,
                                                                                   parts);
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
