// Device building blocks of the ghost-zone exchange (Section 2, Boundary conditions,
// static refinement), shared by the fill kernels and the persistent fused stage kernel:
// one pair of pass-1 plan entries (same-level copies, restrictions), one pass-2 entry
// (prolongation), and a bounded barrier across the CTAs of a cooperative launch.
// Reads of the register go through L2 only (ld.global.cg): in the fused kernel other
// CTAs write ghost cells between the phases, so no stale line may sit in an L1.
#pragma once

#include "ak_internal.cuh"

namespace ak {

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldcg2(const double* p) {
  return __ldcg(reinterpret_cast<const double2*>(p));
}

// minmod of two differences with its sign and magnitude tests on the integer pipe:
// 0 unless a and b are nonzero with one sign, else the one of smaller magnitude
__device__ __forceinline__ double minmod(double a, double b) {
  const long long ba = __double_as_longlong(a), bb = __double_as_longlong(b);
  if ((ba ^ bb) < 0 || (ba << 1) == 0 || (bb << 1) == 0) return 0.0;
  return (ba & 0x7fffffffffffffffll) < (bb & 0x7fffffffffffffffll) ? a : b;
}

// Pass 1 of the exchange plan, entries 2p and 2p+1: same-level copies and restrictions
// (mean of the 2x2x2 fine cells).  The plan lists ghost cells row by row (x fastest) in
// runs of even length, so two consecutive copies whose destinations and sources are both
// contiguous and 16-byte aligned move as one 16-byte load and store per variable;
// anything else goes cell by cell.  vstride/srow/splane: per-level element strides.
__device__ __forceinline__ void xfer_pass1_pair(double* reg, const ak_meshdev& md, long long p,
                                                const long long* vstride, const int* srow,
                                                const int* splane) {
  const long long t0 = 2 * p;
  if (t0 >= md.nxa) return;
  const ak_xfer x = md.xa[t0];
  if (t0 + 1 < md.nxa) {
    const ak_xfer y = md.xa[t0 + 1];
    if ((x.info & 3) == 0 && (y.info & 3) == 0 && y.dst == x.dst + 1 && y.src == x.src + 1 &&
        ((x.dst | x.src) & 1) == 0 && x.info == y.info) {
      const long long vd = vstride[(x.info >> 2) & 0xff], vs = vstride[(x.info >> 10) & 0xff];
#pragma unroll
      for (int v = 0; v < AK_NVAR; ++v)
        *reinterpret_cast<double2*>(reg + x.dst + v * vd) = ldcg2(reg + x.src + v * vs);
      return;
    }
  }
  for (long long t = t0; t < t0 + 2 && t < md.nxa; ++t) {
    const ak_xfer z = t == t0 ? x : md.xa[t];
    const int ld = (z.info >> 2) & 0xff, ls = (z.info >> 10) & 0xff;
    const long long vd = vstride[ld], vs = vstride[ls];
    if ((z.info & 3) == 0) {
#pragma unroll
      for (int v = 0; v < AK_NVAR; ++v) reg[z.dst + v * vd] = ldcg(reg + z.src + v * vs);
    } else {
      const int row = srow[ls], plane = splane[ls];
#pragma unroll
      for (int v = 0; v < AK_NVAR; ++v) {
        const double* f = reg + z.src + v * vs;
        double s = 0.0;
        for (int dz = 0; dz < 2; ++dz)
          for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) s += ldcg(f + dz * plane + dy * row + dx);
        reg[z.dst + v * vd] = s / 8.0;
      }
    }
  }
}

__device__ __forceinline__ void xf_cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void xf_cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// Pass 1 over pairs p0, p0 + step, ..., p0 + (B-1) step (those below npairs).  The plain
// 16-byte copies are staged through this thread's own B x 5 slots of shared memory
// (buf) with asynchronous copies, all issued before any store, so that a thread keeps
// B pairs of loads in flight without holding them in registers: the fused stage kernel
// runs this phase at the stage's low occupancy, where one pair per thread and trip
// leaves HBM latency exposed.  Other entries (restrictions, unaligned copies) go
// through xfer_pass1_pair.
template <int B>
__device__ __forceinline__ void xfer_pass1_staged(double* reg, const ak_meshdev& md,
                                                  long long p0, long long step, double2* buf,
                                                  const long long* vstride, const int* srow,
                                                  const int* splane) {
  const long long npairs = (md.nxa + 1) / 2;
  long long dst[B], vd[B];
  unsigned fast = 0u;
#pragma unroll
  for (int u = 0; u < B; ++u) {
    const long long p = p0 + u * step;
    if (p >= npairs || 2 * p + 1 >= md.nxa) continue;
    const ak_xfer x = md.xa[2 * p], y = md.xa[2 * p + 1];
    if ((x.info & 3) == 0 && (y.info & 3) == 0 && y.dst == x.dst + 1 && y.src == x.src + 1 &&
        ((x.dst | x.src) & 1) == 0 && x.info == y.info) {
      fast |= 1u << u;
      dst[u] = x.dst;
      vd[u] = vstride[(x.info >> 2) & 0xff];
      const long long vs = vstride[(x.info >> 10) & 0xff];
#pragma unroll
      for (int v = 0; v < AK_NVAR; ++v) xf_cp_async16(&buf[u * AK_NVAR + v], reg + x.src + v * vs);
    }
  }
  xf_cp_async_wait_all();
#pragma unroll
  for (int u = 0; u < B; ++u) {
    const long long p = p0 + u * step;
    if ((fast >> u) & 1u) {
#pragma unroll
      for (int v = 0; v < AK_NVAR; ++v)
        *reinterpret_cast<double2*>(reg + dst[u] + v * vd[u]) = buf[u * AK_NVAR + v];
    } else if (p < npairs) {
      xfer_pass1_pair(reg, md, p, vstride, srow, splane);
    }
  }
}

// Pass 2 of the exchange plan, entry t: one coarse cell's three minmod slopes, then every
// fine ghost child it owns, U_f = U_c + sum_d (+-1/4) s_d (added in the order x, y, z).
__device__ __forceinline__ void xfer_prolong(double* reg, const ak_meshdev& md, long long t) {
  const ak_xfer x = md.xb[t];
  const ak_level D = md.levels[(x.info >> 2) & 0xff];
  const ak_level C = md.levels[(x.info >> 10) & 0xff];
  const int mask = (x.info >> 18) & 0xff;
  const long long st[3] = {1, C.row, C.plane};
#pragma unroll
  for (int v = 0; v < AK_NVAR; ++v) {
    const double* c = reg + x.src + v * C.var_stride;
    const double uc = ldcg(c);
    double s[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) s[d] = 0.25 * minmod(ldcg(c + st[d]) - uc, uc - ldcg(c - st[d]));
    double* f = reg + x.dst + v * D.var_stride;
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
      if (!((mask >> ch) & 1)) continue;
      double u = uc;
      u += (ch & 1) ? s[0] : -s[0];
      u += (ch & 2) ? s[1] : -s[1];
      u += (ch & 4) ? s[2] : -s[2];
      f[(ch & 1) + ((ch >> 1) & 1) * (long long)D.row + ((ch >> 2) & 1) * (long long)D.plane] = u;
    }
  }
}

// Barrier of all CTAs of a cooperative launch (all of them are resident).  One thread per
// CTA arrives on sc->bar_count; the last one resets it and advances sc->bar_gen, which
// the others wait for.  The wait is bounded (2e9 clocks, about a second at the maximum
// SM clock): a CTA that gives up counts a timeout (AK_ETIMEOUT on the host) and goes on.
__device__ __forceinline__ void grid_barrier(ak_dev_scalars* sc) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &sc->bar_gen;
    const unsigned g0 = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&sc->bar_count, 1u) + 1u;
    if (arrived == gridDim.x) {
      sc->bar_count = 0u;
      __threadfence();
      atomicAdd(&sc->bar_gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g0) {
        if (clock64() - t0 > 2000000000ll) {
          atomicAdd(&sc->counters[2], 1ull);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

}  // namespace ak
