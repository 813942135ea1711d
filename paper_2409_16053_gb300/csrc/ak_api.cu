// C-ABI of libak (declarations and argument conventions in include/ak.h).
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <unordered_map>
#include <unordered_set>
#include <vector>


#include "ak_internal.cuh"

static thread_local char g_err[512] = "";

void ak_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

extern "C" const char* ak_last_error(void) { return g_err; }

#define AK_CUDA_TRY(call)                                                        \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      ak_set_error("%s failed: %s", #call, cudaGetErrorString(e_));              \
      return AK_ECUDA;                                                           \
    }                                                                            \
  } while (0)

static ak_status einval(const char* msg) {
  ak_set_error("%s", msg);
  return AK_EINVAL;
}

static int stage_in_reg(int rk, int s) { return s == 1 ? 0 : (rk == 2 ? 1 : s - 1); }
static int stage_out_reg(int rk, int s) { return s == rk ? 0 : s; }
static bool tile_ok(const ak_mesh* m, int tile);
// a stage needs ghost cells filled first: a refined mesh (level boundaries) or FOFC
static bool stage_fill(const ak_mesh* m) { return m->md.nxa > 0 || m->md.nxb > 0; }

namespace {

// Host view of the levels and leaf maps while a mesh is built.
struct HostIndex {
  int nlev = 0, ng = 0;
  int N[AK_MAX_LEVELS][3];
  int bs[AK_MAX_LEVELS][3];
  int md[AK_MAX_LEVELS][3];
  int off[AK_MAX_LEVELS + 1];
  std::vector<int32_t> map;
  const int32_t* B = nullptr;

  static long long wrap(long long v, long long n) {
    long long r = v % n;
    return r < 0 ? r + n : r;
  }
  // leaf containing level-l cell (x, y, z) (wrapped), or -1
  int leaf(int l, long long x, long long y, long long z) const {
    if (l < 0 || l >= nlev || bs[l][0] == 0) return -1;
    long long c[3] = {wrap(x, N[l][0]) / bs[l][0], wrap(y, N[l][1]) / bs[l][1],
                      wrap(z, N[l][2]) / bs[l][2]};
    return map[off[l] + (c[2] * md[l][1] + c[1]) * md[l][0] + c[0]];
  }
};

}  // namespace

extern "C" ak_status ak_mesh_create(const ak_mesh_desc* d, void* cuda_stream, ak_mesh** out) {
  if (!d || !out) return einval("ak_mesh_create: NULL argument");
  *out = nullptr;
  if (d->nblocks < 1 || !d->blocks) return einval("ak_mesh_create: need nblocks >= 1 and a block table");
  if (d->recon != AK_PLM && d->recon != AK_PPM4 && d->recon != AK_WENOZ && d->recon != AK_PPMX)
    return einval("ak_mesh_create: recon must be AK_PLM, AK_PPM4, AK_WENOZ or AK_PPMX");
  const int ng = d->recon == AK_PLM ? 2 : 3;
  if (d->nghost != ng) return einval("ak_mesh_create: nghost must be 2 for PLM and 3 for PPM4 / WENO-Z / PPMX");
  if (d->rk != 2 && d->rk != 3) return einval("ak_mesh_create: rk must be 2 or 3");
  if (d->precision != AK_FP64 && d->precision != AK_MIXED)
    return einval("ak_mesh_create: precision must be AK_FP64 or AK_MIXED");
  if (d->riemann != AK_HLLC && d->riemann != AK_HLLE && d->riemann != AK_LLF)
    return einval("ak_mesh_create: riemann must be AK_HLLC, AK_HLLE or AK_LLF");
  if (d->fofc != 0 && d->fofc != 1) return einval("ak_mesh_create: fofc must be 0 or 1");
  if (!(d->gamma > 1.0)) return einval("ak_mesh_create: gamma must be > 1");
  if (!(d->cfl > 0.0 && d->cfl <= 1.0)) return einval("ak_mesh_create: cfl must be in (0, 1]");
  if (d->precision == AK_MIXED && !(d->ref_rho > 0.0 && d->ref_p > 0.0))
    return einval("ak_mesh_create: mixed precision needs ref_rho > 0 and ref_p > 0");
  for (int a = 0; a < 3; ++a) {
    if (!(d->xmax[a] > d->xmin[a])) return einval("ak_mesh_create: xmax must exceed xmin");
    if (d->root_nx[a] < 1) return einval("ak_mesh_create: root_nx must be positive");
  }

  // ---- levels, block sizes, leaf maps ------------------------------------------------
  HostIndex X;
  X.ng = ng;
  X.B = d->blocks;
  const int nb = d->nblocks;
  for (int b = 0; b < nb; ++b) {
    const int32_t* e = d->blocks + (size_t)AK_BLOCK_INTS * b;
    if (e[0] < 0 || e[0] >= AK_MAX_LEVELS) return einval("ak_mesh_create: level out of range");
    if (e[0] + 1 > X.nlev) X.nlev = e[0] + 1;
  }
  memset(X.bs, 0, sizeof(X.bs));
  for (int l = 0; l < X.nlev; ++l)
    for (int a = 0; a < 3; ++a) {
      const long long n = (long long)d->root_nx[a] << l;
      if (n > (1ll << 30)) return einval("ak_mesh_create: level index space too large");
      X.N[l][a] = (int)n;
    }
  for (int b = 0; b < nb; ++b) {
    const int32_t* e = d->blocks + (size_t)AK_BLOCK_INTS * b;
    const int l = e[0];
    for (int a = 0; a < 3; ++a) {
      if (e[4 + a] < ng) return einval("ak_mesh_create: block sizes must be >= nghost");
      if (X.bs[l][a] == 0) X.bs[l][a] = e[4 + a];
      if (X.bs[l][a] != e[4 + a])
        return einval("ak_mesh_create: all blocks of one level must have the same size");
      if (e[1 + a] < 0 || e[1 + a] >= X.N[l][a] || e[1 + a] % e[4 + a])
        return einval("ak_mesh_create: block origin not on its level's block lattice");
      if (X.N[l][a] % e[4 + a]) return einval("ak_mesh_create: blocks must tile each level");
      if (X.N[l][a] < e[4 + a] + 2 * ng && X.nlev > 1)
        return einval("ak_mesh_create: a refined mesh needs more than one block per level and direction");
      if (X.nlev > 1 && (e[4 + a] % 2 || e[1 + a] % 2))
        return einval("ak_mesh_create: refined meshes need even block sizes and origins");
    }
  }
  X.off[0] = 0;
  for (int l = 0; l < X.nlev; ++l) {
    long long cnt = 1;
    for (int a = 0; a < 3; ++a) {
      X.md[l][a] = X.bs[l][a] ? X.N[l][a] / X.bs[l][a] : 0;
      cnt *= X.md[l][a];
    }
    if (X.off[l] + cnt > (1ll << 28)) return einval("ak_mesh_create: too many block slots");
    X.off[l + 1] = X.off[l] + (int)cnt;
  }
  X.map.assign((size_t)X.off[X.nlev], -1);
  for (int b = 0; b < nb; ++b) {
    const int32_t* e = d->blocks + (size_t)AK_BLOCK_INTS * b;
    const int l = e[0];
    const long long c = ((long long)(e[3] / X.bs[l][2]) * X.md[l][1] + e[2] / X.bs[l][1]) * X.md[l][0] +
                        e[1] / X.bs[l][0];
    int32_t& slot = X.map[X.off[l] + c];
    if (slot != -1) return einval("ak_mesh_create: overlapping blocks");
    slot = b;
  }
  // exact tiling: no leaf inside a coarser leaf, and the volumes add up to the box
  {
    const int L = X.nlev - 1;
    long long vol = 0, box = (long long)X.N[L][0] * X.N[L][1] * X.N[L][2];
    for (int b = 0; b < nb; ++b) {
      const int32_t* e = d->blocks + (size_t)AK_BLOCK_INTS * b;
      const int l = e[0];
      vol += (long long)e[4] * e[5] * e[6] << (3 * (L - l));
      for (int lc = 0; lc < l; ++lc)
        for (int c = 0; c < 8; ++c) {
          const int sh = l - lc;
          long long x = (e[1] + ((c & 1) ? e[4] - 1 : 0)) >> sh;
          long long y = (e[2] + ((c & 2) ? e[5] - 1 : 0)) >> sh;
          long long z = (e[3] + ((c & 4) ? e[6] - 1 : 0)) >> sh;
          if (X.leaf(lc, x, y, z) >= 0) return einval("ak_mesh_create: a block overlaps a coarser block");
        }
    }
    if (vol != box) return einval("ak_mesh_create: the blocks do not tile the domain");
  }
  // ghost zones: neighbours at most one level apart, and prolongation stencils that only
  // read coarse cells filled by copies or restrictions
  if (X.nlev > 1) {
    for (int b = 0; b < nb; ++b) {
      const int32_t* e = d->blocks + (size_t)AK_BLOCK_INTS * b;
      const int l = e[0];
      for (int k = -ng; k < e[6] + ng; ++k)
        for (int j = -ng; j < e[5] + ng; ++j)
          for (int i = -ng; i < e[4] + ng; ++i) {
            if (i >= 0 && i < e[4] && j >= 0 && j < e[5] && k >= 0 && k < e[6]) continue;
            const long long x = e[1] + i, y = e[2] + j, z = e[3] + k;
            if (X.leaf(l, x, y, z) >= 0) continue;
            if (X.leaf(l + 1, 2 * x, 2 * y, 2 * z) >= 0) continue;
            const long long cx = HostIndex::wrap(x, X.N[l][0]) >> 1,
                            cy = HostIndex::wrap(y, X.N[l][1]) >> 1,
                            cz = HostIndex::wrap(z, X.N[l][2]) >> 1;
            if (X.leaf(l - 1, cx, cy, cz) < 0)
              return einval("ak_mesh_create: neighbouring blocks differ by more than one level");
            for (int a = 0; a < 3; ++a)
              for (int s2 = -1; s2 <= 1; s2 += 2) {
                long long q[3] = {cx, cy, cz};
                q[a] += s2;
                if (X.leaf(l - 1, q[0], q[1], q[2]) < 0 &&
                    X.leaf(l, 2 * q[0], 2 * q[1], 2 * q[2]) < 0)
                  return einval("ak_mesh_create: refinement not properly nested (prolongation "
                                "stencil reaches two levels down)");
              }
          }
    }
  }

  // ---- the mesh object, block table, flux-correction faces, work list ------------------
  ak_mesh* m = (ak_mesh*)aligned_alloc(64, (sizeof(ak_mesh) + 63) / 64 * 64);
  if (!m) return AK_ENOMEM;
  memset(m, 0, sizeof(ak_mesh));
  m->desc = *d;
  m->stream = (cudaStream_t)cuda_stream;
  m->nreg = d->rk == 3 ? 3 : 2;
  m->ng = ng;
  m->nlev = X.nlev;
  m->multilevel = X.nlev > 1;
  m->nblocks = nb;
  m->h_blocks = (int32_t*)malloc(sizeof(int32_t) * AK_BLOCK_INTS * nb);
  m->h_offsets = (int64_t*)malloc(sizeof(int64_t) * nb);
  m->h_blk = (ak_block*)calloc(nb, sizeof(ak_block));
  if (!m->h_blocks || !m->h_offsets || !m->h_blk) {
    ak_mesh_destroy(m);
    return AK_ENOMEM;
  }
  memcpy(m->h_blocks, d->blocks, sizeof(int32_t) * AK_BLOCK_INTS * nb);
  m->desc.blocks = m->h_blocks;
  const long long front = (4 - ng % 4) % 4;
  long long reg_elems = 0;
  std::vector<long long> pack_off(nb + 1, 0), pad_off(nb + 1, 0);
  std::vector<int4> fc;
  long long fc_cells = 0;
  for (int b = 0; b < nb; ++b) {
    const int32_t* e = d->blocks + (size_t)AK_BLOCK_INTS * b;
    ak_block& B = m->h_blk[b];
    B.level = e[0];
    B.lx1 = e[1];
    B.lx2 = e[2];
    B.lx3 = e[3];
    B.nx1 = e[4];
    B.nx2 = e[5];
    B.nx3 = e[6];
    B.p1 = B.nx1 + 2 * ng;
    B.p2 = B.nx2 + 2 * ng;
    B.p3 = B.nx3 + 2 * ng;
    B.s1 = (B.p1 + 3) / 4 * 4;
    B.var_stride = (long long)B.s1 * B.p2 * B.p3;
    B.off = reg_elems + front;
    reg_elems += ((front + AK_NVAR * B.var_stride + 31) / 32) * 32;
    m->h_offsets[b] = B.off;
    B.dx1 = (d->xmax[0] - d->xmin[0]) / X.N[B.level][0];
    B.dx2 = (d->xmax[1] - d->xmin[1]) / X.N[B.level][1];
    B.dx3 = (d->xmax[2] - d->xmin[2]) / X.N[B.level][2];
    pack_off[b + 1] = pack_off[b] + (long long)B.nx1 * B.nx2 * B.nx3;
    pad_off[b + 1] = pad_off[b] + B.var_stride;
    // faces next to a refined region: whole face or nothing
    const int n[3] = {B.nx1, B.nx2, B.nx3};
    for (int f = 0; f < 6; ++f) {
      B.ovr[f] = -1;
      if (!m->multilevel) continue;
      const int dd = f / 2, side = f % 2;
      const int a1 = dd == 0 ? 1 : 0, a2 = dd == 2 ? 1 : 2;  // face cell = t2 * n[a1] + t1
      int refined = 0, total = 0;
      for (int t2 = 0; t2 < n[a2]; ++t2)
        for (int t1 = 0; t1 < n[a1]; ++t1) {
          long long q[3];
          q[dd] = (long long)(side ? n[dd] : -1) + e[1 + dd];
          q[a1] = (long long)t1 + e[1 + a1];
          q[a2] = (long long)t2 + e[1 + a2];
          ++total;
          if (X.leaf(B.level, q[0], q[1], q[2]) < 0 &&
              X.leaf(B.level + 1, 2 * q[0], 2 * q[1], 2 * q[2]) >= 0)
            ++refined;
        }
      if (refined != 0 && refined != total) {
        ak_mesh_destroy(m);
        return einval("ak_mesh_create: a block face is only partly next to a refined region");
      }
      if (refined) {
        B.ovr[f] = (int)fc_cells;
        fc.push_back(make_int4(b, f, (int)fc_cells, total));
        fc_cells += total;
      }
    }
  }
  m->reg_bytes = sizeof(double) * (size_t)reg_elems;
  m->interior_cells = pack_off[nb];
  m->padded_cells = pad_off[nb];
  m->nfc = (int)fc.size();
  m->fc_cells = fc_cells;
  // default stage schedule: 16x16 column tiles, x3 split so that the GPU is filled a
  // few times over, blocks in table order (ak_mesh_autotune may change it)
  int seg = 1;
  {
    long long tiles = 0;
    int minz = 1 << 30;
    for (int b = 0; b < nb; ++b) {
      tiles += (long long)((m->h_blk[b].nx1 + 15) / 16) * ((m->h_blk[b].nx2 + 15) / 16);
      minz = m->h_blk[b].nx3 < minz ? m->h_blk[b].nx3 : minz;
    }
    while (tiles * seg < 4 * 152 && minz / (2 * seg) >= 8) seg *= 2;
  }
  // exchange plan: every ghost cell of every block, with its source
  std::vector<ak_xfer> xa, xb;
  std::unordered_set<long long> pro_reads;
  {
    auto el0 = [&](const ak_block& B, long long i, long long j, long long k) {
      return B.off + ((k + ng) * B.p2 + (j + ng)) * (long long)B.s1 + (i + ng);
    };
    std::unordered_map<long long, size_t> pro;  // coarse cell -> its entry (one block)
    // coarse elements next to a prolonged cell: its minmod slopes read them, so the copies
    // into those (ghost) cells must precede pass 2 even with direct halo reads
    std::unordered_set<long long>& pread = pro_reads;
    for (int b = 0; b < nb; ++b) {
      const ak_block& B = m->h_blk[b];
      const int l = B.level;
      for (int k = -ng; k < B.nx3 + ng; ++k)
        for (int j = -ng; j < B.nx2 + ng; ++j)
          for (int i = -ng; i < B.nx1 + ng; ++i) {
            if (i >= 0 && i < B.nx1 && j >= 0 && j < B.nx2 && k >= 0 && k < B.nx3) continue;
            const long long gx = HostIndex::wrap(B.lx1 + i, X.N[l][0]),
                            gy = HostIndex::wrap(B.lx2 + j, X.N[l][1]),
                            gz = HostIndex::wrap(B.lx3 + k, X.N[l][2]);
            ak_xfer t;
            t.dst = el0(B, i, j, k);
            t.pad = 0;
            const int same = X.leaf(l, gx, gy, gz);
            if (same >= 0) {
              const ak_block& S = m->h_blk[same];
              t.src = el0(S, gx - S.lx1, gy - S.lx2, gz - S.lx3);
              t.info = 0 | (l << 2) | (l << 10);
              xa.push_back(t);
              continue;
            }
            const int fine = X.leaf(l + 1, 2 * gx, 2 * gy, 2 * gz);
            if (fine >= 0) {
              const ak_block& F = m->h_blk[fine];
              t.src = el0(F, 2 * gx - F.lx1, 2 * gy - F.lx2, 2 * gz - F.lx3);
              t.info = 1 | (l << 2) | ((l + 1) << 10);
              xa.push_back(t);
              continue;
            }
            const int coarse = X.leaf(l - 1, gx >> 1, gy >> 1, gz >> 1);
            if (coarse < 0) {  // excluded by the validation above
              ak_mesh_destroy(m);
              return einval("ak_mesh_create: ghost cell without a source");
            }
            // one entry per (fine block, coarse cell): the ghost children form a mask and
            // dst is the element of the child with the lower half in every direction
            const ak_block& C = m->h_blk[coarse];
            t.src = el0(C, (gx >> 1) - C.lx1, (gy >> 1) - C.lx2, (gz >> 1) - C.lx3);
            const int child = (int)((gx & 1) | ((gy & 1) << 1) | ((gz & 1) << 2));
            auto it = pro.find(t.src);
            if (it == pro.end()) {
              t.dst = el0(B, i - (gx & 1), j - (gy & 1), k - (gz & 1));
              t.info = 2 | (l << 2) | ((l - 1) << 10);
              it = pro.emplace(t.src, xb.size()).first;
              xb.push_back(t);
              const long long st[3] = {1, C.s1, (long long)C.s1 * C.p2};
              for (int a = 0; a < 3; ++a) {
                pread.insert(t.src - st[a]);
                pread.insert(t.src + st[a]);
              }
            }
            xb[it->second].info |= 1 << (18 + child);
          }
      pro.clear();
    }
  }
  // Direct halo reads (meshes without FOFC): the stage kernels read the halo cells that
  // lie in a same-level leaf straight from its interior, so the fill before a stage keeps
  // only the restrictions, the prolongations, and the copies into coarse ghost cells that
  // a prolongation's slopes read (xs); ak_fill_ghosts still runs the whole plan.
  const bool direct = !d->fofc;
  std::vector<ak_xfer> xs;
  if (direct) {
    for (const ak_xfer& t : xa)
      if ((t.info & 3) != 0 || pro_reads.count(t.dst)) xs.push_back(t);
  }
  // Per block and direction t = (dx + 1) + 3 (dy + 1) + 9 (dz + 1): the element base of its
  // halo region, so that padded cell (ip, jp) of interior plane kp (of any direction) is
  // element base + ((kp + ng) p2 + jp) s1 + ip.  For a same-level neighbour leaf that is
  // its offset shifted back by the block extents (blocks of one level share their
  // geometry); for a region at another level, and for t = 13, the block's own offset (its
  // ghost cells, filled by restriction or prolongation).
  std::vector<long long> nbase(27 * (size_t)nb);
  for (int b = 0; b < nb; ++b) {
    const ak_block& B = m->h_blk[b];
    const int l = B.level;
    for (int t = 0; t < 27; ++t) {
      const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
      long long base = B.off;
      if (t != 13) {
        const int s = X.leaf(l, B.lx1 + (dx < 0 ? -1 : dx * B.nx1),
                             B.lx2 + (dy < 0 ? -1 : dy * B.nx2), B.lx3 + (dz < 0 ? -1 : dz * B.nx3));
        if (s >= 0)
          base = m->h_blk[s].off - dx * (long long)B.nx1 - dy * (long long)B.nx2 * B.s1 -
                 dz * (long long)B.nx3 * B.p2 * B.s1;
      }
      nbase[27 * (size_t)b + t] = base;
    }
  }
  // level table
  ak_level lev[AK_MAX_LEVELS];
  for (int l = 0; l < X.nlev; ++l) {
    lev[l].n1 = X.N[l][0];
    lev[l].n2 = X.N[l][1];
    lev[l].n3 = X.N[l][2];
    lev[l].bs1 = X.bs[l][0];
    lev[l].bs2 = X.bs[l][1];
    lev[l].bs3 = X.bs[l][2];
    lev[l].md1 = X.md[l][0];
    lev[l].md2 = X.md[l][1];
    lev[l].md3 = X.md[l][2];
    lev[l].map_off = X.off[l];
    lev[l].var_stride = 0;
    lev[l].row = lev[l].plane = 0;
    if (X.bs[l][0]) {
      const int p1 = X.bs[l][0] + 2 * ng, p2 = X.bs[l][1] + 2 * ng, p3 = X.bs[l][2] + 2 * ng;
      const int s1 = (p1 + 3) / 4 * 4;
      lev[l].row = s1;
      lev[l].plane = s1 * p2;
      lev[l].var_stride = (long long)s1 * p2 * p3;
    }
  }

  cudaError_t e = cudaSuccess;
  auto dmalloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes < 8 ? 8 : bytes);
  };
  auto h2d = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  dmalloc((void**)&m->d_blk, sizeof(ak_block) * nb);
  dmalloc((void**)&m->d_lev, sizeof(ak_level) * X.nlev);
  dmalloc((void**)&m->d_map, sizeof(int32_t) * X.map.size());
  dmalloc((void**)&m->d_fc, sizeof(int4) * fc.size());
  dmalloc((void**)&m->d_fcbuf, sizeof(double) * AK_NVAR * (size_t)fc_cells);
  dmalloc((void**)&m->d_pack_off, sizeof(long long) * (nb + 1));
  dmalloc((void**)&m->d_pad_off, sizeof(long long) * (nb + 1));
  dmalloc((void**)&m->d_sc, sizeof(ak_dev_scalars));
  dmalloc((void**)&m->d_xa, sizeof(ak_xfer) * xa.size());
  dmalloc((void**)&m->d_xb, sizeof(ak_xfer) * xb.size());
  dmalloc((void**)&m->d_xs, sizeof(ak_xfer) * xs.size());
  dmalloc((void**)&m->d_nbase, sizeof(long long) * nbase.size());
  h2d(m->d_xa, xa.data(), sizeof(ak_xfer) * xa.size());
  h2d(m->d_xb, xb.data(), sizeof(ak_xfer) * xb.size());
  h2d(m->d_xs, xs.data(), sizeof(ak_xfer) * xs.size());
  h2d(m->d_nbase, nbase.data(), sizeof(long long) * nbase.size());
  h2d(m->d_blk, m->h_blk, sizeof(ak_block) * nb);
  h2d(m->d_lev, lev, sizeof(ak_level) * X.nlev);
  h2d(m->d_map, X.map.data(), sizeof(int32_t) * X.map.size());
  h2d(m->d_fc, fc.data(), sizeof(int4) * fc.size());
  h2d(m->d_pack_off, pack_off.data(), sizeof(long long) * (nb + 1));
  h2d(m->d_pad_off, pad_off.data(), sizeof(long long) * (nb + 1));
  m->md.blocks = m->d_blk;
  m->md.levels = m->d_lev;
  m->md.map = m->d_map;
  m->md.fc = m->d_fc;
  m->md.fcbuf = m->d_fcbuf;
  m->md.nblocks = nb;
  m->md.nlev = X.nlev;
  m->md.ng = ng;
  m->md.nfc = m->nfc;
  m->md.fc_cells = m->fc_cells;
  m->md.gamma = d->gamma;
  m->nxa_full = (long long)xa.size();
  m->md.xa = direct ? m->d_xs : m->d_xa;
  m->md.xb = m->d_xb;
  m->md.nxa = direct ? (long long)xs.size() : (long long)xa.size();
  m->md.nxb = (long long)xb.size();
  m->md.nbase = m->d_nbase;
  m->md.cell_off = m->d_pack_off;
  m->md.direct = direct;
  if (d->fofc) {
    // flagged cells are rare: a list of cells/64 entries (at least 65536)
    const long long cap = std::max(65536ll, m->interior_cells / 64);
    m->md.fcap = (int)std::min(cap, (long long)INT32_MAX);
    m->md.fofc = 1;
    dmalloc((void**)&m->d_fflag, (size_t)m->interior_cells);
    dmalloc((void**)&m->d_flist, sizeof(int4) * (size_t)m->md.fcap);
    dmalloc((void**)&m->d_fu0, sizeof(double) * 5 * (size_t)m->md.fcap);
    if (e == cudaSuccess) e = cudaMemset(m->d_fflag, 0, (size_t)m->interior_cells);
    m->md.fflag = m->d_fflag;
    m->md.flist = m->d_flist;
    m->md.fu0 = m->d_fu0;
  }
  if (e == cudaSuccess) e = ak_build_work(m, tile_ok(m, 0) ? 0 : 2, seg, 0);
  if (e == cudaSuccess) e = ak_stage_prepare(m);
  if (e == cudaSuccess) {
    ak_dev_scalars s;
    memset(&s, 0, sizeof(s));
    s.dtmin_bits = 0x7ff0000000000000ull;
    e = cudaMemcpy(m->d_sc, &s, sizeof(s), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    ak_set_error("ak_mesh_create: %s", cudaGetErrorString(e));
    ak_mesh_destroy(m);
    return e == cudaErrorMemoryAllocation ? AK_ENOMEM : AK_ECUDA;
  }
  *out = m;
  return AK_OK;
}

// Stage tile variants of a mesh's form: FP64 0 (16x16 columns); mixed 0 (paired
// 16x16), 2 (16x16 columns), and for PLM also 1 (32x8 columns).  The paired kernel stages
// rows in 16-byte chunks that must not straddle a block boundary, so it needs an even
// number of cells in x1 in every block.
static bool even_x1(const ak_mesh* m) {
  for (int b = 0; b < m->nblocks; ++b)
    if (m->h_blk[b].nx1 % 2) return false;
  return true;
}
static bool tile_ok(const ak_mesh* m, int tile) {
  if (m->desc.precision != AK_MIXED) return tile == 0;
  if (tile == 0) return even_x1(m);
  return tile == 2 || (tile == 1 && m->desc.recon == AK_PLM);
}

cudaError_t ak_build_work(ak_mesh* m, int tile, int nseg, int order) {
  const int TX = tile == 1 ? 32 : 16, TY = tile == 1 ? 8 : 16;
  std::vector<ak_work> work;
  std::vector<long long> cost;
  for (int b = 0; b < m->nblocks; ++b) {
    const ak_block& B = m->h_blk[b];
    int seg = nseg;
    while (seg > 1 && B.nx3 / seg < 4) seg >>= 1;
    const int kseg = (B.nx3 + seg - 1) / seg;
    for (int s = 0; s < seg; ++s)
      for (int j0 = 0; j0 < B.nx2; j0 += TY)
        for (int i0 = 0; i0 < B.nx1; i0 += TX) {
          ak_work w;
          w.block = b;
          w.i0 = i0;
          w.j0 = j0;
          w.k0 = s * kseg;
          w.k1 = (s + 1) * kseg < B.nx3 ? (s + 1) * kseg : B.nx3;
          w.pad = 0;
          if (w.k0 < w.k1) {
            work.push_back(w);
            cost.push_back((long long)(w.k1 - w.k0 + 2 * m->ng));
          }
        }
  }
  if (order == 1) {  // longest column segments first (a static block-to-SM schedule)
    std::vector<size_t> idx(work.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
    std::vector<ak_work> w2(work.size());
    for (size_t i = 0; i < idx.size(); ++i) w2[i] = work[idx[i]];
    work.swap(w2);
  }
  if (m->d_work) cudaFree(m->d_work);
  m->d_work = nullptr;
  cudaError_t e = cudaMalloc(&m->d_work, sizeof(ak_work) * (work.size() ? work.size() : 1));
  if (e == cudaSuccess)
    e = cudaMemcpy(m->d_work, work.data(), sizeof(ak_work) * work.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  m->nwork = (int)work.size();
  m->tile = tile;
  m->nseg = nseg;
  m->order = order;
  return cudaSuccess;
}

extern "C" void ak_mesh_destroy(ak_mesh* m) {
  if (!m) return;
  if (m->graph_exec) cudaGraphExecDestroy(m->graph_exec);
  if (m->graph) cudaGraphDestroy(m->graph);
  cudaFree(m->d_blk);
  cudaFree(m->d_lev);
  cudaFree(m->d_map);
  cudaFree(m->d_fc);
  cudaFree(m->d_fcbuf);
  cudaFree(m->d_pack_off);
  cudaFree(m->d_pad_off);
  cudaFree(m->d_xa);
  cudaFree(m->d_xb);
  cudaFree(m->d_xs);
  cudaFree(m->d_nbase);
  cudaFree(m->d_fflag);
  cudaFree(m->d_flist);
  cudaFree(m->d_fu0);
  cudaFree(m->d_work);
  cudaFree(m->d_sc);
  cudaFree(m->d_staging);
  free(m->h_blocks);
  free(m->h_offsets);
  free(m->h_blk);
  free(m);
}

extern "C" ak_status ak_mesh_layout(const ak_mesh* m, int32_t* nregisters, size_t* register_bytes,
                                    int64_t* block_offset, int64_t strides[4]) {
  if (!m) return einval("ak_mesh_layout: NULL mesh");
  if (nregisters) *nregisters = m->nreg;
  if (register_bytes) *register_bytes = m->reg_bytes;
  if (block_offset) memcpy(block_offset, m->h_offsets, sizeof(int64_t) * m->nblocks);
  if (strides) {  // of block 0; blocks of other sizes follow the same rule
    strides[0] = m->h_blk[0].var_stride;
    strides[1] = (int64_t)m->h_blk[0].s1 * m->h_blk[0].p2;
    strides[2] = m->h_blk[0].s1;
    strides[3] = 1;
  }
  return AK_OK;
}

static void invalidate_graph(ak_mesh* m) {
  if (m->graph_exec) cudaGraphExecDestroy(m->graph_exec);
  if (m->graph) cudaGraphDestroy(m->graph);
  m->graph_exec = nullptr;
  m->graph = nullptr;
  m->graph_ready = 0;
}

extern "C" ak_status ak_mesh_bind(ak_mesh* m, int32_t reg, double* p) {
  if (!m) return einval("ak_mesh_bind: NULL mesh");
  if (reg < 0 || reg >= m->nreg) return einval("ak_mesh_bind: register index out of range");
  if (!p || ((uintptr_t)p & 255u)) return einval("ak_mesh_bind: pointer NULL or not 256-byte aligned");
  m->reg[reg] = p;
  invalidate_graph(m);
  return AK_OK;
}

static ak_status need_reg(const ak_mesh* m, int reg, const char* who) {
  if (reg < 0 || reg >= m->nreg) {
    ak_set_error("%s: register index out of range", who);
    return AK_EINVAL;
  }
  if (!m->reg[reg]) {
    ak_set_error("%s: register %d not bound", who, reg);
    return AK_ESTATE;
  }
  return AK_OK;
}

extern "C" ak_status ak_fill_ghosts(ak_mesh* m, int32_t reg) {
  if (!m) return einval("ak_fill_ghosts: NULL mesh");
  ak_status s = need_reg(m, reg, "ak_fill_ghosts");
  if (s != AK_OK) return s;
  AK_CUDA_TRY(ak_launch_fill_ghosts(m, m->reg[reg], true));
  return AK_OK;
}

static ak_status enqueue_stage(ak_mesh* m, int stage) {
  const int rk = m->desc.rk;
  const int in = stage_in_reg(rk, stage), outr = stage_out_reg(rk, stage);
  AK_CUDA_TRY(ak_launch_stage(m, stage, m->reg[in], m->reg[0], m->reg[outr], stage == rk));
  if (m->md.fofc)
    AK_CUDA_TRY(ak_launch_fofc(m, stage, m->reg[in], m->reg[outr], stage == rk));
  return AK_OK;
}

extern "C" ak_status ak_stage(ak_mesh* m, int32_t stage, double dt) {
  if (!m) return einval("ak_stage: NULL mesh");
  if (stage < 1 || stage > m->desc.rk) return einval("ak_stage: stage out of range");
  if (dt != dt) return einval("ak_stage: dt is NaN");
  for (int r = 0; r < m->nreg; ++r) {
    ak_status s = need_reg(m, r, "ak_stage");
    if (s != AK_OK) return s;
  }
  if (dt > 0.0) AK_CUDA_TRY(ak_launch_set_dt(m, dt));
  if (m->nfc && !m->fused)
    AK_CUDA_TRY(ak_launch_flux_correction(m, m->reg[stage_in_reg(m->desc.rk, stage)]));
  ak_status s = enqueue_stage(m, stage);
  if (s != AK_OK) return s;
  if (stage == m->desc.rk) AK_CUDA_TRY(ak_launch_finalize_dt(m, 0));
  return AK_OK;
}

// Reads the device scalars (synchronizes) and maps new timeouts of bounded device waits
// to AK_ETIMEOUT, flagged cells beyond the FOFC list to AK_EOVERFLOW and new floor /
// non-finite counts to AK_ENEGATIVE.
static ak_status read_scalars(ak_mesh* m, ak_dev_scalars* s) {
  AK_CUDA_TRY(cudaMemcpyAsync(s, m->d_sc, sizeof(*s), cudaMemcpyDeviceToHost, m->stream));
  AK_CUDA_TRY(cudaStreamSynchronize(m->stream));
  ak_status st = AK_OK;
  if (s->counters[2] != s->reported[2]) {
    ak_set_error("bounded device waits that gave up: %llu (since mesh creation)", s->counters[2]);
    st = AK_ETIMEOUT;
  } else if (s->fofc_dropped != 0) {
    ak_set_error("FOFC: %u flagged cells beyond the list's %d entries were not corrected",
                 s->fofc_dropped, m->md.fcap);
    st = AK_EOVERFLOW;
  } else if (s->counters[0] != s->reported[0] || s->counters[1] != s->reported[1]) {
    ak_set_error("floors applied: %llu, non-finite cells: %llu (since mesh creation)",
                 s->counters[0], s->counters[1]);
    st = AK_ENEGATIVE;
  }
  if (st != AK_OK) {
    // mark as reported (device copy of the counters is the source of truth)
    unsigned long long rep[4] = {s->counters[0], s->counters[1], s->counters[2], s->counters[3]};
    AK_CUDA_TRY(cudaMemcpyAsync(&m->d_sc->reported, rep, sizeof(rep), cudaMemcpyHostToDevice,
                                m->stream));
    // an overflow is reported once: the drop count starts again from zero
    const unsigned int zero = 0;
    if (st == AK_EOVERFLOW)
      AK_CUDA_TRY(cudaMemcpyAsync(&m->d_sc->fofc_dropped, &zero, sizeof(zero),
                                  cudaMemcpyHostToDevice, m->stream));
    AK_CUDA_TRY(cudaStreamSynchronize(m->stream));
  }
  return st;
}

extern "C" ak_status ak_new_dt(ak_mesh* m, int32_t reg, double* dt_out) {
  if (!m || !dt_out) return einval("ak_new_dt: NULL argument");
  ak_status s = need_reg(m, reg, "ak_new_dt");
  if (s != AK_OK) return s;
  AK_CUDA_TRY(ak_launch_cfl(m, m->reg[reg]));
  AK_CUDA_TRY(ak_launch_finalize_dt(m, 1));
  ak_dev_scalars sc;
  s = read_scalars(m, &sc);
  *dt_out = sc.dt_next;
  return s;
}

static ak_status enqueue_step(ak_mesh* m) {
  for (int st = 1; st <= m->desc.rk; ++st) {
    double* in = m->reg[stage_in_reg(m->desc.rk, st)];
    if (stage_fill(m) && !m->fused) AK_CUDA_TRY(ak_launch_fill_ghosts(m, in, false));
    if (m->nfc && !m->fused) AK_CUDA_TRY(ak_launch_flux_correction(m, in));
    ak_status s = enqueue_stage(m, st);
    if (s != AK_OK) return s;
  }
  AK_CUDA_TRY(ak_launch_finalize_dt(m, 1));
  return AK_OK;
}

extern "C" ak_status ak_step(ak_mesh* m, double dt, double* dt_next) {
  if (!m) return einval("ak_step: NULL mesh");
  for (int r = 0; r < m->nreg; ++r) {
    ak_status s = need_reg(m, r, "ak_step");
    if (s != AK_OK) return s;
  }
  if (dt > 0.0) AK_CUDA_TRY(ak_launch_set_dt(m, dt));
  if (m->stream != nullptr) {
    if (!m->graph_ready) {
      AK_CUDA_TRY(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
      ak_status s = enqueue_step(m);
      cudaGraph_t graph = nullptr;
      cudaError_t ce = cudaStreamEndCapture(m->stream, &graph);
      if (s != AK_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
      }
      if (ce != cudaSuccess) {
        ak_set_error("ak_step: graph capture failed: %s", cudaGetErrorString(ce));
        return AK_ECUDA;
      }
      cudaGraphExec_t exec = nullptr;
      ce = cudaGraphInstantiate(&exec, graph, 0);
      if (ce != cudaSuccess) {
        cudaGraphDestroy(graph);
        ak_set_error("ak_step: graph instantiate failed: %s", cudaGetErrorString(ce));
        return AK_ECUDA;
      }
      m->graph = graph;
      m->graph_exec = exec;
      m->graph_ready = 1;
    }
    AK_CUDA_TRY(cudaGraphLaunch(m->graph_exec, m->stream));
  } else {
    ak_status s = enqueue_step(m);
    if (s != AK_OK) return s;
  }
  if (dt_next) {
    ak_dev_scalars sc;
    ak_status s = read_scalars(m, &sc);
    *dt_next = sc.dt_next;
    return s;
  }
  return AK_OK;
}

extern "C" ak_status ak_mesh_autotune(ak_mesh* m, int32_t result[5]) {
  if (!m) return einval("ak_mesh_autotune: NULL mesh");
  for (int r = 0; r < 2; ++r) {
    ak_status s = need_reg(m, r, "ak_mesh_autotune");
    if (s != AK_OK) return s;
  }
  const int fused0 = m->fused;
  m->fused = 0;
  AK_CUDA_TRY(ak_launch_fill_ghosts(m, m->reg[0], true));
  if (m->nfc) AK_CUDA_TRY(ak_launch_flux_correction(m, m->reg[0]));
  cudaEvent_t ev[2];
  AK_CUDA_TRY(cudaEventCreate(&ev[0]));
  AK_CUDA_TRY(cudaEventCreate(&ev[1]));
  int best_tile = m->tile, best_seg = m->nseg, best_order = m->order;
  float best = 1e30f;
  cudaError_t e = cudaSuccess;
  const int fofc = m->md.fofc;
  m->md.fofc = 0;  // the timed launches flag no cells (their output is discarded)
  for (int tile = 0; tile < 3 && e == cudaSuccess; ++tile)
    for (int seg = 1; seg <= 16 && e == cudaSuccess && tile_ok(m, tile); seg *= 2)
      for (int order = 0; order < 2 && e == cudaSuccess; ++order) {
        e = ak_build_work(m, tile, seg, order);
        float t = 1e30f;
        for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
          e = cudaEventRecord(ev[0], m->stream);
          if (e == cudaSuccess) e = ak_launch_stage(m, 1, m->reg[0], m->reg[0], m->reg[1], 0);
          if (e == cudaSuccess) e = cudaEventRecord(ev[1], m->stream);
          if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
          float ms = 0.f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
          if (rep >= 2 && ms < t) t = ms;  // two warm-up launches
        }
        if (e == cudaSuccess && t < best) {
          best = t;
          best_tile = tile;
          best_seg = seg;
          best_order = order;
        }
      }
  // meshes with a ghost fill: separate fill / flux-correction / stage launches against
  // the persistent fused launch, with the chosen schedule
  int best_fused = 0;
  if (e == cudaSuccess) e = ak_build_work(m, best_tile, best_seg, best_order);
  if (stage_fill(m) && e == cudaSuccess) {
    float tf[2] = {1e30f, 1e30f};
    for (int fu = 0; fu < 2 && e == cudaSuccess; ++fu) {
      m->fused = fu;
      for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(ev[0], m->stream);
        if (e == cudaSuccess && !fu) e = ak_launch_fill_ghosts(m, m->reg[0], false);
        if (e == cudaSuccess && !fu && m->nfc) e = ak_launch_flux_correction(m, m->reg[0]);
        if (e == cudaSuccess) e = ak_launch_stage(m, 1, m->reg[0], m->reg[0], m->reg[1], 0);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], m->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (rep >= 2 && ms < tf[fu]) tf[fu] = ms;
      }
    }
    best_fused = tf[1] < tf[0];
    best = tf[best_fused];
  }
  m->fused = e == cudaSuccess ? best_fused : fused0;
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  m->md.fofc = fofc;
  if (e != cudaSuccess) {
    ak_set_error("ak_mesh_autotune: %s", cudaGetErrorString(e));
    return AK_ECUDA;
  }
  invalidate_graph(m);
  if (result) {
    result[0] = best_tile;
    result[1] = best_seg;
    result[2] = best_order;
    result[3] = (int32_t)(best * 1000.0f);
    result[4] = m->fused;
  }
  return AK_OK;
}

extern "C" ak_status ak_selftest_barrier(ak_mesh* m, int32_t absent) {
  if (!m) return einval("ak_selftest_barrier: NULL mesh");
  if (absent != 0 && absent != 1) return einval("ak_selftest_barrier: absent must be 0 or 1");
  AK_CUDA_TRY(ak_launch_barrier_selftest(m, absent));
  // a barrier that ran out leaves its arrival count behind: clear it for the next one
  AK_CUDA_TRY(cudaMemsetAsync(&m->d_sc->bar_count, 0, sizeof(unsigned int), m->stream));
  ak_dev_scalars sc;
  return read_scalars(m, &sc);
}

extern "C" ak_status ak_mesh_fuse(ak_mesh* m, int32_t fused) {
  if (!m) return einval("ak_mesh_fuse: NULL mesh");
  if (fused != 0 && fused != 1) return einval("ak_mesh_fuse: fused must be 0 or 1");
  if (fused && !stage_fill(m))
    return einval("ak_mesh_fuse: this mesh has no ghost fill to fuse (uniform, no FOFC)");
  m->fused = fused;
  invalidate_graph(m);
  return AK_OK;
}

extern "C" ak_status ak_mesh_schedule(ak_mesh* m, int32_t tile, int32_t nseg, int32_t order) {
  if (!m) return einval("ak_mesh_schedule: NULL mesh");
  if (!tile_ok(m, tile)) {
    ak_set_error("ak_mesh_schedule: tile %d not available for this form (FP64: 0; mixed PLM: "
                 "0, 1, 2; mixed with 3 ghost cells: 0, 2)", tile);
    return AK_EINVAL;
  }
  if (nseg < 1 || nseg > 64) {
    ak_set_error("ak_mesh_schedule: nseg %d not in 1..64", nseg);
    return AK_EINVAL;
  }
  if (order != 0 && order != 1) {
    ak_set_error("ak_mesh_schedule: order %d not 0 or 1", order);
    return AK_EINVAL;
  }
  AK_CUDA_TRY(ak_build_work(m, tile, nseg, order));
  invalidate_graph(m);
  return AK_OK;
}

static ak_status ensure_staging(ak_mesh* m) {
  const size_t need = sizeof(double) * (size_t)AK_NVAR * m->interior_cells;
  if (m->d_staging && m->staging_bytes >= need) return AK_OK;
  cudaFree(m->d_staging);
  m->d_staging = nullptr;
  cudaError_t e = cudaMalloc(&m->d_staging, need);
  if (e != cudaSuccess) {
    ak_set_error("staging allocation of %zu bytes failed: %s", need, cudaGetErrorString(e));
    return AK_ENOMEM;
  }
  m->staging_bytes = need;
  return AK_OK;
}

// Device address of a host buffer that the GPU reaches directly: page-locked memory
// mapped into the device's address space (cudaHostAlloc / cudaMallocHost, or
// cudaHostRegister with mapping, on a system with unified addressing).  nullptr for
// anything else (pageable memory), which goes through the staging buffer.
static void* mapped_host(const void* host) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
    cudaGetLastError();  // clear the error of an unknown pointer
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

extern "C" ak_status ak_upload(ak_mesh* m, int32_t reg, const double* host) {
  if (!m || !host) return einval("ak_upload: NULL argument");
  ak_status s = need_reg(m, reg, "ak_upload");
  if (s != AK_OK) return s;
  // mapped page-locked memory: the unpack kernel reads it over the host link itself, one
  // pass instead of a copy into the staging buffer and a second pass over HBM
  if (const void* dh = mapped_host(host)) {
    AK_CUDA_TRY(ak_launch_unpack(m, static_cast<const double*>(dh), m->reg[reg]));
    return AK_OK;
  }
  if ((s = ensure_staging(m)) != AK_OK) return s;
  AK_CUDA_TRY(cudaMemcpyAsync(m->d_staging, host, m->staging_bytes, cudaMemcpyHostToDevice, m->stream));
  AK_CUDA_TRY(ak_launch_unpack(m, m->d_staging, m->reg[reg]));
  return AK_OK;
}

extern "C" ak_status ak_download(ak_mesh* m, int32_t reg, double* host) {
  if (!m || !host) return einval("ak_download: NULL argument");
  ak_status s = need_reg(m, reg, "ak_download");
  if (s != AK_OK) return s;
  if (void* dh = mapped_host(host)) {  // the pack kernel writes the host buffer itself
    AK_CUDA_TRY(ak_launch_pack(m, m->reg[reg], static_cast<double*>(dh)));
    AK_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return AK_OK;
  }
  if ((s = ensure_staging(m)) != AK_OK) return s;
  AK_CUDA_TRY(ak_launch_pack(m, m->reg[reg], m->d_staging));
  AK_CUDA_TRY(cudaMemcpyAsync(host, m->d_staging, m->staging_bytes, cudaMemcpyDeviceToHost, m->stream));
  AK_CUDA_TRY(cudaStreamSynchronize(m->stream));
  return AK_OK;
}

extern "C" ak_status ak_status_counters(ak_mesh* m, int64_t out[4]) {
  if (!m || !out) return einval("ak_status_counters: NULL argument");
  ak_dev_scalars s;
  AK_CUDA_TRY(cudaMemcpyAsync(&s, m->d_sc, sizeof(s), cudaMemcpyDeviceToHost, m->stream));
  AK_CUDA_TRY(cudaStreamSynchronize(m->stream));
  for (int i = 0; i < 4; ++i) out[i] = (int64_t)s.counters[i];
  return AK_OK;
}
