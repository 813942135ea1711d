// C-ABI of libak (declarations and argument conventions in include/ak.h).
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include <cudaTypedefs.h>

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

extern "C" ak_status ak_mesh_create(const ak_mesh_desc* d, void* cuda_stream, ak_mesh** out) {
  if (!d || !out) return einval("ak_mesh_create: NULL argument");
  *out = nullptr;
  if (d->nblocks < 1 || !d->blocks) return einval("ak_mesh_create: need nblocks >= 1 and a block table");
  if (d->recon != AK_PLM && d->recon != AK_PPM4) return einval("ak_mesh_create: recon must be AK_PLM or AK_PPM4");
  const int ng_need = d->recon == AK_PLM ? 2 : 3;
  if (d->nghost != ng_need) return einval("ak_mesh_create: nghost must be 2 for PLM and 3 for PPM4");
  if (d->rk != 2 && d->rk != 3) return einval("ak_mesh_create: rk must be 2 or 3");
  if (d->precision != AK_FP64 && d->precision != AK_MIXED)
    return einval("ak_mesh_create: precision must be AK_FP64 or AK_MIXED");
  if (!(d->gamma > 1.0)) return einval("ak_mesh_create: gamma must be > 1");
  if (!(d->cfl > 0.0 && d->cfl <= 1.0)) return einval("ak_mesh_create: cfl must be in (0, 1]");
  if (d->precision == AK_MIXED && !(d->ref_rho > 0.0 && d->ref_p > 0.0))
    return einval("ak_mesh_create: mixed precision needs ref_rho > 0 and ref_p > 0");
  for (int a = 0; a < 3; ++a) {
    if (!(d->xmax[a] > d->xmin[a])) return einval("ak_mesh_create: xmax must exceed xmin");
    if (d->root_nx[a] < 1) return einval("ak_mesh_create: root_nx must be positive");
  }
  // this version: a uniform level-0 mesh of equal blocks tiling root_nx
  const int32_t* B = d->blocks;
  const int nx1 = B[4], nx2 = B[5], nx3 = B[6];
  if (nx1 < ng_need || nx2 < ng_need || nx3 < ng_need)
    return einval("ak_mesh_create: block sizes must be >= nghost");
  if (d->root_nx[0] % nx1 || d->root_nx[1] % nx2 || d->root_nx[2] % nx3)
    return einval("ak_mesh_create: blocks must tile root_nx");
  const int nb1 = d->root_nx[0] / nx1, nb2 = d->root_nx[1] / nx2, nb3 = d->root_nx[2] / nx3;
  if ((long long)nb1 * nb2 * nb3 != d->nblocks)
    return einval("ak_mesh_create: nblocks does not match root_nx / block size");
  std::vector<int32_t> map((size_t)nb1 * nb2 * nb3, -1), loc((size_t)3 * d->nblocks);
  for (int b = 0; b < d->nblocks; ++b) {
    const int32_t* e = B + (size_t)AK_BLOCK_INTS * b;
    if (e[0] != 0) return einval("ak_mesh_create: only level-0 (uniform) meshes are supported");
    if (e[4] != nx1 || e[5] != nx2 || e[6] != nx3)
      return einval("ak_mesh_create: all blocks must have the same size");
    if (e[1] % nx1 || e[2] % nx2 || e[3] % nx3 || e[1] < 0 || e[2] < 0 || e[3] < 0 ||
        e[1] >= d->root_nx[0] || e[2] >= d->root_nx[1] || e[3] >= d->root_nx[2])
      return einval("ak_mesh_create: block origin not on the block lattice");
    const int bx = e[1] / nx1, by = e[2] / nx2, bz = e[3] / nx3;
    int32_t& slot = map[((size_t)bz * nb2 + by) * nb1 + bx];
    if (slot != -1) return einval("ak_mesh_create: overlapping blocks");
    slot = b;
    loc[3 * b] = bx;
    loc[3 * b + 1] = by;
    loc[3 * b + 2] = bz;
  }

  // 64-byte alignment: the embedded tensor maps require it
  ak_mesh* m = (ak_mesh*)aligned_alloc(64, (sizeof(ak_mesh) + 63) / 64 * 64);
  if (!m) return AK_ENOMEM;
  memset(m, 0, sizeof(ak_mesh));
  m->desc = *d;
  m->stream = (cudaStream_t)cuda_stream;
  m->nreg = d->rk == 3 ? 3 : 2;
  ak_geom& g = m->geom;
  g.nx1 = nx1;
  g.nx2 = nx2;
  g.nx3 = nx3;
  g.ng = ng_need;
  g.p1 = nx1 + 2 * g.ng;
  g.p2 = nx2 + 2 * g.ng;
  g.p3 = nx3 + 2 * g.ng;
  g.s1 = (g.p1 + 3) / 4 * 4;
  g.front = (4 - g.ng % 4) % 4;
  g.var_stride = (long long)g.s1 * g.p2 * g.p3;
  g.block_stride = ((g.front + AK_NVAR * g.var_stride + 31) / 32) * 32;
  g.nblocks = d->nblocks;
  g.nbx1 = nb1;
  g.nbx2 = nb2;
  g.nbx3 = nb3;
  g.dx1 = (d->xmax[0] - d->xmin[0]) / d->root_nx[0];
  g.dx2 = (d->xmax[1] - d->xmin[1]) / d->root_nx[1];
  g.dx3 = (d->xmax[2] - d->xmin[2]) / d->root_nx[2];
  g.gamma = d->gamma;
  m->reg_bytes = sizeof(double) * (size_t)g.block_stride * g.nblocks;
  m->h_blocks = (int32_t*)malloc(sizeof(int32_t) * AK_BLOCK_INTS * d->nblocks);
  m->h_offsets = (int64_t*)malloc(sizeof(int64_t) * d->nblocks);
  if (!m->h_blocks || !m->h_offsets) {
    ak_mesh_destroy(m);
    return AK_ENOMEM;
  }
  memcpy(m->h_blocks, B, sizeof(int32_t) * AK_BLOCK_INTS * d->nblocks);
  m->desc.blocks = m->h_blocks;
  for (int b = 0; b < d->nblocks; ++b) m->h_offsets[b] = (int64_t)b * g.block_stride + g.front;
  // x3 segments per block: enough CTAs to fill the GPU a few times over
  {
    const long long tiles = (long long)d->nblocks * ((nx1 + 15) / 16) * ((nx2 + 15) / 16);
    int seg = 1;
    while (tiles * seg < 4 * 152 && nx3 / (2 * seg) >= 8) seg *= 2;
    m->seg3 = seg;
  }
  cudaError_t e = cudaMalloc(&m->d_block_map, sizeof(int32_t) * map.size());
  if (e == cudaSuccess) e = cudaMalloc(&m->d_block_loc, sizeof(int32_t) * loc.size());
  if (e == cudaSuccess) e = cudaMalloc(&m->d_sc, sizeof(ak_dev_scalars));
  if (e == cudaSuccess)
    e = cudaMemcpy(m->d_block_map, map.data(), sizeof(int32_t) * map.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(m->d_block_loc, loc.data(), sizeof(int32_t) * loc.size(), cudaMemcpyHostToDevice);
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

extern "C" void ak_mesh_destroy(ak_mesh* m) {
  if (!m) return;
  if (m->graph_exec) cudaGraphExecDestroy(m->graph_exec);
  if (m->graph) cudaGraphDestroy(m->graph);
  cudaFree(m->d_block_map);
  cudaFree(m->d_block_loc);
  cudaFree(m->d_sc);
  cudaFree(m->d_staging);
  free(m->h_blocks);
  free(m->h_offsets);
  free(m);
}

extern "C" ak_status ak_mesh_layout(const ak_mesh* m, int32_t* nregisters, size_t* register_bytes,
                                    int64_t* block_offset, int64_t strides[4]) {
  if (!m) return einval("ak_mesh_layout: NULL mesh");
  if (nregisters) *nregisters = m->nreg;
  if (register_bytes) *register_bytes = m->reg_bytes;
  if (block_offset) memcpy(block_offset, m->h_offsets, sizeof(int64_t) * m->geom.nblocks);
  if (strides) {
    strides[0] = m->geom.var_stride;
    strides[1] = (int64_t)m->geom.s1 * m->geom.p2;
    strides[2] = m->geom.s1;
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
  m->tmap_ok[reg] = ak_encode_register_tmap(m, reg) == 0;
  invalidate_graph(m);
  return AK_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
int ak_encode_register_tmap(ak_mesh* m, int reg) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return 1;
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const ak_geom& g = m->geom;
  char* base = (char*)m->reg[reg] + sizeof(double) * g.front;
  if (((uintptr_t)base & 15u) != 0) return 2;
  cuuint64_t dims[5] = {(cuuint64_t)g.p1, (cuuint64_t)g.p2, (cuuint64_t)g.p3, 5,
                        (cuuint64_t)g.nblocks};
  cuuint64_t strides[4] = {sizeof(double) * (cuuint64_t)g.s1,
                           sizeof(double) * (cuuint64_t)g.s1 * g.p2,
                           sizeof(double) * (cuuint64_t)g.var_stride,
                           sizeof(double) * (cuuint64_t)g.block_stride};
  cuuint32_t box[5] = {16, 16, 1, 5, 1};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult r = encode(&m->tmap[reg], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, base, dims, strides, box,
                      estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : 3;
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
  AK_CUDA_TRY(ak_launch_fill_ghosts(m, m->reg[reg]));
  return AK_OK;
}

static ak_status enqueue_stage(ak_mesh* m, int stage) {
  const int rk = m->desc.rk;
  const int in = stage_in_reg(rk, stage), outr = stage_out_reg(rk, stage);
  AK_CUDA_TRY(ak_launch_stage(m, stage, m->reg[in], m->reg[0], m->reg[outr], outr, stage == rk));
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
  ak_status s = enqueue_stage(m, stage);
  if (s != AK_OK) return s;
  if (stage == m->desc.rk) AK_CUDA_TRY(ak_launch_finalize_dt(m, 0));
  return AK_OK;
}

// Reads the device scalars (synchronizes) and maps new floor / non-finite counts to
// AK_ENEGATIVE.
static ak_status read_scalars(ak_mesh* m, ak_dev_scalars* s) {
  AK_CUDA_TRY(cudaMemcpyAsync(s, m->d_sc, sizeof(*s), cudaMemcpyDeviceToHost, m->stream));
  AK_CUDA_TRY(cudaStreamSynchronize(m->stream));
  ak_status st = AK_OK;
  if (s->counters[0] != s->reported[0] || s->counters[1] != s->reported[1]) {
    ak_set_error("floors applied: %llu, non-finite cells: %llu (since mesh creation)",
                 s->counters[0], s->counters[1]);
    st = AK_ENEGATIVE;
    // mark as reported (device copy of the counters is the source of truth)
    unsigned long long rep[4] = {s->counters[0], s->counters[1], s->counters[2], s->counters[3]};
    AK_CUDA_TRY(cudaMemcpyAsync(&m->d_sc->reported, rep, sizeof(rep), cudaMemcpyHostToDevice,
                                m->stream));
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
    AK_CUDA_TRY(ak_launch_fill_ghosts(m, m->reg[stage_in_reg(m->desc.rk, st)]));
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

static ak_status ensure_staging(ak_mesh* m) {
  const size_t need = sizeof(double) * (size_t)m->geom.nblocks * AK_NVAR * m->geom.nx1 *
                      m->geom.nx2 * m->geom.nx3;
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

extern "C" ak_status ak_upload(ak_mesh* m, int32_t reg, const double* host) {
  if (!m || !host) return einval("ak_upload: NULL argument");
  ak_status s = need_reg(m, reg, "ak_upload");
  if (s != AK_OK) return s;
  if ((s = ensure_staging(m)) != AK_OK) return s;
  AK_CUDA_TRY(cudaMemcpyAsync(m->d_staging, host, m->staging_bytes, cudaMemcpyHostToDevice, m->stream));
  AK_CUDA_TRY(ak_launch_unpack(m, m->d_staging, m->reg[reg]));
  return AK_OK;
}

extern "C" ak_status ak_download(ak_mesh* m, int32_t reg, double* host) {
  if (!m || !host) return einval("ak_download: NULL argument");
  ak_status s = need_reg(m, reg, "ak_download");
  if (s != AK_OK) return s;
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
  out[3] = 0;
  return AK_OK;
}
