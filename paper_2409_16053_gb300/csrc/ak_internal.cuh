// Internal declarations of libak: the mesh object, device scalars and the kernel
// launchers shared by the translation units of the library.
#pragma once

#include <cuda.h>  // CUtensorMap (tensor maps are encoded through the runtime's entry point)
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ak.h"

#define AK_NVAR 5
#define AK_MAX_REG 3

// Floors of the primitive recovery (counted when applied).  The paper gives no hydro
// floor values; these are the library's choice.
#define AK_RHO_FLOOR 1.0e-12
#define AK_UG_FLOOR 1.0e-15

// Device-resident scalars of one mesh.  Kept in device memory so that a whole step
// (and a loop of steps) runs without a host round trip.
struct ak_dev_scalars {
  double dt;                        // dt used by the stage kernels
  double dt_next;                   // cfl * min(dx / (|v| + c_s)) of the last reduction
  unsigned long long dtmin_bits;    // running min of dx / (|v| + c_s), as bits (>= 0)
  unsigned long long counters[4];   // floors, non-finite cells, timeouts, reserved
  unsigned long long reported[4];   // counters already reported to the host
};

// Geometry of a uniform mesh of equal blocks, passed by value to kernels.
struct ak_geom {
  int nx1, nx2, nx3;     // interior cells per block
  int ng;                // ghost cells per side
  int p1, p2, p3;        // padded extents nx + 2 ng
  int s1;                // row pitch: p1 rounded up to a multiple of 4 elements
  long long front;       // elements before a block's first ghost cell, chosen so that
                         // every row's interior starts on a 32-byte boundary
  long long var_stride;  // s1 * p2 * p3
  long long block_stride;
  int nblocks;
  int nbx1, nbx2, nbx3;  // blocks per direction
  double dx1, dx2, dx3;
  double gamma;
};

struct ak_mesh {
  CUtensorMap tmap[AK_MAX_REG];  // bulk-tensor (TMA) view of each bound register
  int tmap_ok[AK_MAX_REG];
  ak_mesh_desc desc;
  cudaStream_t stream;
  ak_geom geom;
  int nreg;
  double* reg[AK_MAX_REG];
  size_t reg_bytes;
  int32_t* d_block_map;     // [nbx3][nbx2][nbx1] -> block id
  int32_t* d_block_loc;     // [nblocks][3] block coordinates (in blocks)
  int32_t* h_blocks;        // copy of the desc's block table
  int64_t* h_offsets;       // element offset of each block
  ak_dev_scalars* d_sc;
  double* d_staging;        // interior staging buffer for ak_upload / ak_download
  size_t staging_bytes;
  cudaGraph_t graph;
  cudaGraphExec_t graph_exec;
  int graph_ready;
  int seg3;                 // x3 segments per block for the stage launch
};

// Error message of the last failing call on this thread.
void ak_set_error(const char* fmt, ...);

// ---- launchers (return cudaSuccess or the launch error) ----
cudaError_t ak_launch_fill_ghosts(const ak_mesh* m, double* reg);
cudaError_t ak_launch_pack(const ak_mesh* m, const double* reg, double* packed);
cudaError_t ak_launch_unpack(const ak_mesh* m, const double* packed, double* reg);
cudaError_t ak_launch_stage(const ak_mesh* m, int stage, const double* u_in, const double* u0,
                            double* u_out, int out_reg, int last_stage);
cudaError_t ak_launch_cfl(const ak_mesh* m, const double* reg);
cudaError_t ak_launch_finalize_dt(const ak_mesh* m, int use_next_as_dt);
cudaError_t ak_launch_set_dt(const ak_mesh* m, double dt);
cudaError_t ak_stage_prepare(const ak_mesh* m);
// Encodes m->tmap[reg] for register `reg` (5-D: x, y, z, var, block of doubles, box of
// one 16x16 tile plane of all 5 variables); returns 0 on success.
int ak_encode_register_tmap(ak_mesh* m, int reg);
