// Internal declarations of libak: the mesh object, its device tables, the device
// scalars and the kernel launchers shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ak.h"

#define AK_NVAR 5
#define AK_MAX_REG 3
#define AK_MAX_LEVELS 16

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
  unsigned long long counters[4];   // floors, non-finite cells, timeouts, FOFC cells
  unsigned long long reported[4];   // counters already reported to the host
  unsigned int fofc_n;              // cells flagged by FOFC in the current stage
  unsigned int fofc_dropped;        // flagged cells beyond the list's capacity
  unsigned long long sink[2];       // counts nobody reads (recomputations)
  unsigned int bar_count;           // grid barrier of the fused stage kernel: arrivals
  unsigned int bar_gen;             //   and generation
  unsigned int work_next;           // next stage tile of the fused kernel's loop
};

// One leaf MeshBlock (device table entry).
struct ak_block {
  long long off;         // element offset of the block's first ghost cell in a register
  long long var_stride;  // s1 * p2 * p3
  int nx1, nx2, nx3;     // interior cells
  int lx1, lx2, lx3;     // first interior cell in its level's index space
  int level;
  int p1, p2, p3;        // padded extents nx + 2 ng
  int s1;                // row pitch: p1 rounded up to a multiple of 4 elements
  int ovr[6];            // flux-correction faces (x1-, x1+, x2-, x2+, x3-, x3+): offset (in
                         // face cells) of the face's corrected fluxes, or -1
  double dx1, dx2, dx3;
};

// One refinement level: its cell count, block size and leaf map, and the strides of its
// blocks (all leaves of a level have one size).
struct ak_level {
  int n1, n2, n3;        // cells per direction in this level's index space
  int bs1, bs2, bs3;     // block size of the level's leaves (0 if the level is empty)
  int md1, md2, md3;     // map extent in blocks
  int map_off;           // start of the level's map in the map table
  long long var_stride;  // element strides inside a block of this level
  int row, plane;        // (row = s1, plane = s1 * p2)
};

// One entry of the exchange plan (built once per mesh on the host).  Copies and
// restrictions (pass 1): one ghost cell -- the element of variable 0 of the ghost cell and
// of its source (same-level cell, or the first of the 2x2x2 fine cells).  Prolongations
// (pass 2): one coarse cell and a fine block -- the coarse element, and the element of the
// fine child with the lower half in every direction (it may itself lie outside the
// ghost zone); bits 18..25 of info mark the children (x | y << 1 | z << 2) that are ghost
// cells of that block.  info = kind | dst level << 2 | src level << 10 | ...
// (kind 0 copy, 1 restriction, 2 prolongation).
struct ak_xfer {
  long long dst, src;
  int info, pad;
};

// One CTA of the stage kernel: a column tile of one block over planes [k0, k1).
struct ak_work {
  int block, i0, j0, k0, k1, pad;
};

// Everything the kernels need about the mesh, passed by value.
struct ak_meshdev {
  const ak_block* blocks;
  const ak_level* levels;
  const int32_t* map;   // leaf id or -1, per level per block slot
  const int4* fc;       // flux-correction faces: (block, face, first face cell, n cells)
  double* fcbuf;        // corrected coarse-face fluxes, [face cell][5]
  const ak_xfer* xa;    // exchange plan, pass 1 before a stage: copies and restrictions
                        // (with direct halo reads only the entries a stage needs)
  const ak_xfer* xb;    // exchange plan, pass 2: prolongations
  long long nxa, nxb;
  const long long* nbase;  // direct halo reads: per block, 27 element bases (see
                           // neighbour_table)
  const long long* cell_off;  // first interior cell of each block in the global count
  unsigned char* fflag; // FOFC: 1 for a flagged interior cell (global count), else 0
  int4* flist;          // FOFC: flagged cells (block, i, j, k) of the current stage
  double* fu0;          // FOFC: U0 of each listed cell, [entry][5] (stages that use U0)
  int fcap;             // capacity of flist
  int fofc;             // FOFC on
  int direct;           // stage kernels read halo cells of same-level neighbours from
                        // their interiors (meshes without FOFC): a stage needs no copies,
                        // only the restrictions and prolongations at level boundaries
  int nblocks, nlev, ng, nfc;
  long long fc_cells;   // face cells of all flux-correction faces
  double gamma;
};

struct ak_mesh {
  ak_mesh_desc desc;
  cudaStream_t stream;
  int nreg;
  double* reg[AK_MAX_REG];
  size_t reg_bytes;
  int ng, nlev, multilevel;
  int nblocks;
  long long interior_cells;     // over all blocks
  long long padded_cells;       // over all blocks
  int32_t* h_blocks;            // copy of the desc's block table
  int64_t* h_offsets;           // element offset of each block
  ak_block* h_blk;              // host copy of the block table
  ak_block* d_blk;
  ak_level* d_lev;
  int32_t* d_map;
  int4* d_fc;
  double* d_fcbuf;
  long long* d_pack_off;        // interior prefix sums per block (nblocks + 1)
  long long* d_pad_off;         // padded-cell prefix sums per block (nblocks + 1)
  unsigned char* d_fflag;       // FOFC flags and list (see ak_meshdev)
  int4* d_flist;
  double* d_fu0;
  ak_xfer* d_xa;                // exchange plan (see ak_xfer): every ghost cell
  ak_xfer* d_xb;
  ak_xfer* d_xs;                // pass-1 entries a stage needs with direct halo reads
  long long nxa_full;           // entries of d_xa
  long long* d_nbase;           // direct halo reads: 27 element bases per block
  ak_work* d_work;
  int nwork;
  int tile;                     // stage tile: 0 = 16x16 columns, 1 = 32x8
  int nseg;                     // x3 segments per block (upper bound)
  int order;                    // 0 = block order, 1 = longest work first
  int fused;                    // 1: meshes with a ghost fill run each stage as one
                                // persistent cooperative launch (fill, flux correction
                                // and stage fused); 0: separate launches
  int nfc;
  long long fc_cells;
  ak_meshdev md;
  ak_dev_scalars* d_sc;
  double* d_staging;            // interior staging buffer for ak_upload / ak_download
  size_t staging_bytes;
  cudaGraph_t graph;
  cudaGraphExec_t graph_exec;
  int graph_ready;
};

// Error message of the last failing call on this thread.
void ak_set_error(const char* fmt, ...);

// ---- launchers (return cudaSuccess or the launch error) ----
// full: every ghost cell (ak_fill_ghosts); else the fill a stage needs (md.xa, md.xb)
cudaError_t ak_launch_fill_ghosts(const ak_mesh* m, double* reg, bool full);
cudaError_t ak_launch_flux_correction(const ak_mesh* m, const double* reg);
cudaError_t ak_launch_pack(const ak_mesh* m, const double* reg, double* packed);
cudaError_t ak_launch_unpack(const ak_mesh* m, const double* packed, double* reg);
cudaError_t ak_launch_stage(const ak_mesh* m, int stage, const double* u_in, const double* u0,
                            double* u_out, int last_stage);
cudaError_t ak_launch_cfl(const ak_mesh* m, const double* reg);
// First-order flux correction after a stage launch (FOFC meshes): corrects the stage's
// output for the cells it flagged and their neighbours, then clears the flags.
cudaError_t ak_launch_fofc(const ak_mesh* m, int stage, const double* u_in, double* u_out,
                           int last_stage);
cudaError_t ak_launch_finalize_dt(const ak_mesh* m, int use_next_as_dt);
cudaError_t ak_launch_set_dt(const ak_mesh* m, double dt);
// Two-CTA cooperative launch meeting at the fused kernel's grid barrier (CTA 1 stays away
// when absent != 0, so the wait runs out).
cudaError_t ak_launch_barrier_selftest(const ak_mesh* m, int absent);
cudaError_t ak_stage_prepare(const ak_mesh* m);
// (Re)builds the stage work list for a tile shape, x3 segment count and CTA order.
cudaError_t ak_build_work(ak_mesh* m, int tile, int nseg, int order);

