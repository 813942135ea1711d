/*
 * ak.h -- C-ABI of the GB300 hydro-stage library (libak).
 *
 * One Runge-Kutta stage of the Godunov finite-volume update for 3D adiabatic
 * Newtonian hydrodynamics on a mesh of MeshBlocks, as AthenaK states it
 * (arXiv 2409.16053):
 *   - conservation law dU/dt + div F(W) = 0 ............ Section 3, Eq. (1) (S = 0)
 *   - U = (rho, rho v, E), F, W = (rho, v, u_g),
 *     E = u_g + rho v^2/2, p = (gamma-1) u_g ............ Section 3.1, Eq. (4)
 *   - reconstruction on primitives (PLM, PPM4, PPMX,
 *     WENO-Z) ........................................ Section 3
 *   - HLLC, HLLE and LLF Riemann solvers ............... Section 3
 *   - method of lines with SSP Runge-Kutta ............. Section 3
 *   - CFL time step, min over all cells and dims ....... Section 3, Eq. (3)
 *   - MeshBlocks aggregated per device, one launch
 *     covers all blocks ................................ Section 2 (MeshBlockPacks)
 *   - ghost zones filled by device copies .............. Section 2 (Boundary conditions)
 *   - uniform time step across levels .................. Section 2
 *
 * Conventions
 *   - All calls are ordered on the CUDA stream given to ak_mesh_create.  Calls that
 *     return a device result to the host (ak_new_dt, ak_step with dt_next, ak_download,
 *     ak_status_counters) synchronize that stream; the others only enqueue work.
 *   - Device pointers are plain `double*` in device memory.  Registers (the state
 *     arrays) are owned by the caller (e.g. torch tensors) and only borrowed by
 *     ak_mesh_bind; the library never frees them.  The library allocates only its own
 *     small tables, device scalars and, for ak_upload/ak_download, a staging buffer of
 *     one register's interior size; ak_mesh_destroy frees them.
 *   - Argument errors are returned synchronously.  Device-side problems (density or
 *     internal energy below the floors, non-finite states) are counted in a device
 *     status word and reported by the next synchronizing call as AK_ENEGATIVE (a
 *     bounded device wait that gave up as AK_ETIMEOUT, an overflowing FOFC list as
 *     AK_EOVERFLOW, in that order of precedence); the counters stay readable through
 *     ak_status_counters.
 *   - A mesh object is not thread safe; distinct meshes may be used from distinct
 *     host threads.
 *
 * Register layout (the library's choice, reported by ak_mesh_layout):
 *   register = blocks one after another (each with its own size on a refined mesh);
 *   inside a block the layout is
 *   [var 0..4][k][j][i] with i fastest, each dimension padded by nghost ghost cells on
 *   both sides (extents nx1+2g, nx2+2g, nx3+2g), var = (rho, M1, M2, M3, E).  Rows are
 *   stored with a pitch s1 = round_up(nx1 + 2g, 4) elements, and block b's first ghost
 *   cell is at element block_offset[b] = b * S + f, with f = (4 - g % 4) % 4 and
 *   S = round_up(f + 5 * s1 * (nx2+2g) * (nx3+2g), 32): every row's interior then starts
 *   on a 32-byte boundary.  The interior cell (i, j, k), 0 <= i < nx1, of block b,
 *   variable v is element
 *     block_offset[b] + ((v*(nx3+2g) + k+g)*(nx2+2g) + j+g)*s1 + i+g.
 */
#ifndef AK_H
#define AK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AK_OK = 0,
  AK_EINVAL = -1,     /* invalid argument or unsupported configuration */
  AK_ENOMEM = -2,     /* a library allocation failed */
  AK_ECUDA = -3,      /* a CUDA runtime call failed (see ak_last_error) */
  AK_ENEGATIVE = -4,  /* rho or u_g fell below the floors (see ak_status_counters) */
  AK_ETIMEOUT = -5,   /* a bounded device wait gave up */
  AK_ESTATE = -6,     /* call out of order (e.g. a register not bound) */
  AK_EOVERFLOW = -7   /* FOFC: a stage flagged more cells than its list holds
                         (max(65536, interior cells / 64)); the cells beyond it kept
                         their uncorrected state */
} ak_status;

enum { AK_PLM = 0, AK_PPM4 = 1, AK_WENOZ = 2, AK_PPMX = 3 };  /* reconstruction (Section 3) */
enum { AK_FP64 = 0, AK_MIXED = 1 };   /* arithmetic form of the stage */
enum { AK_HLLC = 0, AK_HLLE = 1, AK_LLF = 2 };  /* Riemann solver (Section 3) */

/* Number of int32 entries per block in ak_mesh_desc.blocks. */
#define AK_BLOCK_INTS 7

typedef struct ak_mesh ak_mesh;

typedef struct {
  int32_t nblocks;        /* number of MeshBlocks (Section 2), >= 1 */
  int32_t nghost;         /* ghost cells per side: 2 for PLM, 3 for PPM4, WENO-Z, PPMX */
  const int32_t* blocks;  /* host array, AK_BLOCK_INTS ints per leaf block:
                             level, lx1, lx2, lx3, nx1, nx2, nx3 -- (lx1, lx2, lx3) is the
                             block's first cell in the cell index space of its level
                             (root_nx * 2^level cells per direction).  Level 0 only is a
                             uniform mesh; several levels are a static refinement
                             (Section 2) whose leaves advance with one dt.  Copied at
                             create time; the caller keeps ownership. */
  double xmin[3], xmax[3];  /* domain, periodic in all three directions */
  int32_t root_nx[3];       /* level-0 cells per direction; the blocks must tile it */
  int32_t recon;            /* AK_PLM (van Leer), AK_PPM4 (Colella & Woodward limiters),
                               AK_WENOZ (Borges et al.) or AK_PPMX (extremum-preserving
                               limiters of Colella & Sekora / McCorquodale & Colella) */
  int32_t rk;               /* SSP-RK order: 2 (Heun) or 3 (Shu-Osher) */
  int32_t precision;        /* AK_FP64 or AK_MIXED */
  int32_t riemann;          /* AK_HLLC (0: HLLC with PVRS speeds bounded by the Davis
                               speeds), AK_HLLE (HLL with Einfeldt's Roe-average speeds)
                               or AK_LLF (Rusanov) */
  int32_t fofc;             /* 1: first-order flux correction (Section 3): in every RK
                               stage, a cell whose density or internal energy would not
                               be positive gets first-order (piecewise-constant) LLF
                               fluxes on all its faces, before the level flux correction
                               on refined meshes (a fine face at a level boundary turns
                               first-order when the fine or the coarse cell is flagged;
                               the coarse side takes the fine mean).  The flagged
                               cells of one stage go to a list of max(65536, interior
                               cells / 64) entries; cells beyond it are not corrected
                               and the next synchronizing call returns AK_EOVERFLOW.
                               0: off. */
  double gamma;             /* gamma-law EOS, > 1 */
  double cfl;               /* Courant number of Eq. (3), in (0, 1] */
  double ref_rho, ref_p;    /* AK_MIXED only: background density and pressure that are
                               subtracted (in FP64) before the FP32 arithmetic; any
                               positive values are valid, values close to the flow's
                               typical state give the smallest rounding error. */
} ak_mesh_desc;

/* A mesh of MeshBlocks aggregated on one device (Section 2, "MeshBlockPacks": all
 * MeshBlocks on a device form one structure, so one launch covers them all; static
 * refinement follows Section 2's block-based design with uniform time steps across
 * levels).  Validates `desc`, copies the block table to the device and allocates the
 * device scalars.  `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
 * A valid mesh: blocks of one level share one size; origins lie on the level's block
 * lattice; the leaves tile the periodic box exactly (no overlap within or across
 * levels); and, with several levels, sizes and origins are even, ghost zones see at
 * most one level jump, prolongation stencils reach at most one level down (proper
 * nesting), and a block face next to a finer region is so over its whole extent.
 * Returns AK_EINVAL for an invalid description (with the violated rule in
 * ak_last_error), AK_ENOMEM / AK_ECUDA on allocation failure.  On success *out owns the
 * mesh (free with ak_mesh_destroy). */
ak_status ak_mesh_create(const ak_mesh_desc* desc, void* cuda_stream, ak_mesh** out);

/* Frees what ak_mesh_create allocated (Section 2's MeshBlockPack goes away with it);
 * bound registers are not touched.  NULL is a no-op. */
void ak_mesh_destroy(ak_mesh* mesh);

/* Layout of the dependent variables (Section 2, "Data locality": one device array per
 * variable set, with the MeshBlock index as an extra dimension, kept on the device).
 * Reports the number of registers the configured integrator needs (2 for RK2, 3 for
 * RK3), bytes of one register, (if block_offset != NULL) the element offset of every block's first
 * ghost cell (nblocks entries), and (if strides != NULL) the element strides of
 * (var, k, j, i) inside block 0 (blocks of other sizes follow the same rule).  Any output pointer may be NULL.  Register 0 holds
 * U^n before ak_step and U^{n+1} after it. */
ak_status ak_mesh_layout(const ak_mesh* mesh, int32_t* nregisters, size_t* register_bytes,
                         int64_t* block_offset, int64_t strides[4]);

/* Binds device memory as one register (Section 2, "Data locality": the state lives in
 * device memory and is never moved to the host by a step).  Borrows `dev_ptr` (device
 * memory of register_bytes bytes, 256-byte aligned) as register `reg` in
 * [0, nregisters); the caller keeps ownership.  AK_EINVAL for a bad index, NULL or misaligned
 * pointer. */
ak_status ak_mesh_bind(ak_mesh* mesh, int32_t reg, double* dev_ptr);

/* Ghost-zone fill of register `reg` (Section 2, Boundary conditions): every ghost
 * cell of every block receives the periodic image of its position, copied from the
 * neighbouring block on the same device (same level), restricted as the mean of the
 * 2x2x2 cells of a finer neighbour, or prolonged from a coarser neighbour (coarse value
 * plus minmod-limited slopes of the conserved variables, +-1/4 of a coarse slope per
 * direction; done after the copies and restrictions).  One launch per pass covers all
 * blocks.  Edge and corner ghosts are filled too.
 * Without FOFC the stage kernels read every halo cell that lies in a same-level block
 * straight from that block's interior, so ak_step fills only the ghost cells at level
 * boundaries before a stage (restrictions, prolongations, and the copies a
 * prolongation's slopes read) and none on a uniform mesh; this call still fills every
 * ghost cell (e.g. for output, or before ak_stage on a refined mesh). */
ak_status ak_fill_ghosts(ak_mesh* mesh, int32_t reg);

/* One RK stage s in [1, rk] with time step dt (Section 3); dt <= 0 uses the
 * device-resident dt (the last CFL reduction, or the last dt given):
 *   U_out = a_s * U0 + b_s * (U_in + dt * L(U_in)),   L = -div F (Eq. (1)),
 * RK2: (a, b) = (0, 1), (1/2, 1/2); RK3: (0, 1), (3/4, 1/4), (1/3, 2/3).
 * Registers: RK2 stage 1: in 0, out 1; stage 2: in 1, U0 = 0, out 0.
 *            RK3 stage 1: in 0, out 1; stage 2: in 1, out 2; stage 3: in 2, out 0.
 * The ghost zones of the input register must be current (ak_fill_ghosts).  On a
 * refined mesh the call first computes, for every coarse face next to a finer region,
 * the mean of the 2x2 fine fluxes through it, and the coarse update uses that mean
 * (flux correction at level boundaries, Section 2), so the update stays conservative.
 * Only interior cells of the output are written.  The last stage also accumulates the
 * CFL minimum of the new state (over all levels, each with its dx) for ak_new_dt's
 * device-resident value. */
ak_status ak_stage(ak_mesh* mesh, int32_t stage, double dt);

/* CFL time step of register `reg` (Section 3, Eq. (3)):
 *   dt = cfl * min over interior cells and d of dx_d / (|v_d| + c_s),
 *   c_s = sqrt(gamma p / rho).  Synchronizes the stream and writes *dt_out.  The value
 * also becomes the device-resident dt that ak_step uses when called with dt <= 0.
 * Returns AK_ENEGATIVE if any floor was hit since the last check (the dt is still
 * written). */
ak_status ak_new_dt(ak_mesh* mesh, int32_t reg, double* dt_out);

/* One full RK step of register 0: for each stage, ghost fill of its input then
 * ak_stage; the new CFL dt is reduced in the last stage.  dt > 0 uses that dt;
 * dt <= 0 uses the device-resident dt (from ak_new_dt or the previous ak_step), so a
 * time loop needs no host round trip.  If dt_next != NULL the stream is synchronized
 * and the CFL dt of the new state is written there.  The step's launches are captured
 * into a CUDA graph on the first call and replayed afterwards. */
ak_status ak_step(ak_mesh* mesh, double dt, double* dt_next);

/* Picks, by timing stage launches on this mesh, the schedule of the stage kernel: the
 * column-tile variant (see ak_mesh_schedule), the number of x3 segments per MeshBlock, and the order in which CTAs take the (block, tile, segment) work items
 * (block order, or longest first) -- the block-to-SM schedule.  The paper finds the
 * MeshBlock size decisive for throughput (Section 5.1); this tunes how a given mesh is
 * cut into GPU work.  Results are bitwise independent of the choice.  Registers 0 and 1
 * must be bound and register 0 must hold a valid state (its ghosts are refilled);
 * register 1 is overwritten.  Synchronizes the stream; do not call during a stream
 * capture.  On a mesh with a ghost fill (static refinement, or FOFC) it then times a
 * stage as separate fill / flux-correction / stage launches against the persistent fused
 * launch (ak_mesh_fuse) and keeps the faster.  result (may be NULL): tile, segments,
 * order (as for ak_mesh_schedule), the chosen stage time in microseconds (with the fill
 * and flux correction on such meshes), and 1 if the fused launch was chosen. */
ak_status ak_mesh_autotune(ak_mesh* mesh, int32_t result[5]);

/* Fused stage for meshes with a ghost fill (Section 2: static refinement; or FOFC).
 *   fused = 1: each stage is ONE persistent cooperative launch of at most one resident
 *              wave of CTAs: the ghost fill (copies / restrictions, then prolongations)
 *              and the flux correction run first, spread over the whole grid and
 *              separated by grid barriers (bounded waits: a barrier that times out counts
 *              in ak_status_counters' timeouts, AK_ETIMEOUT), then the CTAs loop over
 *              the stage work list;
 *   fused = 0: separate fill, flux-correction and stage launches (default).
 * Results are bitwise the same either way.  AK_EINVAL for fused = 1 on a mesh without
 * a ghost fill (one level, no FOFC: its stage reads halos from the neighbour blocks). */
ak_status ak_mesh_fuse(ak_mesh* mesh, int32_t fused);

/* Self-test of the bounded device waits (failure detection without a GPU fault): a
 * cooperative launch of two CTAs meets at the grid barrier the fused stage uses; with
 * absent = 1 the second CTA never arrives, so the first one's wait runs out after about
 * a second, counts a timeout and returns.  Synchronizes the stream.  Returns AK_OK when
 * every wait was met, AK_ETIMEOUT when one ran out (the count is in ak_status_counters);
 * the mesh stays usable either way. */
ak_status ak_selftest_barrier(ak_mesh* mesh, int32_t absent);

/* Sets the stage kernel's schedule explicitly (what ak_mesh_autotune picks by timing).
 *   tile:  0 = 16x16 column tiles (for the mixed form: the variant with paired x1/x2
 *          work, 288 threads); 2 = 16x16 tiles with one thread per column (mixed form
 *          only); 1 = 32x8 tiles with one thread per column (mixed PLM form only);
 *   nseg:  x3 segments per MeshBlock, 1..64 (fewer for blocks thinner than 4 cells per
 *          segment);
 *   order: 0 = block order, 1 = longest work items first.
 * Results are bitwise independent of the schedule.  AK_EINVAL for a value out of range;
 * synchronous (rebuilds a small device table), not during a stream capture. */
ak_status ak_mesh_schedule(ak_mesh* mesh, int32_t tile, int32_t nseg, int32_t order);

/* Host <-> device state transfer (Section 2, "Data locality": data reaches the host
 * only for outputs).  The host array is the interior only, packed block after block:
 * [block][var][k][j][i], i fastest (nblocks * 5 * nx1*nx2*nx3 doubles for equal
 * blocks), and must hold that many doubles.  Page-locked host memory that is mapped
 * into the device's address space (cudaMallocHost / cudaHostAlloc, or cudaHostRegister
 * with mapping, on a system with unified addressing) is read or written by the library's
 * (un)pack kernel directly over the host link; ak_upload then returns before the data
 * has moved, so keep the buffer until the stream has finished.  Other (pageable) memory
 * goes through a library staging buffer (allocated on first use).  ak_download
 * synchronizes the stream. */
ak_status ak_upload(ak_mesh* mesh, int32_t reg, const double* host_interior);
ak_status ak_download(ak_mesh* mesh, int32_t reg, double* host_interior);

/* Positivity and failure counters (Section 3: density and internal energy must stay
 * positive; cells that would not are corrected by FOFC, else floored).  Synchronizes the
 * stream.  out[0] floors applied, out[1] non-finite cells seen, out[2] bounded waits
 * that timed out, out[3] cells corrected by FOFC (summed over stages).  The counters
 * accumulate over the mesh's lifetime. */
ak_status ak_status_counters(ak_mesh* mesh, int64_t out[4]);

/* Largest number of MeshBlocks ak_cfl_dt_noalloc accepts: the size of its static
 * device scratch (AK_NOALLOC_MAX_BLOCKS + 1 doubles, 512 KiB per GPU). */
#define AK_NOALLOC_MAX_BLOCKS 65536

/* CFL time step of a register, computed without allocating any memory.
 *
 * The paper has no counterpart to this call; it exists for callers that cannot call
 * cudaMalloc -- e.g. a host code whose own pool allocator owns all device memory
 * (so a library may not allocate behind its back), or a monitoring / recovery path
 * that must still report a time step when the device is out of memory.  It needs no
 * ak_mesh (creating one allocates): the caller passes the register and its geometry.
 *
 * reg       device pointer to one register in the layout described above (and by
 *           ak_mesh_layout) for a mesh of `nblocks` equal blocks of
 *           nx[0] x nx[1] x nx[2] interior cells with `nghost` ghost cells per side;
 *           only interior cells are read.  Not modified; the caller keeps ownership.
 * dx        cell widths; gamma, cfl as in ak_mesh_desc.
 * dt_out    host pointer; receives cfl * min over interior cells and d of
 *           dx_d / (|v_d| + c_s), the same value ak_new_dt returns for that register.
 * cuda_stream  the work runs on this stream, which the call synchronizes.
 *
 * Scratch: a file-scope static __device__ array (AK_NOALLOC_MAX_BLOCKS + 1 doubles)
 * that every GPU loading the library keeps until the process exits.  Every call looks
 * up that array's device address (cudaGetSymbolAddress) with the device current, which
 * allocates nothing.  With CUDA's lazy module loading (the default), the first use of
 * the library's device code on a device -- this call or any other of the library --
 * loads it there, and that load places the array and the kernels in device memory: make
 * one warm-up call per device while memory is still free (not when the device is
 * already out of memory) and before any stream capture.  Every call on a device shares
 * the array and leaves its last contents there, so calls that overlap on the GPU
 * (concurrent streams, threads) race: serialize them.  No call of this function runs
 * cudaMalloc, cudaFree or any other allocating routine.
 * Errors: AK_EINVAL for NULL pointers, invalid sizes, or nblocks outside
 * [1, AK_NOALLOC_MAX_BLOCKS]; AK_ECUDA if a CUDA call fails. */
ak_status ak_cfl_dt_noalloc(const double* reg, int32_t nblocks, const int32_t nx[3],
                            int32_t nghost, const double dx[3], double gamma, double cfl,
                            void* cuda_stream, double* dt_out);

/* Measured FP64 rate of the current device: fused multiply-adds per second that its
 * FP64 unit sustains (every thread runs eight independent chains, so the pipe, not the
 * latency of one chain, limits it).  A measurement aid for the roofline of the FP64
 * form, whose stage kernels are bound by the FP64 unit rather than by HBM (Section 3's
 * update in double precision); DADD and DMUL issue on the same pipe.  Runs four
 * launches of about 10 ms on `cuda_stream` (a cudaStream_t, NULL = legacy default
 * stream), synchronizes it, and writes the fastest of the last three to *dfma_per_s.
 * Allocates no device memory.  AK_EINVAL for a NULL output, AK_ECUDA if a CUDA call
 * fails. */
ak_status ak_probe_fp64_rate(void* cuda_stream, double* dfma_per_s);

/* Message of the last error returned on this host thread ("" if none). */
const char* ak_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AK_H */
