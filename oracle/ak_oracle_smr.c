/*
 * FP64 CPU oracle for the static-refinement (SMR) form of the hydro RK stage: leaf
 * MeshBlocks on several levels with uniform time stepping across levels (AthenaK,
 * arXiv 2409.16053, Section 2: block-based AMR design with communication between
 * levels only at boundaries, flux corrections at level boundaries, uniform time
 * stepping; prolongation and restriction when filling ghost zones between levels).
 *
 * TEST INFRASTRUCTURE ONLY (see ak_oracle.c).  Shares no code with the CUDA path.
 *
 * Readings (the paper defers these to its references):
 *   - restriction: a coarse ghost cell takes the mean of the 2x2x2 fine cells it
 *     covers;
 *   - prolongation: a fine ghost cell takes the coarse cell value plus minmod-limited
 *     slopes of the conserved variables, U_f = U_c + sum_d (+-1/4) s_d, so that the
 *     eight fine cells average back to U_c;
 *   - flux correction: on a coarse face whose neighbour region is refined, the coarse
 *     flux is replaced by the mean of the 2x2 fine fluxes computed by the fine block
 *     on the same face (before the coarse update, so the update is conservative);
 *   - one global dt: min over all leaves of CFL dx_l / (|v| + c_s);
 *   - FOFC (Section 3: applied before the level flux correction): a face of a leaf
 *     takes the LLF flux of the piecewise-constant states when the cell on either
 *     side is flagged; a ghost cell carries the flag of the same-level or coarser leaf
 *     cell it lies in, so a fine face at a level boundary turns first-order when the
 *     fine cell or the coarse cell across is flagged.  The coarse side of such a face
 *     then takes the mean of the fine fluxes, as without FOFC.
 * Ghost zones are filled in two passes: same-level copies and restrictions first, then
 * prolongations level by level from coarse to fine, so that every coarse value a
 * prolongation reads (including coarse ghost cells) is already final.
 *
 * Storage: every leaf block is a padded array [5][n3+2g][n2+2g][n1+2g] (x1 fastest),
 * block b at element offset off[b]; the interior cell (i,j,k) of block b, variable v
 * is U[off[b] + ((v*(n3+2g) + k+g)*(n2+2g) + j+g)*(n1+2g) + i+g].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NV 5

/* from ak_oracle.c */
void orc_cons_to_prim(const double u[5], double w[5], int64_t* nfloor);
double orc_plm_slope(double qm, double q0, double qp);
void orc_ppm4_edges(const double q[5], double* qlo, double* qhi);
void orc_wenoz_edges(const double q[5], double* qlo, double* qhi);
void orc_ppmx_edges(const double q[5], double* qlo, double* qhi);
void orc_riemann(int solver, const double wl[5], const double wr[5], double gamma,
                 double f[5]);

typedef struct {
  int32_t nblocks, ng, recon, flux_correction;
  const int32_t* blocks; /* nblocks x 7: level, lx1, lx2, lx3, nx1, nx2, nx3 */
  int32_t root_nx[3];
  double length[3]; /* domain side lengths */
  double gamma;
  int32_t riemann;   /* 0 HLLC, 1 HLLE, 2 LLF */
  int32_t fofc;      /* 1: first-order flux correction in every RK stage */
} orc_smr;

typedef struct {
  const orc_smr* m;
  int nlev;
  int64_t* off;     /* per block */
  int32_t* bs;      /* block size per level (uniform within a level), 3 per level */
  int32_t* mapdim;  /* blocks per direction per level, 3 per level */
  int64_t* mapoff;  /* start of each level's map */
  int32_t* map;     /* leaf id or -1 */
} smr_index;

static int64_t block_elems(const orc_smr* m, int b) {
  const int32_t* e = m->blocks + 7 * b;
  int64_t g = m->ng;
  return NV * (e[4] + 2 * g) * (e[5] + 2 * g) * (e[6] + 2 * g);
}

int64_t orc_smr_storage(const orc_smr* m) {
  int64_t n = 0;
  for (int b = 0; b < m->nblocks; ++b) n += block_elems(m, b);
  return n;
}

static int64_t lvl_n(const orc_smr* m, int l, int d) { return (int64_t)m->root_nx[d] << l; }

static int64_t wrapl(int64_t i, int64_t n) {
  int64_t r = i % n;
  return r < 0 ? r + n : r;
}

static int leaf_at(const smr_index* x, int l, const int64_t G[3]);

/* builds the leaf maps; returns 0 or -1 on an inconsistent mesh (blocks of one level of
 * different sizes, two leaves in one slot, or a leaf overlapping a coarser one) */
static int index_build(const orc_smr* m, smr_index* x) {
  memset(x, 0, sizeof(*x));
  x->m = m;
  int nlev = 0;
  for (int b = 0; b < m->nblocks; ++b)
    if (m->blocks[7 * b] + 1 > nlev) nlev = m->blocks[7 * b] + 1;
  x->nlev = nlev;
  x->off = (int64_t*)malloc(sizeof(int64_t) * m->nblocks);
  x->bs = (int32_t*)calloc(3 * nlev, sizeof(int32_t));
  x->mapdim = (int32_t*)calloc(3 * nlev, sizeof(int32_t));
  x->mapoff = (int64_t*)calloc(nlev + 1, sizeof(int64_t));
  int64_t o = 0;
  for (int b = 0; b < m->nblocks; ++b) {
    x->off[b] = o;
    o += block_elems(m, b);
    const int32_t* e = m->blocks + 7 * b;
    for (int d = 0; d < 3; ++d) {
      if (x->bs[3 * e[0] + d] == 0) x->bs[3 * e[0] + d] = e[4 + d];
      if (x->bs[3 * e[0] + d] != e[4 + d]) return -1;
    }
  }
  for (int l = 0; l < nlev; ++l) {
    int64_t cnt = 1;
    for (int d = 0; d < 3; ++d) {
      int s = x->bs[3 * l + d] ? x->bs[3 * l + d] : 1;
      x->mapdim[3 * l + d] = (int32_t)(lvl_n(m, l, d) / s);
      cnt *= x->mapdim[3 * l + d];
    }
    x->mapoff[l + 1] = x->mapoff[l] + cnt;
  }
  x->map = (int32_t*)malloc(sizeof(int32_t) * x->mapoff[nlev]);
  for (int64_t i = 0; i < x->mapoff[nlev]; ++i) x->map[i] = -1;
  for (int b = 0; b < m->nblocks; ++b) {
    const int32_t* e = m->blocks + 7 * b;
    int l = e[0];
    int64_t c[3];
    for (int d = 0; d < 3; ++d) c[d] = e[1 + d] / x->bs[3 * l + d];
    int64_t id = x->mapoff[l] + (c[2] * x->mapdim[3 * l + 1] + c[1]) * x->mapdim[3 * l] + c[0];
    if (x->map[id] >= 0) return -1; /* two leaves in one slot */
    x->map[id] = b;
  }
  /* leaves must not overlap: no cell of a leaf lies in a leaf of a coarser level */
  for (int b = 0; b < m->nblocks; ++b) {
    const int32_t* e = m->blocks + 7 * b;
    for (int l = e[0] - 1; l >= 0; --l) {
      int sh = e[0] - l;
      for (int64_t k = e[3]; k < e[3] + e[6]; ++k)
        for (int64_t j = e[2]; j < e[2] + e[5]; ++j)
          for (int64_t i = e[1]; i < e[1] + e[4]; ++i) {
            int64_t G[3] = {i >> sh, j >> sh, k >> sh};
            if (x->bs[3 * l] && leaf_at(x, l, G) >= 0) return -1;
          }
    }
  }
  return 0;
}

static void index_free(smr_index* x) {
  free(x->off);
  free(x->bs);
  free(x->mapdim);
  free(x->mapoff);
  free(x->map);
}

/* leaf containing level-l cell G (wrapped), or -1 */
static int leaf_at(const smr_index* x, int l, const int64_t G[3]) {
  if (l < 0 || l >= x->nlev || x->bs[3 * l] == 0) return -1;
  int64_t c[3];
  for (int d = 0; d < 3; ++d) c[d] = wrapl(G[d], lvl_n(x->m, l, d)) / x->bs[3 * l + d];
  return x->map[x->mapoff[l] + (c[2] * x->mapdim[3 * l + 1] + c[1]) * x->mapdim[3 * l] + c[0]];
}

/* element index of level-l cell G (wrapped) in leaf b, variable v; local offsets may
 * reach into the ghost zone by `extra` cells */
static int64_t elem(const smr_index* x, int b, int v, const int64_t G[3]) {
  const orc_smr* m = x->m;
  const int32_t* e = m->blocks + 7 * b;
  int64_t g = m->ng, loc[3];
  for (int d = 0; d < 3; ++d) {
    int64_t n = lvl_n(m, e[0], d);
    int64_t r = wrapl(G[d] - e[1 + d], n);  /* in [0, n) */
    if (r >= n - g) r -= n;                   /* just below the block: negative offset */
    loc[d] = r;
  }
  int64_t p1 = e[4] + 2 * g, p2 = e[5] + 2 * g, p3 = e[6] + 2 * g;
  return x->off[b] + ((v * p3 + loc[2] + g) * p2 + loc[1] + g) * p1 + loc[0] + g;
}

static double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return fabs(a) < fabs(b) ? a : b;
}

/* Prolongation of one fine cell: coarse centre value uc, coarse neighbours um[d],
 * up[d] along d, fine cell in the upper (hi[d] = 1) or lower half along d. */
double orc_prolong(double uc, const double um[3], const double up[3], const int hi[3]) {
  double u = uc;
  for (int d = 0; d < 3; ++d) {
    double s = minmod(up[d] - uc, uc - um[d]);
    u += (hi[d] ? 0.25 : -0.25) * s;
  }
  return u;
}

/* Restriction: mean of the eight fine cells. */
double orc_restrict(const double f[8]) {
  double s = 0.0;
  for (int i = 0; i < 8; ++i) s += f[i];
  return s / 8.0;
}

static void fill_ghosts(const smr_index* x, double* U, int pass, int level_only) {
  const orc_smr* m = x->m;
  int g = m->ng;
  for (int b = 0; b < m->nblocks; ++b) {
    const int32_t* e = m->blocks + 7 * b;
    int l = e[0];
    if (pass == 2 && l != level_only) continue;
    for (int k = -g; k < e[6] + g; ++k)
      for (int j = -g; j < e[5] + g; ++j)
        for (int i = -g; i < e[4] + g; ++i) {
          if (i >= 0 && i < e[4] && j >= 0 && j < e[5] && k >= 0 && k < e[6]) continue;
          int64_t G[3] = {e[1] + i, e[2] + j, e[3] + k};
          for (int d = 0; d < 3; ++d) G[d] = wrapl(G[d], lvl_n(m, l, d));
          int64_t dst[NV];
          {
            int64_t p1 = e[4] + 2 * g, p2 = e[5] + 2 * g, p3 = e[6] + 2 * g;
            for (int v = 0; v < NV; ++v)
              dst[v] = x->off[b] + ((v * p3 + k + g) * p2 + j + g) * p1 + i + g;
          }
          int same = leaf_at(x, l, G);
          if (pass == 1) {
            if (same >= 0) {
              for (int v = 0; v < NV; ++v) U[dst[v]] = U[elem(x, same, v, G)];
              continue;
            }
            int64_t F[3] = {2 * G[0], 2 * G[1], 2 * G[2]};
            int fine = leaf_at(x, l + 1, F);
            if (fine >= 0) {
              for (int v = 0; v < NV; ++v) {
                double f[8];
                int n = 0;
                for (int dz = 0; dz < 2; ++dz)
                  for (int dy = 0; dy < 2; ++dy)
                    for (int dx = 0; dx < 2; ++dx) {
                      int64_t Q[3] = {F[0] + dx, F[1] + dy, F[2] + dz};
                      f[n++] = U[elem(x, fine, v, Q)];
                    }
                U[dst[v]] = orc_restrict(f);
              }
            }
          } else if (same < 0) {
            int64_t C[3] = {G[0] >> 1, G[1] >> 1, G[2] >> 1};
            int coarse = leaf_at(x, l - 1, C);
            if (coarse < 0) continue;
            int hi[3] = {(int)(G[0] & 1), (int)(G[1] & 1), (int)(G[2] & 1)};
            for (int v = 0; v < NV; ++v) {
              double um[3], up[3];
              for (int d = 0; d < 3; ++d) {
                int64_t Cm[3] = {C[0], C[1], C[2]}, Cp[3] = {C[0], C[1], C[2]};
                Cm[d] -= 1;
                Cp[d] += 1;
                um[d] = U[elem(x, coarse, v, Cm)];
                up[d] = U[elem(x, coarse, v, Cp)];
              }
              U[dst[v]] = orc_prolong(U[elem(x, coarse, v, C)], um, up, hi);
            }
          }
        }
  }
}

/* Ghost zones of every leaf: copies and restrictions, then prolongations from coarse to
 * fine levels. */
int orc_smr_fill_ghosts(const orc_smr* m, double* U) {
  smr_index x;
  if (index_build(m, &x) != 0) {
    index_free(&x);
    return -1;
  }
  fill_ghosts(&x, U, 1, 0);
  for (int l = 1; l < x.nlev; ++l) fill_ghosts(&x, U, 2, l);
  index_free(&x);
  return 0;
}

/* Face fluxes of one block: F[d] has (n_d + 1) faces along d, full extent in the other
 * directions, layout [v][k][j][i] with the face index along d. */
static void block_fluxes(const smr_index* x, int b, const double* U, double* F[3],
                         const unsigned char* flag) {
  const orc_smr* m = x->m;
  const int32_t* e = m->blocks + 7 * b;
  int g = m->ng;
  int64_t p1 = e[4] + 2 * g, p2 = e[5] + 2 * g, p3 = e[6] + 2 * g;
  int64_t np = p1 * p2 * p3;
  double* W = (double*)malloc(sizeof(double) * NV * np);
  int64_t nf = 0;
  for (int64_t c = 0; c < np; ++c) {
    double u[5], w[5];
    for (int v = 0; v < NV; ++v) u[v] = U[x->off[b] + v * np + c];
    orc_cons_to_prim(u, w, &nf);
    for (int v = 0; v < NV; ++v) W[v * np + c] = w[v];
  }
  for (int d = 0; d < 3; ++d) {
    int n[3] = {e[4], e[5], e[6]};
    n[d] += 1;
    int perm[5] = {0, 1 + d, 1 + (d + 1) % 3, 1 + (d + 2) % 3, 4};
    int64_t st[3] = {1, p1, p1 * p2};
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          /* face below cell (i,j,k) along d */
          int64_t c0 = ((int64_t)(k + g) * p2 + j + g) * p1 + i + g;
          double wl[5], wr[5], f[5];
          const unsigned char* fb = flag ? flag + x->off[b] / NV : NULL;
          if (fb && (fb[c0 - st[d]] || fb[c0])) {
            /* FOFC: LLF flux of the two cells' own states */
            for (int q = 0; q < NV; ++q) {
              wl[q] = W[(int64_t)perm[q] * np + c0 - st[d]];
              wr[q] = W[(int64_t)perm[q] * np + c0];
            }
            orc_riemann(2, wl, wr, m->gamma, f);
            int64_t fi = ((int64_t)k * n[1] + j) * n[0] + i;
            int64_t fn = (int64_t)n[0] * n[1] * n[2];
            for (int q = 0; q < NV; ++q) F[d][(int64_t)perm[q] * fn + fi] = f[q];
            continue;
          }
          for (int q = 0; q < NV; ++q) {
            const double* w = W + (int64_t)perm[q] * np;
            if (m->recon == 0) {
              double qm2 = w[c0 - 2 * st[d]], qm1 = w[c0 - st[d]], q0 = w[c0], qp1 = w[c0 + st[d]];
              wl[q] = qm1 + 0.5 * orc_plm_slope(qm2, qm1, q0);
              wr[q] = q0 - 0.5 * orc_plm_slope(qm1, q0, qp1);
            } else {
              double s[6], lo, hi, lo2, hi2;
              for (int t = 0; t < 6; ++t) s[t] = w[c0 + (t - 3) * st[d]];
              if (m->recon == 2) {
                orc_wenoz_edges(&s[0], &lo, &hi);
                orc_wenoz_edges(&s[1], &lo2, &hi2);
              } else if (m->recon == 3) {
                orc_ppmx_edges(&s[0], &lo, &hi);
                orc_ppmx_edges(&s[1], &lo2, &hi2);
              } else {
                orc_ppm4_edges(&s[0], &lo, &hi);
                orc_ppm4_edges(&s[1], &lo2, &hi2);
              }
              wl[q] = hi;
              wr[q] = lo2;
            }
          }
          orc_riemann(m->riemann, wl, wr, m->gamma, f);
          int64_t fi = ((int64_t)k * n[1] + j) * n[0] + i;
          int64_t fn = (int64_t)n[0] * n[1] * n[2];
          for (int q = 0; q < NV; ++q) F[d][(int64_t)perm[q] * fn + fi] = f[q];
        }
  }
  free(W);
}

/* FOFC flags of the ghost cells of every leaf: the flag of the same-level leaf cell, or
 * of the coarser leaf cell, the ghost cell lies in; 0 over a finer region (those ghost
 * cells only border level-boundary faces, whose coarse flux the fine mean replaces).
 * flag: one byte per padded cell, block b from off[b] / NV. */
static void fill_flag_ghosts(const smr_index* x, unsigned char* flag) {
  const orc_smr* m = x->m;
  int g = m->ng;
  for (int b = 0; b < m->nblocks; ++b) {
    const int32_t* e = m->blocks + 7 * b;
    int l = e[0];
    int64_t p1 = e[4] + 2 * g, p2 = e[5] + 2 * g;
    for (int k = -g; k < e[6] + g; ++k)
      for (int j = -g; j < e[5] + g; ++j)
        for (int i = -g; i < e[4] + g; ++i) {
          if (i >= 0 && i < e[4] && j >= 0 && j < e[5] && k >= 0 && k < e[6]) continue;
          int64_t G[3] = {e[1] + i, e[2] + j, e[3] + k};
          for (int d = 0; d < 3; ++d) G[d] = wrapl(G[d], lvl_n(m, l, d));
          unsigned char f = 0;
          int same = leaf_at(x, l, G);
          if (same >= 0) {
            f = flag[x->off[same] / NV + (elem(x, same, 0, G) - x->off[same])];
          } else {
            int64_t C[3] = {G[0] >> 1, G[1] >> 1, G[2] >> 1};
            int coarse = leaf_at(x, l - 1, C);
            if (coarse >= 0) f = flag[x->off[coarse] / NV + (elem(x, coarse, 0, C) - x->off[coarse])];
          }
          flag[x->off[b] / NV + ((int64_t)(k + g) * p2 + j + g) * p1 + i + g] = f;
        }
  }
}

/* L(U) for every leaf (interior cells, layout of U; ghost entries of L are zero).
 * flag != NULL: FOFC flags (ghosts filled) select first-order LLF faces. */
static int64_t smr_rhs_impl(const orc_smr* m, const double* U, double* L,
                            const unsigned char* flag) {
  smr_index x;
  if (index_build(m, &x) != 0) {
    index_free(&x);
    return -1;
  }
  int g = m->ng;
  double** Fb = (double**)malloc(sizeof(double*) * 3 * m->nblocks);
  for (int b = 0; b < m->nblocks; ++b) {
    const int32_t* e = m->blocks + 7 * b;
    for (int d = 0; d < 3; ++d) {
      int64_t n = (int64_t)(e[4] + (d == 0)) * (e[5] + (d == 1)) * (e[6] + (d == 2));
      Fb[3 * b + d] = (double*)malloc(sizeof(double) * NV * n);
    }
  }
#pragma omp parallel for schedule(dynamic)
  for (int b = 0; b < m->nblocks; ++b) block_fluxes(&x, b, U, &Fb[3 * b], flag);

  /* flux correction: coarse faces next to a refined region take the fine mean */
  if (m->flux_correction) {
    for (int b = 0; b < m->nblocks; ++b) {
      const int32_t* e = m->blocks + 7 * b;
      int l = e[0];
      for (int d = 0; d < 3; ++d)
        for (int side = 0; side < 2; ++side) {
          int n[3] = {e[4], e[5], e[6]};
          int a1 = (d + 1) % 3, a2 = (d + 2) % 3;
          for (int t2 = 0; t2 < n[a2]; ++t2)
            for (int t1 = 0; t1 < n[a1]; ++t1) {
              int loc[3];
              loc[d] = side ? n[d] - 1 : 0;
              loc[a1] = t1;
              loc[a2] = t2;
              int64_t N[3] = {e[1] + loc[0], e[2] + loc[1], e[3] + loc[2]};
              N[d] += side ? 1 : -1;
              if (leaf_at(&x, l, N) >= 0) continue;
              int64_t F0[3] = {2 * N[0], 2 * N[1], 2 * N[2]};
              int fine = leaf_at(&x, l + 1, F0);
              if (fine < 0) continue;
              const int32_t* ef = m->blocks + 7 * fine;
              int nf[3] = {ef[4], ef[5], ef[6]};
              nf[d] += 1;
              int64_t fn = (int64_t)nf[0] * nf[1] * nf[2];
              /* the fine cells next to the interface, and their face towards it */
              int64_t fine_layer = side ? 2 * N[d] : 2 * N[d] + 1;
              double sum[5] = {0, 0, 0, 0, 0};
              for (int u2 = 0; u2 < 2; ++u2)
                for (int u1 = 0; u1 < 2; ++u1) {
                  int64_t Q[3];
                  Q[d] = fine_layer;
                  Q[a1] = 2 * N[a1] + u1;
                  Q[a2] = 2 * N[a2] + u2;
                  int64_t fl[3];
                  for (int q = 0; q < 3; ++q)
                    fl[q] = wrapl(Q[q] - ef[1 + q], lvl_n(m, l + 1, q));
                  if (!side) fl[d] += 1; /* upper face of the fine cell */
                  int64_t fi = (fl[2] * nf[1] + fl[1]) * nf[0] + fl[0];
                  for (int v = 0; v < NV; ++v) sum[v] += Fb[3 * fine + d][v * fn + fi];
                }
              int nc[3] = {e[4], e[5], e[6]};
              nc[d] += 1;
              int64_t cn = (int64_t)nc[0] * nc[1] * nc[2];
              int cf[3] = {loc[0], loc[1], loc[2]};
              if (side) cf[d] += 1;
              int64_t ci = ((int64_t)cf[2] * nc[1] + cf[1]) * nc[0] + cf[0];
              for (int v = 0; v < NV; ++v) Fb[3 * b + d][v * cn + ci] = 0.25 * sum[v];
            }
        }
    }
  }

  for (int64_t i = 0, n = orc_smr_storage(m); i < n; ++i) L[i] = 0.0;
  for (int b = 0; b < m->nblocks; ++b) {
    const int32_t* e = m->blocks + 7 * b;
    int l = e[0];
    int64_t p1 = e[4] + 2 * g, p2 = e[5] + 2 * g, p3 = e[6] + 2 * g;
    for (int d = 0; d < 3; ++d) {
      double dx = m->length[d] / (double)lvl_n(m, l, d);
      int nc[3] = {e[4], e[5], e[6]};
      nc[d] += 1;
      int64_t fn = (int64_t)nc[0] * nc[1] * nc[2];
      for (int k = 0; k < e[6]; ++k)
        for (int j = 0; j < e[5]; ++j)
          for (int i = 0; i < e[4]; ++i) {
            int64_t f0 = ((int64_t)k * nc[1] + j) * nc[0] + i;
            int64_t f1 = ((int64_t)(k + (d == 2)) * nc[1] + j + (d == 1)) * nc[0] + i + (d == 0);
            for (int v = 0; v < NV; ++v) {
              int64_t c = x.off[b] + ((v * p3 + k + g) * p2 + j + g) * p1 + i + g;
              L[c] -= (Fb[3 * b + d][v * fn + f1] - Fb[3 * b + d][v * fn + f0]) / dx;
            }
          }
    }
  }
  for (int b = 0; b < 3 * m->nblocks; ++b) free(Fb[b]);
  free(Fb);
  index_free(&x);
  return 0;
}

int64_t orc_smr_rhs(const orc_smr* m, const double* U, double* L) {
  return smr_rhs_impl(m, U, L, NULL);
}

/* L(U) with FOFC flags (Section 3): flag holds one byte per interior cell, block after
 * block as [block][k][j][i]; the ghost cells take the flags of fill_flag_ghosts, and every
 * face next to a flagged cell takes the LLF flux of the two cells' own states.  U's ghost
 * cells must be filled. */
int64_t orc_smr_rhs_flagged(const orc_smr* m, const double* U, double* L,
                            const unsigned char* flag_packed) {
  smr_index x;
  if (index_build(m, &x) != 0) {
    index_free(&x);
    return -1;
  }
  int64_t n = orc_smr_storage(m);
  unsigned char* flag = (unsigned char*)calloc(n / NV, 1);
  int g = m->ng;
  int64_t o = 0;
  for (int b = 0; b < m->nblocks; ++b) {
    const int32_t* e = m->blocks + 7 * b;
    int64_t p1 = e[4] + 2 * g, p2 = e[5] + 2 * g;
    for (int k = 0; k < e[6]; ++k)
      for (int j = 0; j < e[5]; ++j)
        for (int i = 0; i < e[4]; ++i)
          flag[x.off[b] / NV + ((int64_t)(k + g) * p2 + j + g) * p1 + i + g] = flag_packed[o++];
  }
  fill_flag_ghosts(&x, flag);
  int64_t rc = smr_rhs_impl(m, U, L, flag);
  free(flag);
  index_free(&x);
  return rc;
}

/* One SSP-RK step of every leaf with one dt: ghost fill, then U <- a U0 + b (U + dt L)
 * on interior cells, for each stage.  With m->fofc, each stage first makes the update
 * tentatively, flags the cells whose density or internal energy would not be positive,
 * and recomputes L with first-order LLF faces around them; *nfofc (if given) receives
 * the number of flagged cells summed over the stages. */
int64_t orc_smr_rk_step_fofc(const orc_smr* m, double* U, double dt, int rk,
                             int64_t* nfofc) {
  static const double a2[2] = {0.0, 0.5}, b2[2] = {1.0, 0.5};
  static const double a3[3] = {0.0, 0.75, 1.0 / 3.0}, b3[3] = {1.0, 0.25, 2.0 / 3.0};
  const double* a = rk == 3 ? a3 : a2;
  const double* bb = rk == 3 ? b3 : b2;
  int ns = rk == 3 ? 3 : 2;
  int64_t n = orc_smr_storage(m);
  double* U0 = (double*)malloc(sizeof(double) * n);
  double* L = (double*)malloc(sizeof(double) * n);
  unsigned char* flag = m->fofc ? (unsigned char*)calloc(n / NV, 1) : NULL;
  memcpy(U0, U, sizeof(double) * n);
  int64_t rc = 0, nflag = 0;
  smr_index x;
  if (index_build(m, &x) != 0) rc = -1;
  int g = m->ng;
  for (int s = 0; s < ns && rc == 0; ++s) {
    if (orc_smr_fill_ghosts(m, U) != 0 || smr_rhs_impl(m, U, L, NULL) != 0) {
      rc = -1;
      break;
    }
    if (m->fofc) {
      int64_t nst = 0;
      memset(flag, 0, n / NV);
      for (int b = 0; b < m->nblocks; ++b) {
        const int32_t* e = m->blocks + 7 * b;
        int64_t p1 = e[4] + 2 * g, p2 = e[5] + 2 * g, p3 = e[6] + 2 * g, np = p1 * p2 * p3;
        for (int k = 0; k < e[6]; ++k)
          for (int j = 0; j < e[5]; ++j)
            for (int i = 0; i < e[4]; ++i) {
              int64_t c = ((int64_t)(k + g) * p2 + j + g) * p1 + i + g;
              double u[5];
              for (int v = 0; v < NV; ++v) {
                int64_t cv = x.off[b] + v * np + c;
                u[v] = a[s] * U0[cv] + bb[s] * (U[cv] + dt * L[cv]);
              }
              double ug = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0];
              unsigned char f = !(u[0] > 0.0) || !(ug > 0.0);
              flag[x.off[b] / NV + c] = f;
              nst += f;
            }
      }
      if (nst) {
        nflag += nst;
        fill_flag_ghosts(&x, flag);
        if (smr_rhs_impl(m, U, L, flag) != 0) {
          rc = -1;
          break;
        }
      }
    }
    int64_t o = 0;
    for (int b = 0; b < m->nblocks; ++b) {
      const int32_t* e = m->blocks + 7 * b;
      int64_t p1 = e[4] + 2 * g, p2 = e[5] + 2 * g, p3 = e[6] + 2 * g;
      for (int v = 0; v < NV; ++v)
        for (int k = 0; k < e[6]; ++k)
          for (int j = 0; j < e[5]; ++j)
            for (int i = 0; i < e[4]; ++i) {
              int64_t c = o + ((v * p3 + k + g) * p2 + j + g) * p1 + i + g;
              U[c] = a[s] * U0[c] + bb[s] * (U[c] + dt * L[c]);
            }
      o += block_elems(m, b);
    }
  }
  index_free(&x);
  free(U0);
  free(L);
  free(flag);
  if (nfofc) *nfofc = nflag;
  return rc;
}

int64_t orc_smr_rk_step(const orc_smr* m, double* U, double dt, int rk) {
  return orc_smr_rk_step_fofc(m, U, dt, rk, NULL);
}

/* Global CFL dt over every leaf's interior (Section 3 Eq. (3), uniform across levels). */
double orc_smr_new_dt(const orc_smr* m, const double* U, double cfl) {
  int g = m->ng;
  double best = INFINITY;
  int64_t o = 0;
  for (int b = 0; b < m->nblocks; ++b) {
    const int32_t* e = m->blocks + 7 * b;
    int64_t p1 = e[4] + 2 * g, p2 = e[5] + 2 * g, p3 = e[6] + 2 * g, np = p1 * p2 * p3;
    for (int k = 0; k < e[6]; ++k)
      for (int j = 0; j < e[5]; ++j)
        for (int i = 0; i < e[4]; ++i) {
          int64_t c = o + ((int64_t)(k + g) * p2 + j + g) * p1 + i + g;
          double u[5], w[5];
          int64_t nf = 0;
          for (int v = 0; v < NV; ++v) u[v] = U[c + v * np];
          orc_cons_to_prim(u, w, &nf);
          double cs = sqrt(m->gamma * (m->gamma - 1.0) * w[4] / w[0]);
          for (int d = 0; d < 3; ++d) {
            double dx = m->length[d] / (double)lvl_n(m, e[0], d);
            double t = dx / (fabs(w[1 + d]) + cs);
            if (t < best) best = t;
          }
        }
    o += block_elems(m, b);
  }
  return cfl * best;
}
