/*
 * CPU oracle for the extruded-mesh numbering and par_loop.
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow, serial FP64 restatement of the
 * paper's algorithms, used to check the CUDA library.  Nothing in the CUDA
 * path includes, links or calls this file.  Compiled with -O2
 * -ffp-contract=off (no fused multiply-add, no fast-math).
 *
 * Sections followed:
 *   - entities and adjacency of the base mesh: Sec. 2.2 (all adjacencies are
 *     derivable from cell-vertex; edges are derived here);
 *   - extruded entity sets V_{d1,d2}, 0 <= l <= lambda - d2: Sec. 3.1.3;
 *   - Algorithm 1 (vertical-innermost numbering): Sec. 3.2;
 *   - explicit lists reduced to the bottom layer, Algorithm 2 (offsets) and
 *     Algorithm 3 (iteration of a stencil over the extruded mesh): Sec. 3.3;
 *   - the residual I = int f v dx with the coordinate field as a vector at
 *     every vertex: Sec. 4.1.1; the element pairs of Sec. 4.1.2.
 *
 * Readings where the paper is silent (stated once here, used throughout):
 *   - base entities are visited dimension-major (vertices, edges, cells),
 *     index ascending, in Algorithm 1;
 *   - the stencil of a cell lists its local base entities in the order
 *     vertices, edges, cell interior; per entity: the delta(d,0) DoFs of the
 *     bottom horizontal entity, the delta(d,0) DoFs of the top one, then the
 *     delta(d,1) DoFs of the vertical entity;
 *   - local edge e_k joins local vertices k and (k+1) mod nvc;
 *   - quadrature: prisms use the 3-point degree-2 triangle rule times the
 *     2-point Gauss rule; hexahedra use the n-point Gauss rule per direction
 *     (n = 4 unless changed), which integrates every integrand used here
 *     exactly on straight-sided columns.
 */
#include "oracle.h"

#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Base-mesh edges (Sec. 2.2: derivable from cell-vertex adjacency).        */
/* An open-addressing table keyed by the unordered vertex pair; a pair seen */
/* for the first time gets the next edge number.                           */
/* ------------------------------------------------------------------------ */
int64_t oracle_derive_edges(int32_t nvc, int64_t ncells, const int32_t *cell_verts,
                            int64_t nverts, int32_t *cell_edges) {
  int64_t cap = 16;
  while (cap < 4 * ncells * nvc + 16) cap *= 2;
  int64_t *key_lo = (int64_t *)malloc(sizeof(int64_t) * cap);
  int64_t *key_hi = (int64_t *)malloc(sizeof(int64_t) * cap);
  int64_t *val = (int64_t *)malloc(sizeof(int64_t) * cap);
  if (!key_lo || !key_hi || !val) {
    free(key_lo); free(key_hi); free(val);
    return -1;
  }
  for (int64_t s = 0; s < cap; ++s) key_lo[s] = -1;
  int64_t nedges = 0;
  for (int64_t c = 0; c < ncells; ++c) {
    for (int32_t k = 0; k < nvc; ++k) {
      int64_t a = cell_verts[c * nvc + k];
      int64_t b = cell_verts[c * nvc + (k + 1) % nvc];
      if (a < 0 || b < 0 || a >= nverts || b >= nverts) {
        free(key_lo); free(key_hi); free(val);
        return -1;
      }
      int64_t lo = a < b ? a : b, hi = a < b ? b : a;
      uint64_t h = (uint64_t)lo * 1000003ULL + (uint64_t)hi * 998244353ULL;
      int64_t s = (int64_t)(h & (uint64_t)(cap - 1));
      while (key_lo[s] != -1 && !(key_lo[s] == lo && key_hi[s] == hi)) s = (s + 1) & (cap - 1);
      if (key_lo[s] == -1) {
        key_lo[s] = lo;
        key_hi[s] = hi;
        val[s] = nedges++;
      }
      cell_edges[c * nvc + k] = (int32_t)val[s];
    }
  }
  free(key_lo); free(key_hi); free(val);
  return nedges;
}

/* ------------------------------------------------------------------------ */
/* The numbering of Sec. 3.2 (Algorithm 1), written from the property it    */
/* establishes rather than as the algorithm's loop.  Base entity g (index   */
/* dimension-major: vertices, edges, cells, each ascending) owns one column */
/* of extruded entities.  Along that column every extruded entity has a     */
/* height rank s counted from the bottom: the horizontal copy at level l    */
/* has s = 2l, the vertical entity spanning layer l has s = 2l + 1, so a    */
/* column with levels lo..hi has ranks 2 lo .. 2 hi.  The numbers are       */
/* handed out in increasing (g, s), each extruded entity taking as many     */
/* consecutive numbers as it carries DoFs.  A column is then one contiguous */
/* range, ordered from its bottom to its top (vertical innermost).          */
/* lo/hi NULL: every column spans 0..layers; dent NULL: an extruded entity  */
/* of type t = 2 d1 + d2 carries delta[t] DoFs, else entity g carries        */
/* dent[2g + d2].                                                           */
/* ------------------------------------------------------------------------ */
static int64_t number_by_rank(const int64_t N[3], int32_t maxlevel, const int32_t *lo, const int32_t *hi,
                              const int32_t *delta, const int32_t *dent, int64_t *const first[6]) {
  int64_t next = 0, g = 0;
  for (int d1 = 0; d1 <= 2; ++d1) {
    for (int64_t i = 0; i < N[d1]; ++i, ++g) {
      const int64_t s_lo = 2 * (int64_t)(lo ? lo[g] : 0), s_hi = 2 * (int64_t)(hi ? hi[g] : maxlevel);
      for (int64_t s = s_lo; s <= s_hi; ++s) {
        const int d2 = (int)(s % 2);    /* odd rank: a vertical entity */
        const int64_t level = s / 2;    /* its level (horizontal) or layer (vertical) */
        const int t = 2 * d1 + d2;
        if (first[t]) first[t][i * (maxlevel + 1 - d2) + level] = next;
        next += dent ? dent[2 * g + d2] : delta[t];
      }
    }
  }
  return next;
}

int64_t oracle_alg1(const int64_t N[3], int32_t layers, const int32_t delta[6],
                    int64_t *const first[6]) {
  return number_by_rank(N, layers, NULL, NULL, delta, NULL, first);
}

static int32_t nentities(int32_t nvc, int d) { return d == 2 ? 1 : nvc; }

int32_t oracle_stencil_size(int32_t nvc, const int32_t delta[6]) {
  int32_t k = 0;
  for (int d = 0; d <= 2; ++d) k += nentities(nvc, d) * (2 * delta[2 * d] + delta[2 * d + 1]);
  return k;
}

int oracle_base_map(int32_t nvc, int64_t ncells, const int32_t *cell_verts,
                    const int32_t *cell_edges, int32_t layers, const int32_t delta[6],
                    int64_t *const first[6], int32_t *map) {
  int32_t k = oracle_stencil_size(nvc, delta);
  for (int64_t c = 0; c < ncells; ++c) {
    int32_t j = 0;
    for (int d = 0; d <= 2; ++d) {
      for (int32_t e = 0; e < nentities(nvc, d); ++e) {
        int64_t id;
        if (d == 0) id = cell_verts[c * nvc + e];
        else if (d == 1) {
          if ((delta[2] || delta[3]) && !cell_edges) return -1;
          id = (delta[2] || delta[3]) ? cell_edges[c * nvc + e] : 0;
        } else id = c;
        /* bottom horizontal entity ((d,0),(id,0)) */
        for (int32_t q = 0; q < delta[2 * d]; ++q)
          map[c * k + j++] = (int32_t)(first[2 * d][id * (layers + 1) + 0] + q);
        /* top horizontal entity ((d,0),(id,1)) */
        for (int32_t q = 0; q < delta[2 * d]; ++q)
          map[c * k + j++] = (int32_t)(first[2 * d][id * (layers + 1) + 1] + q);
        /* vertical entity ((d,1),(id,0)) */
        for (int32_t q = 0; q < delta[2 * d + 1]; ++q)
          map[c * k + j++] = (int32_t)(first[2 * d + 1][id * layers + 0] + q);
      }
    }
  }
  return 0;
}

/* Offsets (Sec. 3.3, Algorithm 2), from what they are for: the explicit
 * list of a cell at layer l + 1 is its list at layer l plus the offsets.
 * One base cell with its own nvc vertices and nvc edges is numbered over two
 * layers, its explicit lists at layers 0 and 1 are read off the tables, and
 * the offsets are their differences. */
static void list_at_layer(int32_t nvc, int32_t layers, const int32_t delta[6], int64_t *const first[6],
                          int32_t l, int64_t *list) {
  int32_t j = 0;
  for (int d = 0; d <= 2; ++d)
    for (int32_t e = 0; e < nentities(nvc, d); ++e) {
      for (int32_t q = 0; q < delta[2 * d]; ++q) list[j++] = first[2 * d][e * (layers + 1) + l] + q;
      for (int32_t q = 0; q < delta[2 * d]; ++q) list[j++] = first[2 * d][e * (layers + 1) + l + 1] + q;
      for (int32_t q = 0; q < delta[2 * d + 1]; ++q) list[j++] = first[2 * d + 1][e * layers + l] + q;
    }
}

void oracle_alg2(int32_t nvc, const int32_t delta[6], int32_t *offset) {
  const int64_t N[3] = {nvc, nvc, 1};
  int64_t tab[6][2 * 3 * 4];  /* at most 4 entities per dimension, 3 levels */
  int64_t *first[6];
  for (int t = 0; t < 6; ++t) first[t] = tab[t];
  number_by_rank(N, 2, NULL, NULL, delta, NULL, first);
  const int32_t k = oracle_stencil_size(nvc, delta);
  int64_t *l0 = (int64_t *)malloc(sizeof(int64_t) * (k > 0 ? k : 1));
  int64_t *l1 = (int64_t *)malloc(sizeof(int64_t) * (k > 0 ? k : 1));
  list_at_layer(nvc, 2, delta, first, 0, l0);
  list_at_layer(nvc, 2, delta, first, 1, l1);
  for (int32_t i = 0; i < k; ++i) offset[i] = (int32_t)(l1[i] - l0[i]);
  free(l0);
  free(l1);
}

/* ------------------------------------------------------------------------ */
/* Variable layers per column (Sec. 3.1 footnote; Sec. 5: a constant number */
/* of layers is not needed by the numbering).  Base cell c spans the levels */
/* cell_first[c] .. cell_first[c] + cell_layers[c]; a vertex or edge column  */
/* spans the levels from the lowest bottom to the highest top of the cells  */
/* that contain it.  Entity ranges lo..hi are indexed dimension-major:      */
/* vertices, then edges, then cells.                                         */
/* ------------------------------------------------------------------------ */
int oracle_var_ranges(int32_t nvc, const int64_t N[3], const int32_t *cell_verts,
                      const int32_t *cell_edges, const int32_t *cell_first,
                      const int32_t *cell_layers, int32_t *lo, int32_t *hi) {
  const int64_t nent = N[0] + N[1] + N[2];
  for (int64_t e = 0; e < nent; ++e) {
    lo[e] = -1;
    hi[e] = -1;
  }
  for (int64_t c = 0; c < N[2]; ++c) {
    const int32_t bottom = cell_first[c], top = cell_first[c] + cell_layers[c];
    if (cell_first[c] < 0 || cell_layers[c] < 1) return -1;
    for (int d = 0; d <= 2; ++d) {
      for (int32_t e = 0; e < nentities(nvc, d); ++e) {
        int64_t id;
        if (d == 0) id = cell_verts[c * nvc + e];
        else if (d == 1) {
          if (!cell_edges) continue;
          id = N[0] + cell_edges[c * nvc + e];
        } else id = N[0] + N[1] + c;
        if (lo[id] < 0 || bottom < lo[id]) lo[id] = bottom;
        if (hi[id] < 0 || top > hi[id]) hi[id] = top;
      }
    }
  }
  for (int64_t e = 0; e < N[0]; ++e)
    if (lo[e] < 0) return -2; /* a vertex that no cell contains */
  if (cell_edges)
    for (int64_t e = N[0]; e < N[0] + N[1]; ++e)
      if (lo[e] < 0) return -2;
  return 0;
}

/* The numbering over per-entity level ranges: the same order of height
 * ranks, each column running from its own lowest level to its highest.
 * first[t] is indexed by absolute level: i * (maxlevel + 1 - d2) + l. */
int64_t oracle_alg1_var(const int64_t N[3], int32_t maxlevel, const int32_t *lo,
                        const int32_t *hi, const int32_t delta[6], int64_t *const first[6]) {
  return number_by_rank(N, maxlevel, lo, hi, delta, NULL, first);
}

/* Explicit lists L(c) at the bottom layer of each column (level
 * cell_first[c]), read off the tables of oracle_alg1_var. */
int oracle_base_map_var(int32_t nvc, int64_t ncells, const int32_t *cell_verts,
                        const int32_t *cell_edges, int32_t maxlevel, const int32_t *cell_first,
                        const int32_t delta[6], int64_t *const first[6], int32_t *map) {
  int32_t k = oracle_stencil_size(nvc, delta);
  for (int64_t c = 0; c < ncells; ++c) {
    const int64_t s = cell_first[c];
    int32_t j = 0;
    for (int d = 0; d <= 2; ++d) {
      for (int32_t e = 0; e < nentities(nvc, d); ++e) {
        int64_t id;
        if (d == 0) id = cell_verts[c * nvc + e];
        else if (d == 1) {
          if ((delta[2] || delta[3]) && !cell_edges) return -1;
          id = (delta[2] || delta[3]) ? cell_edges[c * nvc + e] : 0;
        } else id = c;
        for (int32_t q = 0; q < delta[2 * d]; ++q)
          map[c * k + j++] = (int32_t)(first[2 * d][id * (maxlevel + 1) + s] + q);
        for (int32_t q = 0; q < delta[2 * d]; ++q)
          map[c * k + j++] = (int32_t)(first[2 * d][id * (maxlevel + 1) + s + 1] + q);
        for (int32_t q = 0; q < delta[2 * d + 1]; ++q)
          map[c * k + j++] = (int32_t)(first[2 * d + 1][id * maxlevel + s] + q);
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Horizontal facets (the (2,0) entities, iterated with d2 = 0 in           */
/* Algorithm 3).  The explicit list of facet ((2,0),(c,l)) is its closure:  */
/* per base entity of the cell (vertices, edges, cell) the delta(d,0) DoFs  */
/* of that entity's horizontal copy at level l.  Algorithm 2's rule gives   */
/* every facet DoF the offset delta(d,0) + delta(d,1).                      */
/* ------------------------------------------------------------------------ */
int32_t oracle_hfacet_size(int32_t nvc, const int32_t delta[6]) {
  int32_t k = 0;
  for (int d = 0; d <= 2; ++d) k += nentities(nvc, d) * delta[2 * d];
  return k;
}

int oracle_hfacet_map(int32_t nvc, int64_t ncells, const int32_t *cell_verts,
                      const int32_t *cell_edges, int32_t maxlevel, const int32_t *cell_first,
                      const int32_t delta[6], int64_t *const first[6], int32_t *map) {
  int32_t k = oracle_hfacet_size(nvc, delta);
  for (int64_t c = 0; c < ncells; ++c) {
    const int64_t s = cell_first ? cell_first[c] : 0;
    int32_t j = 0;
    for (int d = 0; d <= 2; ++d) {
      for (int32_t e = 0; e < nentities(nvc, d); ++e) {
        int64_t id;
        if (d == 0) id = cell_verts[c * nvc + e];
        else if (d == 1) {
          if (delta[2] && !cell_edges) return -1;
          id = delta[2] ? cell_edges[c * nvc + e] : 0;
        } else id = c;
        for (int32_t q = 0; q < delta[2 * d]; ++q)
          map[c * k + j++] = (int32_t)(first[2 * d][id * (maxlevel + 1) + s] + q);
      }
    }
  }
  return 0;
}

/* Facet offsets, like the cell offsets, as the difference between the
 * facet's lists at levels 1 and 0 of one base cell numbered over two layers. */
void oracle_hfacet_alg2(int32_t nvc, const int32_t delta[6], int32_t *offset) {
  const int64_t N[3] = {nvc, nvc, 1};
  int64_t tab[6][2 * 3 * 4];
  int64_t *first[6];
  for (int t = 0; t < 6; ++t) first[t] = tab[t];
  number_by_rank(N, 2, NULL, NULL, delta, NULL, first);
  int32_t i = 0;
  for (int d = 0; d <= 2; ++d)
    for (int32_t e = 0; e < nentities(nvc, d); ++e)
      for (int32_t q = 0; q < delta[2 * d]; ++q, ++i)
        offset[i] = (int32_t)(first[2 * d][e * 3 + 1] - first[2 * d][e * 3 + 0]);
}

/* ------------------------------------------------------------------------ */
/* Per-entity DoF counts (Sec. 5: the numbering needs neither a constant    */
/* number of layers nor a constant number of DoFs per entity type).  Entity */
/* g (dimension-major index: vertices, edges, cells) carries dent[2g] DoFs  */
/* on each of its horizontal copies and dent[2g+1] on each vertical one.     */
/* ------------------------------------------------------------------------ */
int64_t oracle_alg1_ragged(const int64_t N[3], int32_t maxlevel, const int32_t *lo,
                           const int32_t *hi, const int32_t *dent, int64_t *const first[6]) {
  return number_by_rank(N, maxlevel, lo, hi, NULL, dent, first);
}

/* Ragged explicit lists at each column's bottom layer (level cell_first[c],
 * or 0): row c holds, per base entity of the cell (vertices, edges, cell),
 * the dent[2g] DoFs of its bottom horizontal copy, the dent[2g] of its top
 * copy and the dent[2g+1] of its vertical copy; the offset of each entry is
 * its entity's dent[2g] + dent[2g+1] (Algorithm 2's rule).  rowptr (ncells +
 * 1) is always filled; map and offset (rowptr[ncells] entries) may be NULL. */
int oracle_ragged_map(int32_t nvc, int64_t ncells, const int32_t *cell_verts,
                      const int32_t *cell_edges, int32_t maxlevel, const int32_t *cell_first,
                      const int64_t N[3], const int32_t *dent, int64_t *const first[6],
                      int64_t *rowptr, int32_t *map, int32_t *offset) {
  rowptr[0] = 0;
  for (int64_t c = 0; c < ncells; ++c) {
    const int64_t s = cell_first ? cell_first[c] : 0;
    int64_t j = rowptr[c];
    for (int d = 0; d <= 2; ++d) {
      for (int32_t e = 0; e < nentities(nvc, d); ++e) {
        int64_t id;
        if (d == 0) id = cell_verts[c * nvc + e];
        else if (d == 1) {
          if (!cell_edges) return -1;
          id = cell_edges[c * nvc + e];
        } else id = c;
        const int64_t g = (d == 0 ? 0 : (d == 1 ? N[0] : N[0] + N[1])) + id;
        const int32_t a = dent[2 * g], b = dent[2 * g + 1];
        for (int part = 0; part < 3; ++part) {
          const int32_t n = part < 2 ? a : b;
          for (int32_t q = 0; q < n; ++q, ++j) {
            if (!map) continue;
            if (part == 0) map[j] = (int32_t)(first[2 * d][id * (maxlevel + 1) + s] + q);
            else if (part == 1) map[j] = (int32_t)(first[2 * d][id * (maxlevel + 1) + s + 1] + q);
            else map[j] = (int32_t)(first[2 * d + 1][id * maxlevel + s] + q);
            offset[j] = a + b;
          }
        }
      }
    }
    rowptr[c + 1] = j;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Reference elements.                                                      */
/* ------------------------------------------------------------------------ */

/* Gauss-Legendre rule on [0,1]: roots of P_n by Newton's method from the
 * Chebyshev-like initial guesses, weights 2/((1-t^2) P_n'(t)^2) halved. */
void oracle_gauss_legendre(int32_t n, double *x, double *w) {
  const double pi = 3.14159265358979323846;
  for (int32_t i = 0; i < n; ++i) {
    double t = cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int32_t k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dp;
      t -= dt;
      if (fabs(dt) < 1e-17) break;
    }
    /* recompute derivative at the converged root */
    {
      double p0 = 1.0, p1 = t;
      for (int32_t k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
    }
    /* t in (-1,1) descending with i; map to [0,1] ascending */
    x[n - 1 - i] = 0.5 * (1.0 + t);
    w[n - 1 - i] = 0.5 * 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

static int32_t g_hex_rule = 4;
void oracle_set_hex_rule(int32_t n) { g_hex_rule = (n >= 1 && n <= 16) ? n : 4; }

/* Prism P1 x P1 (triangle (0,0),(1,0),(0,1) times [0,1]).  Stencil DoF
 * i = 2a + b: vertex a of the triangle, b = 0 bottom / 1 top. */
static double tri_lam(int a, double xi, double eta) {
  return a == 0 ? 1.0 - xi - eta : (a == 1 ? xi : eta);
}
static void tri_dlam(int a, double *dxi, double *deta) {
  if (a == 0) { *dxi = -1.0; *deta = -1.0; }
  else if (a == 1) { *dxi = 1.0; *deta = 0.0; }
  else { *dxi = 0.0; *deta = 1.0; }
}
static double lin(int b, double z) { return b == 0 ? 1.0 - z : z; }
static double dlin(int b) { return b == 0 ? -1.0 : 1.0; }

static void prism_basis(double xi, double eta, double zeta, double phi[6], double grad[6][3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 2; ++b) {
      double dx, de;
      tri_dlam(a, &dx, &de);
      phi[2 * a + b] = tri_lam(a, xi, eta) * lin(b, zeta);
      grad[2 * a + b][0] = dx * lin(b, zeta);
      grad[2 * a + b][1] = de * lin(b, zeta);
      grad[2 * a + b][2] = tri_lam(a, xi, eta) * dlin(b);
    }
}

/* 6-point prism rule: triangle points (1/6,1/6),(2/3,1/6),(1/6,2/3) with
 * weights 1/6 each, times 2-point Gauss on [0,1] (weights 1/2). */
static void prism_rule(double pts[6][3], double wts[6]) {
  const double tp[3][2] = {{1.0 / 6.0, 1.0 / 6.0}, {2.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 3.0}};
  double gz[2], gw[2];
  oracle_gauss_legendre(2, gz, gw);
  int q = 0;
  for (int t = 0; t < 3; ++t)
    for (int g = 0; g < 2; ++g) {
      pts[q][0] = tp[t][0];
      pts[q][1] = tp[t][1];
      pts[q][2] = gz[g];
      wts[q] = (1.0 / 6.0) * gw[g];
      ++q;
    }
}

/* Hexahedron, reference [0,1]^3.  Geometry is Q1 x P1: coordinate stencil
 * DoF 2a+b, base-quad vertex a -> (0,0),(1,0),(1,1),(0,1), b bottom/top. */
static const int quad_vx[4] = {0, 1, 1, 0};
static const int quad_vy[4] = {0, 0, 1, 1};
static void hex_geom_basis(double xi, double eta, double zeta, double phi[8], double grad[8][3]) {
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 2; ++b) {
      double nx = lin(quad_vx[a], xi), ny = lin(quad_vy[a], eta);
      int i = 2 * a + b;
      phi[i] = nx * ny * lin(b, zeta);
      grad[i][0] = dlin(quad_vx[a]) * ny * lin(b, zeta);
      grad[i][1] = nx * dlin(quad_vy[a]) * lin(b, zeta);
      grad[i][2] = nx * ny * dlin(b);
    }
}

/* 1-D P2 Lagrange basis on nodes t0 = 0, t1 = 1, t2 = 1/2. */
static double p2(int k, double t) {
  const double nodes[3] = {0.0, 1.0, 0.5};
  double v = 1.0;
  for (int m = 0; m < 3; ++m)
    if (m != k) v *= (t - nodes[m]) / (nodes[k] - nodes[m]);
  return v;
}

/* Q2 x P2 on the hexahedron.  Stencil DoF i = 3e + v: horizontal entity e in
 * the order (v0,v1,v2,v3, e0=(v0v1), e1=(v1v2), e2=(v2v3), e3=(v3v0), centre),
 * vertical node v in the order (bottom, top, middle).  Horizontal nodes as
 * 1-D node index pairs (0 -> 0, 1 -> 1, 2 -> 1/2).  The same 27 functions in
 * the same order are the DG2 basis (all DoFs interior to the cell). */
static const int q2_ix[9] = {0, 1, 1, 0, 2, 1, 2, 0, 2};
static const int q2_iy[9] = {0, 0, 1, 1, 0, 2, 1, 2, 2};
static void q2_basis(double xi, double eta, double zeta, double phi[27]) {
  for (int e = 0; e < 9; ++e)
    for (int v = 0; v < 3; ++v) phi[3 * e + v] = p2(q2_ix[e], xi) * p2(q2_iy[e], eta) * p2(v, zeta);
}

static double det3(const double J[3][3]) {
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
         J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

/* |det J| at reference point from coordinate values X[i][r] and geometry
 * basis gradients. */
static double abs_detJ(int ngeo, const double *X, double grad[][3]) {
  double J[3][3] = {{0}};
  for (int i = 0; i < ngeo; ++i)
    for (int r = 0; r < 3; ++r)
      for (int s = 0; s < 3; ++s) J[r][s] += X[3 * i + r] * grad[i][s];
  return fabs(det3(J));
}

/* ------------------------------------------------------------------------ */
/* Local kernels (the stencil function S of Algorithm 3).                   */
/* vals[a] holds the gathered values of argument a (k x ncomp); outputs are  */
/* written into out[a] (zeroed by the driver), |contributions| into absv[a]. */
/* ------------------------------------------------------------------------ */

/* int f phi_i dx on a P1xP1 prism with general (possibly non-straight)
 * coordinates; used for both the RHS (f interpolated) and the mass action. */
static void k_mass_prism(double *const *vals, double *const *out, double *const *absv) {
  double pts[6][3], wts[6];
  prism_rule(pts, wts);
  const double *X = vals[0], *f = vals[1];
  for (int q = 0; q < 6; ++q) {
    double phi[6], grad[6][3];
    prism_basis(pts[q][0], pts[q][1], pts[q][2], phi, grad);
    double dj = abs_detJ(6, X, grad);
    double fq = 0.0, fa = 0.0;
    for (int j = 0; j < 6; ++j) {
      fq += phi[j] * f[j];
      fa += fabs(phi[j] * f[j]);
    }
    for (int i = 0; i < 6; ++i) {
      out[2][i] += wts[q] * dj * fq * phi[i];
      absv[2][i] += wts[q] * dj * fa * fabs(phi[i]);
    }
  }
}

/* Nodal interpolation of a P1xP1 field into DG1xDG1: DG1 node j = 2a+b sits
 * at prism vertex a, level b; its value is the P1xP1 field evaluated there. */
static void k_interp(double *const *vals, double *const *out) {
  const double node[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 2; ++b) {
      double phi[6], grad[6][3];
      prism_basis(node[a][0], node[a][1], (double)b, phi, grad);
      double v = 0.0;
      for (int j = 0; j < 6; ++j)
        if (phi[j] != 0.0) v += phi[j] * vals[0][j];
      out[1][2 * a + b] = v;
    }
}

/* Quadrature points/weights and basis tables for int u^2 v on prism or hex. */
typedef struct {
  int nq, nb, ngeo;
  double w[16 * 16 * 16];
  double phi[16 * 16 * 16][27];
  double ggrad[16 * 16 * 16][8][3];
} u2v_tab;

static void u2v_setup(int32_t nvc, u2v_tab *T) {
  if (nvc == 3) {
    double pts[6][3], wts[6];
    prism_rule(pts, wts);
    T->nq = 6; T->nb = 6; T->ngeo = 6;
    for (int q = 0; q < 6; ++q) {
      double phi[6], grad[6][3];
      prism_basis(pts[q][0], pts[q][1], pts[q][2], phi, grad);
      T->w[q] = wts[q];
      for (int i = 0; i < 6; ++i) {
        T->phi[q][i] = phi[i];
        for (int s = 0; s < 3; ++s) T->ggrad[q][i][s] = grad[i][s];
      }
    }
  } else {
    int n = g_hex_rule;
    double gx[16], gw[16];
    oracle_gauss_legendre(n, gx, gw);
    T->nq = n * n * n; T->nb = 27; T->ngeo = 8;
    int q = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) {
          double phi8[8], grad8[8][3];
          T->w[q] = gw[i] * gw[j] * gw[k];
          q2_basis(gx[i], gx[j], gx[k], T->phi[q]);
          hex_geom_basis(gx[i], gx[j], gx[k], phi8, grad8);
          for (int a = 0; a < 8; ++a)
            for (int s = 0; s < 3; ++s) T->ggrad[q][a][s] = grad8[a][s];
          ++q;
        }
  }
}

/* F_i += sum_q w_q |detJ_q| u(x_q)^2 phi_i(x_q). */
static void k_u2v(const u2v_tab *T, double *const *vals, double *const *out, double *const *absv) {
  const double *X = vals[0], *u = vals[1];
  for (int q = 0; q < T->nq; ++q) {
    double dj = abs_detJ(T->ngeo, X, (double(*)[3])T->ggrad[q]);
    double uq = 0.0, ua = 0.0;
    for (int j = 0; j < T->nb; ++j) {
      uq += T->phi[q][j] * u[j];
      ua += fabs(T->phi[q][j] * u[j]);
    }
    for (int i = 0; i < T->nb; ++i) {
      out[2][i] += T->w[q] * dj * uq * uq * T->phi[q][i];
      absv[2][i] += T->w[q] * dj * ua * ua * fabs(T->phi[q][i]);
    }
  }
}

/* Adjoint of k_u2v applied to a cotangent w on F's space:
 * g_j += sum_q w_q |detJ_q| 2 u(x_q) w(x_q) phi_j(x_q)  (the transpose of
 * dF_i/du_j = sum_q w_q |detJ_q| 2 u(x_q) phi_j(x_q) phi_i(x_q)). */
static void k_u2v_adj(const u2v_tab *T, double *const *vals, double *const *out, double *const *absv) {
  const double *X = vals[0], *u = vals[1], *w = vals[2];
  for (int q = 0; q < T->nq; ++q) {
    double dj = abs_detJ(T->ngeo, X, (double(*)[3])T->ggrad[q]);
    double uq = 0.0, ua = 0.0, wq = 0.0, wa = 0.0;
    for (int j = 0; j < T->nb; ++j) {
      uq += T->phi[q][j] * u[j];
      ua += fabs(T->phi[q][j] * u[j]);
      wq += T->phi[q][j] * w[j];
      wa += fabs(T->phi[q][j] * w[j]);
    }
    for (int j = 0; j < T->nb; ++j) {
      out[3][j] += T->w[q] * dj * 2.0 * uq * wq * T->phi[q][j];
      absv[3][j] += T->w[q] * dj * 2.0 * ua * wa * fabs(T->phi[q][j]);
    }
  }
}

/* Tensor-product spaces on the prism (Sec. 4.1.2: the pairs (h, v) of
 * CG1, DG0, DG1).  The horizontal element carries dh[d] DoFs on each base
 * entity of dimension d (CG1: one per vertex; DG0: one per cell; DG1: three
 * per cell, at the vertex positions); the vertical element carries dv0 DoFs
 * on each interval end and dv1 inside (CG1: 1, 0; DG0: 0, 1; DG1: 0, 2 at
 * the two end positions).  The space's delta is dh[d1] * (dv0, dv1)[d2].  A
 * local DoF is identified by walking the stencil as ext_number/oracle_base_map
 * do: entities in order (vertices, edges, cell), per entity the bottom
 * horizontal DoFs, the top horizontal DoFs, then the vertical entity's DoFs
 * (horizontal index major, vertical index minor). */
static int32_t g_tp_h = ORC_CG1, g_tp_v = ORC_CG1;
void oracle_set_tp_element(int32_t h, int32_t v) {
  g_tp_h = h;
  g_tp_v = v;
}

/* hfun[i]: horizontal basis of local DoF i (0..2 = barycentric lambda_a, 3 =
 * constant); vfun[i]: vertical basis (0 = 1 - zeta, 1 = zeta, 2 = constant).
 * Returns the number of local DoFs. */
static int tp_layout(int h, int v, int hfun[27], int vfun[27]) {
  const int dh[3] = {h == ORC_CG1 ? 1 : 0, 0, h == ORC_DG0 ? 1 : (h == ORC_DG1 ? 3 : 0)};
  const int dv0 = v == ORC_CG1 ? 1 : 0;
  const int dv1 = v == ORC_DG0 ? 1 : (v == ORC_DG1 ? 2 : 0);
  int i = 0;
  for (int d = 0; d <= 2; ++d)
    for (int e = 0; e < (d == 2 ? 1 : 3); ++e) {
      /* horizontal function of the entity's j-th horizontal DoF */
      for (int part = 0; part < 3; ++part) {
        const int nv = part < 2 ? dv0 : dv1;
        for (int j = 0; j < dh[d]; ++j)
          for (int beta = 0; beta < nv; ++beta) {
            int hf;
            if (h == ORC_DG0) hf = 3;
            else if (d == 0) hf = e;  /* CG1 vertex */
            else hf = j;              /* DG1 node at vertex j */
            int vf;
            if (part == 0) vf = 0;
            else if (part == 1) vf = 1;
            else vf = (v == ORC_DG0) ? 2 : beta;
            hfun[i] = hf;
            vfun[i] = vf;
            ++i;
          }
      }
    }
  return i;
}

static double tp_phi(int hf, int vf, double xi, double eta, double zeta, double g[3]) {
  double H, Hx, He, V, Vz;
  if (hf == 3) { H = 1.0; Hx = 0.0; He = 0.0; }
  else { H = tri_lam(hf, xi, eta); tri_dlam(hf, &Hx, &He); }
  if (vf == 2) { V = 1.0; Vz = 0.0; }
  else { V = lin(vf, zeta); Vz = dlin(vf); }
  g[0] = Hx * V;
  g[1] = He * V;
  g[2] = H * Vz;
  return H * V;
}

/* int f phi_i dx on one prism of a tensor-product space; the coordinates are
 * the P1xP1 vector field (stencil DoF 2a+b) and define a general Jacobian. */
static void k_mass_tp_hv(int h, int v, double *const *vals, double *const *out, double *const *absv) {
  int hfun[27], vfun[27];
  const int k = tp_layout(h, v, hfun, vfun);
  double pts[6][3], wts[6];
  prism_rule(pts, wts);
  const double *X = vals[0], *f = vals[1];
  for (int q = 0; q < 6; ++q) {
    double gphi[6], ggrad[6][3];
    prism_basis(pts[q][0], pts[q][1], pts[q][2], gphi, ggrad);
    const double dj = abs_detJ(6, X, ggrad);
    double phi[27], fq = 0.0, fa = 0.0;
    for (int j = 0; j < k; ++j) {
      double g[3];
      phi[j] = tp_phi(hfun[j], vfun[j], pts[q][0], pts[q][1], pts[q][2], g);
      fq += phi[j] * f[j];
      fa += fabs(phi[j] * f[j]);
    }
    for (int i = 0; i < k; ++i) {
      out[2][i] += wts[q] * dj * fq * phi[i];
      absv[2][i] += wts[q] * dj * fa * fabs(phi[i]);
    }
  }
}

/* Degree-2 rule on the reference triangle (exact for products of two
 * linear functions), shared by the facet kernels. */
static const double tri_pts[3][2] = {{1.0 / 6.0, 1.0 / 6.0}, {2.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 3.0}};
static const double tri_w = 1.0 / 6.0;

/* Area element |dx/dxi x dx/deta| of the flat triangle through P0, P1, P2
 * (three consecutive 3-vectors at P, stride `stride` doubles). */
static double tri_area_element(const double *P, int stride) {
  double e1[3], e2[3];
  for (int r = 0; r < 3; ++r) {
    e1[r] = P[stride + r] - P[r];
    e2[r] = P[2 * stride + r] - P[r];
  }
  const double n0 = e1[1] * e2[2] - e1[2] * e2[1];
  const double n1 = e1[2] * e2[0] - e1[0] * e2[2];
  const double n2 = e1[0] * e2[1] - e1[1] * e2[0];
  return sqrt(n0 * n0 + n1 * n1 + n2 * n2);
}

/* int_F f phi_i ds on a horizontal facet F, for the spaces whose DoFs sit on
 * horizontal facets (vertical element CG1; horizontal CG1, DG0 or DG1).  The
 * facet list holds the closure DoFs (CG1: one per vertex; DG0: one; DG1:
 * three at the vertex positions); the coordinate list holds the facet's three
 * vertices. */
static void k_hfacet_mass(double *const *vals, double *const *out, double *const *absv) {
  const double *X = vals[0], *f = vals[1];
  const double ds = tri_area_element(X, 3);
  const int k = g_tp_h == ORC_DG0 ? 1 : 3;
  for (int q = 0; q < 3; ++q) {
    double phi[3], fq = 0.0, fa = 0.0;
    for (int j = 0; j < k; ++j) {
      phi[j] = (g_tp_h == ORC_DG0) ? 1.0 : tri_lam(j, tri_pts[q][0], tri_pts[q][1]);
      fq += phi[j] * f[j];
      fa += fabs(phi[j] * f[j]);
    }
    for (int i = 0; i < k; ++i) {
      out[2][i] += tri_w * ds * fq * phi[i];
      absv[2][i] += tri_w * ds * fa * fabs(phi[i]);
    }
  }
}

/* Interior horizontal facet between the cell below (first k DoFs of the
 * two-cell list) and the cell above (last k): the jump term
 *   r_i += int_F [u] [phi_i] ds,   [w] = w(below, zeta = 1) - w(above, zeta = 0),
 * on the tensor-product space chosen by oracle_set_tp_element.  The facet is
 * the top face of the cell below (coordinate DoFs 2a+1 of the first cell). */
static void k_hfacet_jump(int k, double *const *vals, double *const *out, double *const *absv) {
  int hfun[27], vfun[27];
  tp_layout(g_tp_h, g_tp_v, hfun, vfun);
  const double *X = vals[0], *u = vals[1];
  const double ds = tri_area_element(X + 3, 6);
  for (int q = 0; q < 3; ++q) {
    double pb[27], pa[27], g[3], jump = 0.0, ja = 0.0;
    for (int j = 0; j < k; ++j) {
      pb[j] = tp_phi(hfun[j], vfun[j], tri_pts[q][0], tri_pts[q][1], 1.0, g);
      pa[j] = tp_phi(hfun[j], vfun[j], tri_pts[q][0], tri_pts[q][1], 0.0, g);
      jump += u[j] * pb[j] - u[k + j] * pa[j];
      ja += fabs(u[j] * pb[j]) + fabs(u[k + j] * pa[j]);
    }
    for (int i = 0; i < k; ++i) {
      out[2][i] += tri_w * ds * jump * pb[i];
      out[2][k + i] -= tri_w * ds * jump * pa[i];
      absv[2][i] += tri_w * ds * ja * fabs(pb[i]);
      absv[2][k + i] += tri_w * ds * ja * fabs(pa[i]);
    }
  }
}

static void k_mass_tp(double *const *vals, double *const *out, double *const *absv) {
  k_mass_tp_hv(g_tp_h, g_tp_v, vals, out, absv);
}

/* p-adaptive DG: every cell carries its own element, one of the spaces
 * discontinuous in both directions, told apart by the cell's DoF count:
 * 1 DG0xDG0, 2 DG0xDG1, 3 DG1xDG0, 6 DG1xDG1.  Returns -1 for other counts. */
static int k_mass_dgp(int k, double *const *vals, double *const *out, double *const *absv) {
  int h, v;
  if (k == 1) { h = ORC_DG0; v = ORC_DG0; }
  else if (k == 2) { h = ORC_DG0; v = ORC_DG1; }
  else if (k == 3) { h = ORC_DG1; v = ORC_DG0; }
  else if (k == 6) { h = ORC_DG1; v = ORC_DG1; }
  else return -1;
  k_mass_tp_hv(h, v, vals, out, absv);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3: for every base cell, read its explicit list once; for every */
/* layer apply the stencil function, then add the vertical offsets.         */
/* ------------------------------------------------------------------------ */
#define ORC_MAXARGS 6
#define ORC_MAXVALS (2 * 27 * 3)

/* Cells (d2 = 1) are visited at l = 0 .. lambda_c - 1; horizontal facets
 * (d2 = 0) at l = 0 .. lambda_c; interior horizontal facets at
 * l = 1 .. lambda_c - 1 with the two-cell list (L(c), L(c) + offset), which
 * advances by (offset, offset).  lambda_c = cell_layers[c] (or `layers`), and
 * level s + l of a column has z = (s + l) / layers with s = cell_first[c]
 * (or 0). */
static int par_loop_impl(int32_t kernel, int32_t nvc, int64_t ncells, const int64_t *cell_ids,
                         const int32_t *cell_first, const int32_t *cell_layers, int32_t layers,
                         const int32_t *cell_verts, const double *base_xy, int32_t nargs,
                         const orc_arg *args) {
  if (nargs < 1 || nargs > ORC_MAXARGS || layers < 1) return -1;
  for (int a = 0; a < nargs; ++a)
    if ((!args[a].rowptr && (args[a].k < 1 || args[a].k > 27)) || args[a].ncomp < 1 || args[a].ncomp > 3)
      return -2;
  if (kernel == ORC_K_HFACET_MASS && (g_tp_v != ORC_CG1 || nvc != 3)) return -5;
  if (kernel == ORC_K_HFACET_JUMP && nvc != 3) return -5;
  const int twocell = kernel == ORC_K_HFACET_JUMP;
  u2v_tab *T = NULL;
  if (kernel == ORC_K_U2V || kernel == ORC_K_U2V_ADJ) {
    T = (u2v_tab *)malloc(sizeof(u2v_tab));
    if (!T) return -3;
    u2v_setup(nvc, T);
  }
  int64_t dofs[ORC_MAXARGS][2 * 27], offs[ORC_MAXARGS][2 * 27];
  int kk[ORC_MAXARGS], kc[ORC_MAXARGS];
  double vbuf[ORC_MAXARGS][ORC_MAXVALS], obuf[ORC_MAXARGS][ORC_MAXVALS], abuf[ORC_MAXARGS][ORC_MAXVALS];
  double *vals[ORC_MAXARGS], *outv[ORC_MAXARGS], *absv[ORC_MAXARGS];
  for (int a = 0; a < ORC_MAXARGS; ++a) {
    vals[a] = vbuf[a];
    outv[a] = obuf[a];
    absv[a] = abuf[a];
  }
  for (int a = 0; a < nargs; ++a)
    if (args[a].rowptr && twocell) return -6; /* ragged lists: cell loops only */
  for (int64_t ci = 0; ci < ncells; ++ci) {
    const int64_t c = cell_ids ? cell_ids[ci] : ci; /* the cells visited: all, or a given list */
    /* list length and offsets of this cell (ragged lists vary per cell) */
    const int32_t *lst[ORC_MAXARGS];
    for (int a = 0; a < nargs; ++a) {
      const int64_t r0 = args[a].rowptr ? args[a].rowptr[c] : c * (int64_t)args[a].k;
      kc[a] = args[a].rowptr ? (int)(args[a].rowptr[c + 1] - r0) : args[a].k;
      if (kc[a] < 1 || kc[a] > 27) return -2;
      lst[a] = args[a].map + r0;
      kk[a] = twocell ? 2 * kc[a] : kc[a];
      for (int j = 0; j < kk[a]; ++j)
        offs[a][j] = args[a].rowptr ? args[a].offset[r0 + j] : args[a].offset[j % args[a].k];
    }
    const int32_t s = cell_first ? cell_first[c] : 0;
    const int32_t lam = cell_layers ? cell_layers[c] : layers;
    int32_t l0 = 0, l1 = lam;                       /* cells: d2 = 1        */
    if (kernel == ORC_K_HFACET_MASS) l1 = lam + 1;  /* facets: d2 = 0       */
    if (twocell) l0 = 1;                            /* interior facets only */
    /* (dof_0 .. dof_{k-1}) <- L(v) */
    for (int a = 0; a < nargs; ++a)
      for (int j = 0; j < kk[a]; ++j)
        dofs[a][j] = lst[a][j % kc[a]] + (j >= kc[a] ? offs[a][j] : 0);
    for (int32_t l = l0; l < l1; ++l) {
      for (int a = 0; a < nargs; ++a) {
        int n = kk[a] * args[a].ncomp;
        for (int t = 0; t < n; ++t) obuf[a][t] = abuf[a][t] = 0.0;
        if (args[a].access == ORC_READ)
          for (int j = 0; j < kk[a]; ++j)
            for (int r = 0; r < args[a].ncomp; ++r)
              vbuf[a][j * args[a].ncomp + r] = args[a].data[dofs[a][j] * args[a].ncomp + r];
      }
      switch (kernel) {
        case ORC_K_EXTRUDE: {
          /* stencil DoF 2a+b of the coordinate space: vertex a, level s+l+b */
          for (int a = 0; a < nvc; ++a)
            for (int b = 0; b < 2; ++b) {
              int64_t v = cell_verts[c * nvc + a];
              obuf[0][3 * (2 * a + b) + 0] = base_xy[2 * v + 0];
              obuf[0][3 * (2 * a + b) + 1] = base_xy[2 * v + 1];
              obuf[0][3 * (2 * a + b) + 2] = (double)(s + l + b) / (double)layers;
            }
          break;
        }
        case ORC_K_COPY:
          for (int j = 0; j < kc[1]; ++j) obuf[1][j] = vbuf[0][j];
          break;
        case ORC_K_MASS:
          k_mass_prism(vals, outv, absv);
          break;
        case ORC_K_INTERP:
          k_interp(vals, outv);
          break;
        case ORC_K_U2V:
          k_u2v(T, vals, outv, absv);
          break;
        case ORC_K_U2V_ADJ:
          k_u2v_adj(T, vals, outv, absv);
          break;
        case ORC_K_MASS_TP:
          k_mass_tp(vals, outv, absv);
          break;
        case ORC_K_HFACET_MASS:
          k_hfacet_mass(vals, outv, absv);
          break;
        case ORC_K_HFACET_JUMP:
          k_hfacet_jump(kc[1], vals, outv, absv);
          break;
        case ORC_K_MASS_DGP:
          if (k_mass_dgp(kc[1], vals, outv, absv) != 0) {
            free(T);
            return -7;
          }
          break;
        default:
          free(T);
          return -4;
      }
      /* write back */
      for (int a = 0; a < nargs; ++a) {
        if (args[a].access == ORC_READ) continue;
        for (int j = 0; j < kk[a]; ++j)
          for (int r = 0; r < args[a].ncomp; ++r) {
            int64_t g = dofs[a][j] * args[a].ncomp + r;
            int t = j * args[a].ncomp + r;
            if (args[a].access == ORC_INC) args[a].data[g] += obuf[a][t];
            else args[a].data[g] = obuf[a][t];
            if (args[a].absdata) {
              if (args[a].access == ORC_INC) args[a].absdata[g] += abuf[a][t];
              else args[a].absdata[g] = abuf[a][t];
            }
          }
      }
      /* dof_j <- dof_j + offset(j) */
      for (int a = 0; a < nargs; ++a)
        for (int j = 0; j < kk[a]; ++j) dofs[a][j] += offs[a][j];
    }
  }
  free(T);
  return 0;
}

int oracle_par_loop(int32_t kernel, int32_t nvc, int64_t ncells, int32_t layers,
                    const int32_t *cell_verts, const double *base_xy, int32_t nargs,
                    const orc_arg *args) {
  return par_loop_impl(kernel, nvc, ncells, NULL, NULL, NULL, layers, cell_verts, base_xy, nargs, args);
}

int oracle_par_loop_var(int32_t kernel, int32_t nvc, int64_t ncells, const int32_t *cell_first,
                        const int32_t *cell_layers, int32_t maxlevel, const int32_t *cell_verts,
                        const double *base_xy, int32_t nargs, const orc_arg *args) {
  if (!cell_first || !cell_layers) return -1;
  for (int64_t c = 0; c < ncells; ++c)
    if (cell_first[c] < 0 || cell_layers[c] < 1 || cell_first[c] + cell_layers[c] > maxlevel) return -1;
  return par_loop_impl(kernel, nvc, ncells, NULL, cell_first, cell_layers, maxlevel, cell_verts, base_xy, nargs,
                       args);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3 on several host cores (a CPU baseline, not a check): the     */
/* base cells are grouped in colours such that no two cells of a colour     */
/* share a vertex (greedy, in cell order), so the cells of one colour write */
/* disjoint DoFs of every space whose DoFs sit on vertices or cells; the    */
/* colours run one after another, the cells of a colour split evenly over   */
/* the threads.  Each thread runs the serial loop above on its share.       */
/* ------------------------------------------------------------------------ */
int32_t oracle_color_cells(int32_t nvc, int64_t ncells, const int32_t *cell_verts, int64_t nverts,
                           int32_t *color) {
  uint64_t *used = (uint64_t *)calloc((size_t)(nverts > 0 ? nverts : 1), sizeof(uint64_t));
  if (!used) return -1;
  int32_t ncolors = 0;
  for (int64_t c = 0; c < ncells; ++c) {
    uint64_t taken = 0;
    for (int32_t a = 0; a < nvc; ++a) taken |= used[cell_verts[c * nvc + a]];
    int32_t k = 0;
    while (k < 64 && (taken >> k & 1u)) ++k;
    if (k == 64) {
      free(used);
      return -2;
    }
    color[c] = k;
    for (int32_t a = 0; a < nvc; ++a) used[cell_verts[c * nvc + a]] |= (uint64_t)1 << k;
    if (k + 1 > ncolors) ncolors = k + 1;
  }
  free(used);
  return ncolors;
}

int32_t oracle_max_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

int oracle_par_loop_colored(int32_t kernel, int32_t nvc, int32_t layers, const int32_t *cell_verts,
                            const double *base_xy, int32_t nargs, const orc_arg *args, int32_t ncolors,
                            const int64_t *color_ptr, const int64_t *color_cells, int32_t nthreads) {
  int err = 0;
  for (int32_t k = 0; k < ncolors; ++k) {
    const int64_t n = color_ptr[k + 1] - color_ptr[k];
    const int64_t *ids = color_cells + color_ptr[k];
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads) reduction(| : err)
    {
      const int64_t t = omp_get_thread_num(), T = omp_get_num_threads();
      const int64_t lo = n * t / T, hi = n * (t + 1) / T;
      if (hi > lo)
        err |= par_loop_impl(kernel, nvc, hi - lo, ids + lo, NULL, NULL, layers, cell_verts, base_xy, nargs,
                             args) != 0;
    }
#else
    (void)nthreads;
    err |= par_loop_impl(kernel, nvc, n, ids, NULL, NULL, layers, cell_verts, base_xy, nargs, args) != 0;
#endif
  }
  return err ? -1 : 0;
}
