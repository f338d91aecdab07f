/*
 * CPU oracle for the extruded-mesh numbering and par_loop.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, serial FP64 implementation
 * written from the paper (Bercea et al., "A structure-exploiting numbering
 * algorithm for finite elements on extruded meshes"): Algorithm 1 (Sec. 3.2),
 * Algorithm 2 and Algorithm 3 (Sec. 3.3), and the residual I = int f v dx of
 * Sec. 4.1.1 plus the nonlinear residual int u^2 v dx and its adjoint.  Only
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it; the
 * CUDA library never does, and the two share no code.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Access descriptors of Algorithm 3 arguments. */
enum { ORC_READ = 0, ORC_WRITE = 1, ORC_INC = 2 };

/* Local kernels available to oracle_par_loop. */
enum {
  ORC_K_EXTRUDE = 0, /* coords WRITE: (x_v, y_v, level/layers)                   */
  ORC_K_COPY = 1,    /* in READ, out WRITE: out_j = in_j                           */
  ORC_K_MASS = 2,    /* coords READ, f READ, b INC: b_i += int f phi_i (P1xP1)     */
  ORC_K_INTERP = 3,  /* x READ (P1xP1), out WRITE (DG1xDG1): nodal interpolation   */
  ORC_K_U2V = 4,     /* coords READ, u READ, F INC|WRITE: F_i += int u^2 phi_i     */
  ORC_K_U2V_ADJ = 5, /* coords READ, u READ, w READ, g INC|WRITE: (dF/du)^T w      */
  ORC_K_MASS_TP = 6, /* coords READ, f READ, b INC: b_i += int f phi_i on a prism
                        tensor-product space chosen by oracle_set_tp_element      */
  ORC_K_HFACET_MASS = 7, /* horizontal facets, l = 0 .. lambda (d2 = 0), facet lists:
                            coords READ, f READ, b INC: b_i += int_F f phi_i ds;
                            space (h, CG1) chosen by oracle_set_tp_element         */
  ORC_K_HFACET_JUMP = 8, /* interior horizontal facets, l = 1 .. lambda-1, two-cell
                            lists built from the cell lists: coords READ, u READ,
                            r INC: r_i += int_F [u][phi_i] ds                      */
  ORC_K_MASS_DGP = 9     /* coords READ, f READ, b INC on a p-adaptive DG space
                            (ragged lists): each cell's element by its DoF count,
                            1 DG0xDG0, 2 DG0xDG1, 3 DG1xDG0, 6 DG1xDG1            */
};

/* Horizontal / vertical elements of the prism spaces of Sec. 4.1.2. */
enum { ORC_CG1 = 0, ORC_DG0 = 1, ORC_DG1 = 2 };

typedef struct {
  const int32_t *map;    /* ncells x k, the layer-0 explicit lists L(c)          */
  const int32_t *offset; /* k vertical offsets (Algorithm 2)                     */
  int32_t k;             /* DoFs per stencil                                      */
  int32_t ncomp;         /* values per DoF (3 for coordinates, else 1)           */
  double *data;          /* field values, ndofs x ncomp                          */
  double *absdata;       /* optional: accumulates |contribution| for INC outputs */
  int32_t access;        /* ORC_READ / ORC_WRITE / ORC_INC                        */
  const int64_t *rowptr; /* ragged lists (NULL: k per cell): cell c's entries are
                            map[rowptr[c] .. rowptr[c+1]), offsets alongside     */
} orc_arg;

/* Edges of the base mesh, numbered by first appearance when cells are scanned
 * in order and local edges e_k = (v_k, v_{(k+1) mod nvc}) in order.  Writes
 * cell_edges (ncells x nvc); returns the number of edges or -1. */
int64_t oracle_derive_edges(int32_t nvc, int64_t ncells, const int32_t *cell_verts,
                            int64_t nverts, int32_t *cell_edges);

/* Algorithm 1.  first[2*d1+d2] (may be NULL when delta[2*d1+d2]==0) receives
 * N[d1] x (layers+1-d2) int64 entries: the first global number given to entity
 * ((d1,d2),(i,l)) at index i*(layers+1-d2)+l.  Returns the number of DoFs. */
int64_t oracle_alg1(const int64_t N[3], int32_t layers, const int32_t delta[6],
                    int64_t *const first[6]);

/* Stencil length k of a cell with nvc vertices for the given delta. */
int32_t oracle_stencil_size(int32_t nvc, const int32_t delta[6]);

/* Explicit layer-0 lists L(c) read off the entity tables of oracle_alg1. */
int oracle_base_map(int32_t nvc, int64_t ncells, const int32_t *cell_verts,
                    const int32_t *cell_edges, int32_t layers, const int32_t delta[6],
                    int64_t *const first[6], int32_t *map);

/* Algorithm 2. */
void oracle_alg2(int32_t nvc, const int32_t delta[6], int32_t *offset);

/* Algorithm 3 over cells [0, ncells) with the chosen local kernel.  For
 * ORC_K_EXTRUDE, base_xy (nverts x 2) and cell_verts are read; otherwise they
 * may be NULL.  Returns 0 or a negative error. */
int oracle_par_loop(int32_t kernel, int32_t nvc, int64_t ncells, int32_t layers,
                    const int32_t *cell_verts, const double *base_xy, int32_t nargs,
                    const orc_arg *args);

/* Variable layers per column: base cell c spans levels cell_first[c] ..
 * cell_first[c] + cell_layers[c] (cell_layers[c] >= 1).  oracle_var_ranges
 * writes the level range lo..hi of every base entity (dimension-major index:
 * vertices, edges, cells; a vertex or edge spans its cells' union hull); it
 * returns -2 if a vertex or edge belongs to no cell.  cell_edges may be NULL
 * when no edge carries DoFs (edge ranges are then left at -1). */
int oracle_var_ranges(int32_t nvc, const int64_t N[3], const int32_t *cell_verts,
                      const int32_t *cell_edges, const int32_t *cell_first,
                      const int32_t *cell_layers, int32_t *lo, int32_t *hi);

/* Algorithm 1 over per-entity level ranges; first[t] (t = 2*d1+d2) has
 * N[d1] x (maxlevel + 1 - d2) entries indexed by absolute level. */
int64_t oracle_alg1_var(const int64_t N[3], int32_t maxlevel, const int32_t *lo,
                        const int32_t *hi, const int32_t delta[6], int64_t *const first[6]);

/* Explicit lists at each column's bottom layer (level cell_first[c]). */
int oracle_base_map_var(int32_t nvc, int64_t ncells, const int32_t *cell_verts,
                        const int32_t *cell_edges, int32_t maxlevel, const int32_t *cell_first,
                        const int32_t delta[6], int64_t *const first[6], int32_t *map);

/* Explicit lists of the horizontal facets at each column's bottom level
 * (cell_first NULL: level 0): the closure DoFs delta(d,0) of the cell's
 * vertices, edges and cell at that level; oracle_hfacet_alg2 gives their
 * offsets by Algorithm 2's rule. */
int32_t oracle_hfacet_size(int32_t nvc, const int32_t delta[6]);
int oracle_hfacet_map(int32_t nvc, int64_t ncells, const int32_t *cell_verts,
                      const int32_t *cell_edges, int32_t maxlevel, const int32_t *cell_first,
                      const int32_t delta[6], int64_t *const first[6], int32_t *map);
void oracle_hfacet_alg2(int32_t nvc, const int32_t delta[6], int32_t *offset);

/* Algorithm 3 with lambda_c = cell_layers[c] layers in column c, starting at
 * level cell_first[c]; maxlevel is the highest level (coordinates use
 * z = level / maxlevel). */
int oracle_par_loop_var(int32_t kernel, int32_t nvc, int64_t ncells, const int32_t *cell_first,
                        const int32_t *cell_layers, int32_t maxlevel, const int32_t *cell_verts,
                        const double *base_xy, int32_t nargs, const orc_arg *args);

/* Per-entity DoF counts: entity g (dimension-major) carries dent[2g] DoFs on
 * each horizontal copy and dent[2g+1] on each vertical copy.  Algorithm 1 over
 * the level ranges lo..hi (constant layers: lo = 0, hi = layers). */
int64_t oracle_alg1_ragged(const int64_t N[3], int32_t maxlevel, const int32_t *lo,
                           const int32_t *hi, const int32_t *dent, int64_t *const first[6]);

/* Ragged explicit lists and their offsets; rowptr has ncells + 1 entries;
 * map/offset (rowptr[ncells] entries each) may be NULL to size them. */
int oracle_ragged_map(int32_t nvc, int64_t ncells, const int32_t *cell_verts,
                      const int32_t *cell_edges, int32_t maxlevel, const int32_t *cell_first,
                      const int64_t N[3], const int32_t *dent, int64_t *const first[6],
                      int64_t *rowptr, int32_t *map, int32_t *offset);

/* n-point Gauss-Legendre rule on [0,1] (Newton iteration on P_n). */
void oracle_gauss_legendre(int32_t n, double *x, double *w);

/* Select the 1-D Gauss rule used by the hexahedral kernels (default 4). */
void oracle_set_hex_rule(int32_t n);

/* Select the space of ORC_K_MASS_TP: horizontal element h on the triangle and
 * vertical element v on the interval, each ORC_CG1, ORC_DG0 or ORC_DG1. */
void oracle_set_tp_element(int32_t h, int32_t v);

/* CPU baseline on several cores: greedy vertex-disjoint colouring of the
 * base cells (returns the colour count, or a negative error), the number of
 * threads OpenMP would use (1 without OpenMP), and Algorithm 3 over the
 * cells listed per colour (color_ptr: ncolors + 1 offsets into color_cells),
 * colours in sequence, the cells of a colour split over nthreads threads. */
int32_t oracle_color_cells(int32_t nvc, int64_t ncells, const int32_t *cell_verts, int64_t nverts,
                           int32_t *color);
int32_t oracle_max_threads(void);
int oracle_par_loop_colored(int32_t kernel, int32_t nvc, int32_t layers, const int32_t *cell_verts,
                            const double *base_xy, int32_t nargs, const orc_arg *args, int32_t ncolors,
                            const int64_t *color_ptr, const int64_t *color_cells, int32_t nthreads);

#ifdef __cplusplus
}
#endif
#endif
