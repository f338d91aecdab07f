// Internal declarations of the extmesh CUDA library (not installed; the public
// ABI is include/extmesh.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/extmesh.h"

#define EXT_MAXK 64  // longest stencil handled (Q2/DG2 hexahedra use 27)
#ifndef EXT_GATHER_MIN_LAYERS
#define EXT_GATHER_MIN_LAYERS 32  // constant layers: the probe and the gather forms from this many layers
#endif

// Bits of the device error word (ext_sync_check maps them to statuses).
enum : unsigned int {
  EXT_DERR_TIMEOUT = 1u,   // a bounded spin-wait gave up
  EXT_DERR_BOUNDS = 2u,    // an index failed a device-side range check
  EXT_DERR_INPUT = 4u      // an input a kernel cannot handle (e.g. bad map row)
};

// FP64 constants the kernels take as arguments: a product and a sum are
// issued as DFMA, a b + (-0) and a (+-1) + b, which round exactly like DMUL
// and DADD but issue at the DFMA rate (GB300 issues DADD and DMUL at about
// 5/6 of it).  Literal constants would let the compiler fold them back.
struct Fp64Ones {
  double one, mone, mzero;  // 1, -1, -0
};
inline Fp64Ones fp64_ones() { return Fp64Ones{1.0, -1.0, -0.0}; }
#ifdef __CUDACC__
__device__ __forceinline__ double fmul(double a, double b, const Fp64Ones &k) { return fma(a, b, k.mzero); }
__device__ __forceinline__ double fadd(double a, double b, const Fp64Ones &k) { return fma(a, k.one, b); }
__device__ __forceinline__ double fsub(double a, double b, const Fp64Ones &k) { return fma(b, k.mone, a); }

// Programmatic dependent launch: a kernel started by launch_dependent may
// begin (its launch and block dispatch overlapping the tail of the kernel
// before it in the stream) before that kernel has finished; it must wait here
// before it reads anything the earlier kernel writes.  Returns at once when
// the kernel was launched the ordinary way.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch `kernel` on stream s as a programmatic dependent of the kernel
// before it (see grid_dep_wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}
#endif

// Element recognised from a space's delta table.
enum ElemKind : int {
  ELEM_GENERIC = 0,
  ELEM_P1P1 = 1,    // delta(0,0)=1 only: CG1 x CG1 (coordinates when ncomp=3)
  ELEM_DGCELL = 2,  // only delta(2,1) > 0: every DoF interior to the cell
  ELEM_Q2P2 = 3,    // all six deltas 1 on quadrilateral base: Q2 x P2
};

struct ext_mesh {
  int32_t kind;        // vertices per base cell (3 or 4)
  int64_t N[3];        // base entity counts: vertices, edges, cells
  int32_t layers;      // lambda; with variable layers the highest level
  int device;
  int32_t *d_cell_verts = nullptr;  // ncells x kind
  int32_t *d_cell_edges = nullptr;  // ncells x kind
  double *d_base_xy = nullptr;      // nverts x 2 (may be null)
  bool has_xy = false;              // base coordinates were given
  // variable layers per column: cell c spans levels first[c] .. first[c] + layers[c]
  bool var = false;
  int32_t *d_cell_first = nullptr;   // ncells
  int32_t *d_cell_layers = nullptr;  // ncells
  int32_t *d_ent_lo = nullptr;       // level range of every base entity,
  int32_t *d_ent_hi = nullptr;       // dimension-major (vertices, edges, cells)
  double mean_layers = 0.0;
  void *host = nullptr;             // host-side copies (ext_api.cu)
  // triangle meshes with constant layers: the sparsity pattern of the P1
  // mass matrix of the base triangulation as vertex rows (row a: a itself,
  // then its neighbours in ascending order), each entry holding the first
  // DoF j (layers + 1) of vertex j's CG1xCG1 column and the one or two cells
  // on edge (a, j) (ascending; -1 where absent, both -1 on the diagonal), and
  // the cells around every vertex in ascending order.  Topology only: the
  // P1xP1 gather form computes the weights from the coordinate field of each
  // launch.
  int32_t *d_vrow = nullptr;    // nverts + 1
  int32_t *d_vnbr = nullptr;    // d_vrow[nverts] entries
  int2 *d_vedge = nullptr;      // d_vrow[nverts] entries
  int32_t *d_vcrow = nullptr;   // nverts + 1
  int32_t *d_vcells = nullptr;  // 3 ncells
  int64_t n_vent = 0;           // d_vrow[nverts]
};

struct ext_space {
  const ext_mesh *mesh;
  int32_t delta[6];
  int32_t ncomp;
  int32_t k;
  int64_t ndofs;
  int32_t *d_map = nullptr;     // ncells x k
  int32_t *d_offset = nullptr;  // k
  int32_t h_offset[EXT_MAXK];
  int elem;
  cudaStream_t stream;  // creation stream (map ready after it)
  // per-entity DoF counts: ragged lists (k = 0; d_map holds nentries values)
  bool ragged = false;
  int64_t nentries = 0;
  int64_t *d_rowptr = nullptr;  // ncells + 1
  int32_t *d_roff = nullptr;    // nentries: offset of every list entry
  bool dg_cells = false;        // DoFs only inside cells (copyable column by column)
  bool dgp = false;             // and every cell is DG0|DG1 x DG0|DG1 (1, 2, 3 or 6 DoFs)
  int32_t *d_cells_by_k[4] = {nullptr, nullptr, nullptr, nullptr};  // dgp: cells with 1, 2, 3, 6 DoFs
  int64_t ncells_by_k[4] = {0, 0, 0, 0};
};

// ---------------------------------------------------------------------------
// error reporting (ext_api.cu)
ext_status ext_fail(ext_status st, const char *fmt, ...);
unsigned int *ext_device_error_word();  // per-device word, allocated lazily

// ---------------------------------------------------------------------------
// kernel launchers; each returns cudaGetLastError() after the launch.

// Closed-form Algorithm 1 / Algorithm 2 for one space (k_number.cu).
struct NumberLaunch {
  int64_t ncells;
  int32_t nvc, k;
  int64_t block_start[3];  // first number of dimension-d entities
  int64_t colsize[3];      // numbers per column of a dimension-d entity
  int8_t slot_dim[EXT_MAXK];
  int8_t slot_ent[EXT_MAXK];
  int32_t slot_add[EXT_MAXK];  // position inside the column at layer 0
  const int32_t *cell_verts, *cell_edges;
  int32_t *map;
  // variable layers: entity column starts (dimension-major global entity
  // index), entity bottom levels, the cells' bottom levels; null otherwise
  const int64_t *ent_start = nullptr;
  const int32_t *ent_lo = nullptr, *cell_first = nullptr;
  int64_t ent_base[3];   // global index of the first entity of dimension d
  int32_t colstep[3];    // delta(d,0) + delta(d,1)
};
cudaError_t launch_number(const NumberLaunch &p, cudaStream_t s);

// Variable layers (k_number.cu, k_scan.cu): entity level ranges from the
// cells' ranges, entity column sizes, and an exclusive int64 prefix sum with
// the total written to data[n].
cudaError_t launch_var_ranges(const ext_mesh *m, cudaStream_t s);
cudaError_t launch_var_colsize(const ext_mesh *m, const int32_t delta[6], int64_t *sizes, cudaStream_t s);
cudaError_t launch_scan_i64(int64_t *data, int64_t n, int64_t *scratch, cudaStream_t s);
int64_t scan_scratch_elems(int64_t n);

// Per-entity DoF counts (k_number.cu): column sizes from dent (2 per entity,
// dimension-major) and the entity ranges (variable layers) or `layers`; row
// lengths of the ragged lists; the lists and their offsets.
struct RaggedLaunch {
  int64_t N[3];
  int64_t ncells;
  int32_t nvc, layers;
  const int32_t *dent;                      // (N0+N1+N2) x 2
  const int32_t *ent_lo = nullptr, *ent_hi = nullptr, *cell_first = nullptr;  // variable layers
  const int32_t *cell_verts, *cell_edges;
  const int64_t *ent_start;                 // column starts (exclusive scan of the sizes)
  int64_t *rowptr;                          // ncells + 1 (row lengths before the scan)
  int32_t *map, *roff;
};
cudaError_t launch_ragged_colsize(const RaggedLaunch &p, int64_t *sizes, cudaStream_t s);
cudaError_t launch_ragged_rowlen(const RaggedLaunch &p, cudaStream_t s);
cudaError_t launch_ragged_map(const RaggedLaunch &p, cudaStream_t s);

struct ExtrudeLaunch {
  int64_t ncells;
  int32_t nvc, layers;
  const int32_t *cell_verts;
  const double *base_xy;
  const int32_t *map;  // coords space, k = 2 nvc
  int32_t off;         // vertical offset of every slot (1 for CG1xCG1)
  double *X;
  const int32_t *cell_first = nullptr, *cell_layers = nullptr;  // variable layers
};
cudaError_t launch_extrude(const ExtrudeLaunch &p, cudaStream_t s);

// DG copy and DG1 interpolation (k_dg.cu).
struct CopyDGLaunch {
  int64_t ncells;
  int32_t k, layers;
  const int32_t *map;
  const double *in;
  double *out;
  const int32_t *cell_layers = nullptr;  // variable layers
  const int64_t *rowptr = nullptr;       // ragged lists: k of cell c = rowptr[c+1] - rowptr[c]
};
cudaError_t launch_copy_dg(const CopyDGLaunch &p, cudaStream_t s);

struct InterpDG1Launch {
  int64_t ncells;
  int32_t layers;
  const int32_t *xmap;  // CG1xCG1 map, k = 6
  int32_t xoff;         // vertical offset of every slot (Algorithm 2: 1 for CG1xCG1)
  const int32_t *omap;  // DG1xDG1 map, k = 6
  const double *x;
  double *out;
  const int32_t *cell_layers = nullptr;  // variable layers
};
cudaError_t launch_interp_dg1(const InterpDG1Launch &p, cudaStream_t s);

// P1 x P1 prism mass action / RHS (k_p1.cu).
struct MassP1Launch {
  int64_t ncells;
  int32_t layers;
  const int32_t *cmap, *fmap, *bmap;  // coords, input, output maps (k = 6)
  int32_t coff[6], foff[6], boff[6];
  const double *X, *f;
  double *b;
  unsigned int *err;
  const int32_t *cell_layers = nullptr;  // variable layers
  double mean_layers = 0.0;
  int64_t nf = 0;  // DoFs of the f space (CG1xCG1 numbering shared with the coordinates)
  const double *base_xy = nullptr;  // the mesh's base coordinates (nverts x 2), if it has them
  bool overwrite = false;           // b = M f (EXT_WRITE) instead of b += M f (EXT_INC)
  // the mesh's vertex rows (ext_mesh::d_vrow ...), null when it has none
  const int32_t *vrow = nullptr, *vnbr = nullptr;
  const int2 *vedge = nullptr;
  const int32_t *vcrow = nullptr, *vcells = nullptr;
  int32_t nverts = 0;
  int64_t nvent = 0;  // entries of the vertex rows
};

// Form of the P1xP1 launch (ext_set_option(EXT_OPT_P1_FORM, ...)) and of its
// flat gather (EXT_OPT_P1_FLAT).
int p1_form();
int p1_flat();
cudaError_t launch_mass_p1(const MassP1Launch &p, cudaStream_t s);

// Mass action on the nine prism tensor-product spaces (k_tp.cu).
struct MassTPLaunch {
  int64_t ncells;
  int32_t layers;
  int32_t nh, nv;        // horizontal nodes (1: DG0, 3: CG1/DG1), vertical nodes (1: DG0, 2: CG1/DG1)
  int32_t k;             // stencil length of the f/b space
  const int32_t *cmap;   // coords map (k = 6)
  int32_t coff[6];
  const int32_t *fmap;   // f and b share this numbering
  int32_t slot[6];       // stencil slot of node (a, b), index a * nv + b
  int32_t off[6];        // vertical offsets of those slots
  double scale;          // 1/2 x (1/12 if nh = 3) x (1/6 if nv = 2)
  const double *X, *f;
  double *b;
  const int32_t *cell_layers = nullptr;  // variable layers
  double mean_layers = 0.0;
  const double *base_xy = nullptr;       // the mesh's base coordinates, if it has them
  int64_t ncoord = 0;                    // DoFs of the coordinate space (V (layers + 1))
  int64_t nf = 0;                        // DoFs of the f / b space
  // filled by launch_mass_tp when it runs the flagged form
  const uint32_t *vflags = nullptr;      // bit d: coordinate DoF d verified straight
  const double *hlay = nullptr;          // |z_{l+1} - z_l| of the reference column
  const int32_t *badv = nullptr;         // optimistic form: per CTA of its first launch, a DoF not verified straight
  int32_t nbadv = 0;
  Fp64Ones k1;                           // fp64_ones(): products and sums of the closed forms issued as DFMA
  // CG1 x DG on the gather path (launch_mass_cgdg): the mesh's vertex rows
  const int32_t *vrow = nullptr, *vnbr = nullptr;
  const int2 *vedge = nullptr;
  const int32_t *vcrow = nullptr, *vcells = nullptr;
  int32_t nverts = 0;
  int64_t nvent = 0;
  unsigned int *err = nullptr;           // the device error word
  const unsigned int *mode = nullptr;    // cell kernel: run only when this probe word is in cell-loop mode
  bool overwrite = false;                // b = M f (EXT_WRITE) instead of b += M f (EXT_INC)
  bool hown = false;                     // horizontal DG0/DG1: every DoF belongs to one cell column
  bool vcont = false;                    // vertical CG1: layers l and l + 1 share their facet DoFs
};
cudaError_t launch_mass_tp(const MassTPLaunch &p, cudaStream_t s);
// CG1 x DG0 / CG1 x DG1 with WRITE through the P1xP1 gather machinery
// (k_p1.cu), and its two nine-space kernels (k_tp.cu): the general rule on the
// recorded DoFs, and the cell kernel gated on the probe's cell-loop mode.
cudaError_t launch_mass_cgdg(const MassTPLaunch &p, cudaStream_t s);
cudaError_t launch_cgdg_general(const MassTPLaunch &p, const int2 *list, const unsigned int *count, unsigned int cap,
                                cudaStream_t s);
cudaError_t launch_tp_cells_gated(const MassTPLaunch &p, const unsigned int *mode, cudaStream_t s);

// p-adaptive DG right-hand side (k_tp.cu): every cell's element is DG0|DG1 x
// DG0|DG1 by its DoF count (1 DG0xDG0, 2 DG0xDG1, 3 DG1xDG0, 6 DG1xDG1); the
// cell's DoFs are consecutive, layer after layer (Algorithm 1).
struct MassDGPLaunch {
  int64_t ncells;        // cells in `cells` (one element kind per launch)
  const int32_t *cells;  // base cells of this element kind
  int32_t kind;          // DoFs per cell-layer: 1, 2, 3 or 6
  int32_t layers;
  const int32_t *cmap;   // coords map (k = 6)
  int32_t coff[6];
  const int64_t *rowptr; // ragged lists of the f/b space
  const int32_t *fmap;
  const double *X, *f;
  double *b;
  const int32_t *cell_layers = nullptr;  // variable layers
  double mean_layers = 0.0;
};
cudaError_t launch_mass_dgp(const MassDGPLaunch &p, cudaStream_t s);

// Horizontal-facet loops (k_facet.cu).  Facet m of a column (m = 0..lambda)
// reads the bottom stencil slots at layer m, or the top slots of the last
// layer for m = lambda.  FACET_MASS: b_a += int_F f phi_a ds on a space
// (h, CG1); FACET_JUMP: r += int_F [u][phi] ds over the interior facets
// m = 1..lambda-1 on a prism tensor-product space.
struct FacetLaunch {
  int64_t ncells;
  int32_t layers;
  int32_t nh;             // horizontal nodes: 1 (DG0) or 3 (CG1, DG1)
  int32_t jump;           // 0: facet mass, 1: interior-facet jump
  int32_t nv;             // vertical nodes of the space: 1 (DG0) or 2 (CG1, DG1)
  int32_t mode;           // jump: 0 facet-centric atomics, 1 cell-owned DoFs (DG x DG), 2 none (CG1 vertical)
  const int32_t *cmap;    // coords map (k = 6)
  int32_t coff[6];
  const int32_t *fmap;    // f/u and b/r share this numbering
  int32_t k;
  // facet mass: slot of node a at the bottom (lo) and top (hi) of a layer
  // jump: slot of node a's trace from below (lo: top of the cell under the
  // facet) and from above (hi: bottom of the cell over it)
  int32_t slot_lo[3], slot_hi[3];
  int32_t off_lo[3], off_hi[3];
  const double *X, *f;
  double *b;
  const int32_t *cell_layers = nullptr;  // variable layers
  double mean_layers = 0.0;
};
cudaError_t launch_facet(const FacetLaunch &p, cudaStream_t s);

// u^2 v residual and adjoint (k_u2v.cu): prisms (P1 x P1) and hexahedra (Q2 x P2, DG2).
struct U2VLaunch {
  int64_t ncells;
  int32_t layers;
  int32_t nvc;         // 3: prism P1xP1, 4: hexahedron Q2/DG2
  int32_t dg;          // outputs WRITE (DG2) instead of INC
  int32_t mode;        // bit 0: forward F, bit 1: adjoint g
  const int32_t *cmap; // coords map (k = 2 nvc)
  int32_t coff[8];
  const int32_t *umap; // u/w/F/g map (same space)
  int32_t uoff[27];
  int32_t k;
  const double *X, *u, *w;
  double *F, *g;
  unsigned int *err;
};
cudaError_t launch_u2v(const U2VLaunch &p, cudaStream_t s);

// Batched persistent u^2 v on prisms (k_batch.cu).  Descriptors are opaque
// to the host code: batch_fill_desc writes one into a host array of
// nmesh * batch_desc_size() bytes, which is then copied to the device.
size_t batch_desc_size();
void batch_fill_desc(void *host_descs, int mi, int64_t ncells, int64_t item_begin, int32_t layers,
                     int32_t ncol_items, int32_t nlay_items, const int32_t *cells, const int32_t *cmap,
                     const int32_t *umap, const int32_t coff[6], const int32_t uoff[6], const double *X,
                     const double *u, const double *w, double *F, double *G);
cudaError_t launch_batch_phase(const void *d_descs, int nmesh, int64_t nitems, int mode, bool colour,
                               int cpi, int lt, unsigned long long *counter, int threads, int grid,
                               cudaStream_t s);

// Helpers for the batched launch that runs without allocating (k_batch.cu).
ext_status ext_batch_validate(int32_t nmesh, const ext_mesh *const *meshes, int32_t kernel_id, int32_t nargs,
                              const ext_arg *args, int *mode_out);
const int32_t *ext_space_map_dev(const ext_space *s);
const int32_t *ext_space_offsets_host(const ext_space *s);
int64_t ext_mesh_ncells(const ext_mesh *m);
int32_t ext_mesh_layers(const ext_mesh *m);

// Range checks of the checked build (k_number.cu): stencil maps of a space
// over its mesh's layers, and the vertex rows of the gather form.
cudaError_t launch_check_map(const ext_space *sp, const int32_t *cell_layers, int32_t layers, unsigned int *err,
                             cudaStream_t s);
cudaError_t launch_check_rows(const ext_mesh *m, int64_t ndofs, unsigned int *err, cudaStream_t s);
