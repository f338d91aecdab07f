/*
 * extmesh: numbering and parallel iteration (par_loop) over extruded meshes on
 * one GB300 GPU.  C ABI.
 *
 * Method: Bercea et al., "A structure-exploiting numbering algorithm for
 * finite elements on extruded meshes, and its performance evaluation in
 * Firedrake".  An extruded mesh is a base mesh replicated over `layers`
 * intervals (Sec. 3.1); the degrees of freedom (DoFs) of a function space are
 * numbered vertical-innermost (Algorithm 1, Sec. 3.2) so that only the
 * bottom-layer stencil list of each column is stored; the DoFs of layer l are
 * base_map[c][i] + l * offset[i] (Algorithm 2 and the direct-addressing
 * formula, Sec. 3.3), and a stencil (local kernel) is applied to every cell of
 * every column with the layers innermost (Algorithm 3, Sec. 3.3).
 *
 * Conventions shared by every entry point:
 *   - Pointers named *_host are host memory; every other data pointer is
 *     device memory of the current CUDA device.  Field data are FP64.
 *   - The library owns meshes, spaces, stencil maps and batch plans (device
 *     copies included); destroy functions free them.  The caller owns field
 *     buffers and streams; `stream` is a cudaStream_t (NULL = legacy default
 *     stream).
 *   - Launches are asynchronous on the given stream.  A validation error
 *     returns before anything is launched (nothing is partially applied).
 *     Device-side conditions (bounded waits that expired, inputs a kernel
 *     cannot handle) set a device error word that ext_sync_check reports.
 *   - Every function returns EXT_OK or an error code; ext_last_error() gives
 *     a message for the calling thread's most recent error.
 *   - Entity and DoF indices are int32; a space with 2^31 or more DoFs is
 *     rejected with EXT_EOVERFLOW.
 */
#ifndef EXTMESH_H
#define EXTMESH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EXT_ABI_VERSION 1

typedef enum {
  EXT_OK = 0,
  EXT_EINVAL = 1,        /* invalid argument or inconsistent inputs        */
  EXT_ENOMEM = 2,        /* device or host allocation failed               */
  EXT_ECUDA = 3,         /* a CUDA runtime call failed                     */
  EXT_EOVERFLOW = 4,     /* a count does not fit the int32 index type      */
  EXT_ETIMEOUT = 5,      /* a bounded device-side wait expired             */
  EXT_EDEVICE = 6,       /* the device error word reported a condition     */
  EXT_EUNSUPPORTED = 7   /* valid request this build does not implement    */
} ext_status;

/* Base-mesh cell kinds: triangles extrude to prisms, quadrilaterals to
 * hexahedra (tensor-product cells, Sec. 3.1.1). */
typedef enum { EXT_TRI = 3, EXT_QUAD = 4 } ext_cell_kind;

/* Access descriptors of a par_loop argument (Sec. 3.3, PyOP2 semantics):
 * READ is never written; WRITE overwrites every DoF the loop reaches; INC
 * adds into the existing values (the caller zeroes them first).  A WRITE or
 * INC argument's data must not overlap any other argument's data
 * (EXT_EINVAL). */
typedef enum { EXT_READ = 0, EXT_WRITE = 1, EXT_INC = 2 } ext_access;

/* Local kernels (stencil functions S of Algorithm 3).  Each fixes its
 * argument list; spaces are identified by their delta table:
 *   CG1xCG1  delta = {1,0, 0,0, 0,0}          (P1 x P1, "coords" with ncomp 3)
 *   DG0xDG0  delta = {0,0, 0,0, 0,1}
 *   DG1xDG1  delta = {0,0, 0,0, 0,6}          (prisms)
 *   Q2xP2    delta = {1,1, 1,1, 1,1}          (hexahedra, continuous)
 *   DG2      delta = {0,0, 0,0, 0,27}         (hexahedra, discontinuous)
 *
 * EXT_K_EXTRUDE     [coords WRITE]                       coordinates (x_v, y_v, level/layers)
 *                   of the unit-height column over every base vertex (Sec. 4.1.1).
 * EXT_K_COPY_DG     [in READ, out WRITE], one space with DoFs only on cells
 *                   (delta(2,1) > 0, all other deltas 0): out = in.
 * EXT_K_RHS_P1P1    [coords READ, f READ, b INC|WRITE] on prisms, all CG1xCG1:
 *                   b_i += int_cell f_h phi_i dx  (the residual I_1, Sec. 4.1.1);
 *                   with WRITE, b is overwritten with the assembled result
 *                   (every DoF set, no zeroing needed beforehand).
 * EXT_K_MASS_P1P1   same arguments and operator: y += M x (mass-matrix action).
 *                   Forms (ext_set_option(EXT_OPT_P1_FORM); the default picks
 *                   by size and geometry; all agree within rounding):
 *                   - gather form (constant layers on a triangle mesh, from
 *                     32 layers; chosen when a probe of the coordinates of
 *                     about 4,096 sampled vertex columns, every level, finds a
 *                     straight extrusion with flat levels, or, with a
 *                     depth-weighted base matrix, terrain-following levels
 *                     z = z0 + sigma_l D(x, y)): per launch, a table of the level
 *                     heights (column of vertex 0), the area of every
 *                     level-0 triangle and from them the weights of the base
 *                     triangulation's P1 mass matrix Mh on the mesh's vertex
 *                     rows; the column mass matrix applied per vertex level
 *                     (w = Mv f); b = Mh w per level, every DoF written by
 *                     one thread in a fixed order (the same bits from launch
 *                     to launch); and a pass over the DoFs whose stencil
 *                     holds a prism that is not straight with flat levels,
 *                     or a NaN (the 6-point rule on both layers of every
 *                     cell around the vertex);
 *                   - cell loop (any other coordinate field, e.g.
 *                     terrain-following levels or leaning columns):
 *                     Algorithm 3 over the cell columns, one element vector
 *                     per prism with the 6-point rule (a closed form of the
 *                     rule for prisms with vertical edges, the general
 *                     Jacobian otherwise), FP64 atomic adds;
 *                   - factored / unfactored cell pass over vertical sums (the
 *                     default below 32 layers: from 3 / at 1 or 2 layers)
 *                     (vertex area sums, vertical sums per vertex level, the
 *                     cell pass with FP64 atomic adds, and a pass over the
 *                     warp steps that met a prism which is not straight);
 *                     variable layers always take this form;
 *                   - single pass (under a million (column, level) items, or
 *                     when the scratch cannot be allocated): every cell forms
 *                     its own vertical sums.
 *                   Scratch (vertical sums, level table, areas, row weights,
 *                   recorded steps: 8 bytes per DoF of f plus 8 per cell and
 *                   8 per row entry in the gather form, 16 per DoF plus 8
 *                   per vertex in the factored one, 24 per DoF on variable
 *                   layers, none in the cell loop, plus at most 1 byte per
 *                   item) comes from the device's default stream-ordered pool
 *                   (cudaMallocAsync / cudaFreeAsync on `stream`), so
 *                   launches on different streams never share it and the
 *                   launch can be captured in a CUDA graph.  Coordinates
 *                   must be finite.
 * EXT_K_INTERP_DG1  [x READ (CG1xCG1), out WRITE (DG1xDG1)] on prisms: nodal
 *                   interpolation, out at DG1 node (vertex a, level b) = x there.
 * EXT_K_U2V_FWD     [coords READ, u READ, F INC|WRITE]: F_i += int u_h^2 phi_i dx,
 *                   u and F on the same space: CG1xCG1 on prisms, Q2xP2 or DG2 on
 *                   hexahedra; INC for continuous spaces, WRITE for DG2.
 * EXT_K_U2V_ADJ     [coords READ, u READ, w READ, g INC|WRITE]: g = (dF/du)^T w,
 *                   the hand-written adjoint of EXT_K_U2V_FWD (gathers become
 *                   scatter-adds; F's INC output becomes the READ cotangent w).
 * EXT_K_U2V_FWDADJ  [coords READ, u READ, w READ, F INC|WRITE, g INC|WRITE]:
 *                   both of the above in one pass.
 * EXT_K_MASS_TP     [coords READ, f READ, b INC|WRITE] on prisms: b_i += int f_h phi_i dx
 *                   on any of the nine spaces h x v, h, v in {CG1, DG0, DG1}, of
 *                   Sec. 4.1.2 (delta: CG1xCG1 {1,0,0,0,0,0}, CG1xDG0 {0,1,..},
 *                   CG1xDG1 {0,2,..}, DG0xCG1 {..,1,0}, DG0xDG0 {..,0,1},
 *                   DG0xDG1 {..,0,2}, DG1xCG1 {..,3,0}, DG1xDG0 {..,0,3},
 *                   DG1xDG1 {..,0,6}); f and b share one numbering.  From a
 *                   million (column, layer) items on a mesh with base
 *                   coordinates and constant layers, a first kernel sets one
 *                   straightness bit per coordinate DoF (scratch from the
 *                   stream-ordered pool: 1 bit per coordinate DoF and two
 *                   level tables), and the cell kernel tests those bits
 *                   instead of comparing each prism's coordinates; without
 *                   the scratch, or with EXTMESH_TP_FLAGS=0, it compares them.
 *                   WRITE overwrites b with the result.  Where every DoF
 *                   belongs to one cell-layer (DG x DG) each is stored once;
 *                   the other spaces add with FP64 atomics, b cleared first
 *                   for WRITE (EXTMESH_TP_LEVELS=1, read once per process:
 *                   DG0 x CG1 and DG1 x CG1 on constant layers instead walk a
 *                   column's levels and form each DoF from the two layers
 *                   that share it in registers).
 * EXT_K_HFACET_MASS [coords READ, f READ, b INC] on prisms, over the horizontal
 *                   facets ((2,0),(c,m)), m = 0..lambda, of every column
 *                   (Algorithm 3 with d2 = 0): b_i += int_F f_h phi_i ds on the
 *                   spaces whose DoFs sit on horizontal facets, CG1xCG1, DG0xCG1,
 *                   DG1xCG1.  A facet's DoFs are the bottom horizontal DoFs of
 *                   layer m (the top ones of the last layer for m = lambda).
 * EXT_K_HFACET_JUMP [coords READ, u READ, r INC] on prisms, over the interior
 *                   horizontal facets m = 1..lambda-1 of every column, each with
 *                   the two cells it separates: r_i += int_F [u_h] [phi_i] ds,
 *                   [w] = w(cell below, at the facet) - w(cell above, at the
 *                   facet), on any of the nine spaces of EXT_K_MASS_TP (zero for
 *                   the vertically continuous ones); u and r share one numbering.
 * EXT_K_MASS_DGP    [coords READ, f READ, b INC] on prisms, f and b on one space
 *                   from ext_number_dofs_ragged whose DoFs all sit inside the
 *                   cells: b_i += int f_h phi_i dx where every cell carries its
 *                   own element, told apart by its DoF count: 1 DG0xDG0, 2
 *                   DG0xDG1, 3 DG1xDG0, 6 DG1xDG1 (p-adaptive DG).
 * EXT_K_COPY_DG also takes a space from ext_number_dofs_ragged whose DoFs all
 * sit inside the cells (any count per cell).
 * Quadrature: prisms use the 6-point rule (3-point degree-2 triangle rule x
 * 2-point Gauss); hexahedra use 4x4x4 Gauss points; facets are flat triangles
 * whose P1 surface integrals are evaluated exactly. */
typedef enum {
  EXT_K_EXTRUDE = 0,
  EXT_K_COPY_DG = 1,
  EXT_K_RHS_P1P1 = 2,
  EXT_K_MASS_P1P1 = 3,
  EXT_K_INTERP_DG1 = 4,
  EXT_K_U2V_FWD = 5,
  EXT_K_U2V_ADJ = 6,
  EXT_K_U2V_FWDADJ = 7,
  EXT_K_MASS_TP = 8,
  EXT_K_HFACET_MASS = 9,
  EXT_K_HFACET_JUMP = 10,
  EXT_K_MASS_DGP = 11
} ext_kernel_id;

typedef struct ext_mesh ext_mesh;
typedef struct ext_space ext_space;
typedef struct ext_batch ext_batch;

/* One par_loop argument: a field on `space` (data: device, FP64,
 * ndofs * ncomp values, DoF-major) with its access descriptor. */
typedef struct {
  const ext_space *space;
  void *data;
  int32_t access; /* ext_access */
} ext_arg;

/* Launch parameters of the batched persistent loop (and its autotuner). */
typedef struct {
  int32_t cols_per_item; /* base columns per work item                    */
  int32_t layer_tile;    /* layers per work item; 0 = the whole column     */
  int32_t use_atomics;   /* 1: FP64 atomic increments; 0: colour phases    */
  int32_t threads;       /* threads per CTA                                */
  int32_t ctas_per_sm;   /* resident CTAs per SM of the persistent grid    */
} ext_tune_params;

/* Library ABI version (EXT_ABI_VERSION of the build). */
int32_t ext_abi_version(void);

/* Message of the calling thread's most recent error ("" if none).  The
 * string stays valid until the thread's next failing call. */
const char *ext_last_error(void);

/* Creates an extruded mesh (Sec. 3.1): the base mesh's cell-vertex lists
 * (the only topology input; every other adjacency is derived from it, Sec.
 * 2.2) and the number of layers lambda >= 1.
 *   kind            EXT_TRI or EXT_QUAD
 *   nverts, ncells  base vertex and cell counts (ncells may be 0)
 *   cell_verts_host ncells x kind int32, vertex ids in [0, nverts), counter-
 *                   clockwise when base_xy_host is given
 *   base_xy_host    nverts x 2 FP64 vertex coordinates, or NULL (then
 *                   EXT_K_EXTRUDE is unavailable and orientation is unchecked)
 * Edges are numbered by first appearance when scanning cells in order with
 * local edge k = (vertex k, vertex k+1 mod kind).  The topology is copied to
 * the device (synchronously).  A triangle mesh with base coordinates also
 * gets, on the device, the rows of its base P1 mass matrix per vertex (the
 * vertex itself and its neighbours, weighted by |2A|/144 of the cells on each
 * edge, 16 bytes per entry, about 7 entries per vertex) and the cells around
 * every vertex, which the P1xP1 loops' gather form reads.  Errors: EXT_EINVAL
 * (ids out of range, repeated
 * vertex in a cell, clockwise or degenerate cell, layers < 1), EXT_EOVERFLOW,
 * EXT_ENOMEM, EXT_ECUDA. */
ext_status ext_mesh_create(int32_t kind, int64_t nverts, int64_t ncells,
                           const int32_t *cell_verts_host, const double *base_xy_host,
                           int32_t layers, ext_mesh **out);

/* Creates an extruded mesh whose columns have their own layer ranges: base
 * cell c spans the levels cell_first_host[c] .. cell_first_host[c] +
 * cell_layers_host[c] (the paper fixes one lambda for exposition and notes
 * that this is not a limitation of the method, Sec. 3.1 footnote and Sec. 5).
 * A vertex or edge column spans the hull of the ranges of the cells containing
 * it, so Algorithm 1 gives entity columns their own sizes; the numbering
 * prefix-sums those sizes on the device.  Each cell's stencil list is taken at
 * its own bottom layer, and a par_loop visits layers 0..cell_layers[c]-1 of
 * column c.  Entity levels inside the hull that no cell around spans (a gap
 * between disjoint ranges) are numbered but reached by no stencil.
 *   cell_first_host   ncells int32 >= 0
 *   cell_layers_host  ncells int32 >= 1
 * The highest level first + layers over all cells is reported as the mesh's
 * `layers` by ext_mesh_info, and EXT_K_EXTRUDE places level l at z = l / that
 * level.  Other arguments and errors as ext_mesh_create, plus EXT_EINVAL when
 * a vertex belongs to no cell.  Kernels on such meshes: EXT_K_EXTRUDE,
 * EXT_K_COPY_DG, EXT_K_RHS_P1P1, EXT_K_MASS_P1P1, EXT_K_INTERP_DG1,
 * EXT_K_MASS_TP, EXT_K_HFACET_MASS, EXT_K_HFACET_JUMP (others, and batches,
 * return EXT_EUNSUPPORTED). */
ext_status ext_mesh_create_var(int32_t kind, int64_t nverts, int64_t ncells,
                               const int32_t *cell_verts_host, const double *base_xy_host,
                               const int32_t *cell_first_host, const int32_t *cell_layers_host,
                               ext_mesh **out);

/* Entity counts N_0, N_1, N_2 (vertices, edges, cells) of the base mesh, the
 * cell kind and the number of layers (Sec. 2.2, 3.1); for a mesh with
 * variable layers, the highest level. */
ext_status ext_mesh_info(const ext_mesh *mesh, int32_t *kind, int64_t n[3], int32_t *layers);

void ext_mesh_destroy(ext_mesh *mesh);

/* Numbers the DoFs of a function space (Algorithm 1, Sec. 3.2) and builds its
 * bottom-layer stencil map and vertical offsets (Sec. 3.3, Algorithm 2).
 *   delta_host  6 int32: delta((d1,d2)) at index 2*d1+d2, DoFs per extruded
 *               entity of horizontal dimension d1 and vertical dimension d2
 *   ncomp       values per DoF (1, or 3 for a coordinate field)
 * Numbering: base entities dimension-major (vertices, edges, cells), index
 * ascending; in each column, layer by layer, the horizontal entity's
 * delta(d,0) numbers then the vertical entity's delta(d,1) numbers, and the
 * top horizontal entity last.  Stencil order: the cell's vertices, edges,
 * then the cell itself; per entity the bottom horizontal DoFs, the top
 * horizontal DoFs, then the vertical DoFs.  The map is computed by a kernel
 * on `stream` (asynchronous).  Errors: EXT_EINVAL, EXT_EOVERFLOW (2^31 DoFs or
 * more), EXT_ENOMEM, EXT_ECUDA. */
ext_status ext_number_dofs(ext_mesh *mesh, const int32_t delta_host[6], int32_t ncomp,
                           void *stream, ext_space **out);

/* Numbers a space whose DoF counts vary per base entity (the paper fixes one
 * count per entity type for exposition and notes that the numbering does not
 * need it, Sec. 5): Algorithm 1 with entity g's column holding
 * lambda_g (dent[2g] + dent[2g+1]) + dent[2g] numbers, on constant or
 * variable layers.  The column starts and the list lengths are prefix sums on
 * the device.
 *   dent_host  (N_0 + N_1 + N_2) x 2 int32 in [0, 4096]: DoFs of entity g on
 *              each horizontal copy and on each vertical copy; entities
 *              dimension-major (vertices, edges, cells), index ascending
 * The lists are ragged: row c (cell c at its bottom layer) holds, per entity
 * of the cell (vertices, edges, cell), the bottom horizontal DoFs, the top
 * horizontal DoFs and the vertical DoFs; each entry's vertical offset is its
 * entity's dent[2g] + dent[2g+1] (Algorithm 2's rule).  ext_space_info
 * reports k = 0; ext_space_ragged_info / ext_space_copy_ragged_to_host give
 * the row pointers (ncells + 1 int64), the entries and their offsets.
 * Synchronous on `stream`.  Errors: EXT_EINVAL (negative or too large count,
 * no DoFs), EXT_EOVERFLOW, EXT_ENOMEM, EXT_ECUDA. */
ext_status ext_number_dofs_ragged(ext_mesh *mesh, const int32_t *dent_host, int32_t ncomp, void *stream,
                                  ext_space **out);

/* Device row pointers (ncells + 1), entries and per-entry offsets of a space
 * from ext_number_dofs_ragged (EXT_EINVAL for a space with one length k). */
ext_status ext_space_ragged_info(const ext_space *space, int64_t *nentries, const int64_t **rowptr_dev,
                                 const int32_t **map_dev, const int32_t **offset_dev);

/* Copies them to host arrays (ncells + 1, nentries, nentries; any may be
 * NULL).  Synchronous. */
ext_status ext_space_copy_ragged_to_host(const ext_space *space, int64_t *rowptr_host, int32_t *map_host,
                                         int32_t *offset_host);

/* DoF count, stencil length k, ncomp and the device stencil data of a space:
 * base_map (ncells x k int32, row-major, global DoFs at layer 0) and offset
 * (k int32).  Any output pointer may be NULL.  The device arrays belong to the
 * space. */
ext_status ext_space_info(const ext_space *space, int64_t *ndofs, int32_t *k, int32_t *ncomp,
                          const int32_t **base_map_dev, const int32_t **offset_dev);

/* Copies the stencil map (ncells x k) and offsets (k) to host arrays
 * (synchronous on the space's creation stream; either pointer may be NULL). */
ext_status ext_space_copy_map_to_host(const ext_space *space, int32_t *map_host, int32_t *offset_host);

void ext_space_destroy(ext_space *space);

/* Algorithm 3: applies local kernel `kernel_id` to every cell of every column
 * of `mesh`, columns in parallel and layers innermost, reading each column's
 * stencil lists once and reaching layer l by base_map + l * offset.  `args`
 * must match the kernel's argument list (spaces of this mesh, access
 * descriptors).  Asynchronous on `stream`.  Errors: EXT_EINVAL (argument
 * list, spaces or modes do not match), EXT_EUNSUPPORTED, EXT_ECUDA. */
ext_status ext_par_loop(const ext_mesh *mesh, int32_t kernel_id, int32_t nargs,
                        const ext_arg *args, void *stream);

/* Batched form: one persistent launch applies `kernel_id` over `nmesh`
 * extruded meshes of different base sizes and layer counts.  `args` holds
 * nmesh x nargs entries (mesh-major).  Work items are (mesh, column range,
 * layer range) tiles taken from a device work counter; every spin-wait in
 * the kernel is bounded.  `params` NULL selects parameters by autotuning
 * (timed trial launches on `stream`, which overwrite the INC/WRITE outputs;
 * the caller zeroes INC outputs before each real launch).  The launch is
 * captured into a CUDA graph; ext_batch_launch replays it.  Supported
 * kernels: EXT_K_U2V_FWD, EXT_K_U2V_ADJ, EXT_K_U2V_FWDADJ on CG1xCG1 prisms.
 * Errors: as ext_par_loop, plus EXT_ENOMEM. */
ext_status ext_batch_create(int32_t nmesh, const ext_mesh *const *meshes, int32_t kernel_id,
                            int32_t nargs, const ext_arg *args, const ext_tune_params *params,
                            void *stream, ext_batch **out);

/* Replays the captured batched launch on `stream`. */
ext_status ext_batch_launch(ext_batch *batch, void *stream);

/* Runs the batched work queue with an uncaptured launch and explicit
 * parameters (used by the autotuner; also a plain entry point). */
ext_status ext_batch_launch_params(ext_batch *batch, const ext_tune_params *params, void *stream);

/* Parameters in use by the batch (chosen or autotuned). */
ext_status ext_batch_params(const ext_batch *batch, ext_tune_params *out);

/* Where the batch's parameters came from (*source: 0 given by the caller,
 * 1 autotuned by ext_batch_create, 2 read from the tuning cache) and the host
 * time ext_batch_create took, in seconds; either pointer may be NULL.
 * Tuning cache: with params NULL, ext_batch_create first looks up the
 * parameters tuned earlier for the same GPU (name, SM count), kernel and
 * power-of-two buckets of the prism count, mean layer count and mesh count,
 * in memory and in a file of JSON lines (EXTMESH_TUNE_CACHE, else
 * $XDG_CACHE_HOME/extmesh/batch_tune.jsonl or $HOME/.cache/extmesh/
 * batch_tune.jsonl); it autotunes and records the result only on a miss.
 * EXTMESH_TUNE=force re-tunes and replaces the entry, EXTMESH_TUNE=off
 * neither reads nor writes the cache.  The environment is read at every
 * ext_batch_create.  (The autotuner and its cache are this library's; the
 * paper has no counterpart.) */
ext_status ext_batch_plan_info(const ext_batch *batch, int32_t *source, double *setup_seconds);

void ext_batch_destroy(ext_batch *batch);

/* Batched launch for callers that cannot allocate device memory (the paper
 * has no counterpart; this is a deployment variant of ext_batch_launch).
 * Some callers cannot call cudaMalloc: code running under a device-memory
 * budget owned by someone else (a framework's caching allocator that has
 * reserved the device, or a service that forbids allocation after start-up),
 * and latency-sensitive loops that cannot take cudaMalloc's implicit device
 * synchronisation.  This entry point runs the batched u^2 v work-queue kernel
 * (FP64-atomic form only) directly, without a plan, and allocates nothing:
 * its scratch (work counter and per-mesh descriptors) lives in a 64 KiB
 * static device array of the library, which every GPU that loads the library
 * holds until the process exits.
 *   nmesh <= EXT_NOALLOC_MAX_MESHES; larger batches fail with EXT_EINVAL.
 *   args, kernels and argument rules: as ext_batch_create.  INC outputs are
 *   added to; the caller zeroes them.
 *   params NULL = {cols_per_item 4, layer_tile 0, use_atomics 1, threads 256,
 *   ctas_per_sm 4}; use_atomics must be 1 (EXT_EUNSUPPORTED otherwise).
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  Every call
 * on a device shares the array and it keeps the last call's contents, so calls
 * whose launches overlap on the GPU race: order them (e.g. one stream).
 * The per-mesh descriptors travel to the array as kernel parameters (16 per
 * small staging launch), so the call reads no host memory after it returns
 * and does not wait for `stream`.  Every mesh must live on the current device,
 * and no written argument may overlap another argument of its mesh
 * (EXT_EINVAL).  Asynchronous on `stream`; errors as ext_batch_create. */
#define EXT_NOALLOC_MAX_MESHES 256
#define EXT_NOALLOC_SCRATCH_BYTES 65536
ext_status ext_batch_run_noalloc(int32_t nmesh, const ext_mesh *const *meshes, int32_t kernel_id,
                                 int32_t nargs, const ext_arg *args, const ext_tune_params *params,
                                 void *stream);

/* Measured FP64 rates of this GPU, in G operations per second:
 * gops_host[0] DFMA, [1] DADD, [2] DMUL issued by the SMs (eight independent
 * chains per thread, 4 CTAs of 256 threads per SM), [3] FP64 atomic adds
 * executed by L2 (coalesced, to a 64 MiB buffer resident in L2); best of two
 * timed launches each.  A measurement helper for the roofline of the FP64
 * assembly kernels; the paper has no counterpart.  Synchronous on `stream`;
 * allocates and frees scratch buffers. */
ext_status ext_fp64_rates(double gops_host[4], void *stream);

/* Process-wide options.  EXT_OPT_P1_FORM selects the form of the
 * EXT_K_RHS_P1P1 / EXT_K_MASS_P1P1 launch (all forms give the same result
 * within the rounding of their summation orders):
 *   EXT_P1_AUTO (default)  the single-pass kernel under a million
 *                          (column, level) items, else EXT_P1_SPLIT;
 *   EXT_P1_SPLIT           a probe of the coordinate field picks the gather
 *                          form on a straight extrusion with flat levels and
 *                          the cell loop on any other geometry;
 *   EXT_P1_GATHER          the gather form without the probe;
 *   EXT_P1_FACTORED        the cell pass over vertical sums with the area
 *                          pass; EXT_P1_UNFACTORED without it;
 *   EXT_P1_CELLS           the cell loop (Algorithm 3, one element vector
 *                          per prism);
 *   EXT_P1_SINGLE          the single-pass kernel.
 * The initial value comes from the environment variable EXTMESH_P1_FORM
 * (auto, split, gather, factored, unfactored, cells, single), read at the
 * first query.  ext_set_option returns EXT_EINVAL for an unknown option or
 * value; it affects launches issued after it returns. */
typedef enum { EXT_OPT_P1_FORM = 1, EXT_OPT_P1_FLAT = 2 } ext_option;
/* EXT_OPT_P1_FLAT: how the flat gather runs.  EXT_P1_FLAT_OPTIMISTIC
 * (default): with WRITE access one pass forms b_{a,m} = Mv applied to
 * g = Mh f per level (lanes along a column's levels) for every DoF as if the
 * mesh were a straight flat extrusion, while the same launch sets one
 * straightness bit per coordinate DoF; a second launch sends every DoF whose
 * stencil holds a DoF that is not straight to the general path (and exits at
 * once when there is none), so the coordinate field, f and b each cross HBM
 * once; with INC access the split form runs.  EXT_P1_FLAT_SPLIT: the vertex
 * pass w = Mv f stored, then b = Mh w (w written and read back).
 * EXT_P1_FLAT_FUSED: one pass with the straightness of every row entry
 * checked while walking the rows (three coordinate loads per entry).
 * Initial value from EXTMESH_P1_FLAT (optimistic, split, fused). */
typedef enum { EXT_P1_FLAT_FUSED = 0, EXT_P1_FLAT_SPLIT = 1, EXT_P1_FLAT_OPTIMISTIC = 2 } ext_p1_flat;
typedef enum {
  EXT_P1_AUTO = 0,
  EXT_P1_SPLIT = 1,
  EXT_P1_GATHER = 2,
  EXT_P1_FACTORED = 3,
  EXT_P1_UNFACTORED = 4,
  EXT_P1_CELLS = 5,
  EXT_P1_SINGLE = 6
} ext_p1_form;
ext_status ext_set_option(int32_t option, int32_t value);
ext_status ext_get_option(int32_t option, int32_t *value);

/* Range check of a space's stencil lists on the device: every index that
 * Algorithm 3 forms from them (base_map[c][i] + l * offset[i] for every layer
 * l of column c; for a CG1xCG1 space also the gather form's vertex rows) must
 * lie in [0, ndofs).  Synchronous on `stream`; EXT_OK, or EXT_EDEVICE when an
 * index is out of range (the error word is cleared again) or when the device
 * error word was already set.  The checked build of the library
 * (libextmesh_checked.so, compiled with EXT_CHECKED) runs the same checks on
 * every argument of ext_par_loop before launching and launches nothing when
 * one fails.  A debugging aid of this library; the paper has no counterpart. */
ext_status ext_space_check(const ext_space *space, void *stream);

/* Waits for `stream`, then reads and clears the device error word:
 * EXT_OK, EXT_ETIMEOUT (a bounded wait expired), EXT_EDEVICE (another device
 * condition; see ext_last_error), or EXT_ECUDA (an asynchronous CUDA error). */
ext_status ext_sync_check(void *stream);

#ifdef __cplusplus
}
#endif
#endif /* EXTMESH_H */
