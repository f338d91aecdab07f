// Numbering (Algorithm 1 in closed form, Algorithm 2) and coordinate
// extrusion kernels.
#include "ext_internal.cuh"

// Algorithm 1 assigns numbers entity column by entity column, dimension-major
// and index ascending, so the counter when entity (d, i) starts is
//   block_start[d] + i * colsize[d],
//   colsize[d] = layers * (delta(d,0) + delta(d,1)) + delta(d,0),
// and inside that column layer l's horizontal entity starts at
// l * (delta(d,0) + delta(d,1)) and its vertical entity delta(d,0) later; the
// top horizontal entity starts at layers * (delta(d,0) + delta(d,1)).
// One thread writes one entry of the layer-0 stencil map (Sec. 3.3: the
// explicit lists are kept for the bottom of each column only).
__global__ void __launch_bounds__(256) k_number(const NumberLaunch p) {
  const int64_t total = p.ncells * p.k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / p.k;
    const int i = (int)(t - c * p.k);
    const int d = p.slot_dim[i];
    const int e = p.slot_ent[i];
    int64_t id;
    if (d == 0) id = p.cell_verts[c * p.nvc + e];
    else if (d == 1) id = p.cell_edges[c * p.nvc + e];
    else id = c;
    p.map[t] = (int32_t)(p.block_start[d] + id * p.colsize[d] + p.slot_add[i]);
  }
}

// Variable layers: entity (d, id) has the column start ent_start[g] (g its
// dimension-major global index, a prefix sum of the column sizes) and bottom
// level ent_lo[g]; cell c's list is taken at its own bottom level first[c],
// (first[c] - ent_lo[g]) layers of (delta(d,0) + delta(d,1)) numbers above
// the entity's bottom.
__global__ void __launch_bounds__(256) k_number_var(const NumberLaunch p) {
  const int64_t total = p.ncells * p.k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / p.k;
    const int i = (int)(t - c * p.k);
    const int d = p.slot_dim[i];
    const int e = p.slot_ent[i];
    int64_t id;
    if (d == 0) id = p.cell_verts[c * p.nvc + e];
    else if (d == 1) id = p.cell_edges[c * p.nvc + e];
    else id = c;
    const int64_t g = p.ent_base[d] + id;
    const int64_t lift = (int64_t)(p.cell_first[c] - p.ent_lo[g]) * p.colstep[d];
    p.map[t] = (int32_t)(p.ent_start[g] + lift + p.slot_add[i]);
  }
}

cudaError_t launch_number(const NumberLaunch &p, cudaStream_t s) {
  const int64_t total = p.ncells * p.k;
  if (total == 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (p.ent_start) k_number_var<<<(unsigned)blocks, 256, 0, s>>>(p);
  else k_number<<<(unsigned)blocks, 256, 0, s>>>(p);
  return cudaGetLastError();
}

// Level range of every base entity: a cell spans first .. first + layers; a
// vertex or edge the hull of the ranges of the cells containing it (integer
// atomics, so the result does not depend on the order).
__global__ void __launch_bounds__(256) k_var_ranges(int64_t ncells, int nvc, int64_t nv, int64_t ne,
                                                    const int32_t *cell_verts, const int32_t *cell_edges,
                                                    const int32_t *first, const int32_t *layers, int32_t *lo,
                                                    int32_t *hi) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncells;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = first[c], t = first[c] + layers[c];
    for (int a = 0; a < nvc; ++a) {
      const int64_t v = cell_verts[c * nvc + a];
      const int64_t e = nv + cell_edges[c * nvc + a];
      atomicMin(lo + v, b);
      atomicMax(hi + v, t);
      atomicMin(lo + e, b);
      atomicMax(hi + e, t);
    }
    lo[nv + ne + c] = b;
    hi[nv + ne + c] = t;
  }
}

cudaError_t launch_var_ranges(const ext_mesh *m, cudaStream_t s) {
  const int64_t nent = m->N[0] + m->N[1] + m->N[2];
  cudaError_t e = cudaMemsetAsync(m->d_ent_lo, 0x7f, sizeof(int32_t) * nent, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->d_ent_hi, 0xff, sizeof(int32_t) * nent, s);
  if (e != cudaSuccess || m->N[2] == 0) return e;
  int64_t blocks = (m->N[2] + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_var_ranges<<<(unsigned)blocks, 256, 0, s>>>(m->N[2], m->kind, m->N[0], m->N[1], m->d_cell_verts,
                                                 m->d_cell_edges, m->d_cell_first, m->d_cell_layers,
                                                 m->d_ent_lo, m->d_ent_hi);
  return cudaGetLastError();
}

// Column size of every entity: (hi - lo) (delta(d,0) + delta(d,1)) + delta(d,0).
__global__ void __launch_bounds__(256) k_var_colsize(int64_t n0, int64_t n01, int64_t nent, const int32_t *lo,
                                                     const int32_t *hi, int4 a, int4 b, int64_t *sizes) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nent;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int d = g < n0 ? 0 : (g < n01 ? 1 : 2);
    const int h = d == 0 ? a.x : (d == 1 ? a.y : a.z);
    const int v = d == 0 ? b.x : (d == 1 ? b.y : b.z);
    sizes[g] = (int64_t)(hi[g] - lo[g]) * (h + v) + h;
  }
}

cudaError_t launch_var_colsize(const ext_mesh *m, const int32_t delta[6], int64_t *sizes, cudaStream_t s) {
  const int64_t nent = m->N[0] + m->N[1] + m->N[2];
  if (nent == 0) return cudaSuccess;
  int64_t blocks = (nent + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_var_colsize<<<(unsigned)blocks, 256, 0, s>>>(m->N[0], m->N[0] + m->N[1], nent, m->d_ent_lo, m->d_ent_hi,
                                                  make_int4(delta[0], delta[2], delta[4], 0),
                                                  make_int4(delta[1], delta[3], delta[5], 0), sizes);
  return cudaGetLastError();
}

// EXT_K_EXTRUDE as Algorithm 3 over cells, one item per (cell, vertex level m),
// m = 0..layers: the coordinate DoF of local vertex a at level m is the bottom
// slot 2a plus m offsets (m < layers) or the top slot 2a+1 at layer
// layers-1.  Neighbouring cells write identical values to shared vertices.
__global__ void __launch_bounds__(256) k_extrude(const ExtrudeLaunch p) {
  const int L1 = p.layers + 1;
  const int64_t total = p.ncells * L1;
  const int k = 2 * p.nvc;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / L1;
    const int m = (int)(t - c * L1);
    const double z = (double)m / (double)p.layers;
    for (int a = 0; a < p.nvc; ++a) {
      const int v = p.cell_verts[c * p.nvc + a];
      const int64_t dof = (m < p.layers)
                              ? (int64_t)p.map[c * k + 2 * a] + (int64_t)m * p.off
                              : (int64_t)p.map[c * k + 2 * a + 1] + (int64_t)(p.layers - 1) * p.off;
      p.X[3 * dof + 0] = p.base_xy[2 * (int64_t)v + 0];
      p.X[3 * dof + 1] = p.base_xy[2 * (int64_t)v + 1];
      p.X[3 * dof + 2] = z;
    }
  }
}

// Variable layers: one warp per cell, lanes along the levels m = 0..layers[c]
// of the column; level m sits at z = (first[c] + m) / maxlevel.
__global__ void __launch_bounds__(256) k_extrude_var(const ExtrudeLaunch p) {
  const int lane = threadIdx.x & 31;
  const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t c = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); c < p.ncells; c += wstride) {
    const int lay = p.cell_layers[c], f0 = p.cell_first[c];
    const int k = 2 * p.nvc;
    for (int m = lane; m <= lay; m += 32) {
      const double z = (double)(f0 + m) / (double)p.layers;
      for (int a = 0; a < p.nvc; ++a) {
        const int v = p.cell_verts[c * p.nvc + a];
        const int64_t dof = (m < lay) ? (int64_t)p.map[c * k + 2 * a] + (int64_t)m * p.off
                                      : (int64_t)p.map[c * k + 2 * a + 1] + (int64_t)(lay - 1) * p.off;
        p.X[3 * dof + 0] = p.base_xy[2 * (int64_t)v + 0];
        p.X[3 * dof + 1] = p.base_xy[2 * (int64_t)v + 1];
        p.X[3 * dof + 2] = z;
      }
    }
  }
}

cudaError_t launch_extrude(const ExtrudeLaunch &p, cudaStream_t s) {
  if (p.cell_layers) {
    if (p.ncells == 0) return cudaSuccess;
    int64_t blocks = (p.ncells + 7) / 8;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_extrude_var<<<(unsigned)blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
  }
  const int64_t total = p.ncells * (p.layers + 1);
  if (total == 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_extrude<<<(unsigned)blocks, 256, 0, s>>>(p);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-entity DoF counts (ragged lists).  Entity g (dimension-major) carries
// dent[2g] DoFs on each horizontal copy and dent[2g+1] on each vertical one;
// its column holds (hi - lo)(dent[2g] + dent[2g+1]) + dent[2g] numbers.

__global__ void __launch_bounds__(256) k_ragged_colsize(const RaggedLaunch p, int64_t nent, int64_t *sizes) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nent; g += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = p.dent[2 * g], b = p.dent[2 * g + 1];
    const int64_t lay = p.ent_lo ? (int64_t)(p.ent_hi[g] - p.ent_lo[g]) : (int64_t)p.layers;
    sizes[g] = lay * (a + b) + a;
  }
}

cudaError_t launch_ragged_colsize(const RaggedLaunch &p, int64_t *sizes, cudaStream_t s) {
  const int64_t nent = p.N[0] + p.N[1] + p.N[2];
  if (nent == 0) return cudaSuccess;
  int64_t blocks = (nent + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_ragged_colsize<<<(unsigned)blocks, 256, 0, s>>>(p, nent, sizes);
  return cudaGetLastError();
}

// global entity index of local entity e of dimension d of cell c
__device__ __forceinline__ int64_t ragged_entity(const RaggedLaunch &p, int64_t c, int d, int e) {
  if (d == 0) return p.cell_verts[c * p.nvc + e];
  if (d == 1) return p.N[0] + p.cell_edges[c * p.nvc + e];
  return p.N[0] + p.N[1] + c;
}

// row length of cell c: sum over its entities of 2 dent_h + dent_v
__global__ void __launch_bounds__(256) k_ragged_rowlen(const RaggedLaunch p) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < p.ncells;
       c += (int64_t)gridDim.x * blockDim.x) {
    int64_t len = 0;
    for (int d = 0; d <= 2; ++d)
      for (int e = 0; e < (d == 2 ? 1 : p.nvc); ++e) {
        const int64_t g = ragged_entity(p, c, d, e);
        len += 2 * p.dent[2 * g] + p.dent[2 * g + 1];
      }
    p.rowptr[c] = len;
  }
}

cudaError_t launch_ragged_rowlen(const RaggedLaunch &p, cudaStream_t s) {
  if (p.ncells == 0) return cudaSuccess;
  int64_t blocks = (p.ncells + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_ragged_rowlen<<<(unsigned)blocks, 256, 0, s>>>(p);
  return cudaGetLastError();
}

// Row c at the cell's bottom layer: per entity the bottom horizontal DoFs,
// the top horizontal DoFs and the vertical DoFs; each entry's offset is its
// entity's dent_h + dent_v (Algorithm 2's rule).
__global__ void __launch_bounds__(256) k_ragged_map(const RaggedLaunch p) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < p.ncells;
       c += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = p.rowptr[c];
    for (int d = 0; d <= 2; ++d)
      for (int e = 0; e < (d == 2 ? 1 : p.nvc); ++e) {
        const int64_t g = ragged_entity(p, c, d, e);
        const int32_t a = p.dent[2 * g], b = p.dent[2 * g + 1];
        const int64_t lift = p.ent_lo ? (int64_t)(p.cell_first[c] - p.ent_lo[g]) * (a + b) : 0;
        const int64_t s0 = p.ent_start[g] + lift;
        for (int32_t q = 0; q < a; ++q, ++j) { p.map[j] = (int32_t)(s0 + q); p.roff[j] = a + b; }
        for (int32_t q = 0; q < a; ++q, ++j) { p.map[j] = (int32_t)(s0 + a + b + q); p.roff[j] = a + b; }
        for (int32_t q = 0; q < b; ++q, ++j) { p.map[j] = (int32_t)(s0 + a + q); p.roff[j] = a + b; }
      }
  }
}

cudaError_t launch_ragged_map(const RaggedLaunch &p, cudaStream_t s) {
  if (p.ncells == 0) return cudaSuccess;
  int64_t blocks = (p.ncells + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_ragged_map<<<(unsigned)blocks, 256, 0, s>>>(p);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Range check of a stencil map (the checked build, EXT_CHECKED, runs it for
// every argument before a launch): every index Algorithm 3 forms,
// map[c][i] + l offset[i] for l = 0 .. lambda_c - 1, must lie in [0, ndofs).
// The map is linear in l, so checking l = 0 and l = lambda_c - 1 covers all
// layers.  A failure sets EXT_DERR_BOUNDS in the error word; the kernel reads
// only the map, the offsets and the layer counts, all in range.
__global__ void __launch_bounds__(256) k_check_map(const int32_t *__restrict__ map, const int64_t *__restrict__ rowptr,
                                                   const int32_t *__restrict__ roff, int32_t k,
                                                   const int32_t *__restrict__ offset, int64_t ncells, int32_t layers,
                                                   const int32_t *__restrict__ cell_layers, int64_t ndofs,
                                                   unsigned int *err) {
  const int64_t n = rowptr ? rowptr[ncells] : ncells * (int64_t)k;
  int bad = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t c;
    int32_t off;
    if (rowptr) {  // ragged lists: find the cell of entry e (binary search on the row pointer)
      int64_t lo = 0, hi = ncells - 1;
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (rowptr[mid] <= e) lo = mid;
        else hi = mid - 1;
      }
      c = lo;
      off = roff[e];
    } else {
      c = e / k;
      off = offset[e - c * k];
    }
    const int64_t lay = cell_layers ? cell_layers[c] : layers;
    const int64_t lo_i = map[e], hi_i = lo_i + (lay - 1) * (int64_t)off;
    bad |= (lo_i < 0) | (lo_i >= ndofs) | (hi_i < 0) | (hi_i >= ndofs) | (lay < 1);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, EXT_DERR_BOUNDS);
}

// The vertex rows of the gather form: every entry's column start j (layers +
// 1) plus a level up to `layers` must be a DoF of the CG1xCG1 space, and every
// cell of a row's edge a cell of the mesh.
__global__ void __launch_bounds__(256) k_check_rows(const int32_t *__restrict__ vnbr, const int2 *__restrict__ vedge,
                                                    int64_t nent, int32_t layers, int64_t ndofs, int64_t ncells,
                                                    unsigned int *err) {
  int bad = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nent; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j0 = vnbr[t];
    const int2 e = vedge[t];
    bad |= (j0 < 0) | (j0 + layers >= ndofs) | (e.x >= ncells) | (e.y >= ncells) | (e.x < -1) | (e.y < -1);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, EXT_DERR_BOUNDS);
}

cudaError_t launch_check_map(const ext_space *sp, const int32_t *cell_layers, int32_t layers, unsigned int *err,
                             cudaStream_t s) {
  const int64_t C = sp->mesh->N[2];
  if (C == 0) return cudaSuccess;
  const int64_t n = sp->ragged ? sp->nentries : C * (int64_t)sp->k;
  int64_t g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  k_check_map<<<(unsigned)g, 256, 0, s>>>(sp->d_map, sp->ragged ? sp->d_rowptr : nullptr,
                                          sp->ragged ? sp->d_roff : nullptr, sp->k, sp->d_offset, C, layers,
                                          cell_layers, sp->ndofs, err);
  return cudaGetLastError();
}

cudaError_t launch_check_rows(const ext_mesh *m, int64_t ndofs, unsigned int *err, cudaStream_t s) {
  if (!m->d_vnbr || m->n_vent == 0) return cudaSuccess;
  int64_t g = (m->n_vent + 255) / 256;
  if (g > 4096) g = 4096;
  k_check_rows<<<(unsigned)g, 256, 0, s>>>(m->d_vnbr, m->d_vedge, m->n_vent, m->layers, ndofs, m->N[2], err);
  return cudaGetLastError();
}
