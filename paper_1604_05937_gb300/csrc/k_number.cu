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

cudaError_t launch_number(const NumberLaunch &p, cudaStream_t s) {
  const int64_t total = p.ncells * p.k;
  if (total == 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_number<<<(unsigned)blocks, 256, 0, s>>>(p);
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

cudaError_t launch_extrude(const ExtrudeLaunch &p, cudaStream_t s) {
  const int64_t total = p.ncells * (p.layers + 1);
  if (total == 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_extrude<<<(unsigned)blocks, 256, 0, s>>>(p);
  return cudaGetLastError();
}
