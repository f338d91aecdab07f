// Host implementation of the extmesh C ABI (include/extmesh.h): validation,
// base-mesh entity derivation, space numbering set-up, par_loop dispatch and
// the batched plan (autotuning, colouring, CUDA-graph capture).
#include <algorithm>
#include <unistd.h>
#include <sys/stat.h>
#include <chrono>
#include <string>
#include <map>
#include <atomic>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "ext_internal.cuh"

// ---------------------------------------------------------------------------
// errors

static thread_local std::string g_last_error;

ext_status ext_fail(ext_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

#define EXT_CUDA(call, what)                                                                   \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return ext_fail(EXT_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
  } while (0)

extern "C" const char *ext_last_error(void) { return g_last_error.c_str(); }
extern "C" int32_t ext_abi_version(void) { return EXT_ABI_VERSION; }

// ---------------------------------------------------------------------------
// options
static std::atomic<int> g_p1_form{-1};

int p1_form() {
  int v = g_p1_form.load();
  if (v < 0) {
    static const char *names[] = {"auto", "split", "gather", "factored", "unfactored", "cells", "single"};
    const char *ev = getenv("EXTMESH_P1_FORM");
    int init = EXT_P1_AUTO;
    for (int i = 0; ev && i < 7; ++i)
      if (strcmp(ev, names[i]) == 0) init = i;
    int expect = -1;
    g_p1_form.compare_exchange_strong(expect, init);
    v = g_p1_form.load();
  }
  return v;
}

static std::atomic<int> g_p1_flat{-1};

int p1_flat() {
  int v = g_p1_flat.load();
  if (v < 0) {
    const char *ev = getenv("EXTMESH_P1_FLAT");
    int expect = -1;
    const int init = !ev ? EXT_P1_FLAT_OPTIMISTIC
                         : (strcmp(ev, "fused") == 0 ? EXT_P1_FLAT_FUSED
                                                     : (strcmp(ev, "split") == 0 ? EXT_P1_FLAT_SPLIT
                                                                                 : EXT_P1_FLAT_OPTIMISTIC));
    g_p1_flat.compare_exchange_strong(expect, init);
    v = g_p1_flat.load();
  }
  return v;
}

extern "C" ext_status ext_set_option(int32_t option, int32_t value) {
  if (option == EXT_OPT_P1_FORM) {
    if (value < EXT_P1_AUTO || value > EXT_P1_SINGLE)
      return ext_fail(EXT_EINVAL, "ext_set_option: EXT_OPT_P1_FORM value %d out of range", value);
    g_p1_form.store(value);
    return EXT_OK;
  }
  if (option == EXT_OPT_P1_FLAT) {
    if (value != EXT_P1_FLAT_FUSED && value != EXT_P1_FLAT_SPLIT && value != EXT_P1_FLAT_OPTIMISTIC)
      return ext_fail(EXT_EINVAL, "ext_set_option: EXT_OPT_P1_FLAT value %d out of range", value);
    g_p1_flat.store(value);
    return EXT_OK;
  }
  return ext_fail(EXT_EINVAL, "ext_set_option: unknown option %d", option);
}

extern "C" ext_status ext_get_option(int32_t option, int32_t *value) {
  if (!value) return ext_fail(EXT_EINVAL, "ext_get_option: value is NULL");
  if (option == EXT_OPT_P1_FORM) *value = p1_form();
  else if (option == EXT_OPT_P1_FLAT) *value = p1_flat();
  else return ext_fail(EXT_EINVAL, "ext_get_option: unknown option %d", option);
  return EXT_OK;
}

static std::mutex g_word_mu;
static unsigned int *g_word[128];

unsigned int *ext_device_error_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return nullptr;
  std::lock_guard<std::mutex> lk(g_word_mu);
  if (!g_word[dev]) {
    unsigned int *p = nullptr;
    if (cudaMalloc(&p, sizeof(unsigned int)) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, sizeof(unsigned int)) != cudaSuccess) {
      cudaFree(p);
      return nullptr;
    }
    g_word[dev] = p;
  }
  return g_word[dev];
}

// ---------------------------------------------------------------------------
// mesh

struct ext_mesh_host {
  std::vector<int32_t> cell_verts;
};

// Edges numbered by first appearance (cells in order, local edge k joins
// local vertices k and k+1 mod kind): sort (vertex pair, position) records,
// take each pair's earliest position, and rank pairs by it.
static int64_t derive_edges(int kind, int64_t ncells, const int32_t *cv, std::vector<int32_t> &ce) {
  const int64_t n = ncells * kind;
  std::vector<std::pair<uint64_t, int64_t>> rec((size_t)n);
  for (int64_t c = 0; c < ncells; ++c)
    for (int k = 0; k < kind; ++k) {
      const uint32_t a = (uint32_t)cv[c * kind + k], b = (uint32_t)cv[c * kind + (k + 1) % kind];
      const uint64_t key = a < b ? ((uint64_t)a << 32) | b : ((uint64_t)b << 32) | a;
      rec[(size_t)(c * kind + k)] = {key, c * kind + k};
    }
  std::sort(rec.begin(), rec.end());
  std::vector<std::pair<int64_t, int64_t>> first;  // (earliest position, index of group start)
  for (int64_t i = 0; i < n; ++i)
    if (i == 0 || rec[(size_t)i].first != rec[(size_t)i - 1].first) first.push_back({rec[(size_t)i].second, i});
  std::sort(first.begin(), first.end());
  ce.assign((size_t)n, -1);
  for (size_t id = 0; id < first.size(); ++id) {
    const int64_t s = first[id].second;
    for (int64_t j = s; j < n && rec[(size_t)j].first == rec[(size_t)s].first; ++j)
      ce[(size_t)rec[(size_t)j].second] = (int32_t)id;
  }
  return (int64_t)first.size();
}

// Vertex rows of the P1 mass matrix of a triangulation, topology only (for
// the P1xP1 gather form, which computes the weights from each launch's
// coordinate field): row a lists a itself, then its neighbours j in
// ascending order.  An entry carries, instead of the vertex j, the first DoF
// j col of j's CG1xCG1 column (col = layers + 1 levels; the DoF of level m
// is j col + m), and the cells on edge (a, j) in ascending order (-1 where
// the edge has one cell; both -1 on the diagonal).  Also the cells around
// every vertex, ascending.  Returns false (rows not built) when an edge has
// more than two cells or the entry count does not fit int32.
static bool build_vertex_rows(int64_t nv, int64_t nc, const int32_t *cv, int64_t col, std::vector<int32_t> &vrow,
                              std::vector<int32_t> &vnbr, std::vector<int2> &vedge, std::vector<int32_t> &vcrow,
                              std::vector<int32_t> &vcells) {
  if ((nv - 1) * col + col > (int64_t)INT32_MAX) return false;
  vcrow.assign((size_t)nv + 1, 0);
  for (int64_t c = 0; c < nc; ++c)
    for (int a = 0; a < 3; ++a) ++vcrow[(size_t)cv[3 * c + a] + 1];
  for (int64_t v = 0; v < nv; ++v) vcrow[(size_t)v + 1] += vcrow[(size_t)v];
  vcells.assign((size_t)(3 * nc), 0);
  {
    std::vector<int32_t> cur(vcrow.begin(), vcrow.end() - 1);
    for (int64_t c = 0; c < nc; ++c)
      for (int a = 0; a < 3; ++a) vcells[(size_t)cur[(size_t)cv[3 * c + a]]++] = (int32_t)c;
  }
  vrow.assign((size_t)nv + 1, 0);
  vnbr.clear();
  vedge.clear();
  vnbr.reserve((size_t)(nv + 6 * nc));
  vedge.reserve((size_t)(nv + 6 * nc));
  std::vector<std::pair<int32_t, int32_t>> nb;  // (neighbour, cell)
  for (int64_t a = 0; a < nv; ++a) {
    nb.clear();
    for (int32_t t = vcrow[(size_t)a]; t < vcrow[(size_t)a + 1]; ++t) {
      const int32_t c = vcells[(size_t)t];
      for (int k = 0; k < 3; ++k)
        if (cv[3 * (int64_t)c + k] != a) nb.push_back({cv[3 * (int64_t)c + k], c});
    }
    std::sort(nb.begin(), nb.end());
    vnbr.push_back((int32_t)(a * col));
    vedge.push_back(make_int2(-1, -1));
    for (size_t i = 0; i < nb.size();) {
      size_t e = i + 1;
      while (e < nb.size() && nb[e].first == nb[i].first) ++e;
      if (e - i > 2) return false;
      vnbr.push_back((int32_t)(nb[i].first * col));
      vedge.push_back(make_int2(nb[i].second, e - i == 2 ? nb[i + 1].second : -1));
      i = e;
    }
    if (vnbr.size() >= (size_t)INT32_MAX) return false;
    vrow[(size_t)a + 1] = (int32_t)vnbr.size();
  }
  return true;
}

static void free_mesh(ext_mesh *m) {
  if (!m) return;
  cudaFree(m->d_cell_verts);
  cudaFree(m->d_cell_edges);
  cudaFree(m->d_base_xy);
  cudaFree(m->d_cell_first);
  cudaFree(m->d_cell_layers);
  cudaFree(m->d_ent_lo);
  cudaFree(m->d_ent_hi);
  cudaFree(m->d_vrow);
  cudaFree(m->d_vnbr);
  cudaFree(m->d_vedge);
  cudaFree(m->d_vcrow);
  cudaFree(m->d_vcells);
  delete reinterpret_cast<ext_mesh_host *>(m->host);
  delete m;
}

// Shared by ext_mesh_create and ext_mesh_create_var (first/lay non-null:
// variable layers, `layers` ignored).
static ext_status create_mesh(int32_t kind, int64_t nverts, int64_t ncells, const int32_t *cell_verts_host,
                              const double *base_xy_host, int32_t layers, const int32_t *first,
                              const int32_t *lay, ext_mesh **out) {
  if (!out) return ext_fail(EXT_EINVAL, "ext_mesh_create: out is NULL");
  *out = nullptr;
  if (kind != EXT_TRI && kind != EXT_QUAD) return ext_fail(EXT_EINVAL, "ext_mesh_create: kind must be 3 or 4");
  const bool var = first != nullptr;
  double mean = 0.0;
  if (var) {
    if (ncells > 0 && !lay) return ext_fail(EXT_EINVAL, "ext_mesh_create_var: cell_layers is NULL");
    int64_t top = 1, sum = 0;
    for (int64_t c = 0; c < ncells; ++c) {
      if (first[c] < 0 || lay[c] < 1 || (int64_t)first[c] + lay[c] >= (int64_t)1 << 30)
        return ext_fail(EXT_EINVAL, "ext_mesh_create_var: cell %lld has first %d, layers %d", (long long)c,
                        first[c], lay[c]);
      top = std::max(top, (int64_t)first[c] + lay[c]);
      sum += lay[c];
    }
    layers = (int32_t)top;
    mean = ncells > 0 ? (double)sum / (double)ncells : 1.0;
  }
  if (layers < 1) return ext_fail(EXT_EINVAL, "ext_mesh_create: layers must be >= 1 (got %d)", layers);
  if (nverts < 0 || ncells < 0) return ext_fail(EXT_EINVAL, "ext_mesh_create: negative count");
  if (nverts >= INT32_MAX || ncells * kind >= INT32_MAX)
    return ext_fail(EXT_EOVERFLOW, "ext_mesh_create: base mesh too large for int32 indices");
  if (ncells > 0 && !cell_verts_host) return ext_fail(EXT_EINVAL, "ext_mesh_create: cell_verts is NULL");
  for (int64_t c = 0; c < ncells; ++c) {
    for (int a = 0; a < kind; ++a) {
      const int32_t v = cell_verts_host[c * kind + a];
      if (v < 0 || v >= nverts)
        return ext_fail(EXT_EINVAL, "ext_mesh_create: cell %lld vertex %d = %d out of range", (long long)c, a, v);
      for (int b = 0; b < a; ++b)
        if (cell_verts_host[c * kind + b] == v)
          return ext_fail(EXT_EINVAL, "ext_mesh_create: cell %lld repeats vertex %d", (long long)c, v);
    }
    if (base_xy_host) {
      for (int a = 0; a < kind; ++a) {
        const int64_t p = cell_verts_host[c * kind + a];
        const int64_t n = cell_verts_host[c * kind + (a + 1) % kind];
        const int64_t q = cell_verts_host[c * kind + (a + kind - 1) % kind];
        const double ux = base_xy_host[2 * n] - base_xy_host[2 * p], uy = base_xy_host[2 * n + 1] - base_xy_host[2 * p + 1];
        const double vx = base_xy_host[2 * q] - base_xy_host[2 * p], vy = base_xy_host[2 * q + 1] - base_xy_host[2 * p + 1];
        if (!(ux * vy - uy * vx > 0.0))
          return ext_fail(EXT_EINVAL, "ext_mesh_create: cell %lld is clockwise, non-convex or degenerate", (long long)c);
      }
    }
  }
  if (var) {
    std::vector<char> used((size_t)nverts, 0);
    for (int64_t t = 0; t < ncells * kind; ++t) used[(size_t)cell_verts_host[t]] = 1;
    for (int64_t v = 0; v < nverts; ++v)
      if (!used[(size_t)v])
        return ext_fail(EXT_EINVAL, "ext_mesh_create_var: vertex %lld belongs to no cell", (long long)v);
  }
  std::vector<int32_t> ce;
  const int64_t nedges = derive_edges(kind, ncells, cell_verts_host, ce);

  ext_mesh *m = new ext_mesh();
  m->kind = kind;
  m->N[0] = nverts;
  m->N[1] = nedges;
  m->N[2] = ncells;
  m->layers = layers;
  cudaGetDevice(&m->device);
  auto *h = new ext_mesh_host();
  h->cell_verts.assign(cell_verts_host, cell_verts_host + ncells * kind);
  m->host = h;
  const size_t nb = (size_t)(ncells * kind) * sizeof(int32_t);
  cudaError_t e = cudaSuccess;
  if (nb) {
    if ((e = cudaMalloc(&m->d_cell_verts, nb)) == cudaSuccess &&
        (e = cudaMalloc(&m->d_cell_edges, nb)) == cudaSuccess &&
        (e = cudaMemcpy(m->d_cell_verts, cell_verts_host, nb, cudaMemcpyHostToDevice)) == cudaSuccess)
      e = cudaMemcpy(m->d_cell_edges, ce.data(), nb, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && base_xy_host && nverts > 0) {
    if ((e = cudaMalloc(&m->d_base_xy, (size_t)nverts * 2 * sizeof(double))) == cudaSuccess)
      e = cudaMemcpy(m->d_base_xy, base_xy_host, (size_t)nverts * 2 * sizeof(double), cudaMemcpyHostToDevice);
  }
  m->has_xy = base_xy_host != nullptr;
  if (e == cudaSuccess && kind == EXT_TRI && !var && nverts > 0 && ncells > 0) {
    std::vector<int32_t> vrow, vnbr, vcrow, vcells;
    std::vector<int2> vedge;
    if (build_vertex_rows(nverts, ncells, cell_verts_host, (int64_t)layers + 1, vrow, vnbr, vedge, vcrow, vcells)) {
      const size_t rb = sizeof(int32_t) * vrow.size(), nb4 = sizeof(int32_t) * vnbr.size();
      const size_t eb = sizeof(int2) * vedge.size(), cb = sizeof(int32_t) * vcells.size();
      if ((e = cudaMalloc(&m->d_vrow, rb)) == cudaSuccess && (e = cudaMalloc(&m->d_vnbr, nb4)) == cudaSuccess &&
          (e = cudaMalloc(&m->d_vedge, eb)) == cudaSuccess && (e = cudaMalloc(&m->d_vcrow, rb)) == cudaSuccess &&
          (e = cudaMalloc(&m->d_vcells, cb)) == cudaSuccess &&
          (e = cudaMemcpy(m->d_vrow, vrow.data(), rb, cudaMemcpyHostToDevice)) == cudaSuccess &&
          (e = cudaMemcpy(m->d_vnbr, vnbr.data(), nb4, cudaMemcpyHostToDevice)) == cudaSuccess &&
          (e = cudaMemcpy(m->d_vedge, vedge.data(), eb, cudaMemcpyHostToDevice)) == cudaSuccess &&
          (e = cudaMemcpy(m->d_vcrow, vcrow.data(), rb, cudaMemcpyHostToDevice)) == cudaSuccess)
        e = cudaMemcpy(m->d_vcells, vcells.data(), cb, cudaMemcpyHostToDevice);
      m->n_vent = (int64_t)vnbr.size();
    }
  }
  if (e == cudaSuccess && var) {
    m->var = true;
    m->mean_layers = mean;
    const int64_t nent = nverts + nedges + ncells;
    const size_t cb = sizeof(int32_t) * (size_t)std::max<int64_t>(ncells, 1);
    const size_t eb = sizeof(int32_t) * (size_t)std::max<int64_t>(nent, 1);
    if ((e = cudaMalloc(&m->d_cell_first, cb)) == cudaSuccess && (e = cudaMalloc(&m->d_cell_layers, cb)) == cudaSuccess &&
        (e = cudaMalloc(&m->d_ent_lo, eb)) == cudaSuccess && (e = cudaMalloc(&m->d_ent_hi, eb)) == cudaSuccess &&
        ncells > 0 &&
        (e = cudaMemcpy(m->d_cell_first, first, sizeof(int32_t) * ncells, cudaMemcpyHostToDevice)) == cudaSuccess &&
        (e = cudaMemcpy(m->d_cell_layers, lay, sizeof(int32_t) * ncells, cudaMemcpyHostToDevice)) == cudaSuccess &&
        (e = launch_var_ranges(m, 0)) == cudaSuccess)
      e = cudaStreamSynchronize(0);
  }
  if (e != cudaSuccess) {
    free_mesh(m);
    return ext_fail(e == cudaErrorMemoryAllocation ? EXT_ENOMEM : EXT_ECUDA, "ext_mesh_create: %s",
                    cudaGetErrorString(e));
  }
  *out = m;
  return EXT_OK;
}

extern "C" ext_status ext_mesh_create(int32_t kind, int64_t nverts, int64_t ncells,
                                      const int32_t *cell_verts_host, const double *base_xy_host,
                                      int32_t layers, ext_mesh **out) {
  return create_mesh(kind, nverts, ncells, cell_verts_host, base_xy_host, layers, nullptr, nullptr, out);
}

extern "C" ext_status ext_mesh_create_var(int32_t kind, int64_t nverts, int64_t ncells,
                                          const int32_t *cell_verts_host, const double *base_xy_host,
                                          const int32_t *cell_first_host, const int32_t *cell_layers_host,
                                          ext_mesh **out) {
  if (!cell_first_host && ncells > 0) {
    if (out) *out = nullptr;
    return ext_fail(EXT_EINVAL, "ext_mesh_create_var: cell_first is NULL");
  }
  static const int32_t none = 0;
  return create_mesh(kind, nverts, ncells, cell_verts_host, base_xy_host, 1,
                     cell_first_host ? cell_first_host : &none, cell_layers_host, out);
}

extern "C" ext_status ext_mesh_info(const ext_mesh *mesh, int32_t *kind, int64_t n[3], int32_t *layers) {
  if (!mesh) return ext_fail(EXT_EINVAL, "ext_mesh_info: mesh is NULL");
  if (kind) *kind = mesh->kind;
  if (n) for (int d = 0; d < 3; ++d) n[d] = mesh->N[d];
  if (layers) *layers = mesh->layers;
  return EXT_OK;
}

extern "C" void ext_mesh_destroy(ext_mesh *mesh) { free_mesh(mesh); }

// ---------------------------------------------------------------------------
// spaces

static int classify(const ext_mesh *m, const int32_t d[6]) {
  if (d[0] == 1 && d[1] == 0 && d[2] == 0 && d[3] == 0 && d[4] == 0 && d[5] == 0) return ELEM_P1P1;
  if (d[0] == 0 && d[1] == 0 && d[2] == 0 && d[3] == 0 && d[4] == 0 && d[5] > 0) return ELEM_DGCELL;
  if (m->kind == 4 && d[0] == 1 && d[1] == 1 && d[2] == 1 && d[3] == 1 && d[4] == 1 && d[5] == 1) return ELEM_Q2P2;
  return ELEM_GENERIC;
}

extern "C" ext_status ext_number_dofs(ext_mesh *mesh, const int32_t delta_host[6], int32_t ncomp, void *stream,
                                      ext_space **out) {
  if (!out) return ext_fail(EXT_EINVAL, "ext_number_dofs: out is NULL");
  *out = nullptr;
  if (!mesh || !delta_host) return ext_fail(EXT_EINVAL, "ext_number_dofs: mesh or delta is NULL");
  if (ncomp < 1 || ncomp > 3) return ext_fail(EXT_EINVAL, "ext_number_dofs: ncomp must be 1..3");
  for (int t = 0; t < 6; ++t)
    if (delta_host[t] < 0 || delta_host[t] > 4096) return ext_fail(EXT_EINVAL, "ext_number_dofs: delta[%d] out of range", t);
  const int nvc = mesh->kind;
  const int nent[3] = {nvc, nvc, 1};
  int64_t k = 0;
  for (int d = 0; d < 3; ++d) k += (int64_t)nent[d] * (2 * delta_host[2 * d] + delta_host[2 * d + 1]);
  if (k == 0) return ext_fail(EXT_EINVAL, "ext_number_dofs: the space has no DoFs");
  if (k > EXT_MAXK) return ext_fail(EXT_EUNSUPPORTED, "ext_number_dofs: stencil of %lld DoFs exceeds %d", (long long)k, EXT_MAXK);

  NumberLaunch nl;
  memset(&nl, 0, sizeof(nl));
  const int64_t L = mesh->layers;
  int64_t start = 0;
  for (int d = 0; d < 3; ++d) {
    nl.colsize[d] = L * (delta_host[2 * d] + delta_host[2 * d + 1]) + delta_host[2 * d];
    nl.block_start[d] = start;
    start += mesh->N[d] * nl.colsize[d];
  }
  int64_t ndofs = start;
  // Variable layers: entity column sizes from the entities' level ranges,
  // prefix-summed on the device into column starts (Algorithm 1's counter).
  int64_t *d_starts = nullptr, *d_scratch = nullptr;
  if (mesh->var) {
    const int64_t nent = mesh->N[0] + mesh->N[1] + mesh->N[2];
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc(&d_starts, sizeof(int64_t) * (nent + 1));
    if (e == cudaSuccess) e = cudaMalloc(&d_scratch, sizeof(int64_t) * scan_scratch_elems(nent));
    if (e == cudaSuccess) e = launch_var_colsize(mesh, delta_host, d_starts, st);
    if (e == cudaSuccess) e = launch_scan_i64(d_starts, nent, d_scratch, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ndofs, d_starts + nent, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaFree(d_starts);
      cudaFree(d_scratch);
      return ext_fail(e == cudaErrorMemoryAllocation ? EXT_ENOMEM : EXT_ECUDA, "ext_number_dofs: %s",
                      cudaGetErrorString(e));
    }
    nl.ent_start = d_starts;
    nl.ent_lo = mesh->d_ent_lo;
    nl.cell_first = mesh->d_cell_first;
    nl.ent_base[0] = 0;
    nl.ent_base[1] = mesh->N[0];
    nl.ent_base[2] = mesh->N[0] + mesh->N[1];
    for (int d = 0; d < 3; ++d) nl.colstep[d] = delta_host[2 * d] + delta_host[2 * d + 1];
  }
  if (ndofs >= INT32_MAX || ndofs * ncomp >= INT32_MAX || mesh->N[2] * k >= INT32_MAX) {
    cudaFree(d_starts);
    cudaFree(d_scratch);
    return ext_fail(EXT_EOVERFLOW, "ext_number_dofs: %lld DoFs do not fit int32 indices", (long long)ndofs);
  }

  ext_space *s = new ext_space();
  s->mesh = mesh;
  memcpy(s->delta, delta_host, sizeof(s->delta));
  s->ncomp = ncomp;
  s->k = (int32_t)k;
  s->ndofs = ndofs;
  s->elem = classify(mesh, delta_host);
  s->stream = (cudaStream_t)stream;
  int i = 0;
  for (int d = 0; d < 3; ++d) {
    const int a = delta_host[2 * d], b = delta_host[2 * d + 1];
    for (int e = 0; e < nent[d]; ++e) {
      for (int q = 0; q < a; ++q, ++i) {  // bottom horizontal entity
        nl.slot_dim[i] = (int8_t)d; nl.slot_ent[i] = (int8_t)e; nl.slot_add[i] = q;
        s->h_offset[i] = a + b;
      }
      for (int q = 0; q < a; ++q, ++i) {  // top horizontal entity
        nl.slot_dim[i] = (int8_t)d; nl.slot_ent[i] = (int8_t)e; nl.slot_add[i] = a + b + q;
        s->h_offset[i] = a + b;
      }
      for (int q = 0; q < b; ++q, ++i) {  // vertical entity
        nl.slot_dim[i] = (int8_t)d; nl.slot_ent[i] = (int8_t)e; nl.slot_add[i] = a + q;
        s->h_offset[i] = a + b;
      }
    }
  }
  nl.ncells = mesh->N[2];
  nl.nvc = nvc;
  nl.k = (int32_t)k;
  nl.cell_verts = mesh->d_cell_verts;
  nl.cell_edges = mesh->d_cell_edges;
  cudaError_t e = cudaMalloc(&s->d_offset, sizeof(int32_t) * k);
  if (e == cudaSuccess && nl.ncells > 0) e = cudaMalloc(&s->d_map, sizeof(int32_t) * k * nl.ncells);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_offset, s->h_offset, sizeof(int32_t) * k, cudaMemcpyHostToDevice, s->stream);
  nl.map = s->d_map;
  if (e == cudaSuccess) e = launch_number(nl, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFree(d_starts);
  cudaFree(d_scratch);
  if (e != cudaSuccess) {
    cudaFree(s->d_map);
    cudaFree(s->d_offset);
    delete s;
    return ext_fail(e == cudaErrorMemoryAllocation ? EXT_ENOMEM : EXT_ECUDA, "ext_number_dofs: %s", cudaGetErrorString(e));
  }
  *out = s;
  return EXT_OK;
}

extern "C" ext_status ext_space_info(const ext_space *space, int64_t *ndofs, int32_t *k, int32_t *ncomp,
                                     const int32_t **base_map_dev, const int32_t **offset_dev) {
  if (!space) return ext_fail(EXT_EINVAL, "ext_space_info: space is NULL");
  if (ndofs) *ndofs = space->ndofs;
  if (k) *k = space->k;
  if (ncomp) *ncomp = space->ncomp;
  if (base_map_dev) *base_map_dev = space->d_map;
  if (offset_dev) *offset_dev = space->d_offset;
  return EXT_OK;
}

extern "C" ext_status ext_space_copy_map_to_host(const ext_space *space, int32_t *map_host, int32_t *offset_host) {
  if (!space) return ext_fail(EXT_EINVAL, "ext_space_copy_map_to_host: space is NULL");
  if (space->ragged)
    return ext_fail(EXT_EINVAL, "ext_space_copy_map_to_host: ragged lists (use ext_space_copy_ragged_to_host)");
  if (map_host && space->mesh->N[2] > 0)
    EXT_CUDA(cudaMemcpy(map_host, space->d_map, sizeof(int32_t) * space->k * space->mesh->N[2], cudaMemcpyDeviceToHost),
             "ext_space_copy_map_to_host");
  if (offset_host) memcpy(offset_host, space->h_offset, sizeof(int32_t) * space->k);
  return EXT_OK;
}

extern "C" void ext_space_destroy(ext_space *space) {
  if (!space) return;
  cudaFree(space->d_map);
  cudaFree(space->d_offset);
  cudaFree(space->d_rowptr);
  cudaFree(space->d_roff);
  for (int i = 0; i < 4; ++i) cudaFree(space->d_cells_by_k[i]);
  delete space;
}

enum : int { ELEM_RAGGED = 16 };

extern "C" ext_status ext_number_dofs_ragged(ext_mesh *mesh, const int32_t *dent_host, int32_t ncomp, void *stream,
                                             ext_space **out) {
  if (!out) return ext_fail(EXT_EINVAL, "ext_number_dofs_ragged: out is NULL");
  *out = nullptr;
  if (!mesh) return ext_fail(EXT_EINVAL, "ext_number_dofs_ragged: mesh is NULL");
  if (ncomp < 1 || ncomp > 3) return ext_fail(EXT_EINVAL, "ext_number_dofs_ragged: ncomp must be 1..3");
  const int64_t nent = mesh->N[0] + mesh->N[1] + mesh->N[2];
  if (nent > 0 && !dent_host) return ext_fail(EXT_EINVAL, "ext_number_dofs_ragged: dent is NULL");
  bool dg_cells = true, dgp = true;
  int64_t any = 0;
  for (int64_t g = 0; g < nent; ++g) {
    const int32_t a = dent_host[2 * g], b = dent_host[2 * g + 1];
    if (a < 0 || b < 0 || a > 4096 || b > 4096)
      return ext_fail(EXT_EINVAL, "ext_number_dofs_ragged: entity %lld has counts %d, %d", (long long)g, a, b);
    any += a + b;
    const bool cell = g >= mesh->N[0] + mesh->N[1];
    if ((!cell && (a | b)) || (cell && a)) dg_cells = false;
    if (cell && !(b == 1 || b == 2 || b == 3 || b == 6)) dgp = false;
  }
  if (any == 0) return ext_fail(EXT_EINVAL, "ext_number_dofs_ragged: the space has no DoFs");
  ext_space *sp = new ext_space();
  sp->mesh = mesh;
  memset(sp->delta, 0, sizeof(sp->delta));
  sp->ncomp = ncomp;
  sp->k = 0;
  sp->elem = ELEM_RAGGED;
  sp->ragged = true;
  sp->dg_cells = dg_cells;
  sp->dgp = dg_cells && dgp && mesh->kind == EXT_TRI;
  sp->stream = (cudaStream_t)stream;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t C = mesh->N[2];
  int32_t *d_dent = nullptr;
  int64_t *d_starts = nullptr, *d_scratch = nullptr;
  int64_t ndofs = 0, nentries = 0;
  RaggedLaunch rl;
  memset(&rl, 0, sizeof(rl));
  for (int d = 0; d < 3; ++d) rl.N[d] = mesh->N[d];
  rl.ncells = C;
  rl.nvc = mesh->kind;
  rl.layers = mesh->layers;
  rl.cell_verts = mesh->d_cell_verts;
  rl.cell_edges = mesh->d_cell_edges;
  if (mesh->var) {
    rl.ent_lo = mesh->d_ent_lo;
    rl.ent_hi = mesh->d_ent_hi;
    rl.cell_first = mesh->d_cell_first;
  }
  const int64_t nscr = scan_scratch_elems(nent > C ? nent : C);
  cudaError_t e = cudaMalloc(&d_dent, sizeof(int32_t) * 2 * (nent > 0 ? nent : 1));
  if (e == cudaSuccess) e = cudaMalloc(&d_starts, sizeof(int64_t) * (nent + 1));
  if (e == cudaSuccess) e = cudaMalloc(&d_scratch, sizeof(int64_t) * nscr);
  if (e == cudaSuccess) e = cudaMalloc(&sp->d_rowptr, sizeof(int64_t) * (C + 1));
  if (e == cudaSuccess && nent > 0)
    e = cudaMemcpyAsync(d_dent, dent_host, sizeof(int32_t) * 2 * nent, cudaMemcpyHostToDevice, st);
  rl.dent = d_dent;
  rl.ent_start = d_starts;
  rl.rowptr = sp->d_rowptr;
  // Algorithm 1's counter at each entity column: a prefix sum of the sizes;
  // each row's start: a prefix sum of the row lengths
  if (e == cudaSuccess) e = launch_ragged_colsize(rl, d_starts, st);
  if (e == cudaSuccess) e = launch_scan_i64(d_starts, nent, d_scratch, st);
  if (e == cudaSuccess) e = launch_ragged_rowlen(rl, st);
  if (e == cudaSuccess) e = launch_scan_i64(sp->d_rowptr, C, d_scratch, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ndofs, d_starts + nent, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nentries, sp->d_rowptr + C, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  ext_status bad = EXT_OK;
  if (e == cudaSuccess && (ndofs >= INT32_MAX || ndofs * ncomp >= INT32_MAX))
    bad = ext_fail(EXT_EOVERFLOW, "ext_number_dofs_ragged: %lld DoFs do not fit int32 indices", (long long)ndofs);
  if (e == cudaSuccess && bad == EXT_OK) {
    e = cudaMalloc(&sp->d_map, sizeof(int32_t) * (nentries > 0 ? nentries : 1));
    if (e == cudaSuccess) e = cudaMalloc(&sp->d_roff, sizeof(int32_t) * (nentries > 0 ? nentries : 1));
    rl.map = sp->d_map;
    rl.roff = sp->d_roff;
    if (e == cudaSuccess) e = launch_ragged_map(rl, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(d_dent);
  cudaFree(d_starts);
  cudaFree(d_scratch);
  if (e == cudaSuccess && bad == EXT_OK && sp->dgp) {
    // p-adaptive DG: the cells of each element kind, for one launch per kind
    const int kinds[4] = {1, 2, 3, 6};
    std::vector<int32_t> lst;
    const int64_t cbase = mesh->N[0] + mesh->N[1];
    for (int t = 0; t < 4 && e == cudaSuccess; ++t) {
      lst.clear();
      for (int64_t c = 0; c < C; ++c)
        if (dent_host[2 * (cbase + c) + 1] == kinds[t]) lst.push_back((int32_t)c);
      sp->ncells_by_k[t] = (int64_t)lst.size();
      if (lst.empty()) continue;
      e = cudaMalloc(&sp->d_cells_by_k[t], sizeof(int32_t) * lst.size());
      if (e == cudaSuccess)
        e = cudaMemcpy(sp->d_cells_by_k[t], lst.data(), sizeof(int32_t) * lst.size(), cudaMemcpyHostToDevice);
    }
  }
  if (e != cudaSuccess || bad != EXT_OK) {
    ext_space_destroy(sp);
    if (bad != EXT_OK) return bad;
    return ext_fail(e == cudaErrorMemoryAllocation ? EXT_ENOMEM : EXT_ECUDA, "ext_number_dofs_ragged: %s",
                    cudaGetErrorString(e));
  }
  sp->ndofs = ndofs;
  sp->nentries = nentries;
  *out = sp;
  return EXT_OK;
}

extern "C" ext_status ext_space_ragged_info(const ext_space *space, int64_t *nentries, const int64_t **rowptr_dev,
                                            const int32_t **map_dev, const int32_t **offset_dev) {
  if (!space) return ext_fail(EXT_EINVAL, "ext_space_ragged_info: space is NULL");
  if (!space->ragged) return ext_fail(EXT_EINVAL, "ext_space_ragged_info: the space has one list length k");
  if (nentries) *nentries = space->nentries;
  if (rowptr_dev) *rowptr_dev = space->d_rowptr;
  if (map_dev) *map_dev = space->d_map;
  if (offset_dev) *offset_dev = space->d_roff;
  return EXT_OK;
}

extern "C" ext_status ext_space_copy_ragged_to_host(const ext_space *space, int64_t *rowptr_host, int32_t *map_host,
                                                    int32_t *offset_host) {
  if (!space) return ext_fail(EXT_EINVAL, "ext_space_copy_ragged_to_host: space is NULL");
  if (!space->ragged) return ext_fail(EXT_EINVAL, "ext_space_copy_ragged_to_host: the space has one list length k");
  const int64_t C = space->mesh->N[2];
  if (rowptr_host)
    EXT_CUDA(cudaMemcpy(rowptr_host, space->d_rowptr, sizeof(int64_t) * (C + 1), cudaMemcpyDeviceToHost),
             "ext_space_copy_ragged_to_host");
  if (map_host && space->nentries > 0)
    EXT_CUDA(cudaMemcpy(map_host, space->d_map, sizeof(int32_t) * space->nentries, cudaMemcpyDeviceToHost),
             "ext_space_copy_ragged_to_host");
  if (offset_host && space->nentries > 0)
    EXT_CUDA(cudaMemcpy(offset_host, space->d_roff, sizeof(int32_t) * space->nentries, cudaMemcpyDeviceToHost),
             "ext_space_copy_ragged_to_host");
  return EXT_OK;
}

// ---------------------------------------------------------------------------
// par_loop

// The nine prism spaces of Sec. 4.1.2 by their delta: horizontal element h
// and vertical element v (0 CG1, 1 DG0, 2 DG1); -1 if delta is none of them.
static int prism_pair(const int32_t d[6], int *h, int *v) {
  static const int32_t tab[9][6] = {{1, 0, 0, 0, 0, 0}, {0, 1, 0, 0, 0, 0}, {0, 2, 0, 0, 0, 0},
                                    {0, 0, 0, 0, 1, 0}, {0, 0, 0, 0, 0, 1}, {0, 0, 0, 0, 0, 2},
                                    {0, 0, 0, 0, 3, 0}, {0, 0, 0, 0, 0, 3}, {0, 0, 0, 0, 0, 6}};
  for (int i = 0; i < 9; ++i)
    if (memcmp(tab[i], d, sizeof(tab[i])) == 0) {
      *h = i / 3;
      *v = i % 3;
      return i;
    }
  return -1;
}

// Stencil slot of every (horizontal node, vertical node) of a prism pair,
// following the stencil order of ext_number_dofs: entities vertices, edges,
// cell; per entity bottom, top, then vertical DoFs; horizontal index major.
static void prism_pair_slots(int h, int v, int nh, int nv, int32_t *slot) {
  const int dh[3] = {h == 0 ? 1 : 0, 0, h == 1 ? 1 : (h == 2 ? 3 : 0)};
  const int dv0 = v == 0 ? 1 : 0, dv1 = v == 1 ? 1 : (v == 2 ? 2 : 0);
  int i = 0;
  for (int d = 0; d < 3; ++d)
    for (int e = 0; e < (d == 2 ? 1 : 3); ++e)
      for (int part = 0; part < 3; ++part) {
        const int nvp = part < 2 ? dv0 : dv1;
        for (int j = 0; j < dh[d]; ++j)
          for (int beta = 0; beta < nvp; ++beta, ++i) {
            const int a = nh == 1 ? 0 : (d == 0 ? e : j);
            const int b = nv == 1 ? 0 : (part < 2 ? part : beta);
            slot[a * nv + b] = i;
          }
      }
}

static ext_status check_arg(const ext_mesh *mesh, const ext_arg *args, int i, const char *kn, int elem, int ncomp,
                            int access) {
  const ext_arg &a = args[i];
  if (!a.space) return ext_fail(EXT_EINVAL, "%s: argument %d has no space", kn, i);
  if (a.space->mesh != mesh) return ext_fail(EXT_EINVAL, "%s: argument %d is on another mesh", kn, i);
  if (!a.data && a.space->ndofs > 0) return ext_fail(EXT_EINVAL, "%s: argument %d has no data", kn, i);
  if (elem >= 0 && a.space->elem != elem) return ext_fail(EXT_EINVAL, "%s: argument %d is on the wrong space", kn, i);
  if (a.space->ncomp != ncomp) return ext_fail(EXT_EINVAL, "%s: argument %d must have %d values per DoF", kn, i, ncomp);
  if (a.access != access) {
    static const char *nm[3] = {"READ", "WRITE", "INC"};
    return ext_fail(EXT_EINVAL, "%s: argument %d must be %s", kn, i, (access >= 0 && access < 3) ? nm[access] : "?");
  }
  return EXT_OK;
}

static bool same_numbering(const ext_space *a, const ext_space *b) {
  if (a->ragged || b->ragged) return a == b;  // per-entity counts: the same space object
  return a->mesh == b->mesh && memcmp(a->delta, b->delta, sizeof(a->delta)) == 0;
}

#define EXT_CHECK(x)                   \
  do {                                 \
    ext_status st_ = (x);              \
    if (st_ != EXT_OK) return st_;     \
  } while (0)

// A WRITE or INC argument may share no byte with another argument of the
// same launch (checked from the arguments' base pointers and sizes).
static ext_status check_no_overlap(int32_t nargs, const ext_arg *args, const char *who) {
  for (int i = 0; i < nargs; ++i) {
    if (args[i].access == EXT_READ || !args[i].space || !args[i].data) continue;
    const char *lo_i = (const char *)args[i].data;
    const char *hi_i = lo_i + sizeof(double) * (size_t)args[i].space->ndofs * (size_t)args[i].space->ncomp;
    for (int j = 0; j < nargs; ++j) {
      if (j == i || !args[j].space || !args[j].data) continue;
      const char *lo_j = (const char *)args[j].data;
      const char *hi_j = lo_j + sizeof(double) * (size_t)args[j].space->ndofs * (size_t)args[j].space->ncomp;
      if (lo_i < hi_j && lo_j < hi_i)
        return ext_fail(EXT_EINVAL, "%s: argument %d (written) overlaps argument %d", who, i, j);
    }
  }
  return EXT_OK;
}

extern "C" ext_status ext_space_check(const ext_space *space, void *stream) {
  if (!space || !space->mesh) return ext_fail(EXT_EINVAL, "ext_space_check: space is NULL");
  const ext_mesh *mesh = space->mesh;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned int *w = ext_device_error_word();
  if (!w) return ext_fail(EXT_ECUDA, "ext_space_check: no device error word");
  unsigned int v = 0;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v) return ext_fail(EXT_EDEVICE, "ext_space_check: the device error word is already set (0x%x)", v);
  if (e == cudaSuccess && space->d_map) e = launch_check_map(space, mesh->d_cell_layers, mesh->layers, w, s);
  if (e == cudaSuccess && space->elem == ELEM_P1P1 && space->ncomp == 1) e = launch_check_rows(mesh, space->ndofs, w, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return ext_fail(EXT_ECUDA, "ext_space_check: %s", cudaGetErrorString(e));
  if (v & EXT_DERR_BOUNDS) {
    cudaMemset(w, 0, sizeof(v));
    return ext_fail(EXT_EDEVICE, "ext_space_check: a stencil index of the space is out of range");
  }
  return EXT_OK;
}

extern "C" ext_status ext_par_loop(const ext_mesh *mesh, int32_t kernel_id, int32_t nargs, const ext_arg *args,
                                   void *stream) {
  if (!mesh) return ext_fail(EXT_EINVAL, "ext_par_loop: mesh is NULL");
  if (nargs > 0 && !args) return ext_fail(EXT_EINVAL, "ext_par_loop: args is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t C = mesh->N[2];
  const int L = mesh->layers;
  cudaError_t e = cudaSuccess;
  EXT_CHECK(check_no_overlap(nargs, args, "ext_par_loop"));
#ifdef EXT_CHECKED
  // checked build: every index the launch will form from the stencil maps
  // (and the gather form's vertex rows) is range-checked on the device first;
  // on a failure nothing is launched
  {
    unsigned int *w = ext_device_error_word();
    if (!w) return ext_fail(EXT_ECUDA, "ext_par_loop: no device error word");
    for (int i = 0; i < nargs && e == cudaSuccess; ++i)
      if (args[i].space && args[i].space->d_map && args[i].space->mesh == mesh)
        e = launch_check_map(args[i].space, mesh->d_cell_layers, L, w, s);
    // the vertex rows address the CG1xCG1 space (an argument of another space
    // is refused by the kernel's own validation below)
    if (e == cudaSuccess && (kernel_id == EXT_K_RHS_P1P1 || kernel_id == EXT_K_MASS_P1P1) && nargs > 1 &&
        args[1].space && args[1].space->mesh == mesh && args[1].space->elem == ELEM_P1P1 && args[1].space->ncomp == 1)
      e = launch_check_rows(mesh, args[1].space->ndofs, w, s);
    unsigned int v = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ext_fail(EXT_ECUDA, "ext_par_loop: checked build: %s", cudaGetErrorString(e));
    if (v & EXT_DERR_BOUNDS) {
      cudaMemset(w, 0, sizeof(v));
      return ext_fail(EXT_EDEVICE, "ext_par_loop: checked build: a stencil index is out of range; nothing launched");
    }
  }
#endif
  switch (kernel_id) {
    case EXT_K_EXTRUDE: {
      const char *kn = "EXT_K_EXTRUDE";
      if (nargs != 1) return ext_fail(EXT_EINVAL, "%s: expects 1 argument", kn);
      EXT_CHECK(check_arg(mesh, args, 0, kn, ELEM_P1P1, 3, EXT_WRITE));
      if (!mesh->has_xy) return ext_fail(EXT_EINVAL, "%s: the mesh has no base coordinates", kn);
      ExtrudeLaunch p;
      p.ncells = C;
      p.nvc = mesh->kind;
      p.layers = L;
      p.cell_verts = mesh->d_cell_verts;
      p.base_xy = mesh->d_base_xy;
      p.map = args[0].space->d_map;
      p.off = args[0].space->h_offset[0];
      p.X = (double *)args[0].data;
      p.cell_first = mesh->d_cell_first;
      p.cell_layers = mesh->d_cell_layers;
      e = launch_extrude(p, s);
      break;
    }
    case EXT_K_COPY_DG: {
      const char *kn = "EXT_K_COPY_DG";
      if (nargs != 2) return ext_fail(EXT_EINVAL, "%s: expects 2 arguments", kn);
      const bool rg = args[0].space && args[0].space->ragged;
      if (rg && !args[0].space->dg_cells)
        return ext_fail(EXT_EINVAL, "%s: the space has DoFs outside the cells", kn);
      EXT_CHECK(check_arg(mesh, args, 0, kn, rg ? (int)ELEM_RAGGED : (int)ELEM_DGCELL, 1, EXT_READ));
      EXT_CHECK(check_arg(mesh, args, 1, kn, rg ? (int)ELEM_RAGGED : (int)ELEM_DGCELL, 1, EXT_WRITE));
      if (!same_numbering(args[0].space, args[1].space))
        return ext_fail(EXT_EINVAL, "%s: input and output must share one numbering", kn);
      CopyDGLaunch p;
      p.ncells = C;
      p.k = args[0].space->k;
      p.layers = L;
      p.map = args[0].space->d_map;
      p.in = (const double *)args[0].data;
      p.out = (double *)args[1].data;
      p.cell_layers = mesh->d_cell_layers;
      p.rowptr = rg ? args[0].space->d_rowptr : nullptr;
      e = launch_copy_dg(p, s);
      break;
    }
    case EXT_K_RHS_P1P1:
    case EXT_K_MASS_P1P1: {
      const char *kn = kernel_id == EXT_K_RHS_P1P1 ? "EXT_K_RHS_P1P1" : "EXT_K_MASS_P1P1";
      if (mesh->kind != EXT_TRI) return ext_fail(EXT_EINVAL, "%s: needs a triangular base mesh", kn);
      if (nargs != 3) return ext_fail(EXT_EINVAL, "%s: expects 3 arguments", kn);
      EXT_CHECK(check_arg(mesh, args, 0, kn, ELEM_P1P1, 3, EXT_READ));
      EXT_CHECK(check_arg(mesh, args, 1, kn, ELEM_P1P1, 1, EXT_READ));
      // INC adds M f into b; WRITE overwrites b with M f
      EXT_CHECK(check_arg(mesh, args, 2, kn, ELEM_P1P1, 1, args[2].access == EXT_WRITE ? EXT_WRITE : EXT_INC));
      MassP1Launch p;
      p.ncells = C;
      p.layers = L;
      p.cmap = args[0].space->d_map;
      p.fmap = args[1].space->d_map;
      p.bmap = args[2].space->d_map;
      for (int i = 0; i < 6; ++i) {
        p.coff[i] = args[0].space->h_offset[i];
        p.foff[i] = args[1].space->h_offset[i];
        p.boff[i] = args[2].space->h_offset[i];
      }
      p.X = (const double *)args[0].data;
      p.f = (const double *)args[1].data;
      p.b = (double *)args[2].data;
      p.err = ext_device_error_word();
      p.cell_layers = mesh->d_cell_layers;
      p.mean_layers = mesh->mean_layers;
      p.nf = args[1].space->ndofs;
      p.base_xy = mesh->has_xy ? mesh->d_base_xy : nullptr;
      p.overwrite = args[2].access == EXT_WRITE;
      p.vrow = mesh->d_vrow;
      p.vnbr = mesh->d_vnbr;
      p.vedge = mesh->d_vedge;
      p.nverts = (int32_t)mesh->N[0];
      p.nvent = mesh->n_vent;
      p.vcrow = mesh->d_vcrow;
      p.vcells = mesh->d_vcells;
      e = launch_mass_p1(p, s);
      break;
    }
    case EXT_K_INTERP_DG1: {
      const char *kn = "EXT_K_INTERP_DG1";
      if (mesh->kind != EXT_TRI) return ext_fail(EXT_EINVAL, "%s: needs a triangular base mesh", kn);
      if (nargs != 2) return ext_fail(EXT_EINVAL, "%s: expects 2 arguments", kn);
      EXT_CHECK(check_arg(mesh, args, 0, kn, ELEM_P1P1, 1, EXT_READ));
      EXT_CHECK(check_arg(mesh, args, 1, kn, ELEM_DGCELL, 1, EXT_WRITE));
      if (args[1].space->delta[5] != 6) return ext_fail(EXT_EINVAL, "%s: output must be DG1xDG1 (delta(2,1)=6)", kn);
      InterpDG1Launch p;
      p.ncells = C;
      p.layers = L;
      p.xmap = args[0].space->d_map;
      p.xoff = args[0].space->h_offset[0];
      p.omap = args[1].space->d_map;
      p.x = (const double *)args[0].data;
      p.out = (double *)args[1].data;
      if ((((uintptr_t)p.out) & 15) != 0) return ext_fail(EXT_EINVAL, "%s: output data must be 16-byte aligned", kn);
      p.cell_layers = mesh->d_cell_layers;
      e = launch_interp_dg1(p, s);
      break;
    }
    case EXT_K_U2V_FWD:
    case EXT_K_U2V_ADJ:
    case EXT_K_U2V_FWDADJ: {
      const char *kn = kernel_id == EXT_K_U2V_FWD ? "EXT_K_U2V_FWD"
                                                  : (kernel_id == EXT_K_U2V_ADJ ? "EXT_K_U2V_ADJ" : "EXT_K_U2V_FWDADJ");
      const int mode = kernel_id == EXT_K_U2V_FWD ? 1 : (kernel_id == EXT_K_U2V_ADJ ? 2 : 3);
      const int want = mode == 1 ? 3 : (mode == 2 ? 4 : 5);
      if (mesh->var) return ext_fail(EXT_EUNSUPPORTED, "%s: not available on meshes with variable layers", kn);
      if (nargs != want) return ext_fail(EXT_EINVAL, "%s: expects %d arguments", kn, want);
      EXT_CHECK(check_arg(mesh, args, 0, kn, ELEM_P1P1, 3, EXT_READ));
      const ext_space *us = args[1].space;
      if (!us) return ext_fail(EXT_EINVAL, "%s: argument 1 has no space", kn);
      bool dg = false;
      if (mesh->kind == EXT_TRI) {
        if (us->elem != ELEM_P1P1) return ext_fail(EXT_EUNSUPPORTED, "%s: prisms support CG1xCG1 only", kn);
      } else {
        if (us->elem == ELEM_DGCELL && us->delta[5] == 27) dg = true;
        else if (us->elem != ELEM_Q2P2) return ext_fail(EXT_EUNSUPPORTED, "%s: hexahedra support Q2xP2 and DG2", kn);
      }
      const int out_access = dg ? EXT_WRITE : EXT_INC;
      EXT_CHECK(check_arg(mesh, args, 1, kn, us->elem, 1, EXT_READ));
      int ai = 2;
      if (mode & 2) EXT_CHECK(check_arg(mesh, args, ai++, kn, us->elem, 1, EXT_READ));
      const int fo = ai;
      if (mode & 1) EXT_CHECK(check_arg(mesh, args, ai++, kn, us->elem, 1, out_access));
      const int go = ai;
      if (mode & 2) EXT_CHECK(check_arg(mesh, args, ai++, kn, us->elem, 1, out_access));
      for (int j = 2; j < nargs; ++j)
        if (!same_numbering(us, args[j].space)) return ext_fail(EXT_EINVAL, "%s: u, w, F and g must share one numbering", kn);
      U2VLaunch p;
      memset(&p, 0, sizeof(p));
      p.ncells = C;
      p.layers = L;
      p.nvc = mesh->kind;
      p.dg = dg;
      p.mode = mode;
      p.cmap = args[0].space->d_map;
      for (int i = 0; i < 2 * mesh->kind; ++i) p.coff[i] = args[0].space->h_offset[i];
      p.umap = us->d_map;
      p.k = us->k;
      for (int i = 0; i < us->k && i < 27; ++i) p.uoff[i] = us->h_offset[i];
      p.X = (const double *)args[0].data;
      p.u = (const double *)args[1].data;
      p.w = (mode & 2) ? (const double *)args[2].data : nullptr;
      p.F = (mode & 1) ? (double *)args[fo].data : nullptr;
      p.g = (mode & 2) ? (double *)args[go].data : nullptr;
      p.err = ext_device_error_word();
      e = launch_u2v(p, s);
      break;
    }
    case EXT_K_MASS_TP: {
      const char *kn = "EXT_K_MASS_TP";
      if (mesh->kind != EXT_TRI) return ext_fail(EXT_EINVAL, "%s: needs a triangular base mesh", kn);
      if (nargs != 3) return ext_fail(EXT_EINVAL, "%s: expects 3 arguments", kn);
      EXT_CHECK(check_arg(mesh, args, 0, kn, ELEM_P1P1, 3, EXT_READ));
      EXT_CHECK(check_arg(mesh, args, 1, kn, -1, 1, EXT_READ));
      // INC adds M f into b; WRITE overwrites b with M f
      EXT_CHECK(check_arg(mesh, args, 2, kn, -1, 1, args[2].access == EXT_WRITE ? EXT_WRITE : EXT_INC));
      if (!same_numbering(args[1].space, args[2].space))
        return ext_fail(EXT_EINVAL, "%s: f and b must share one numbering", kn);
      int h = 0, v = 0;
      if (prism_pair(args[1].space->delta, &h, &v) < 0)
        return ext_fail(EXT_EUNSUPPORTED, "%s: not one of the nine CG1/DG0/DG1 prism spaces", kn);
      if (h == 0 && v == 0) return ext_par_loop(mesh, EXT_K_MASS_P1P1, nargs, args, stream);
      MassTPLaunch p;
      memset(&p, 0, sizeof(p));
      p.k1 = fp64_ones();
      p.ncells = C;
      p.layers = L;
      p.nh = h == 1 ? 1 : 3;
      p.nv = v == 1 ? 1 : 2;
      p.k = args[1].space->k;
      p.cmap = args[0].space->d_map;
      for (int i = 0; i < 6; ++i) p.coff[i] = args[0].space->h_offset[i];
      p.fmap = args[1].space->d_map;
      prism_pair_slots(h, v, p.nh, p.nv, p.slot);
      for (int i = 0; i < p.nh * p.nv; ++i) p.off[i] = args[1].space->h_offset[p.slot[i]];
      p.scale = 0.5 * (p.nh == 3 ? 1.0 / 12.0 : 1.0) * (p.nv == 2 ? 1.0 / 6.0 : 1.0);
      p.X = (const double *)args[0].data;
      p.f = (const double *)args[1].data;
      p.b = (double *)args[2].data;
      p.cell_layers = mesh->d_cell_layers;
      p.mean_layers = mesh->mean_layers;
      p.base_xy = mesh->has_xy ? mesh->d_base_xy : nullptr;
      p.ncoord = args[0].space->ndofs;
      p.overwrite = args[2].access == EXT_WRITE;
      p.hown = h != 0;
      p.vcont = v == 0;
      p.nf = args[1].space->ndofs;
      p.vrow = mesh->d_vrow;
      p.vnbr = mesh->d_vnbr;
      p.vedge = mesh->d_vedge;
      p.vcrow = mesh->d_vcrow;
      p.vcells = mesh->d_vcells;
      p.nverts = (int32_t)mesh->N[0];
      p.nvent = mesh->n_vent;
      p.err = ext_device_error_word();
      e = launch_mass_tp(p, s);
      break;
    }
    case EXT_K_MASS_DGP: {
      const char *kn = "EXT_K_MASS_DGP";
      if (mesh->kind != EXT_TRI) return ext_fail(EXT_EINVAL, "%s: needs a triangular base mesh", kn);
      if (nargs != 3) return ext_fail(EXT_EINVAL, "%s: expects 3 arguments", kn);
      EXT_CHECK(check_arg(mesh, args, 0, kn, ELEM_P1P1, 3, EXT_READ));
      EXT_CHECK(check_arg(mesh, args, 1, kn, ELEM_RAGGED, 1, EXT_READ));
      EXT_CHECK(check_arg(mesh, args, 2, kn, ELEM_RAGGED, 1, EXT_INC));
      if (!same_numbering(args[1].space, args[2].space))
        return ext_fail(EXT_EINVAL, "%s: f and b must be on the same space", kn);
      if (!args[1].space->dgp)
        return ext_fail(EXT_EINVAL, "%s: every cell needs 1, 2, 3 or 6 DoFs and no DoF may sit outside the cells", kn);
      MassDGPLaunch p;
      memset(&p, 0, sizeof(p));
      p.layers = L;
      p.cmap = args[0].space->d_map;
      for (int i = 0; i < 6; ++i) p.coff[i] = args[0].space->h_offset[i];
      p.rowptr = args[1].space->d_rowptr;
      p.fmap = args[1].space->d_map;
      p.X = (const double *)args[0].data;
      p.f = (const double *)args[1].data;
      p.b = (double *)args[2].data;
      p.cell_layers = mesh->d_cell_layers;
      p.mean_layers = mesh->mean_layers;
      const int kinds[4] = {1, 2, 3, 6};
      for (int t = 0; t < 4 && e == cudaSuccess; ++t) {
        p.ncells = args[1].space->ncells_by_k[t];
        p.cells = args[1].space->d_cells_by_k[t];
        p.kind = kinds[t];
        e = launch_mass_dgp(p, s);
      }
      break;
    }
    case EXT_K_HFACET_MASS:
    case EXT_K_HFACET_JUMP: {
      const bool jump = kernel_id == EXT_K_HFACET_JUMP;
      const char *kn = jump ? "EXT_K_HFACET_JUMP" : "EXT_K_HFACET_MASS";
      if (mesh->kind != EXT_TRI) return ext_fail(EXT_EINVAL, "%s: needs a triangular base mesh", kn);
      if (nargs != 3) return ext_fail(EXT_EINVAL, "%s: expects 3 arguments", kn);
      EXT_CHECK(check_arg(mesh, args, 0, kn, ELEM_P1P1, 3, EXT_READ));
      EXT_CHECK(check_arg(mesh, args, 1, kn, -1, 1, EXT_READ));
      EXT_CHECK(check_arg(mesh, args, 2, kn, -1, 1, EXT_INC));
      if (!same_numbering(args[1].space, args[2].space))
        return ext_fail(EXT_EINVAL, "%s: input and output must share one numbering", kn);
      int h = 0, v = 0;
      if (prism_pair(args[1].space->delta, &h, &v) < 0)
        return ext_fail(EXT_EUNSUPPORTED, "%s: not one of the nine CG1/DG0/DG1 prism spaces", kn);
      if (!jump && v != 0)
        return ext_fail(EXT_EINVAL, "%s: the space has no DoFs on horizontal facets (vertical element must be CG1)", kn);
      FacetLaunch p;
      memset(&p, 0, sizeof(p));
      p.ncells = C;
      p.layers = L;
      p.nh = h == 1 ? 1 : 3;
      p.jump = jump ? 1 : 0;
      const int nv = v == 1 ? 1 : 2;
      p.nv = nv;
      // a vertically continuous space has no jump across horizontal facets;
      // a space discontinuous in both directions keeps every DoF in one cell
      // (the cell-owned form measured faster than facet-centric atomics for
      // DG1xDG1 only: 3.28 vs 4.37 ms at 1M x 100; slower for the others)
      p.mode = !jump ? 0 : (v == 0 ? 2 : (h == 2 && v == 2 ? 1 : 0));
      if (p.mode == 1 && ((((uintptr_t)args[1].data) | ((uintptr_t)args[2].data)) & 15) != 0)
        p.mode = 0;  // the cell-owned form moves DoF pairs with 16-byte accesses
      int32_t slot[6];
      prism_pair_slots(h, v, p.nh, nv, slot);
      for (int a = 0; a < p.nh; ++a) {
        // facet mass: bottom / top slot of node a; jump: the trace from the
        // cell below (its top node, or its only vertical node) and from above
        p.slot_lo[a] = slot[a * nv + (nv == 2 && jump ? 1 : 0)];
        p.slot_hi[a] = slot[a * nv + (nv == 2 && !jump ? 1 : 0)];
        p.off_lo[a] = args[1].space->h_offset[p.slot_lo[a]];
        p.off_hi[a] = args[1].space->h_offset[p.slot_hi[a]];
      }
      p.k = args[1].space->k;
      p.cmap = args[0].space->d_map;
      for (int i = 0; i < 6; ++i) p.coff[i] = args[0].space->h_offset[i];
      p.fmap = args[1].space->d_map;
      p.X = (const double *)args[0].data;
      p.f = (const double *)args[1].data;
      p.b = (double *)args[2].data;
      p.cell_layers = mesh->d_cell_layers;
      p.mean_layers = mesh->mean_layers;
      e = launch_facet(p, s);
      break;
    }
    default:
      return ext_fail(EXT_EINVAL, "ext_par_loop: unknown kernel id %d", kernel_id);
  }
  if (e != cudaSuccess) return ext_fail(EXT_ECUDA, "ext_par_loop: launch failed: %s", cudaGetErrorString(e));
  return EXT_OK;
}

extern "C" ext_status ext_sync_check(void *stream) {
  EXT_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "ext_sync_check");
  unsigned int *w = ext_device_error_word();
  if (!w) return ext_fail(EXT_ECUDA, "ext_sync_check: no device error word");
  unsigned int v = 0;
  EXT_CUDA(cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost), "ext_sync_check");
  if (v) EXT_CUDA(cudaMemset(w, 0, sizeof(v)), "ext_sync_check");
  if (v & EXT_DERR_TIMEOUT) return ext_fail(EXT_ETIMEOUT, "a bounded device-side wait expired (word 0x%x)", v);
  if (v) return ext_fail(EXT_EDEVICE, "device error word 0x%x", v);
  return EXT_OK;
}

// ---------------------------------------------------------------------------
// batched plan

struct BatchPhaseDev {
  void *d_descs = nullptr;
  int64_t nitems = 0;
};

struct ext_batch {
  int nmesh = 0;
  int mode = 0;
  std::vector<const ext_mesh *> meshes;
  std::vector<ext_arg> args;  // nmesh x nargs
  int nargs = 0;
  // colouring: per mesh, cells sorted by colour and the colour offsets
  std::vector<int32_t *> d_cells;
  std::vector<std::vector<int64_t>> colour_off;
  int ncolours = 0;
  unsigned long long *d_counter = nullptr;
  ext_tune_params params{};
  std::vector<BatchPhaseDev> phases;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int sms = 152;
  bool coloured = false;
  int32_t source = 0;        // 0 parameters given, 1 autotuned, 2 from the tuning cache
  double setup_seconds = 0;  // host time of ext_batch_create
};

static void free_phases(std::vector<BatchPhaseDev> &ph) {
  for (auto &p : ph) cudaFree(p.d_descs);
  ph.clear();
}

// Greedy colouring: each cell takes the smallest colour not yet used by a
// cell sharing one of its vertices.
static int colour_cells(const ext_mesh *m, std::vector<int32_t> &order, std::vector<int64_t> &off) {
  const auto &cv = reinterpret_cast<const ext_mesh_host *>(m->host)->cell_verts;
  const int64_t C = m->N[2];
  const int k = m->kind;
  std::vector<uint64_t> used((size_t)m->N[0], 0);
  std::vector<int> col((size_t)C);
  int ncol = 0;
  for (int64_t c = 0; c < C; ++c) {
    uint64_t mask = 0;
    for (int a = 0; a < k; ++a) mask |= used[(size_t)cv[(size_t)(c * k + a)]];
    int q = 0;
    while (q < 64 && (mask >> q) & 1ull) ++q;
    if (q >= 64) return -1;
    col[(size_t)c] = q;
    for (int a = 0; a < k; ++a) used[(size_t)cv[(size_t)(c * k + a)]] |= 1ull << q;
    ncol = std::max(ncol, q + 1);
  }
  off.assign((size_t)ncol + 1, 0);
  for (int64_t c = 0; c < C; ++c) off[(size_t)col[(size_t)c] + 1]++;
  for (int q = 0; q < ncol; ++q) off[(size_t)q + 1] += off[(size_t)q];
  order.assign((size_t)C, 0);
  std::vector<int64_t> pos(off.begin(), off.end() - 1);
  for (int64_t c = 0; c < C; ++c) order[(size_t)pos[(size_t)col[(size_t)c]]++] = (int32_t)c;
  return ncol;
}

static ext_status build_phases(ext_batch *b, const ext_tune_params &tp, std::vector<BatchPhaseDev> &out) {
  out.clear();
  const bool colour = tp.use_atomics == 0;
  const int nph = colour ? b->ncolours : 1;
  const size_t dsz = batch_desc_size();
  std::vector<unsigned char> host((size_t)b->nmesh * dsz);
  for (int ph = 0; ph < nph; ++ph) {
    int64_t item = 0;
    for (int mi = 0; mi < b->nmesh; ++mi) {
      const ext_mesh *m = b->meshes[(size_t)mi];
      const ext_arg *a = &b->args[(size_t)mi * b->nargs];
      int64_t ncells = m->N[2];
      const int32_t *cells = nullptr;
      if (colour) {
        const auto &off = b->colour_off[(size_t)mi];
        const int64_t lo = ph < (int)off.size() - 1 ? off[(size_t)ph] : 0;
        const int64_t hi = ph < (int)off.size() - 1 ? off[(size_t)ph + 1] : 0;
        ncells = hi - lo;
        cells = b->d_cells[(size_t)mi] + lo;
      }
      const int tile = tp.layer_tile > 0 ? std::min(tp.layer_tile, m->layers) : m->layers;
      const int32_t ncol_items = (int32_t)((ncells + tp.cols_per_item - 1) / tp.cols_per_item);
      const int32_t nlay_items = (m->layers + tile - 1) / tile;
      int ai = 2;
      const double *w = (b->mode & 2) ? (const double *)a[ai++].data : nullptr;
      double *F = (b->mode & 1) ? (double *)a[ai++].data : nullptr;
      double *G = (b->mode & 2) ? (double *)a[ai++].data : nullptr;
      batch_fill_desc(host.data(), mi, ncells, item, m->layers, ncol_items, nlay_items, cells, a[0].space->d_map,
                      a[1].space->d_map, a[0].space->h_offset, a[1].space->h_offset, (const double *)a[0].data,
                      (const double *)a[1].data, w, F, G);
      item += (int64_t)ncol_items * nlay_items;
    }
    BatchPhaseDev pd;
    pd.nitems = item;
    cudaError_t e = cudaMalloc(&pd.d_descs, host.size());
    if (e == cudaSuccess) e = cudaMemcpy(pd.d_descs, host.data(), host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(pd.d_descs);
      free_phases(out);
      return ext_fail(EXT_ENOMEM, "ext_batch: descriptor upload failed: %s", cudaGetErrorString(e));
    }
    out.push_back(pd);
  }
  return EXT_OK;
}

static cudaError_t run_phases(ext_batch *b, const std::vector<BatchPhaseDev> &ph, const ext_tune_params &tp,
                              cudaStream_t s) {
  const int grid = std::max(1, tp.ctas_per_sm) * b->sms;
  for (const auto &p : ph) {
    cudaError_t e = launch_batch_phase(p.d_descs, b->nmesh, p.nitems, b->mode, tp.use_atomics == 0, tp.cols_per_item,
                                       tp.layer_tile, b->d_counter, tp.threads, grid, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static ext_status check_params(const ext_tune_params &tp) {
  if (tp.cols_per_item < 1 || tp.cols_per_item > 32) return ext_fail(EXT_EINVAL, "ext_batch: cols_per_item must be 1..32");
  if (tp.layer_tile < 0) return ext_fail(EXT_EINVAL, "ext_batch: layer_tile must be >= 0");
  if (tp.threads != 64 && tp.threads != 128 && tp.threads != 256)
    return ext_fail(EXT_EINVAL, "ext_batch: threads must be 64, 128 or 256");
  if (tp.ctas_per_sm < 1 || tp.ctas_per_sm > 32) return ext_fail(EXT_EINVAL, "ext_batch: ctas_per_sm must be 1..32");
  return EXT_OK;
}

static void destroy_batch(ext_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  free_phases(b->phases);
  for (auto p : b->d_cells) cudaFree(p);
  cudaFree(b->d_counter);
  delete b;
}

// Colour classes of every mesh of the batch (the colour form's phases), built
// on first use.
static ext_status ensure_colours(ext_batch *b) {
  if (b->coloured) return EXT_OK;
  b->d_cells.assign((size_t)b->nmesh, nullptr);
  b->colour_off.resize((size_t)b->nmesh);
  for (int mi = 0; mi < b->nmesh; ++mi) {
    std::vector<int32_t> order;
    const int nc = colour_cells(b->meshes[(size_t)mi], order, b->colour_off[(size_t)mi]);
    if (nc < 0) return ext_fail(EXT_EUNSUPPORTED, "batched launch: mesh %d needs more than 64 colours", mi);
    b->ncolours = std::max(b->ncolours, nc);
    if (!order.empty()) {
      cudaError_t e = cudaMalloc(&b->d_cells[(size_t)mi], order.size() * sizeof(int32_t));
      if (e == cudaSuccess)
        e = cudaMemcpy(b->d_cells[(size_t)mi], order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return ext_fail(EXT_ENOMEM, "batched launch: %s", cudaGetErrorString(e));
    }
  }
  b->coloured = true;
  return EXT_OK;
}

// ---------------------------------------------------------------------------
// Tuning cache of the batched launch.  Key: GPU name and SM count, kernel
// (forward, adjoint or both), and power-of-two buckets of the prism count,
// the mean layer count and the mesh count; value: the autotuned parameters
// and their time.  Kept in memory for the process and, unless EXTMESH_TUNE=off,
// in a file of JSON lines (EXTMESH_TUNE_CACHE, else
// $XDG_CACHE_HOME/extmesh/batch_tune.jsonl or $HOME/.cache/extmesh/...),
// rewritten through a temporary file and a rename.  EXTMESH_TUNE=force times
// the candidates again and replaces the entry.
static std::mutex g_tune_mu;
static std::map<std::string, ext_tune_params> g_tune_mem;

static int tune_env() {
  const char *ev = getenv("EXTMESH_TUNE");
  if (ev && strcmp(ev, "force") == 0) return 1;
  if (ev && strcmp(ev, "off") == 0) return 2;
  return 0;
}

static std::string tune_path() {
  const char *ev = getenv("EXTMESH_TUNE_CACHE");
  if (ev && ev[0]) return ev;
  const char *xdg = getenv("XDG_CACHE_HOME");
  if (xdg && xdg[0]) return std::string(xdg) + "/extmesh/batch_tune.jsonl";
  const char *home = getenv("HOME");
  if (home && home[0]) return std::string(home) + "/.cache/extmesh/batch_tune.jsonl";
  return std::string();
}

static int log2_bucket(double x) { return x < 1.0 ? 0 : (int)std::floor(std::log2(x)); }

static std::string tune_key(const ext_batch *b) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  std::string name = "unknown";
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
  for (char &c : name)
    if (c == '"' || c == '\\' || c == '|') c = '_';
  double prisms = 0.0, layers = 0.0;
  for (const ext_mesh *m : b->meshes) {
    prisms += (double)m->N[2] * (double)m->layers;
    layers += (double)m->layers;
  }
  char buf[512];
  snprintf(buf, sizeof buf, "%s|sm%d|mode%d|prisms2^%d|layers2^%d|meshes2^%d", name.c_str(), b->sms, b->mode,
           log2_bucket(prisms), log2_bucket(layers / (double)b->nmesh), log2_bucket((double)b->nmesh));
  return buf;
}

// one line: {"key": "...", "params": [cols_per_item, layer_tile, use_atomics, threads, ctas_per_sm], "ms": t}
static bool tune_parse(const std::string &line, std::string &key, ext_tune_params &tp) {
  const size_t k0 = line.find("\"key\": \"");
  if (k0 == std::string::npos) return false;
  const size_t ks = k0 + 8, ke = line.find('"', ks);
  if (ke == std::string::npos) return false;
  key = line.substr(ks, ke - ks);
  const size_t p0 = line.find("\"params\": [", ke);
  if (p0 == std::string::npos) return false;
  int v[5];
  if (sscanf(line.c_str() + p0 + 11, "%d, %d, %d, %d, %d", &v[0], &v[1], &v[2], &v[3], &v[4]) != 5) return false;
  tp.cols_per_item = v[0];
  tp.layer_tile = v[1];
  tp.use_atomics = v[2];
  tp.threads = v[3];
  tp.ctas_per_sm = v[4];
  return true;
}

static bool tune_lookup(const std::string &key, ext_tune_params &out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune_mem.find(key);
  if (it != g_tune_mem.end()) {
    out = it->second;
    return true;
  }
  const std::string path = tune_path();
  if (path.empty()) return false;
  FILE *f = fopen(path.c_str(), "r");
  if (!f) return false;
  bool found = false;
  char buf[1024];
  while (fgets(buf, sizeof buf, f)) {
    std::string k;
    ext_tune_params tp;
    if (tune_parse(buf, k, tp) && check_params(tp) == EXT_OK) {
      g_tune_mem[k] = tp;
      if (k == key) {
        out = tp;
        found = true;
      }
    }
  }
  fclose(f);
  (void)cudaGetLastError();
  return found;
}

static void tune_store(const std::string &key, const ext_tune_params &tp, float ms) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_mem[key] = tp;
  const std::string path = tune_path();
  if (path.empty()) return;
  // keep the other entries of the file, replace this key's
  std::vector<std::string> keep;
  if (FILE *f = fopen(path.c_str(), "r")) {
    char buf[1024];
    while (fgets(buf, sizeof buf, f)) {
      std::string k;
      ext_tune_params t;
      if (tune_parse(buf, k, t) && k != key) keep.push_back(buf);
    }
    fclose(f);
  }
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos) {  // create the directory chain
    for (size_t q = 1; q <= slash; ++q)
      if (path[q] == '/' || q == slash) mkdir(path.substr(0, q == slash ? slash : q).c_str(), 0755);
  }
  const std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
  FILE *f = fopen(tmp.c_str(), "w");
  if (!f) return;
  for (const auto &l : keep) fputs(l.c_str(), f);
  fprintf(f, "{\"key\": \"%s\", \"params\": [%d, %d, %d, %d, %d], \"ms\": %.4f}\n", key.c_str(), tp.cols_per_item,
          tp.layer_tile, tp.use_atomics, tp.threads, tp.ctas_per_sm, (double)ms);
  const bool ok = fclose(f) == 0;
  if (ok) rename(tmp.c_str(), path.c_str());
  else remove(tmp.c_str());
}

static ext_status capture(ext_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  cudaStream_t cs;
  EXT_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "ext_batch: capture stream");
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e2 = run_phases(b, b->phases, b->params, cs);
    e = cudaStreamEndCapture(cs, &b->graph);
    if (e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return ext_fail(EXT_ECUDA, "ext_batch: graph capture failed: %s", cudaGetErrorString(e));
  return EXT_OK;
}

extern "C" ext_status ext_batch_create(int32_t nmesh, const ext_mesh *const *meshes, int32_t kernel_id, int32_t nargs,
                                       const ext_arg *args, const ext_tune_params *params, void *stream,
                                       ext_batch **out) {
  const auto t_start = std::chrono::steady_clock::now();
  if (!out) return ext_fail(EXT_EINVAL, "ext_batch_create: out is NULL");
  *out = nullptr;
  // the same checks as every batched launch: kernel, argument lists,
  // current device, no written argument overlapping another
  int mode = 0;
  EXT_CHECK(ext_batch_validate(nmesh, meshes, kernel_id, nargs, args, &mode));
  if (params) EXT_CHECK(check_params(*params));
  ext_batch *b = new ext_batch();
  b->nmesh = nmesh;
  b->mode = mode;
  b->nargs = nargs;
  b->meshes.assign(meshes, meshes + nmesh);
  b->args.assign(args, args + (size_t)nmesh * nargs);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaMalloc(&b->d_counter, sizeof(unsigned long long));
  if (e != cudaSuccess) {
    destroy_batch(b);
    return ext_fail(EXT_ENOMEM, "ext_batch_create: %s", cudaGetErrorString(e));
  }
  cudaStream_t s = (cudaStream_t)stream;
  const std::string key = tune_key(b);
  const int tune_mode = tune_env();  // 0 use the cache, 1 re-tune and store, 2 no cache
  ext_tune_params cached;
  if (params) {
    b->params = *params;
  } else if (tune_mode == 0 && tune_lookup(key, cached)) {
    b->params = cached;
    b->source = 2;
  } else {
    b->source = 1;
    const ext_status cs = ensure_colours(b);
    if (cs != EXT_OK) {
      destroy_batch(b);
      return cs;
    }
    // autotune: time each candidate once after one warm-up launch
    std::vector<ext_tune_params> cand;
    const int cpis[] = {1, 2, 4, 8};
    const int tiles[] = {0, 32};
    for (int use_atomics = 1; use_atomics >= 0; --use_atomics)
      for (int cpi : cpis)
        for (int t : tiles) {
          if (!use_atomics && cpi < 8) continue;  // colour phases need many columns per item
          ext_tune_params tp;
          tp.cols_per_item = use_atomics ? cpi : 32;
          tp.layer_tile = t;
          tp.use_atomics = use_atomics;
          tp.threads = 256;
          tp.ctas_per_sm = 4;
          cand.push_back(tp);
        }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (const auto &tp : cand) {
      std::vector<BatchPhaseDev> ph;
      if (build_phases(b, tp, ph) != EXT_OK) continue;
      cudaError_t le = run_phases(b, ph, tp, s);
      le = le == cudaSuccess ? cudaEventRecord(e0, s) : le;
      le = le == cudaSuccess ? run_phases(b, ph, tp, s) : le;
      le = le == cudaSuccess ? cudaEventRecord(e1, s) : le;
      le = le == cudaSuccess ? cudaEventSynchronize(e1) : le;
      float ms = 1e30f;
      if (le == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
      free_phases(ph);
      if (le != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        destroy_batch(b);
        return ext_fail(EXT_ECUDA, "ext_batch_create: autotune launch failed: %s", cudaGetErrorString(le));
      }
      if (ms < best) {
        best = ms;
        b->params = tp;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (tune_mode != 2) tune_store(key, b->params, best);
  }
  ext_status st = b->params.use_atomics ? EXT_OK : ensure_colours(b);
  if (st == EXT_OK) st = build_phases(b, b->params, b->phases);
  if (st == EXT_OK) st = capture(b);
  if (st != EXT_OK) {
    destroy_batch(b);
    return st;
  }
  b->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  *out = b;
  return EXT_OK;
}

extern "C" ext_status ext_batch_plan_info(const ext_batch *batch, int32_t *source, double *setup_seconds) {
  if (!batch) return ext_fail(EXT_EINVAL, "ext_batch_plan_info: batch is NULL");
  if (source) *source = batch->source;
  if (setup_seconds) *setup_seconds = batch->setup_seconds;
  return EXT_OK;
}

extern "C" ext_status ext_batch_launch(ext_batch *batch, void *stream) {
  if (!batch || !batch->exec) return ext_fail(EXT_EINVAL, "ext_batch_launch: invalid batch");
  EXT_CUDA(cudaGraphLaunch(batch->exec, (cudaStream_t)stream), "ext_batch_launch");
  return EXT_OK;
}

extern "C" ext_status ext_batch_launch_params(ext_batch *batch, const ext_tune_params *params, void *stream) {
  if (!batch || !params) return ext_fail(EXT_EINVAL, "ext_batch_launch_params: invalid arguments");
  EXT_CHECK(check_params(*params));
  if (!params->use_atomics) EXT_CHECK(ensure_colours(batch));
  std::vector<BatchPhaseDev> ph;
  EXT_CHECK(build_phases(batch, *params, ph));
  cudaError_t e = run_phases(batch, ph, *params, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  free_phases(ph);
  if (e != cudaSuccess) return ext_fail(EXT_ECUDA, "ext_batch_launch_params: %s", cudaGetErrorString(e));
  return EXT_OK;
}

extern "C" ext_status ext_batch_params(const ext_batch *batch, ext_tune_params *out) {
  if (!batch || !out) return ext_fail(EXT_EINVAL, "ext_batch_params: invalid arguments");
  *out = batch->params;
  return EXT_OK;
}

extern "C" void ext_batch_destroy(ext_batch *batch) { destroy_batch(batch); }

// Argument checks of a batched u^2 v launch (the same rules as
// ext_batch_create), for the entry point that runs without allocating.
ext_status ext_batch_validate(int32_t nmesh, const ext_mesh *const *meshes, int32_t kernel_id, int32_t nargs,
                              const ext_arg *args, int *mode_out) {
  if (nmesh < 1 || !meshes || !args) return ext_fail(EXT_EINVAL, "batched launch: no meshes");
  int mode;
  if (kernel_id == EXT_K_U2V_FWD) mode = 1;
  else if (kernel_id == EXT_K_U2V_ADJ) mode = 2;
  else if (kernel_id == EXT_K_U2V_FWDADJ) mode = 3;
  else return ext_fail(EXT_EUNSUPPORTED, "batched launch: kernel %d is not batched", kernel_id);
  const int want = mode == 1 ? 3 : (mode == 2 ? 4 : 5);
  if (nargs != want) return ext_fail(EXT_EINVAL, "batched launch: expects %d arguments per mesh", want);
  int cur = 0;
  const cudaError_t ed = cudaGetDevice(&cur);
  if (ed != cudaSuccess) return ext_fail(EXT_ECUDA, "batched launch: %s", cudaGetErrorString(ed));
  for (int mi = 0; mi < nmesh; ++mi) {
    const ext_mesh *m = meshes[mi];
    const ext_arg *a = args + (size_t)mi * nargs;
    if (!m || m->kind != EXT_TRI) return ext_fail(EXT_EUNSUPPORTED, "batched launch: mesh %d: prisms only", mi);
    if (m->var) return ext_fail(EXT_EUNSUPPORTED, "batched launch: mesh %d has variable layers", mi);
    if (m->device != cur)
      return ext_fail(EXT_EINVAL, "batched launch: mesh %d lives on device %d, the current device is %d", mi,
                      m->device, cur);
    EXT_CHECK(check_no_overlap(nargs, a, "batched launch"));
    EXT_CHECK(check_arg(m, a, 0, "batched launch", ELEM_P1P1, 3, EXT_READ));
    for (int j = 1; j < nargs; ++j) {
      const bool is_out = (mode == 1 && j == 2) || (mode == 2 && j == 3) || (mode == 3 && j >= 3);
      EXT_CHECK(check_arg(m, a, j, "batched launch", ELEM_P1P1, 1, is_out ? EXT_INC : EXT_READ));
    }
  }
  *mode_out = mode;
  return EXT_OK;
}

// Stencil map, offsets and layer count of a space/mesh for code outside this
// file (the entry point that runs without allocating builds its descriptors
// from them).
const int32_t *ext_space_map_dev(const ext_space *s) { return s->d_map; }
const int32_t *ext_space_offsets_host(const ext_space *s) { return s->h_offset; }
int64_t ext_mesh_ncells(const ext_mesh *m) { return m->N[2]; }
int32_t ext_mesh_layers(const ext_mesh *m) { return m->layers; }
