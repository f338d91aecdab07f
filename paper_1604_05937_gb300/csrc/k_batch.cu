// Batched persistent par_loop: the u^2 v residual and/or its adjoint over
// many extruded prism meshes with different base sizes and layer counts in a
// single launch.  Work items are (mesh, run of base columns, range of layers)
// tiles, numbered mesh by mesh; each warp of a persistent grid takes the next
// item index from a device counter (atomicAdd, no waiting), so load balance
// does not depend on the meshes' sizes.  Two increment strategies:
//   - atomics: lanes run along the layers of the tile's columns and every
//     local contribution is an FP64 atomic add executed in L2;
//   - colours: cells of one colour share no vertex, so a colour's tiles can
//     add without atomics; one lane walks one column's layer range, merging
//     the top of layer l with the bottom of layer l+1 in registers, and only
//     the two boundary levels of a layer tile (shared with the neighbouring
//     tiles of the same column) use atomics.  Colours run as separate
//     launches in stream order.
#include "ext_internal.cuh"
#include "prism_u2v.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct BatchDesc {
  int64_t ncells;        // cells of this mesh in this phase
  int64_t item_begin;    // first global work item of this mesh
  int32_t layers;
  int32_t ncol_items;    // column runs
  int32_t nlay_items;    // layer ranges per column run
  int32_t pad;
  const int32_t *cells;  // cell ids of this phase (colour) or null = 0..ncells-1
  const int32_t *cmap, *umap;
  int32_t coff[6], uoff[6];
  const double *X, *u, *w;
  double *F, *G;
};

__device__ __forceinline__ int find_mesh(const BatchDesc *d, int nmesh, int64_t it) {
  int lo = 0, hi = nmesh - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (d[mid].item_begin <= it) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int MODE, bool COLOUR>
__global__ void __launch_bounds__(256) k_batch(const BatchDesc *descs, int nmesh, int64_t nitems, int cpi, int lt,
                        unsigned long long *counter, Fp64Ones k1) {
  __shared__ prism_u2v::ColGeom geo[8][32];  // per warp (<= 8 warps), per column of the tile
  __shared__ int64_t cid[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(counter, 1ull);
    it = __shfl_sync(kFull, it, 0);
    if ((int64_t)it >= nitems) break;
    const int mi = find_mesh(descs, nmesh, (int64_t)it);
    const BatchDesc &d = descs[mi];
    const int64_t local = (int64_t)it - d.item_begin;
    const int64_t ci = local / d.nlay_items;
    const int li = (int)(local - ci * d.nlay_items);
    const int64_t cbeg = ci * cpi;
    const int ncol = (int)(d.ncells - cbeg < cpi ? d.ncells - cbeg : (int64_t)cpi);
    const int layers = d.layers;
    const int tile = lt > 0 ? lt : layers;
    const int l0 = li * tile;
    const int nl = min(tile, layers - l0);

    if (lane < ncol) {
      const int64_t c = d.cells ? (int64_t)d.cells[cbeg + lane] : cbeg + lane;
      cid[warp][lane] = c;
      double x[3], y[3];
      for (int a = 0; a < 3; ++a) {
        const int64_t cd = __ldg(d.cmap + c * 6 + 2 * a);
        x[a] = __ldg(d.X + 3 * cd + 0);
        y[a] = __ldg(d.X + 3 * cd + 1);
      }
      prism_u2v::col_geom(x, y, geo[warp][lane]);
    }
    __syncwarp();

    if (!COLOUR) {
      const int n = ncol * nl;
      int cl = lane / nl, l = lane - (lane / nl) * nl;
      for (int base = 0; base < n; base += 32) {
        if (base + lane < n) {
          const int64_t c = cid[warp][cl];
          int32_t crow[6], urow[6];
          for (int i = 0; i < 6; ++i) {
            crow[i] = __ldg(d.cmap + c * 6 + i);
            urow[i] = __ldg(d.umap + c * 6 + i);
          }
          prism_u2v::cell_layer<MODE>(crow, urow, d.coff, d.uoff, l0 + l, geo[warp][cl], d.X, d.u, d.w,
                                      d.F, d.G, k1);
        }
        l += 32;
        while (l >= nl) { l -= nl; ++cl; }
      }
    } else if (lane < ncol) {
      // one lane per column of this colour: layers in order, level sums in registers
      const int64_t c = cid[warp][lane];
      int32_t crow[6], urow[6];
      for (int i = 0; i < 6; ++i) {
        crow[i] = __ldg(d.cmap + c * 6 + i);
        urow[i] = __ldg(d.umap + c * 6 + i);
      }
      double carryF[3] = {0.0, 0.0, 0.0}, carryG[3] = {0.0, 0.0, 0.0};
      for (int j = 0; j < nl; ++j) {
        const int l = l0 + j;
        double uu[6], ww[6], Xl[6][3];
        int32_t ud[6];
        int ok = 1;
        const prism_u2v::ColGeom &cg = geo[warp][lane];
        for (int i = 0; i < 6; ++i) {
          const int64_t cd = (int64_t)crow[i] + (int64_t)l * d.coff[i];
          Xl[i][0] = __ldg(d.X + 3 * cd + 0);
          Xl[i][1] = __ldg(d.X + 3 * cd + 1);
          Xl[i][2] = __ldg(d.X + 3 * cd + 2);
          ok &= (__double_as_longlong(Xl[i][0]) == cg.rx[i >> 1]) &
                (__double_as_longlong(Xl[i][1]) == cg.ry[i >> 1]);
          ud[i] = urow[i] + l * d.uoff[i];
          uu[i] = __ldg(d.u + ud[i]);
          if (MODE & 2) ww[i] = __ldg(d.w + ud[i]);
        }
        ok &= (__double_as_longlong(Xl[0][2]) == __double_as_longlong(Xl[2][2])) &
              (__double_as_longlong(Xl[0][2]) == __double_as_longlong(Xl[4][2])) &
              (__double_as_longlong(Xl[1][2]) == __double_as_longlong(Xl[3][2])) &
              (__double_as_longlong(Xl[1][2]) == __double_as_longlong(Xl[5][2]));
        double Fo[6], Go[6];
        if (ok) {
          prism_u2v::local_straight<MODE>(uu, ww, fmul(cg.wdet, fabs(fsub(Xl[1][2], Xl[0][2], k1)), k1), Fo, Go,
                                          k1);
        } else {
          double W[6];
          prism_u2v::general_weights(Xl, W);
          prism_u2v::local<MODE>(uu, ww, W, Fo, Go, k1);
        }
        for (int a = 0; a < 3; ++a) {
          const int ib = 2 * a, itp = 2 * a + 1;
          // bottom level of layer l: merged with the carry from layer l-1
          if (MODE & 1) {
            const double v = j == 0 ? Fo[ib] : Fo[ib] + carryF[a];
            if (j == 0) atomicAdd(d.F + ud[ib], v);
            else d.F[ud[ib]] += v;
            carryF[a] = Fo[itp];
          }
          if (MODE & 2) {
            const double v = j == 0 ? Go[ib] : Go[ib] + carryG[a];
            if (j == 0) atomicAdd(d.G + ud[ib], v);
            else d.G[ud[ib]] += v;
            carryG[a] = Go[itp];
          }
          if (j == nl - 1) {  // top level of the tile: shared with the next tile
            if (MODE & 1) atomicAdd(d.F + ud[itp], carryF[a]);
            if (MODE & 2) atomicAdd(d.G + ud[itp], carryG[a]);
          }
        }
      }
    }
    __syncwarp();
  }
}

}  // namespace

size_t batch_desc_size() { return sizeof(BatchDesc); }

// Fills the descriptor of mesh `mi` for one phase (host memory).
void batch_fill_desc(void *host_descs, int mi, int64_t ncells, int64_t item_begin, int32_t layers,
                     int32_t ncol_items, int32_t nlay_items, const int32_t *cells, const int32_t *cmap,
                     const int32_t *umap, const int32_t coff[6], const int32_t uoff[6], const double *X,
                     const double *u, const double *w, double *F, double *G) {
  BatchDesc &d = reinterpret_cast<BatchDesc *>(host_descs)[mi];
  d.ncells = ncells;
  d.item_begin = item_begin;
  d.layers = layers;
  d.ncol_items = ncol_items;
  d.nlay_items = nlay_items;
  d.pad = 0;
  d.cells = cells;
  d.cmap = cmap;
  d.umap = umap;
  for (int i = 0; i < 6; ++i) {
    d.coff[i] = coff[i];
    d.uoff[i] = uoff[i];
  }
  d.X = X;
  d.u = u;
  d.w = w;
  d.F = F;
  d.G = G;
}

cudaError_t launch_batch_phase(const void *d_descs, int nmesh, int64_t nitems, int mode, bool colour,
                               int cpi, int lt, unsigned long long *counter, int threads, int grid,
                               cudaStream_t s) {
  if (nitems == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const BatchDesc *dd = reinterpret_cast<const BatchDesc *>(d_descs);
#define EXT_LAUNCH_BATCH(M, C) k_batch<M, C><<<grid, threads, 0, s>>>(dd, nmesh, nitems, cpi, lt, counter, fp64_ones())
  if (colour) {
    if (mode == 1) EXT_LAUNCH_BATCH(1, true);
    else if (mode == 2) EXT_LAUNCH_BATCH(2, true);
    else EXT_LAUNCH_BATCH(3, true);
  } else {
    if (mode == 1) EXT_LAUNCH_BATCH(1, false);
    else if (mode == 2) EXT_LAUNCH_BATCH(2, false);
    else EXT_LAUNCH_BATCH(3, false);
  }
#undef EXT_LAUNCH_BATCH
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched launch that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs under a device-memory
// budget owned by someone else (a framework's caching allocator that has
// reserved the device, or a service that forbids allocation once it has
// started), and latency-sensitive loops that cannot afford the implicit
// device synchronisation of cudaMalloc/cudaFree.  ext_batch_run_noalloc serves
// them: it runs the same persistent work-queue kernel as a batch plan, in its
// FP64-atomic form, but keeps the kernel's scratch memory -- the work counter
// and the per-mesh descriptor table -- in the file-scope array below instead
// of allocating it.  The array is part of the module image: every GPU that
// loads this library holds its 64 KiB until the process exits.  All calls on
// a device share it and it keeps the last call's contents; calls whose
// launches overlap on the GPU race on it, so issue them in one stream or
// otherwise order them.

#include <cstring>
#include <mutex>

#define EXT_NOALLOC_COUNTER_BYTES 256
static __device__ __align__(256) unsigned char g_noalloc_scratch[EXT_NOALLOC_SCRATCH_BYTES];

static_assert(EXT_NOALLOC_COUNTER_BYTES + EXT_NOALLOC_MAX_MESHES * sizeof(BatchDesc) <= EXT_NOALLOC_SCRATCH_BYTES,
              "scratch array too small for the descriptor table");

// The descriptors reach the array as kernel parameters, kNoallocChunk per
// launch of k_noalloc_stage: no host buffer is read after the entry point
// returns, and the host never waits for the stream.
constexpr int kNoallocChunk = 16;
struct NoallocChunk {
  BatchDesc d[kNoallocChunk];
};

__global__ void k_noalloc_stage(const NoallocChunk chunk, BatchDesc *__restrict__ dst, int count) {
  const int i = threadIdx.x;
  if (i < count) dst[i] = chunk.d[i];
}

static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_dev[128];  // device address of the array, per device

// Device address of the scratch array on the current device.  The host-side
// name g_noalloc_scratch is only a stand-in; the address is looked up once
// per device, with that device current, on the first call.
static ext_status noalloc_scratch(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ext_fail(EXT_ECUDA, "ext_batch_run_noalloc: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= 128) return ext_fail(EXT_EUNSUPPORTED, "ext_batch_run_noalloc: device %d", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_dev[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return ext_fail(EXT_ECUDA, "ext_batch_run_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_noalloc_dev[dev] = reinterpret_cast<unsigned char *>(p);
  }
  *out = g_noalloc_dev[dev];
  return EXT_OK;
}

extern "C" ext_status ext_batch_run_noalloc(int32_t nmesh, const ext_mesh *const *meshes, int32_t kernel_id,
                                            int32_t nargs, const ext_arg *args, const ext_tune_params *params,
                                            void *stream) {
  int mode = 0;
  ext_status st = ext_batch_validate(nmesh, meshes, kernel_id, nargs, args, &mode);
  if (st != EXT_OK) return st;
  if (nmesh > EXT_NOALLOC_MAX_MESHES)
    return ext_fail(EXT_EINVAL, "ext_batch_run_noalloc: %d meshes exceed the limit of %d", nmesh,
                    EXT_NOALLOC_MAX_MESHES);
  ext_tune_params tp;
  if (params) {
    tp = *params;
  } else {
    tp.cols_per_item = 4;
    tp.layer_tile = 0;
    tp.use_atomics = 1;
    tp.threads = 256;
    tp.ctas_per_sm = 4;
  }
  if (tp.use_atomics != 1)
    return ext_fail(EXT_EUNSUPPORTED, "ext_batch_run_noalloc: only the FP64-atomic form runs without allocating");
  if (tp.cols_per_item < 1 || tp.cols_per_item > 32 || tp.layer_tile < 0 ||
      (tp.threads != 64 && tp.threads != 128 && tp.threads != 256) || tp.ctas_per_sm < 1 || tp.ctas_per_sm > 32)
    return ext_fail(EXT_EINVAL, "ext_batch_run_noalloc: invalid launch parameters");
  unsigned char *scratch = nullptr;
  st = noalloc_scratch(&scratch);
  if (st != EXT_OK) return st;

  // descriptors built on the host, then written into the array by
  // k_noalloc_stage, kNoallocChunk at a time, as kernel parameters
  BatchDesc stage[EXT_NOALLOC_MAX_MESHES];
  int64_t item = 0;
  for (int mi = 0; mi < nmesh; ++mi) {
    const ext_arg *a = args + (size_t)mi * nargs;
    const int64_t ncells = ext_mesh_ncells(meshes[mi]);
    const int32_t layers = ext_mesh_layers(meshes[mi]);
    const int tile = tp.layer_tile > 0 ? (tp.layer_tile < layers ? tp.layer_tile : layers) : layers;
    const int32_t ncol_items = (int32_t)((ncells + tp.cols_per_item - 1) / tp.cols_per_item);
    const int32_t nlay_items = (layers + tile - 1) / tile;
    int ai = 2;
    const double *w = (mode & 2) ? (const double *)a[ai++].data : nullptr;
    double *F = (mode & 1) ? (double *)a[ai++].data : nullptr;
    double *G = (mode & 2) ? (double *)a[ai++].data : nullptr;
    batch_fill_desc(stage, mi, ncells, item, layers, ncol_items, nlay_items, nullptr, ext_space_map_dev(a[0].space),
                    ext_space_map_dev(a[1].space), ext_space_offsets_host(a[0].space),
                    ext_space_offsets_host(a[1].space), (const double *)a[0].data, (const double *)a[1].data, w, F,
                    G);
    item += (int64_t)ncol_items * nlay_items;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  BatchDesc *table = reinterpret_cast<BatchDesc *>(scratch + EXT_NOALLOC_COUNTER_BYTES);
  for (int first = 0; first < nmesh && e == cudaSuccess; first += kNoallocChunk) {
    NoallocChunk chunk;
    const int count = nmesh - first < kNoallocChunk ? nmesh - first : kNoallocChunk;
    memcpy(chunk.d, stage + first, sizeof(BatchDesc) * (size_t)count);
    k_noalloc_stage<<<1, kNoallocChunk, 0, s>>>(chunk, table + first, count);
    e = cudaGetLastError();
  }
  int dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // launch_batch_phase zeroes the counter before the launch
  if (e == cudaSuccess)
    e = launch_batch_phase(scratch + EXT_NOALLOC_COUNTER_BYTES, nmesh, item, mode, false, tp.cols_per_item,
                           tp.layer_tile, reinterpret_cast<unsigned long long *>(scratch), tp.threads,
                           tp.ctas_per_sm * sms, s);
  if (e != cudaSuccess) return ext_fail(EXT_ECUDA, "ext_batch_run_noalloc: %s", cudaGetErrorString(e));
  return EXT_OK;
}
