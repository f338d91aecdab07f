// Streaming par_loops over spaces with cell-interior DoFs only: the DG copy
// and the P1xP1 -> DG1xDG1 nodal interpolation.  Neither does floating-point
// arithmetic; both are bound by HBM bandwidth.
//
// For a space whose DoFs all sit on the cells (delta(2,1) = k, every other
// delta 0), Algorithm 1 gives cell c's column the k*layers consecutive
// numbers starting at base_map[c][0], and base_map[c][j] = base_map[c][0] + j
// with offset k, so Algorithm 3's direct addressing base_map[c][j] + l*k
// walks that range in order (t = l*k + j).  The kernels flatten (cell, layer,
// stencil slot) into one index so that consecutive threads touch consecutive
// DoFs and move 16 bytes each.
#include "ext_internal.cuh"
#include "fastdiv.cuh"

namespace {

constexpr int kThreads = 256;
#ifndef EXT_DG_UNROLL
#define EXT_DG_UNROLL 4  // 16-byte moves in flight per thread (copy, flat interpolation)
#endif
constexpr int kUnroll = EXT_DG_UNROLL;
#ifndef EXT_INTERP_TILE
#define EXT_INTERP_TILE 128  // base columns per CTA tile (0: flat grid-stride kernel)
#endif
#ifndef EXT_INTERP_UNROLL
#define EXT_INTERP_UNROLL 8  // pairs in flight per thread in the tiled interpolation
#endif

__device__ __forceinline__ double2 ld_stream2(const double *p) {
  return __ldcs(reinterpret_cast<const double2 *>(p));
}
__device__ __forceinline__ void st_stream2(double *p, double2 v) {
  __stcs(reinterpret_cast<double2 *>(p), v);
}

// out = in over the columns of a cell-interior space.  `pairs` 16-byte pairs
// when the column length is even, single values otherwise.
__global__ void __launch_bounds__(kThreads) k_copy_dg_vec(const CopyDGLaunch p, FastDiv col,
                                                          uint32_t npairs) {
  const uint32_t stride = gridDim.x * kThreads;
  uint32_t v = blockIdx.x * kThreads + threadIdx.x;
  for (; v < npairs; v += kUnroll * stride) {
    double2 val[kUnroll];
    uint32_t dst[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t vv = v + u * stride;
      if (vv < npairs) {
        const uint32_t t = 2u * vv;
        const uint32_t c = fdiv(t, col);
        const uint32_t r = t - c * col.d;
        const uint32_t base = (uint32_t)__ldg(p.map + (int64_t)c * p.k);
        dst[u] = base + r;
        val[u] = ld_stream2(p.in + dst[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t vv = v + u * stride;
      if (vv < npairs) st_stream2(p.out + dst[u], val[u]);
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_copy_dg_scalar(const CopyDGLaunch p, FastDiv col,
                                                             uint32_t n) {
  const uint32_t stride = gridDim.x * kThreads;
  for (uint32_t t = blockIdx.x * kThreads + threadIdx.x; t < n; t += stride) {
    const uint32_t c = fdiv(t, col);
    const uint32_t r = t - c * col.d;
    const uint32_t base = (uint32_t)__ldg(p.map + (int64_t)c * p.k);
    __stcs(p.out + base + r, __ldcs(p.in + base + r));
  }
}

#if EXT_INTERP_TILE == 0
// out(DG1xDG1 node 2a+b of cell c, layer l) = x(vertex a, level l+b).  Pair
// index v covers slots (2a, 2a+1) of one layer: t = 2v = c*6L + 6l + 2a.  The
// P1xP1 DoFs are x_map[c][2a] + l*offset (bottom) and x_map[c][2a+1] +
// l*offset (top), reached by direct addressing as in Algorithm 3 (every slot
// of a CG1xCG1 stencil has the same offset, delta(0,0) = 1).
__global__ void __launch_bounds__(kThreads) k_interp_dg1(const InterpDG1Launch p, FastDiv col,
                                                         FastDiv six, uint32_t npairs) {
  const uint32_t stride = gridDim.x * kThreads;
  uint32_t v = blockIdx.x * kThreads + threadIdx.x;
  for (; v < npairs; v += kUnroll * stride) {
    double2 val[kUnroll];
    uint32_t dst[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t vv = v + u * stride;
      if (vv < npairs) {
        const uint32_t t = 2u * vv;
        const uint32_t c = fdiv(t, col);
        const uint32_t r = t - c * col.d;
        const uint32_t l = fdiv(r, six);
        const uint32_t j = r - 6u * l;  // 0, 2 or 4
        const int32_t *xm = p.xmap + (int64_t)c * 6;
        const int2 xb = __ldg(reinterpret_cast<const int2 *>(xm + j));
        const int ob = __ldg(p.omap + (int64_t)c * 6);
        const double lo = __ldg(p.x + (uint32_t)xb.x + l * (uint32_t)p.xoff);
        const double hi = __ldg(p.x + (uint32_t)xb.y + l * (uint32_t)p.xoff);
        val[u] = make_double2(lo, hi);
        dst[u] = (uint32_t)ob + r;
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t vv = v + u * stride;
      if (vv < npairs) st_stream2(p.out + dst[u], val[u]);
    }
  }
}
#endif

// Tiled form of k_interp_dg1: a CTA takes EXT_INTERP_TILE consecutive base
// columns, stages their two stencil rows in shared memory once, then streams
// the tile's pairs with the same flattened order; the x loads no longer wait
// on a map load.
template <int TILE, int UNROLL>
__global__ void __launch_bounds__(kThreads) k_interp_dg1_tile(const InterpDG1Launch p, FastDiv three,
                                                              int64_t ntiles) {
  __shared__ int32_t xrow[TILE][6];
  __shared__ int32_t obase[TILE];
  const uint32_t npl = 3u * (uint32_t)p.layers;  // pairs per column
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t c0 = tile * TILE;
    const int ncol = (int)(p.ncells - c0 < TILE ? p.ncells - c0 : TILE);
    __syncthreads();
    for (int i = threadIdx.x; i < ncol * 6; i += kThreads) xrow[i / 6][i % 6] = __ldg(p.xmap + c0 * 6 + i);
    for (int i = threadIdx.x; i < ncol; i += kThreads) obase[i] = __ldg(p.omap + (c0 + i) * 6);
    __syncthreads();
    const uint32_t npairs = npl * (uint32_t)ncol;
    for (uint32_t v = threadIdx.x; v < npairs; v += UNROLL * kThreads) {
      double2 val[UNROLL];
      uint32_t dst[UNROLL];
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const uint32_t vv = v + u * kThreads;
        if (vv < npairs) {
          const uint32_t cl = vv / npl;            // column within the tile
          const uint32_t q = vv - cl * npl;        // pair within the column: 3 l + a
          const uint32_t l = fdiv(q, three);
          const uint32_t a = q - 3u * l;
          const double lo = __ldg(p.x + (uint32_t)xrow[cl][2 * a] + l * (uint32_t)p.xoff);
          const double hi = __ldg(p.x + (uint32_t)xrow[cl][2 * a + 1] + l * (uint32_t)p.xoff);
          val[u] = make_double2(lo, hi);
          dst[u] = (uint32_t)obase[cl] + 2u * q;
        }
      }
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const uint32_t vv = v + u * kThreads;
        if (vv < npairs) st_stream2(p.out + dst[u], val[u]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Variable layers: column c has layers[c] layers, so a CTA tile of TILE
// consecutive columns first forms the prefix sums pre[0..ncol] of its
// columns' unit counts (elements for the copy, pairs for the interpolation)
// in shared memory; a flattened unit index v of the tile then belongs to the
// column cl with pre[cl] <= v < pre[cl + 1] (binary search).

// Column c's unit count: its layers (lay[c], or `layers`) times its units
// per layer (rowptr[c+1] - rowptr[c] for ragged lists, or per_layer).
template <int TILE>
__device__ void tile_prefix(const int32_t *lay, int64_t c0, int ncol, uint32_t per_layer, uint32_t *pre,
                            uint32_t *wsum, int layers = 0, const int64_t *rowptr = nullptr) {
  static_assert(TILE % 32 == 0 && TILE <= kThreads, "tile must be whole warps of the CTA");
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  uint32_t x = 0;
  if (t < TILE) {
    if (t < ncol) {
      const uint32_t nl = lay ? (uint32_t)__ldg(lay + c0 + t) : (uint32_t)layers;
      const uint32_t pl = rowptr ? (uint32_t)(__ldg(rowptr + c0 + t + 1) - __ldg(rowptr + c0 + t)) : per_layer;
      x = nl * pl;
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) wsum[w] = x;
  }
  __syncthreads();
  if (t < TILE) {
    uint32_t add = 0;
    for (int j = 0; j < w; ++j) add += wsum[j];
    pre[t + 1] = x + add;
  }
  if (t == 0) pre[0] = 0;
  __syncthreads();
}

template <int TILE>
__device__ __forceinline__ int tile_find(const uint32_t *pre, int ncol, uint32_t v) {
  int lo = 0, hi = ncol;  // pre[lo] <= v < pre[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Variable layers or ragged lists (any number of DoFs per cell).
template <int TILE, int UNROLL>
__global__ void __launch_bounds__(kThreads) k_copy_dg_var(const CopyDGLaunch p, int64_t ntiles) {
  __shared__ uint32_t pre[TILE + 1];
  __shared__ uint32_t wsum[TILE / 32];
  __shared__ int32_t base[TILE];
  __shared__ int contiguous, i0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t c0 = tile * TILE;
    const int ncol = (int)(p.ncells - c0 < TILE ? p.ncells - c0 : TILE);
    __syncthreads();  // the previous tile's readers are done
    if (threadIdx.x == 0) {
      contiguous = 1;
      i0 = TILE;
    }
    for (int i = threadIdx.x; i < ncol; i += kThreads) {
      const int64_t r0 = p.rowptr ? __ldg(p.rowptr + c0 + i) : (c0 + i) * p.k;
      const bool empty = p.rowptr && __ldg(p.rowptr + c0 + i + 1) == r0;
      base[i] = empty ? 0 : __ldg(p.map + r0);
    }
    tile_prefix<TILE>(p.cell_layers, c0, ncol, (uint32_t)p.k, pre, wsum, p.layers, p.rowptr);
    for (int i = threadIdx.x; i < ncol; i += kThreads)
      if (pre[i + 1] > pre[i]) atomicMin(&i0, i);
    __syncthreads();
    // columns numbered back to back (as Algorithm 1 numbers a cell-interior
    // space) make the tile one range: no search
    const int f0 = i0 < ncol ? i0 : 0;
    for (int i = threadIdx.x; i < ncol; i += kThreads)
      if (pre[i + 1] > pre[i] && (uint32_t)(base[i] - base[f0]) != pre[i] - pre[f0]) contiguous = 0;
    __syncthreads();
    const uint32_t total = pre[ncol];
    const bool flat = contiguous != 0;
    for (uint32_t v = threadIdx.x; v < total; v += UNROLL * kThreads) {
      double val[UNROLL];
      uint32_t dst[UNROLL];
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const uint32_t vv = v + u * kThreads;
        if (vv < total) {
          if (flat) {
            dst[u] = (uint32_t)base[f0] - pre[f0] + vv;
          } else {
            const int cl = tile_find<TILE>(pre, ncol, vv);
            dst[u] = (uint32_t)base[cl] + (vv - pre[cl]);
          }
          val[u] = __ldcs(p.in + dst[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const uint32_t vv = v + u * kThreads;
        if (vv < total) __stcs(p.out + dst[u], val[u]);
      }
    }
  }
}

template <int TILE, int UNROLL>
__global__ void __launch_bounds__(kThreads) k_interp_dg1_var(const InterpDG1Launch p, FastDiv three,
                                                             int64_t ntiles) {
  __shared__ uint32_t pre[TILE + 1];
  __shared__ uint32_t wsum[TILE / 32];
  __shared__ int32_t xrow[TILE][6];
  __shared__ int32_t obase[TILE];
  constexpr int kWarps = kThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t c0 = tile * TILE;
    const int ncol = (int)(p.ncells - c0 < TILE ? p.ncells - c0 : TILE);
    __syncthreads();
    for (int i = threadIdx.x; i < ncol * 6; i += kThreads) xrow[i / 6][i % 6] = __ldg(p.xmap + c0 * 6 + i);
    for (int i = threadIdx.x; i < ncol; i += kThreads) obase[i] = __ldg(p.omap + (c0 + i) * 6);
    tile_prefix<TILE>(p.cell_layers, c0, ncol, 3u, pre, wsum);  // three pairs per layer
    const uint32_t npairs = pre[ncol];
    // each warp streams one contiguous eighth of the tile's pairs, lanes on
    // consecutive pairs; a lane finds its column once and then walks forward
    const uint32_t w0 = (uint32_t)(((uint64_t)npairs * warp) / kWarps);
    const uint32_t w1 = (uint32_t)(((uint64_t)npairs * (warp + 1)) / kWarps);
    int cl = tile_find<TILE>(pre, ncol, w0 + lane < npairs ? w0 + lane : (npairs ? npairs - 1 : 0));
    for (uint32_t v = w0 + lane; v < w1; v += UNROLL * 32) {
      double2 val[UNROLL];
      uint32_t dst[UNROLL];
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const uint32_t vv = v + u * 32;
        if (vv < w1) {
          while (pre[cl + 1] <= vv) ++cl;
          const uint32_t q = vv - pre[cl];  // pair within the column: 3 l + a
          const uint32_t l = fdiv(q, three);
          const uint32_t a = q - 3u * l;
          const double lo = __ldg(p.x + (uint32_t)xrow[cl][2 * a] + l * (uint32_t)p.xoff);
          const double hi = __ldg(p.x + (uint32_t)xrow[cl][2 * a + 1] + l * (uint32_t)p.xoff);
          val[u] = make_double2(lo, hi);
          dst[u] = (uint32_t)obase[cl] + 2u * q;
        }
      }
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const uint32_t vv = v + u * 32;
        if (vv < w1) st_stream2(p.out + dst[u], val[u]);
      }
    }
  }
}

unsigned grid_for(uint64_t work, int per_thread) {
  uint64_t blocks = (work + (uint64_t)kThreads * per_thread - 1) / ((uint64_t)kThreads * per_thread);
  const uint64_t cap = 152ull * 16;  // 16 resident CTAs per SM is plenty for a stream
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  return (unsigned)blocks;
}

}  // namespace

cudaError_t launch_copy_dg(const CopyDGLaunch &p, cudaStream_t s) {
  if (p.cell_layers || p.rowptr) {
    if (p.ncells == 0) return cudaSuccess;
    const int64_t ntiles = (p.ncells + 127) / 128;
    const int64_t grid = ntiles < 152 * 8 ? ntiles : 152 * 8;
    k_copy_dg_var<128, 8><<<(unsigned)grid, kThreads, 0, s>>>(p, ntiles);
    return cudaGetLastError();
  }
  const uint64_t colsize = (uint64_t)p.k * p.layers;
  const uint64_t n = colsize * (uint64_t)p.ncells;
  if (n == 0) return cudaSuccess;
  const FastDiv col = make_fastdiv((uint32_t)colsize);
  const bool aligned = ((((uintptr_t)p.in) | ((uintptr_t)p.out)) & 15) == 0;
  if (colsize % 2 == 0 && aligned) {
    const uint32_t npairs = (uint32_t)(n / 2);
    k_copy_dg_vec<<<grid_for(npairs, kUnroll), kThreads, 0, s>>>(p, col, npairs);
  } else {
    k_copy_dg_scalar<<<grid_for(n, 4), kThreads, 0, s>>>(p, col, (uint32_t)n);
  }
  return cudaGetLastError();
}

cudaError_t launch_interp_dg1(const InterpDG1Launch &p, cudaStream_t s) {
  if (p.cell_layers) {
    if (p.ncells == 0) return cudaSuccess;
    const int64_t ntiles = (p.ncells + 127) / 128;
    const int64_t grid = ntiles < 152 * 8 ? ntiles : 152 * 8;
    k_interp_dg1_var<128, EXT_INTERP_UNROLL><<<(unsigned)grid, kThreads, 0, s>>>(p, make_fastdiv(3u), ntiles);
    return cudaGetLastError();
  }
  const uint64_t colsize = 6ull * p.layers;
  const uint64_t n = colsize * (uint64_t)p.ncells;
  if (n == 0) return cudaSuccess;
#if EXT_INTERP_TILE > 0
  const int64_t ntiles = (p.ncells + EXT_INTERP_TILE - 1) / EXT_INTERP_TILE;
  const int64_t grid = ntiles < 152 * 8 ? ntiles : 152 * 8;
  k_interp_dg1_tile<EXT_INTERP_TILE, EXT_INTERP_UNROLL><<<(unsigned)grid, kThreads, 0, s>>>(p, make_fastdiv(3u), ntiles);
#else
  const uint32_t npairs = (uint32_t)(n / 2);
  k_interp_dg1<<<grid_for(npairs, kUnroll), kThreads, 0, s>>>(p, make_fastdiv((uint32_t)colsize),
                                                              make_fastdiv(6u), npairs);
#endif
  return cudaGetLastError();
}
