// Horizontal-facet par_loops: Algorithm 3 with d2 = 0, i.e. over the facets
// ((2,0),(c,m)) of each column at levels m = 0..lambda, and its interior form
// over the facets m = 1..lambda-1 shared by the layers m-1 and m.
//
//   FACET_MASS  b_a += int_F f phi_a ds      on a space (CG1|DG0|DG1) x CG1,
//               whose facet DoFs are the bottom horizontal DoFs of layer m
//               (the top ones of the last layer for m = lambda);
//   FACET_JUMP  r += int_F [u][phi] ds,  [w] = w(below, top) - w(above, bottom),
//               on any prism tensor-product space.
//
// On the flat triangle F with area element |n| = |dx/dxi x dx/deta| (twice
// the area) the P1 surface mass matrix is |n|/24 (1 + [a = b]) and a constant
// integrates to |n|/2, so with c = |n|/24:  v_a = c (g_a + sum_b g_b)  (three
// nodes) or v = |n|/2 g (one node).  One lane per (column, facet) item, lanes
// along the facets of a warp's column group; a straight column (x, y of every
// level bit-equal to level 0, z equal on the three vertices of the facet) uses
// the column's |n| = |2A|, any other facet the cross product of its edges.
// Increments are FP64 atomic adds (executed in L2): facet DoFs of CG1
// horizontal spaces are shared with neighbouring columns, and under the jump
// a vertically-DG0 DoF receives the terms of both of its facets.
#include "ext_internal.cuh"

namespace {

constexpr int kWarps = 8;
constexpr int kMaxCols = 32;
constexpr unsigned kFull = 0xffffffffu;
#ifndef EXT_FACET_ITEMS
#define EXT_FACET_ITEMS 1600  // target items per column group
#endif

struct FacetCol {
  int32_t cb[3], ct[3];  // coords DoF of vertex a at the bottom level, at the top level
  int32_t flo[3], fhi[3];
  double wf;             // |2A| / 24 (three nodes) or |2A| / 2 (one node): the
                         // weight factor of a facet of a straight column
  long long rx[3], ry[3];
  int lay;
};

template <int NH, bool JUMP, bool VAR>
__global__ void __launch_bounds__(kWarps * 32) k_facet(const FacetLaunch p, int cpw) {
  __shared__ FacetCol cols[kWarps][kMaxCols];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ngroups = (p.ncells + cpw - 1) / cpw;
  const int64_t wstride = (int64_t)gridDim.x * kWarps;
  for (int64_t grp = (int64_t)blockIdx.x * kWarps + warp; grp < ngroups; grp += wstride) {
    const int64_t c0 = grp * cpw;
    const int ncol = (int)(p.ncells - c0 < cpw ? p.ncells - c0 : (int64_t)cpw);
    int my_items = 0;
    if (lane < ncol) {
      const int64_t c = c0 + lane;
      FacetCol &ci = cols[warp][lane];
      const int lay = VAR ? __ldg(p.cell_layers + c) : p.layers;
      ci.lay = lay;
      my_items = JUMP ? lay - 1 : lay + 1;
      double x[3], y[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        ci.cb[a] = __ldg(p.cmap + c * 6 + 2 * a);
        ci.ct[a] = __ldg(p.cmap + c * 6 + 2 * a + 1) + (lay - 1) * p.coff[2 * a + 1];
        x[a] = __ldg(p.X + 3 * (int64_t)ci.cb[a] + 0);
        y[a] = __ldg(p.X + 3 * (int64_t)ci.cb[a] + 1);
        ci.rx[a] = __double_as_longlong(x[a]);
        ci.ry[a] = __double_as_longlong(y[a]);
      }
#pragma unroll
      for (int a = 0; a < NH; ++a) {
        ci.flo[a] = __ldg(p.fmap + c * p.k + p.slot_lo[a]);
        ci.fhi[a] = __ldg(p.fmap + c * p.k + p.slot_hi[a]);
      }
      ci.wf = fabs((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0])) * (NH == 3 ? 1.0 / 24.0 : 0.5);
    }
    __syncwarp();
    const int nitems = __reduce_add_sync(kFull, my_items);
    // lane's item: column cl, item index i within the column
    int cl = 0, i = lane;
    while (cl < ncol) {
      const int n = JUMP ? cols[warp][cl].lay - 1 : cols[warp][cl].lay + 1;
      if (i < n) break;
      i -= n;
      ++cl;
    }
    for (int base = 0; base < nitems; base += 32) {
      if (base + lane < nitems) {
        const FacetCol &ci = cols[warp][cl];
        const int lay = ci.lay;
        const int m = JUMP ? i + 1 : i;  // facet level
        double X[3][3];
        int ok = 1;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int64_t cd = m < lay ? (int64_t)ci.cb[a] + (int64_t)m * p.coff[2 * a] : (int64_t)ci.ct[a];
          X[a][0] = __ldg(p.X + 3 * cd + 0);
          X[a][1] = __ldg(p.X + 3 * cd + 1);
          X[a][2] = __ldg(p.X + 3 * cd + 2);
          ok &= (__double_as_longlong(X[a][0]) == ci.rx[a]) & (__double_as_longlong(X[a][1]) == ci.ry[a]);
        }
        ok &= (__double_as_longlong(X[0][2]) == __double_as_longlong(X[1][2])) &
              (__double_as_longlong(X[0][2]) == __double_as_longlong(X[2][2]));
        double cc;  // |n| / 24 (three nodes) or |n| / 2 (one node)
        if (ok) {
          cc = ci.wf;
        } else {
          double e1[3], e2[3];
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            e1[r] = X[1][r] - X[0][r];
            e2[r] = X[2][r] - X[0][r];
          }
          const double n0 = e1[1] * e2[2] - e1[2] * e2[1];
          const double n1 = e1[2] * e2[0] - e1[0] * e2[2];
          const double nz = e1[0] * e2[1] - e1[1] * e2[0];
          cc = sqrt(n0 * n0 + n1 * n1 + nz * nz) * (NH == 3 ? 1.0 / 24.0 : 0.5);
        }
        int32_t dlo[NH], dhi[NH];
        double g[NH];
        if (JUMP) {
#pragma unroll
          for (int a = 0; a < NH; ++a) {
            dlo[a] = ci.flo[a] + (m - 1) * p.off_lo[a];  // top trace of the layer below
            dhi[a] = ci.fhi[a] + m * p.off_hi[a];        // bottom trace of the layer above
            g[a] = __ldg(p.f + dlo[a]) - __ldg(p.f + dhi[a]);
          }
        } else {
#pragma unroll
          for (int a = 0; a < NH; ++a) {
            dlo[a] = m < lay ? ci.flo[a] + m * p.off_lo[a] : ci.fhi[a] + (lay - 1) * p.off_hi[a];
            g[a] = __ldg(p.f + dlo[a]);
          }
        }
        double v[NH];
        if (NH == 3) {
          // c (g_a + sum g): one DMUL and five DFMA
          const double cs = fma(cc, g[0], fma(cc, g[1], cc * g[2]));
#pragma unroll
          for (int a = 0; a < NH; ++a) v[a] = fma(cc, g[a], cs);
        } else {
          v[0] = cc * g[0];
        }
#pragma unroll
        for (int a = 0; a < NH; ++a) {
          atomicAdd(p.b + dlo[a], v[a]);
          if (JUMP) atomicAdd(p.b + dhi[a], -v[a]);
        }
      }
      i += 32;
      while (cl < ncol) {
        const int n = JUMP ? cols[warp][cl].lay - 1 : cols[warp][cl].lay + 1;
        if (i < n) break;
        i -= n;
        ++cl;
      }
    }
    __syncwarp();
  }
}


// Interior-facet jump on a space discontinuous in both directions (used for
// DG1xDG1): every DoF belongs to one cell, so the lane of cell layer l owns
// its DoFs and updates them with plain loads and stores.  It evaluates its
// bottom facet (level l, for l >= 1) from the top trace of the cell below
// (the previous lane's, by shuffle) and its own bottom trace, subtracts that
// term from its bottom-trace DoFs, and adds the term of its top facet, which
// the next lane evaluated, to its top-trace DoFs (for DG0 vertically both are
// the same DoFs).  The cell below a warp step's first lane belongs to the
// previous step's last lane: that one term is added atomically after the
// warp has synchronised.  The atomics of the facet-centric loop fall on a
// 24- or 48-byte stride, which L2 executes one sector at a time.
template <int NH, int NV, bool VAR>
__global__ void __launch_bounds__(kWarps * 32) k_jump_dg(const FacetLaunch p, int cpw) {
  // The cell's K = NH NV DoFs are consecutive (Algorithm 1 numbers a cell
  // entity's DoFs together, layer after layer): node (a, b) is DoF a NV + b of
  // the block, moved with 16-byte accesses when K is even.
  constexpr int K = NH * NV;
  __shared__ FacetCol cols[kWarps][kMaxCols];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ngroups = (p.ncells + cpw - 1) / cpw;
  const int64_t wstride = (int64_t)gridDim.x * kWarps;
  for (int64_t grp = (int64_t)blockIdx.x * kWarps + warp; grp < ngroups; grp += wstride) {
    const int64_t c0 = grp * cpw;
    const int ncol = (int)(p.ncells - c0 < cpw ? p.ncells - c0 : (int64_t)cpw);
    int my_items = 0;
    if (lane < ncol) {
      const int64_t c = c0 + lane;
      FacetCol &ci = cols[warp][lane];
      const int lay = VAR ? __ldg(p.cell_layers + c) : p.layers;
      ci.lay = lay;
      my_items = lay;
      double x[3], y[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        ci.cb[a] = __ldg(p.cmap + c * 6 + 2 * a);
        ci.ct[a] = 0;
        x[a] = __ldg(p.X + 3 * (int64_t)ci.cb[a] + 0);
        y[a] = __ldg(p.X + 3 * (int64_t)ci.cb[a] + 1);
        ci.rx[a] = __double_as_longlong(x[a]);
        ci.ry[a] = __double_as_longlong(y[a]);
      }
      ci.flo[0] = __ldg(p.fmap + c * K);  // the column's first DoF
      ci.wf = fabs((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0])) * (NH == 3 ? 1.0 / 24.0 : 0.5);
    }
    __syncwarp();
    const int nitems = __reduce_add_sync(kFull, my_items);
    int cl = 0, l = lane;
    while (cl < ncol && l >= cols[warp][cl].lay) { l -= cols[warp][cl].lay; ++cl; }
    for (int base = 0; base < nitems; base += 32) {
      const bool valid = base + lane < nitems;
      const FacetCol &ci = cols[warp][valid ? cl : 0];
      const int lay = ci.lay;
      const int64_t blk = (int64_t)ci.flo[0] + (int64_t)l * K;
      double u[K];
#pragma unroll
      for (int j = 0; j < K; ++j) u[j] = 0.0;
      if (valid) {
        if (K % 2 == 0) {
#pragma unroll
          for (int j = 0; j < K; j += 2) {
            const double2 v2 = __ldg(reinterpret_cast<const double2 *>(p.f + blk + j));
            u[j] = v2.x;
            u[j + 1] = v2.y;
          }
        } else {
#pragma unroll
          for (int j = 0; j < K; ++j) u[j] = __ldg(p.f + blk + j);
        }
      }
      double below[NH], vb[NH];
#pragma unroll
      for (int a = 0; a < NH; ++a) {
        below[a] = __shfl_up_sync(kFull, u[a * NV + NV - 1], 1);  // top trace of the cell below
        vb[a] = 0.0;
      }
      const bool has_bot = valid && l >= 1;
      if (has_bot) {
        if (lane == 0) {
#pragma unroll
          for (int a = 0; a < NH; ++a) below[a] = __ldg(p.f + blk - K + a * NV + NV - 1);
        }
        double X[3][3];
        int ok = 1;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int64_t cd = (int64_t)ci.cb[a] + (int64_t)l * p.coff[2 * a];
          X[a][0] = __ldg(p.X + 3 * cd + 0);
          X[a][1] = __ldg(p.X + 3 * cd + 1);
          X[a][2] = __ldg(p.X + 3 * cd + 2);
          ok &= (__double_as_longlong(X[a][0]) == ci.rx[a]) & (__double_as_longlong(X[a][1]) == ci.ry[a]);
        }
        ok &= (__double_as_longlong(X[0][2]) == __double_as_longlong(X[1][2])) &
              (__double_as_longlong(X[0][2]) == __double_as_longlong(X[2][2]));
        double cc;  // |n| / 24 (three nodes) or |n| / 2 (one node)
        if (ok) {
          cc = ci.wf;
        } else {
          double e1[3], e2[3];
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            e1[r] = X[1][r] - X[0][r];
            e2[r] = X[2][r] - X[0][r];
          }
          const double n0 = e1[1] * e2[2] - e1[2] * e2[1];
          const double n1 = e1[2] * e2[0] - e1[0] * e2[2];
          const double nz = e1[0] * e2[1] - e1[1] * e2[0];
          cc = sqrt(n0 * n0 + n1 * n1 + nz * nz) * (NH == 3 ? 1.0 / 24.0 : 0.5);
        }
        double g[NH];
#pragma unroll
        for (int a = 0; a < NH; ++a) g[a] = below[a] - u[a * NV];
        if (NH == 3) {
          const double cs = fma(cc, g[0], fma(cc, g[1], cc * g[2]));
#pragma unroll
          for (int a = 0; a < NH; ++a) vb[a] = fma(cc, g[a], cs);
        } else {
          vb[0] = cc * g[0];
        }
      }
      // the top facet's term, evaluated by the lane of the cell above
      const bool has_top = valid && lane < 31 && l + 1 < lay;
      double vt[NH];
#pragma unroll
      for (int a = 0; a < NH; ++a) {
        vt[a] = __shfl_down_sync(kFull, vb[a], 1);
        if (!has_top) vt[a] = 0.0;
      }
      if (valid && (has_top || has_bot)) {
        double r[K];
        if (K % 2 == 0) {
#pragma unroll
          for (int j = 0; j < K; j += 2) {
            const double2 v2 = *reinterpret_cast<const double2 *>(p.b + blk + j);
            r[j] = v2.x;
            r[j + 1] = v2.y;
          }
        } else {
#pragma unroll
          for (int j = 0; j < K; ++j) r[j] = p.b[blk + j];
        }
#pragma unroll
        for (int a = 0; a < NH; ++a) {
          if (NV == 2) {
            r[a * NV + 1] += vt[a];
            r[a * NV] -= vb[a];
          } else {
            r[a] += vt[a] - vb[a];
          }
        }
        if (K % 2 == 0) {
#pragma unroll
          for (int j = 0; j < K; j += 2) *reinterpret_cast<double2 *>(p.b + blk + j) = make_double2(r[j], r[j + 1]);
        } else {
#pragma unroll
          for (int j = 0; j < K; ++j) p.b[blk + j] = r[j];
        }
      }
      // the cell below this step's first item was the previous step's last
      __syncwarp();
      if (lane == 0 && has_bot) {
#pragma unroll
        for (int a = 0; a < NH; ++a) atomicAdd(p.b + blk - K + a * NV + NV - 1, vb[a]);
      }
      l += 32;
      while (cl < ncol && l >= cols[warp][cl].lay) { l -= cols[warp][cl].lay; ++cl; }
      __syncwarp();
    }
    __syncwarp();
  }
}

template <int NH, bool JUMP, bool VAR>
cudaError_t launch_k(const FacetLaunch &p, cudaStream_t s) {
  const double per = (VAR ? p.mean_layers : (double)p.layers) + (JUMP ? -1.0 : 1.0);
  int cpw = per > 0.5 ? (int)((EXT_FACET_ITEMS + per - 1.0) / per) : kMaxCols;
  if (cpw < 1) cpw = 1;
  if (cpw > kMaxCols) cpw = kMaxCols;
  const int64_t warps = (p.ncells + cpw - 1) / cpw;
  int64_t blocks = (warps + kWarps - 1) / kWarps;
  static int resident = 0, sms = 0;
  if (resident == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_facet<NH, JUMP, VAR>, kWarps * 32, 0);
    if (resident < 1) resident = 1;
  }
  if (blocks > (int64_t)resident * sms) blocks = (int64_t)resident * sms;
  k_facet<NH, JUMP, VAR><<<(unsigned)blocks, kWarps * 32, 0, s>>>(p, cpw);
  return cudaGetLastError();
}

template <bool VAR>
cudaError_t launch_v(const FacetLaunch &p, cudaStream_t s) {
  if (p.jump) return p.nh == 3 ? launch_k<3, true, VAR>(p, s) : launch_k<1, true, VAR>(p, s);
  return p.nh == 3 ? launch_k<3, false, VAR>(p, s) : launch_k<1, false, VAR>(p, s);
}

template <int NH, int NV, bool VAR>
cudaError_t launch_jdg(const FacetLaunch &p, cudaStream_t s) {
  const double per = VAR ? p.mean_layers : (double)p.layers;
  int cpw = (int)((EXT_FACET_ITEMS + per - 1.0) / per);
  if (cpw < 1) cpw = 1;
  if (cpw > kMaxCols) cpw = kMaxCols;
  const int64_t warps = (p.ncells + cpw - 1) / cpw;
  int64_t blocks = (warps + kWarps - 1) / kWarps;
  static int resident = 0, sms = 0;
  if (resident == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_jump_dg<NH, NV, VAR>, kWarps * 32, 0);
    if (resident < 1) resident = 1;
  }
  if (blocks > (int64_t)resident * sms) blocks = (int64_t)resident * sms;
  k_jump_dg<NH, NV, VAR><<<(unsigned)blocks, kWarps * 32, 0, s>>>(p, cpw);
  return cudaGetLastError();
}

template <bool VAR>
cudaError_t launch_jv(const FacetLaunch &p, cudaStream_t s) {
  if (p.nh != 3 || p.nv != 2) return cudaErrorInvalidValue;  // DG1xDG1 only (see ext_par_loop)
  return launch_jdg<3, 2, VAR>(p, s);
}

}  // namespace

cudaError_t launch_facet(const FacetLaunch &p, cudaStream_t s) {
  if (p.ncells == 0) return cudaSuccess;
  if (p.jump && p.mode == 2) return cudaSuccess;  // vertically continuous: every jump is 0
  if (p.jump && p.mode == 1) return p.cell_layers ? launch_jv<true>(p, s) : launch_jv<false>(p, s);
  return p.cell_layers ? launch_v<true>(p, s) : launch_v<false>(p, s);
}
