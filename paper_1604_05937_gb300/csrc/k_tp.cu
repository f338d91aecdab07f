// Mass action / RHS assembly b_i += int f phi_i dx (the residual I_1 of
// Sec. 4.1.1) on the prism spaces of Sec. 4.1.2: horizontal element CG1, DG0
// or DG1 on the triangle times vertical element CG1, DG0 or DG1 on the layer.
// On a straight prism the element matrix is Mh (x) Mv with
//   Mh = A/12 (1 + [a = a'])  (CG1, DG1: three nodes at the vertices) or A (DG0),
//   Mv = h/6 (1 + [b = b'])   (CG1, DG1: nodes at the two ends)      or h (DG0),
// so the kernel is templated on the node counts NH in {1, 3} and NV in {1, 2};
// continuity only changes the addresses (the stencil slots) and whether
// neighbouring cells share a DoF, and every increment is an FP64 atomic add
// executed in L2, which is correct for shared and private DoFs alike.
// One lane per (column, layer) item, lanes along the layers of a warp's
// column group (coalesced column-contiguous accesses); a persistent grid hands
// out column groups round-robin so resident warps sweep the mesh together.
// Straightness is checked exactly as in the P1xP1 kernel; other prisms use the
// 6-point rule with the general Jacobian.
#include <cstdlib>

#include "ext_internal.cuh"
#include "fastdiv.cuh"

namespace {

constexpr int kWarps = 8;
constexpr int kMaxCols = 32;
#ifndef EXT_TP_ITEMS
#define EXT_TP_ITEMS 1600  // target items (column layers) per column group
#endif

struct TPCol {
  double alpha;              // |2A| * (1/2)(1/12 if NH=3)(1/6 if NV=2): c = alpha |h|
  long long rx[3], ry[3];    // level-0 x, y bit patterns
  int32_t cm[6];             // the column's coordinate stencil row (layer 0)
  int32_t fm[6];             // its f/b DoFs of node (a, b) at layer 0
  int lay;                   // layers of this column
  int allok;                 // flagged form: every level of the three vertex columns is straight
};

// element vector of a general prism: out[a*NV+b] = sum_q w_q |detJ| f(x_q) H_a V_b
template <int NH, int NV>
__device__ void tp_general(const double X[6][3], const double f[NH * NV], double out[NH * NV]) {
  const double tp[3][2] = {{1.0 / 6.0, 1.0 / 6.0}, {2.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 3.0}};
  const double gz[2] = {0.5 - 0.28867513459481288225, 0.5 + 0.28867513459481288225};
  for (int i = 0; i < NH * NV; ++i) out[i] = 0.0;
  for (int t = 0; t < 3; ++t) {
    const double lam[3] = {1.0 - tp[t][0] - tp[t][1], tp[t][0], tp[t][1]};
    const double dlx[3] = {-1.0, 1.0, 0.0}, dly[3] = {-1.0, 0.0, 1.0};
    for (int g = 0; g < 2; ++g) {
      const double psi[2] = {1.0 - gz[g], gz[g]};
      const double dpsi[2] = {-1.0, 1.0};
      double J[3][3] = {{0.0}};
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 2; ++b) {
          const double gr[3] = {dlx[a] * psi[b], dly[a] * psi[b], lam[a] * dpsi[b]};
          for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) J[r][s] += X[2 * a + b][r] * gr[s];
        }
      const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                         J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      double phi[NH * NV], fq = 0.0;
      for (int a = 0; a < NH; ++a)
        for (int b = 0; b < NV; ++b) {
          phi[a * NV + b] = (NH == 3 ? lam[a] : 1.0) * (NV == 2 ? psi[b] : 1.0);
          fq += phi[a * NV + b] * f[a * NV + b];
        }
      const double wq = (1.0 / 12.0) * fabs(det) * fq;
      for (int i = 0; i < NH * NV; ++i) out[i] += wq * phi[i];
    }
  }
}

// Flagged form (constant layers, mesh with base coordinates, a million
// (column, layer) items or more): one pass reads the coordinate field once
// and sets bit d of `flags` when coordinate DoF d sits at its vertex's base
// x, y and at the height of its level in the column of vertex 0 (bitwise);
// hlay[l] = |z_{l+1} - z_l| of that column.  A prism whose six vertex levels
// are all flagged is straight with flat faces, so the cell kernel takes its
// element matrix from the column's area and hlay[l] without loading its 18
// coordinates; other prisms load them and take the general 6-point rule.
__global__ void __launch_bounds__(256) k_tp_levels(const double *__restrict__ X, int layers,
                                                   double *__restrict__ ztab, double *__restrict__ hlay) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > layers) return;
  const double z = X[3 * (int64_t)m + 2];
  ztab[m] = z;
  if (m < layers) hlay[m] = fabs(X[3 * (int64_t)(m + 1) + 2] - z);
}

__global__ void __launch_bounds__(256) k_tp_vflags(const double *__restrict__ X, const double *__restrict__ xy,
                                                   const double *__restrict__ ztab, int64_t n, FastDiv col,
                                                   uint32_t *__restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const int64_t nwords = (n + 31) / 32;
  for (int64_t w = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); w < nwords; w += (int64_t)gridDim.x * kWarps) {
    const int64_t d = w * 32 + lane;
    int ok = 0;
    if (d < n) {
      const uint32_t q = fdiv((uint32_t)d, col);
      const uint32_t m = (uint32_t)d - q * col.d;
      ok = (__double_as_longlong(__ldg(X + 3 * d + 0)) == __double_as_longlong(__ldg(xy + 2 * (int64_t)q + 0))) &
           (__double_as_longlong(__ldg(X + 3 * d + 1)) == __double_as_longlong(__ldg(xy + 2 * (int64_t)q + 1))) &
           (__double_as_longlong(__ldg(X + 3 * d + 2)) == __double_as_longlong(__ldg(ztab + m)));
    }
    const unsigned int word = __ballot_sync(0xffffffffu, ok);
    if (lane == 0) flags[w] = word;
  }
}

// Element vector of a straight prism with c = alpha |h|: Mh (x) Mv f in closed
// form for NH horizontal and NV vertical nodes; products and sums go out as
// DFMA (k1), which GB300 issues faster than DMUL and DADD.
template <int NH, int NV>
__device__ __forceinline__ void tp_closed(double cc, const double f[NH * NV], double b[NH * NV], const Fp64Ones &k1) {
  if (NH == 1 && NV == 1) {
    b[0] = fmul(cc, f[0], k1);
  } else if (NH == 1) {  // NV == 2
    const double c2 = fadd(cc, cc, k1);
    b[0] = fma(c2, f[0], fmul(cc, f[1], k1));
    b[1] = fma(c2, f[1], fmul(cc, f[0], k1));
  } else if (NV == 1) {  // NH == 3
    const double cS = fmul(cc, fadd(fadd(f[0], f[1], k1), f[2], k1), k1);
#pragma unroll
    for (int a = 0; a < 3; ++a) b[a] = fma(cc, f[a], cS);
  } else {  // NH == 3, NV == 2: b_{a,beta} = c (t_{a,beta} + T_beta),
            // t_{a,beta} = 2 f_{a,beta} + f_{a,1-beta}, T_beta = sum_a t_{a,beta}
    double t[6];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      t[2 * a] = fma(2.0, f[2 * a], f[2 * a + 1]);
      t[2 * a + 1] = fma(2.0, f[2 * a + 1], f[2 * a]);
    }
    const double K0 = fmul(cc, fadd(fadd(t[0], t[2], k1), t[4], k1), k1);
    const double K1 = fmul(cc, fadd(fadd(t[1], t[3], k1), t[5], k1), k1);
#pragma unroll
    for (int i = 0; i < 6; ++i) b[i] = fma(cc, t[i], (i & 1) ? K1 : K0);
  }
}

#ifndef EXT_TP_UNROLL
#define EXT_TP_UNROLL 4  // (column, layer) items per lane per step of the flagged form
#endif

__device__ __forceinline__ int vflag(const uint32_t *__restrict__ flags, int64_t d) {
  return (int)((__ldg(flags + (d >> 5)) >> (uint32_t)(d & 31)) & 1u);
}

// bits lo .. lo + n - 1 of the flags all set (a whole vertex column straight)
__device__ __forceinline__ int vflags_all(const uint32_t *__restrict__ flags, int64_t lo, int64_t n) {
  const int64_t hi = lo + n;
  for (int64_t w = lo >> 5; w <= (hi - 1) >> 5; ++w) {
    uint32_t need = 0xffffffffu;
    if (w == (lo >> 5)) need &= 0xffffffffu << (uint32_t)(lo & 31);
    if (w == ((hi - 1) >> 5)) need &= 0xffffffffu >> (uint32_t)(31 - ((hi - 1) & 31));
    if ((__ldg(flags + w) & need) != need) return 0;
  }
  return 1;
}

// VAR: column c has cell_layers[c] layers (lists taken at its bottom layer).
// FLAGS: the flagged form (constant layers only); MULTI (with FLAGS): several
// items per lane per step, a separate instantiation so that its registers do
// not lower the occupancy of the one-item loop.
// WR: each DoF belongs to one cell-layer (DG x DG) and b is overwritten:
// plain stores instead of atomic adds.  FIX (with FLAGS and WR): the fix-up
// launch of the optimistic form, which writes only the prisms whose flags are
// not all set (and returns at once when the flag pass found none).
template <int NH, int NV, bool VAR, bool FLAGS, bool MULTI = false, bool WR = false, bool FIX = false>
#ifndef EXT_TP_SMALL_MINB
#define EXT_TP_SMALL_MINB 3  // resident CTAs per SM for one-node elements (DG0xDG0: registers for occupancy)
#endif
__global__ void __launch_bounds__(kWarps * 32, NH * NV == 1 ? EXT_TP_SMALL_MINB : 2) k_mass_tp(const MassTPLaunch p, int cpw) {
  __shared__ TPCol cols[kWarps][kMaxCols];
  if (p.mode && (*p.mode & 3u) != 3u) return;  // gated on the probe's cell-loop mode (CG1 x DG gather path)
  if (FIX) {  // no CTA of the optimistic launch saw a coordinate DoF that is not straight
    grid_dep_wait();  // launched as a dependent of that launch
    int any = 0;
    for (int i = threadIdx.x; i < p.nbadv; i += blockDim.x) any |= __ldg(p.badv + i);
    if (!__syncthreads_or(any)) return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int layers = p.layers;
  const int64_t ngroups = (p.ncells + cpw - 1) / cpw;
  const int64_t wstride = (int64_t)gridDim.x * kWarps;
  for (int64_t grp = (int64_t)blockIdx.x * kWarps + warp; grp < ngroups; grp += wstride) {
    const int64_t c0 = grp * cpw;
    const int ncol = (int)(p.ncells - c0 < cpw ? p.ncells - c0 : (int64_t)cpw);
    int my_items = 0;
    if (lane < ncol) {
      const int64_t c = c0 + lane;
      const int lay = VAR ? __ldg(p.cell_layers + c) : layers;
      cols[warp][lane].lay = lay;
      my_items = lay;
      double x[3], y[3];
#pragma unroll
      for (int i = 0; i < 6; ++i) cols[warp][lane].cm[i] = __ldg(p.cmap + c * 6 + i);
#pragma unroll
      for (int i = 0; i < NH * NV; ++i) cols[warp][lane].fm[i] = __ldg(p.fmap + c * p.k + p.slot[i]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int64_t cd = cols[warp][lane].cm[2 * a];
        if (FLAGS) {  // the base coordinates the flags were checked against (vertex = level-0 DoF / (layers + 1))
          const int64_t v = cd / (layers + 1);
          x[a] = __ldg(p.base_xy + 2 * v + 0);
          y[a] = __ldg(p.base_xy + 2 * v + 1);
        } else {
          x[a] = __ldg(p.X + 3 * cd + 0);
          y[a] = __ldg(p.X + 3 * cd + 1);
        }
        cols[warp][lane].rx[a] = __double_as_longlong(x[a]);
        cols[warp][lane].ry[a] = __double_as_longlong(y[a]);
      }
      const double det2 = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
      cols[warp][lane].alpha = fabs(det2) * p.scale;
      // flagged form: a column whose three vertex columns are straight at
      // every level needs no per-item flag test (Algorithm 3's outer loop
      // does the test once per column)
      int allok = 0;
      if (FLAGS)
        allok = vflags_all(p.vflags, cols[warp][lane].cm[0], layers + 1) &
                vflags_all(p.vflags, cols[warp][lane].cm[2], layers + 1) &
                vflags_all(p.vflags, cols[warp][lane].cm[4], layers + 1);
      cols[warp][lane].allok = allok;
    }
    __syncwarp();
    const int nitems = VAR ? __reduce_add_sync(0xffffffffu, my_items) : ncol * layers;
    int cl, l;
    if (VAR) {
      cl = 0;
      l = lane;
      while (cl < ncol && l >= cols[warp][cl].lay) { l -= cols[warp][cl].lay; ++cl; }
    } else {
      cl = lane / layers;
      l = lane - cl * layers;
    }
    if (FLAGS && !VAR && MULTI) {
      // U items per lane per step, all their loads (straightness bits, layer
      // heights, f) issued before any arithmetic or increment
      constexpr int U = EXT_TP_UNROLL;
      for (int base = 0; base < nitems; base += 32 * U) {
        int32_t dof[U][NH * NV];
        double f[U][NH * NV], hl[U];
        int ok[U], cls[U], ls[U];
        bool valid[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          valid[u] = base + u * 32 + lane < nitems;
          cls[u] = cl;
          ls[u] = l;
          ok[u] = 1;
          hl[u] = 0.0;
          if (valid[u]) {
            const TPCol &ci = cols[warp][cl];
            if (!ci.allok) {
#pragma unroll
              for (int i = 0; i < 6; ++i) ok[u] &= vflag(p.vflags, (int64_t)ci.cm[i] + (int64_t)l * p.coff[i]);
            }
            if (FIX && ok[u]) valid[u] = false;  // written by the optimistic launch
          }
          if (valid[u]) {
            const TPCol &ci = cols[warp][cl];
            if (!FIX) hl[u] = __ldg(p.hlay + l);
#pragma unroll
            for (int i = 0; i < NH * NV; ++i) {
              dof[u][i] = ci.fm[i] + l * p.off[i];
              f[u][i] = __ldg(p.f + dof[u][i]);
            }
          }
          l += 32;
          while (l >= layers) { l -= layers; ++cl; }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (!valid[u]) continue;
          const TPCol &ci = cols[warp][cls[u]];
          double b[NH * NV];
          if (ok[u]) {
            tp_closed<NH, NV>(fmul(ci.alpha, hl[u], p.k1), f[u], b, p.k1);
          } else {
            double Xl[6][3];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
              const int64_t cd = (int64_t)ci.cm[i] + (int64_t)ls[u] * p.coff[i];
              Xl[i][0] = __ldg(p.X + 3 * cd + 0);
              Xl[i][1] = __ldg(p.X + 3 * cd + 1);
              Xl[i][2] = __ldg(p.X + 3 * cd + 2);
            }
            tp_general<NH, NV>(Xl, f[u], b);
          }
#pragma unroll
          for (int i = 0; i < NH * NV; ++i) {
            if (WR) p.b[dof[u][i]] = b[i];
            else atomicAdd(p.b + dof[u][i], b[i]);
          }
        }
      }
      __syncwarp();
      continue;
    }
    for (int base = 0; base < nitems; base += 32) {
      if (base + lane < nitems) {
        const TPCol &ci = cols[warp][cl];
        double Xl[6][3];
        int ok = 1;
        auto load_coords = [&]() {
#pragma unroll
          for (int i = 0; i < 6; ++i) {
            const int64_t cd = (int64_t)ci.cm[i] + (int64_t)l * p.coff[i];
            Xl[i][0] = __ldg(p.X + 3 * cd + 0);
            Xl[i][1] = __ldg(p.X + 3 * cd + 1);
            Xl[i][2] = __ldg(p.X + 3 * cd + 2);
          }
        };
        if (FLAGS) {
          if (!ci.allok) {
#pragma unroll
            for (int i = 0; i < 6; ++i) ok &= vflag(p.vflags, (int64_t)ci.cm[i] + (int64_t)l * p.coff[i]);
          }
        } else {
          load_coords();
#pragma unroll
          for (int i = 0; i < 6; ++i)
            ok &= (__double_as_longlong(Xl[i][0]) == ci.rx[i >> 1]) & (__double_as_longlong(Xl[i][1]) == ci.ry[i >> 1]);
          ok &= (__double_as_longlong(Xl[0][2]) == __double_as_longlong(Xl[2][2])) &
                (__double_as_longlong(Xl[0][2]) == __double_as_longlong(Xl[4][2])) &
                (__double_as_longlong(Xl[1][2]) == __double_as_longlong(Xl[3][2])) &
                (__double_as_longlong(Xl[1][2]) == __double_as_longlong(Xl[5][2]));
        }
        if (!(FIX && ok)) {  // FIX: straight prisms were written by the optimistic launch
          int32_t dof[NH * NV];
          double f[NH * NV], b[NH * NV];
#pragma unroll
          for (int i = 0; i < NH * NV; ++i) {
            dof[i] = ci.fm[i] + l * p.off[i];
            f[i] = __ldg(p.f + dof[i]);
          }
          if (ok) {
            tp_closed<NH, NV>(fmul(ci.alpha, FLAGS ? __ldg(p.hlay + l) : fabs(Xl[1][2] - Xl[0][2]), p.k1), f, b, p.k1);
          } else {
            if (FLAGS) load_coords();
            tp_general<NH, NV>(Xl, f, b);
          }
#pragma unroll
          for (int i = 0; i < NH * NV; ++i) {
            if (WR) p.b[dof[i]] = b[i];
            else atomicAdd(p.b + dof[i], b[i]);
          }
        }
      }
      l += 32;
      if (VAR) {
        while (cl < ncol && l >= cols[warp][cl].lay) { l -= cols[warp][cl].lay; ++cl; }
      } else {
        while (l >= layers) { l -= layers; ++cl; }
      }
    }
    __syncwarp();
  }
}

#ifndef EXT_TP_DGDG_UI1
#define EXT_TP_DGDG_UI1 4  // DG0 x DG0: items per lane per element chunk
#endif
#ifndef EXT_TP_DGDG_UF1
#define EXT_TP_DGDG_UF1 2  // DG0 x DG0: flag words per lane per flag chunk
#endif
#ifndef EXT_TP_DGDG_MINB
#define EXT_TP_DGDG_MINB 4  // DG0 x DG0: resident CTAs per SM
#endif
#ifndef EXT_TP_DGDG_MAX_LAYERS
#define EXT_TP_DGDG_MAX_LAYERS 2048  // the level tables of the optimistic form live in shared memory
#endif
#ifndef EXT_TP_DGCG_MAX_LAYERS
#define EXT_TP_DGCG_MAX_LAYERS 1024  // DG x CG1: four tables per level in shared memory
#endif
// Optimistic WRITE form for DG x DG on constant layers (every DoF of b
// belongs to one cell-layer).  The flagged form's two passes (straightness
// flags over the coordinate field, then the element vectors) have no data
// dependence when the element vector is taken in closed form for every prism
// on the assumption that it is straight: the column's |2A| comes from the
// base coordinates (k_tp_area2, in every launch) and the layer's height from
// the reference column (vertex 0's, coordinate DoFs 0 .. layers).  So one
// launch does both, the
// same warps taking flag chunks and element chunks interleaved in proportion
// to their counts, and the HBM-bound flag work runs beside the FP64-bound
// element work on every SM.  A fix-up launch (k_mass_tp with FIX) then
// rewrites the DoFs of every prism whose six flags are not all set with the
// general rule, and returns at once when no CTA of this launch found such a
// coordinate DoF.  The result is the flagged form's: each DoF is written by
// the closed form exactly when its prism is verified straight.
//
// |2A| of every base cell, formed in every launch from the base coordinates
// the straightness flags are checked against (the vertex of a level-0
// coordinate DoF d is d / (layers + 1)): a prism whose six flags are set has
// exactly these x, y at both of its levels.
// With ztab (the DG x CG1 fix-up's tables): also z of the reference column
// at every level and hlay[l] = |z_{l+1} - z_l| (as k_tp_levels).
__global__ void __launch_bounds__(256) k_tp_area2(const int32_t *__restrict__ cmap, const double *__restrict__ xy,
                                                  FastDiv colv, int64_t ncells, double *__restrict__ area2,
                                                  const double *__restrict__ X = nullptr, int layers = 0,
                                                  double *__restrict__ ztab = nullptr,
                                                  double *__restrict__ hlay = nullptr) {
  if (ztab) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m <= layers) {
      const double z = X[3 * m + 2];
      ztab[m] = z;
      if (m < layers) hlay[m] = fabs(X[3 * (m + 1) + 2] - z);
    }
  }
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x) {
    double x[3], y[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double *bp = xy + 2 * (size_t)fdiv((uint32_t)__ldg(cmap + 6 * c + 2 * a), colv);
      x[a] = __ldg(bp + 0);
      y[a] = __ldg(bp + 1);
    }
    area2[c] = fabs((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]));
  }
}

// flag words per lane per flag chunk, items per lane per element chunk (for
// DG0 x DG0 sized so that 4 CTAs of 256 threads stay resident per SM; 3 CTAs
// for the element vectors of 2, 3 and 6 DoFs)
#ifndef EXT_TP_DGDG_UIK
#define EXT_TP_DGDG_UIK 2  // element vectors of 2, 3 and 6 DoFs: items per lane per element chunk
#endif
#ifndef EXT_TP_DGDG_MINBK
#define EXT_TP_DGDG_MINBK 3  // and their resident CTAs per SM (4 items and 2 CTAs: 13-16 % slower at 100 layers)
#endif
__host__ __device__ constexpr int dgdg_uf(int k) { return k == 1 ? EXT_TP_DGDG_UF1 : 4; }
__host__ __device__ constexpr int dgdg_ui(int k) { return k == 1 ? EXT_TP_DGDG_UI1 : EXT_TP_DGDG_UIK; }

template <int NH, int NV>
__global__ void __launch_bounds__(kWarps * 32, NH * NV == 1 ? EXT_TP_DGDG_MINB : EXT_TP_DGDG_MINBK)
    k_tp_dgdg(const MassTPLaunch p, const double *__restrict__ area2, uint32_t *__restrict__ flags,
              int32_t *__restrict__ badv, FastDiv colv, FastDiv lay, int64_t nfc, int64_t nic) {
  constexpr int UF = dgdg_uf(NH * NV), UI = dgdg_ui(NH * NV), K = NH * NV;
  // level tables of the reference column: z at every level, scaled heights
  // hs[l] = |z_{l+1} - z_l| x (the element's constant)
  extern __shared__ double lvl[];
  double *ztab = lvl, *hs = lvl + p.layers + 1;
  __shared__ int cta_bad;
  for (int m = threadIdx.x; m <= p.layers; m += blockDim.x) ztab[m] = __ldg(p.X + 3 * (int64_t)m + 2);
  if (threadIdx.x == 0) cta_bad = 0;
  __syncthreads();
  for (int m = threadIdx.x; m < p.layers; m += blockDim.x) hs[m] = fabs(ztab[m + 1] - ztab[m]) * p.scale;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t ncoord = (uint32_t)p.ncoord, nwords = (uint32_t)((p.ncoord + 31) / 32);
  const uint32_t nitems = (uint32_t)(p.ncells * (int64_t)p.layers);
  const int64_t nch = nfc + nic;
  const int64_t wstride = (int64_t)gridDim.x * kWarps;
  bool bad = false, waited = false;
  // chunk j is flag chunk fb = floor(j nfc / nch) when floor((j + 1) nfc / nch)
  // > fb, i.e. when r + nfc >= nch with r = j nfc - fb nch, else element
  // chunk j - fb (the flag chunks before it are fb); fb and r advance by the
  // quotient and remainder of wstride nfc / nch from one chunk of the warp to
  // the next (Bresenham's interleave, no division in the loop)
  const int64_t j0 = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  int64_t fb = j0 * nfc / nch, r = j0 * nfc - fb * nch;
  const int64_t qw = wstride * nfc / nch, rw = wstride * nfc - qw * nch;
  for (int64_t j = j0; j < nch; j += wstride) {
    const bool flag_chunk = r + nfc >= nch;
    const int64_t fcur = fb;
    fb += qw;
    r += rw;
    if (r >= nch) {
      r -= nch;
      ++fb;
    }
    if (flag_chunk) {
      // 32-bit indices: the launcher keeps the coordinate DoFs and the items below 2^31
      const uint32_t d0 = (uint32_t)fcur * (uint32_t)(UF * 32) + (uint32_t)lane;
      long long x[UF], y[UF], z[UF], rx[UF], ry[UF], rz[UF];
      bool v[UF];
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const uint32_t d = d0 + (uint32_t)(u * 32);
        v[u] = d < ncoord;
        x[u] = y[u] = z[u] = rx[u] = ry[u] = rz[u] = 0;
        if (v[u]) {
          const uint32_t q = fdiv(d, colv);
          const uint32_t m = d - q * colv.d;
          const double *xp = p.X + 3 * (size_t)d;
          const double *bp = p.base_xy + 2 * (size_t)q;
          x[u] = __double_as_longlong(__ldg(xp + 0));
          y[u] = __double_as_longlong(__ldg(xp + 1));
          z[u] = __double_as_longlong(__ldg(xp + 2));
          rx[u] = __double_as_longlong(__ldg(bp + 0));
          ry[u] = __double_as_longlong(__ldg(bp + 1));
          rz[u] = __double_as_longlong(ztab[m]);
        }
      }
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const uint32_t w = (uint32_t)fcur * (uint32_t)UF + (uint32_t)u;
        const unsigned int word = __ballot_sync(0xffffffffu, v[u] && x[u] == rx[u] && y[u] == ry[u] && z[u] == rz[u]);
        const unsigned int want = __ballot_sync(0xffffffffu, v[u]);
        if (w < nwords) {
          if (lane == 0) flags[w] = word;
          bad |= word != want;
        }
      }
    } else {
      if (!waited) {  // launched as a dependent of k_tp_area2: its |2A| must be complete
        grid_dep_wait();
        waited = true;
      }
      const uint32_t i0 = (uint32_t)(j - fcur) * (uint32_t)(32 * UI) + (uint32_t)lane;
      int32_t dof[UI][K];
      double a2[UI], h[UI], f[UI][K];
      bool v[UI];
#pragma unroll
      for (int u = 0; u < UI; ++u) {
        const uint32_t it = i0 + (uint32_t)(u * 32);
        v[u] = it < nitems;
        a2[u] = h[u] = 0.0;
        if (v[u]) {
          const uint32_t c = fdiv(it, lay);
          const int l = (int)(it - c * lay.d);
          a2[u] = __ldg(area2 + c);
          h[u] = hs[l];
          const int32_t *row = p.fmap + (size_t)c * (uint32_t)p.k;
#pragma unroll
          for (int i = 0; i < K; ++i) dof[u][i] = __ldg(row + p.slot[i]) + l * p.off[i];
        }
      }
#pragma unroll
      for (int u = 0; u < UI; ++u) {
#pragma unroll
        for (int i = 0; i < K; ++i) f[u][i] = v[u] ? __ldg(p.f + (uint32_t)dof[u][i]) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < UI; ++u) {
        if (!v[u]) continue;
        double b[K];
        tp_closed<NH, NV>(fmul(a2[u], h[u], p.k1), f[u], b, p.k1);
#pragma unroll
        for (int i = 0; i < K; ++i) p.b[(uint32_t)dof[u][i]] = b[i];
      }
    }
  }
  // a thread that took only flag chunks still waits for k_tp_area2 before it
  // ends, so that the launches after this one find it complete as well
  if (!waited) grid_dep_wait();
  // one word per CTA (every CTA writes its own, so nothing needs clearing first)
  if (bad && lane == 0) cta_bad = 1;
  __syncthreads();
  if (threadIdx.x == 0) badv[blockIdx.x] = cta_bad;
}

// grid of the optimistic launch: resident CTAs per SM x SMs, at most the chunk count
template <int NH, int NV>
int64_t dgdg_grid(const MassTPLaunch &p, size_t smem) {
  static int resident = 0, sms = 0;
  static size_t at = 0;
  if (resident == 0 || at != smem) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_tp_dgdg<NH, NV>, kWarps * 32, smem);
    if (resident < 1) resident = 1;
    at = smem;
  }
  const int64_t nfc = ((p.ncoord + 31) / 32 + dgdg_uf(NH * NV) - 1) / dgdg_uf(NH * NV);
  const int64_t nic = (p.ncells * (int64_t)p.layers + 32 * dgdg_ui(NH * NV) - 1) / (32 * dgdg_ui(NH * NV));
  int64_t blocks = (nfc + nic + kWarps - 1) / kWarps;
  if (blocks > (int64_t)resident * sms) blocks = (int64_t)resident * sms;
  return blocks < 1 ? 1 : blocks;
}

template <int NH, int NV>
cudaError_t launch_tp_dgdg(const MassTPLaunch &p, const double *area2, uint32_t *flags, int32_t *badv, int64_t blocks,
                           size_t smem, cudaStream_t s) {
  const int64_t nfc = ((p.ncoord + 31) / 32 + dgdg_uf(NH * NV) - 1) / dgdg_uf(NH * NV);
  const int64_t nic = (p.ncells * (int64_t)p.layers + 32 * dgdg_ui(NH * NV) - 1) / (32 * dgdg_ui(NH * NV));
  return launch_dependent(k_tp_dgdg<NH, NV>, dim3((unsigned)blocks), dim3(kWarps * 32), smem, s, p, area2, flags,
                          badv, make_fastdiv((uint32_t)(p.layers + 1)), make_fastdiv((uint32_t)p.layers), nfc, nic);
}

// Optimistic WRITE form for DG x CG1 on constant layers (horizontal DG0 or
// DG1, vertical CG1: the DoFs of a cell column are its own, consecutive
// layers share their facet DoFs).  Summed over the two prisms at level m of a
// straight column, the element vectors give
//   b_{m,a} = coef (g_a + [NH = 3] sum_a' g_a'),
//   g_a = lo_m f_{m-1,a} + mid_m f_{m,a} + hi_m f_{m+1,a}
// with (lo, mid, hi) = (|h_{m-1}|, 2 (|h_{m-1}| + |h_m|), |h_m|) (zero beyond
// the column's ends) and coef = |2A| x the element's constant (1/12 for DG0,
// 1/144 for DG1), so one lane per (column, level) item writes the NH DoFs of
// its level once: no atomics and no clearing of b, 4 (DG0) or 15 (DG1) FP64
// operations per item.  The DoF of node a at level m is the column's first
// DoF + NH m + a (Algorithm 1: the NH facet DoFs of a level together).  As in
// k_tp_dgdg the straightness flags are set in the same launch (flag chunks
// interleaved with item chunks), |2A| comes from k_tp_area2 and the level
// table from the reference column; the fix-up (k_mass_tp_levels with FIX)
// rewrites every column not straight at every level.
template <int NH>
__global__ void __launch_bounds__(kWarps * 32, NH == 1 ? 4 : 3)
    k_dgcg_opt(const MassTPLaunch p, const double *__restrict__ area2, uint32_t *__restrict__ flags,
               int32_t *__restrict__ badv, FastDiv colv, int64_t nfc, int64_t nic) {
  constexpr int UF = 2, UI = 2;  // flag words, items per lane per chunk
  // level table of the reference column: z, lo, mid, hi per level
  extern __shared__ double lvl[];
  const int L1 = p.layers + 1;
  double *ztab = lvl, *tlo = lvl + L1, *tmid = lvl + 2 * L1, *thi = lvl + 3 * L1;
  __shared__ int cta_bad;
  for (int m = threadIdx.x; m < L1; m += blockDim.x) ztab[m] = __ldg(p.X + 3 * (int64_t)m + 2);
  if (threadIdx.x == 0) cta_bad = 0;
  __syncthreads();
  for (int m = threadIdx.x; m < L1; m += blockDim.x) {
    const double lo = m > 0 ? fabs(ztab[m] - ztab[m - 1]) : 0.0;
    const double hi = m < p.layers ? fabs(ztab[m + 1] - ztab[m]) : 0.0;
    tlo[m] = lo;
    thi[m] = hi;
    tmid[m] = 2.0 * (lo + hi);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t ncoord = (uint32_t)p.ncoord, nwords = (uint32_t)((p.ncoord + 31) / 32);
  const uint32_t nitems = (uint32_t)(p.ncells * (int64_t)L1);
  const int64_t nch = nfc + nic;
  const int64_t wstride = (int64_t)gridDim.x * kWarps;
  bool bad = false, waited = false;
  const int64_t j0 = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  int64_t fb = j0 * nfc / nch, r = j0 * nfc - fb * nch;
  const int64_t qw = wstride * nfc / nch, rw = wstride * nfc - qw * nch;
  for (int64_t j = j0; j < nch; j += wstride) {
    const bool flag_chunk = r + nfc >= nch;
    const int64_t fcur = fb;
    fb += qw;
    r += rw;
    if (r >= nch) {
      r -= nch;
      ++fb;
    }
    if (flag_chunk) {
      const uint32_t d0 = (uint32_t)fcur * (uint32_t)(UF * 32) + (uint32_t)lane;
      long long x[UF], y[UF], z[UF], rx[UF], ry[UF], rz[UF];
      bool v[UF];
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const uint32_t d = d0 + (uint32_t)(u * 32);
        v[u] = d < ncoord;
        x[u] = y[u] = z[u] = rx[u] = ry[u] = rz[u] = 0;
        if (v[u]) {
          const uint32_t q = fdiv(d, colv);
          const uint32_t m = d - q * colv.d;
          const double *xp = p.X + 3 * (size_t)d;
          const double *bp = p.base_xy + 2 * (size_t)q;
          x[u] = __double_as_longlong(__ldg(xp + 0));
          y[u] = __double_as_longlong(__ldg(xp + 1));
          z[u] = __double_as_longlong(__ldg(xp + 2));
          rx[u] = __double_as_longlong(__ldg(bp + 0));
          ry[u] = __double_as_longlong(__ldg(bp + 1));
          rz[u] = __double_as_longlong(ztab[m]);
        }
      }
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const uint32_t w = (uint32_t)fcur * (uint32_t)UF + (uint32_t)u;
        const unsigned int word = __ballot_sync(0xffffffffu, v[u] && x[u] == rx[u] && y[u] == ry[u] && z[u] == rz[u]);
        const unsigned int want = __ballot_sync(0xffffffffu, v[u]);
        if (w < nwords) {
          if (lane == 0) flags[w] = word;
          bad |= word != want;
        }
      }
    } else {
      if (!waited) {  // launched as a dependent of k_tp_area2: its |2A| must be complete
        grid_dep_wait();
        waited = true;
      }
      const uint32_t i0 = (uint32_t)(j - fcur) * (uint32_t)(32 * UI) + (uint32_t)lane;
      int64_t dof[UI];
      double fc[UI][NH], fp[UI][NH], fn[UI][NH], co[UI];
      int ms[UI];
      bool v[UI];
#pragma unroll
      for (int u = 0; u < UI; ++u) {
        const uint32_t it = i0 + (uint32_t)(u * 32);
        v[u] = it < nitems;
        co[u] = 0.0;
        ms[u] = 0;
        dof[u] = 0;
        if (v[u]) {
          const uint32_t c = fdiv(it, colv);
          ms[u] = (int)(it - c * colv.d);
          co[u] = fmul(__ldg(area2 + c), p.scale, p.k1);
          dof[u] = (int64_t)__ldg(p.fmap + (int64_t)c * p.k + p.slot[0]) + (int64_t)NH * ms[u];
        }
      }
#pragma unroll
      for (int u = 0; u < UI; ++u) {
#pragma unroll
        for (int a = 0; a < NH; ++a) {
          fc[u][a] = v[u] ? __ldg(p.f + dof[u] + a) : 0.0;
          fp[u][a] = v[u] && ms[u] > 0 ? __ldg(p.f + dof[u] - NH + a) : 0.0;
          fn[u][a] = v[u] && ms[u] < p.layers ? __ldg(p.f + dof[u] + NH + a) : 0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < UI; ++u) {
        if (!v[u]) continue;
        const int m = ms[u];
        double g[NH];
#pragma unroll
        for (int a = 0; a < NH; ++a) g[a] = fma(tlo[m], fp[u][a], fma(tmid[m], fc[u][a], fmul(thi[m], fn[u][a], p.k1)));
        if (NH == 1) {
          p.b[dof[u]] = fmul(co[u], g[0], p.k1);
        } else {
          const double cS = fmul(co[u], fadd(fadd(g[0], g[1 % NH], p.k1), g[2 % NH], p.k1), p.k1);
#pragma unroll
          for (int a = 0; a < NH; ++a) p.b[dof[u] + a] = fma(co[u], g[a], cS);
        }
      }
    }
  }
  if (!waited) grid_dep_wait();  // as in k_tp_dgdg: the later launches rely on k_tp_area2 being complete
  if (bad && lane == 0) cta_bad = 1;
  __syncthreads();
  if (threadIdx.x == 0) badv[blockIdx.x] = cta_bad;
}

template <int NH>
int64_t dgcg_grid(const MassTPLaunch &p, size_t smem) {
  static int resident = 0, sms = 0;
  static size_t at = 0;
  if (resident == 0 || at != smem) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_dgcg_opt<NH>, kWarps * 32, smem);
    if (resident < 1) resident = 1;
    at = smem;
  }
  const int64_t nfc = ((p.ncoord + 31) / 32 + 1) / 2;
  const int64_t nic = (p.ncells * ((int64_t)p.layers + 1) + 63) / 64;
  int64_t blocks = (nfc + nic + kWarps - 1) / kWarps;
  if (blocks > (int64_t)resident * sms) blocks = (int64_t)resident * sms;
  return blocks < 1 ? 1 : blocks;
}

template <int NH, int NV, bool VAR, bool FLAGS, bool MULTI, bool WR = false, bool FIX = false>
cudaError_t launch_tp(const MassTPLaunch &p, cudaStream_t s) {
  const double lay = VAR ? p.mean_layers : (double)p.layers;
  int cpw = (int)((EXT_TP_ITEMS + lay - 1.0) / lay);
  if (cpw < 1) cpw = 1;
  if (cpw > kMaxCols) cpw = kMaxCols;
  const int64_t warps = (p.ncells + cpw - 1) / cpw;
  int64_t blocks = (warps + kWarps - 1) / kWarps;
  static int resident[64] = {0}, sms = 0;
  const int slot = (NH == 3 ? 2 : 0) + (NV == 2 ? 1 : 0) + (VAR ? 4 : 0) + (FLAGS ? 8 : 0) + (MULTI ? 4 : 0) +
                   (WR ? 16 : 0) + (FIX ? 32 : 0);
  if (resident[slot] == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident[slot], k_mass_tp<NH, NV, VAR, FLAGS, MULTI, WR, FIX>,
                                                  kWarps * 32, 0);
    if (resident[slot] < 1) resident[slot] = 1;
  }
  if (blocks > (int64_t)resident[slot] * sms) blocks = (int64_t)resident[slot] * sms;
  if (FIX) return launch_dependent(k_mass_tp<NH, NV, VAR, FLAGS, MULTI, WR, FIX>, dim3((unsigned)blocks),
                                   dim3(kWarps * 32), 0, s, p, cpw);
  k_mass_tp<NH, NV, VAR, FLAGS, MULTI, WR, FIX><<<(unsigned)blocks, kWarps * 32, 0, s>>>(p, cpw);
  return cudaGetLastError();
}

// the flagged form takes several items per lane from EXT_TP_MULTI_LAYERS
// layers on (a warp's group of up to 32 columns then fills the lanes' slots)
#ifndef EXT_TP_MULTI_LAYERS
#define EXT_TP_MULTI_LAYERS 8
#endif
template <bool VAR, bool FLAGS, bool MULTI, bool WR = false, bool FIX = false>
cudaError_t launch_tp_kind(const MassTPLaunch &p, cudaStream_t s) {
  if (p.nh == 1 && p.nv == 1) return launch_tp<1, 1, VAR, FLAGS, MULTI, WR, FIX>(p, s);
  if (p.nh == 1) return launch_tp<1, 2, VAR, FLAGS, MULTI, WR, FIX>(p, s);
  if (p.nv == 1) return launch_tp<3, 1, VAR, FLAGS, MULTI, WR, FIX>(p, s);
  return launch_tp<3, 2, VAR, FLAGS, MULTI, WR, FIX>(p, s);
}
template <bool VAR, bool FLAGS, bool WR = false>
cudaError_t launch_tp_pair(const MassTPLaunch &p, cudaStream_t s) {
  if (FLAGS && !VAR && p.layers >= EXT_TP_MULTI_LAYERS) return launch_tp_kind<VAR, FLAGS, true, WR>(p, s);
  return launch_tp_kind<VAR, FLAGS, false, WR>(p, s);
}

// DG0 x CG1 and DG1 x CG1 on constant layers: the DoFs of a cell column are
// its own (horizontal DG), and layers l and l + 1 share the DoFs of the
// facet between them (vertical CG1).  A warp walks its group's flattened
// items (column, level m), m = 0..layers, lanes along the levels; the lane of
// level m < layers evaluates prism (c, m) once (closed form when its six
// coordinate flags are set, tp_general otherwise), keeps the bottom row
// (level m) and hands the top row (level m + 1) one lane up by a warp
// shuffle (the step's last lane to the next step).  Every DoF is then formed
// in registers by one lane and written once: stored (WR) or added with one
// fire-and-forget reduction.
// FIX (with FLAGS and WR): the fix-up of the optimistic DG x CG1 form, which
// rewrites only the columns not straight at every level (and returns at once
// when no CTA of that launch saw a coordinate DoF that is not straight).
template <int NH, bool FLAGS, bool WR, bool FIX = false>
__global__ void __launch_bounds__(kWarps * 32, 2) k_mass_tp_levels(const MassTPLaunch p, int cpw) {
  __shared__ TPCol cols[kWarps][kMaxCols];
  if (FIX) {
    grid_dep_wait();  // launched as a dependent of the optimistic launch
    int any = 0;
    for (int i = threadIdx.x; i < p.nbadv; i += blockDim.x) any |= __ldg(p.badv + i);
    if (!__syncthreads_or(any)) return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int layers = p.layers, L1 = layers + 1;
  const int64_t ngroups = (p.ncells + cpw - 1) / cpw;
  const int64_t wstride = (int64_t)gridDim.x * kWarps;
  for (int64_t grp = (int64_t)blockIdx.x * kWarps + warp; grp < ngroups; grp += wstride) {
    const int64_t c0 = grp * cpw;
    const int ncol = (int)(p.ncells - c0 < cpw ? p.ncells - c0 : (int64_t)cpw);
    if (lane < ncol) {
      const int64_t c = c0 + lane;
      TPCol &ci = cols[warp][lane];
      ci.lay = layers;
      double x[3], y[3];
#pragma unroll
      for (int i = 0; i < 6; ++i) ci.cm[i] = __ldg(p.cmap + c * 6 + i);
#pragma unroll
      for (int i = 0; i < NH * 2; ++i) ci.fm[i] = __ldg(p.fmap + c * p.k + p.slot[i]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int64_t cd = ci.cm[2 * a];
        if (FLAGS) {
          const int64_t v = cd / L1;
          x[a] = __ldg(p.base_xy + 2 * v + 0);
          y[a] = __ldg(p.base_xy + 2 * v + 1);
        } else {
          x[a] = __ldg(p.X + 3 * cd + 0);
          y[a] = __ldg(p.X + 3 * cd + 1);
        }
        ci.rx[a] = __double_as_longlong(x[a]);
        ci.ry[a] = __double_as_longlong(y[a]);
      }
      ci.alpha = fabs((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0])) * p.scale;
      // all three vertex columns straight at every level: no per-item test
      ci.allok = FLAGS ? vflags_all(p.vflags, ci.cm[0], L1) & vflags_all(p.vflags, ci.cm[2], L1) &
                             vflags_all(p.vflags, ci.cm[4], L1)
                       : 0;
    }
    __syncwarp();
    const int nitems = ncol * L1;
    double carry[NH];
#pragma unroll
    for (int a = 0; a < NH; ++a) carry[a] = 0.0;
    // U steps of 32 items per pass: every load of the pass (flags, layer
    // heights, f at both levels of each prism) is issued before any
    // arithmetic, then the steps are finished in order (the carry runs from
    // one step's last lane to the next step's first)
    constexpr int U = EXT_TP_UNROLL;
    for (int base = 0; base < nitems; base += 32 * U) {
      double f[U][NH * 2], hl[U];
      int ok[U], ms[U], cls[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int it = base + u * 32 + lane;
        const bool valid = it < nitems;
        cls[u] = valid ? it / L1 : 0;
        ms[u] = valid ? it - cls[u] * L1 : L1;
        ok[u] = 1;
        hl[u] = 0.0;
        const TPCol &ci = cols[warp][cls[u]];
        if (ms[u] < layers) {
#pragma unroll
          for (int i = 0; i < NH * 2; ++i) f[u][i] = __ldg(p.f + ci.fm[i] + ms[u] * p.off[i]);
          if (FLAGS) {
            if (!ci.allok) {
#pragma unroll
              for (int i = 0; i < 6; ++i) ok[u] &= vflag(p.vflags, (int64_t)ci.cm[i] + (int64_t)ms[u] * p.coff[i]);
            }
            hl[u] = __ldg(p.hlay + ms[u]);
          }
        } else {
#pragma unroll
          for (int i = 0; i < NH * 2; ++i) f[u][i] = 0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int m = ms[u];
        const TPCol &ci = cols[warp][cls[u]];
        double bot[NH], top[NH];
#pragma unroll
        for (int a = 0; a < NH; ++a) bot[a] = top[a] = 0.0;
        if (m < layers) {
          double b[NH * 2];
          int okp = ok[u];
          double Xl[6][3];
          if (!FLAGS || !okp) {
#pragma unroll
            for (int i = 0; i < 6; ++i) {
              const int64_t cd = (int64_t)ci.cm[i] + (int64_t)m * p.coff[i];
              Xl[i][0] = __ldg(p.X + 3 * cd + 0);
              Xl[i][1] = __ldg(p.X + 3 * cd + 1);
              Xl[i][2] = __ldg(p.X + 3 * cd + 2);
            }
            if (!FLAGS) {
#pragma unroll
              for (int i = 0; i < 6; ++i)
                okp &= (__double_as_longlong(Xl[i][0]) == ci.rx[i >> 1]) &
                       (__double_as_longlong(Xl[i][1]) == ci.ry[i >> 1]);
              okp &= (__double_as_longlong(Xl[0][2]) == __double_as_longlong(Xl[2][2])) &
                     (__double_as_longlong(Xl[0][2]) == __double_as_longlong(Xl[4][2])) &
                     (__double_as_longlong(Xl[1][2]) == __double_as_longlong(Xl[3][2])) &
                     (__double_as_longlong(Xl[1][2]) == __double_as_longlong(Xl[5][2]));
            }
          }
          if (okp) tp_closed<NH, 2>(fmul(ci.alpha, FLAGS ? hl[u] : fabs(Xl[1][2] - Xl[0][2]), p.k1), f[u], b, p.k1);
          else tp_general<NH, 2>(Xl, f[u], b);
#pragma unroll
          for (int a = 0; a < NH; ++a) {
            bot[a] = b[2 * a];
            top[a] = b[2 * a + 1];
          }
        }
        // the top row of the prism below (lane - 1, or the previous step's
        // last lane); at m = 0 the lane below holds the previous column's top
        // level, which has no prism above it and passes zeros
#pragma unroll
        for (int a = 0; a < NH; ++a) {
          double up = __shfl_up_sync(0xffffffffu, top[a], 1);
          const double last = __shfl_sync(0xffffffffu, top[a], 31);
          if (lane == 0) up = carry[a];
          carry[a] = last;
          bot[a] += up;
        }
        if (base + u * 32 + lane < nitems && !(FIX && ci.allok)) {  // FIX: straight columns keep their values
#pragma unroll
          for (int a = 0; a < NH; ++a) {
            const int64_t d = m < layers ? (int64_t)ci.fm[2 * a] + (int64_t)m * p.off[2 * a]
                                         : (int64_t)ci.fm[2 * a + 1] + (int64_t)(layers - 1) * p.off[2 * a + 1];
            if (WR) p.b[d] = bot[a];
            else atomicAdd(p.b + d, bot[a]);
          }
        }
      }
    }
    __syncwarp();
  }
}

template <int NH, bool FLAGS, bool WR, bool FIX = false>
cudaError_t launch_tp_levels(const MassTPLaunch &p, cudaStream_t s) {
  const double L1 = (double)p.layers + 1.0;
  int cpw = (int)((EXT_TP_ITEMS + L1 - 1.0) / L1);
  if (cpw < 1) cpw = 1;
  if (cpw > kMaxCols) cpw = kMaxCols;
  const int64_t warps = (p.ncells + cpw - 1) / cpw;
  int64_t blocks = (warps + kWarps - 1) / kWarps;
  static int resident = 0, sms = 0;
  if (resident == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_mass_tp_levels<NH, FLAGS, WR, FIX>, kWarps * 32, 0);
    if (resident < 1) resident = 1;
  }
  if (blocks > (int64_t)resident * sms) blocks = (int64_t)resident * sms;
  if (FIX)
    return launch_dependent(k_mass_tp_levels<NH, FLAGS, WR, FIX>, dim3((unsigned)blocks), dim3(kWarps * 32), 0, s, p,
                            cpw);
  k_mass_tp_levels<NH, FLAGS, WR, FIX><<<(unsigned)blocks, kWarps * 32, 0, s>>>(p, cpw);
  return cudaGetLastError();
}

template <bool FLAGS>
cudaError_t launch_tp_owned(const MassTPLaunch &p, cudaStream_t s) {
  if (p.vcont) {  // DG x CG1: the level kernel
    if (p.nh == 1) return p.overwrite ? launch_tp_levels<1, FLAGS, true>(p, s) : launch_tp_levels<1, FLAGS, false>(p, s);
    return p.overwrite ? launch_tp_levels<3, FLAGS, true>(p, s) : launch_tp_levels<3, FLAGS, false>(p, s);
  }
  // DG x DG: every DoF in one cell-layer
  return p.overwrite ? launch_tp_pair<false, FLAGS, true>(p, s) : launch_tp_pair<false, FLAGS, false>(p, s);
}



// p-adaptive DG (EXT_K_MASS_DGP): every cell carries its own element, DG0|DG1
// x DG0|DG1, told apart by its DoF count K = NH NV (1, 2, 3, 6).  The library
// keeps the cells of each kind in a list and launches one kernel per kind
// over its list, so a warp never mixes elements.  Node (a, b) is DoF a NV + b
// of the cell's block, and the blocks of a column follow each other layer by
// layer (Algorithm 1), so layer l's block starts at row[0] + l K.  One lane
// per (column, layer) item as in k_mass_tp; the element vector is the closed
// form on a straight prism, tp_general otherwise.  Each block belongs to one
// cell-layer; the increments still go out as reductions (no load of b waits
// on the lane).
struct DGPCol {
  double cc0;              // |2A| / 2 x (1/12 if NH = 3) x (1/6 if NV = 2): cc = cc0 |h|
  long long rx[3], ry[3];
  int32_t cm[6];
  int32_t blk;             // first DoF of the column's block at its bottom layer
  int lay;
};

template <int NH, int NV, bool VAR>
__global__ void __launch_bounds__(kWarps * 32, 2) k_mass_dgp(const MassDGPLaunch p, int cpw) {
  constexpr int K = NH * NV;
  __shared__ DGPCol cols[kWarps][kMaxCols];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int layers = p.layers;
  const int64_t ngroups = (p.ncells + cpw - 1) / cpw;
  const int64_t wstride = (int64_t)gridDim.x * kWarps;
  for (int64_t grp = (int64_t)blockIdx.x * kWarps + warp; grp < ngroups; grp += wstride) {
    const int64_t i0 = grp * cpw;
    const int ncol = (int)(p.ncells - i0 < cpw ? p.ncells - i0 : (int64_t)cpw);
    int my_items = 0;
    if (lane < ncol) {
      const int64_t c = __ldg(p.cells + i0 + lane);
      DGPCol &ci = cols[warp][lane];
      const int lay = VAR ? __ldg(p.cell_layers + c) : layers;
      ci.lay = lay;
      my_items = lay;
      ci.blk = __ldg(p.fmap + __ldg(p.rowptr + c));
      double x[3], y[3];
#pragma unroll
      for (int q = 0; q < 6; ++q) ci.cm[q] = __ldg(p.cmap + c * 6 + q);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        x[a] = __ldg(p.X + 3 * (int64_t)ci.cm[2 * a] + 0);
        y[a] = __ldg(p.X + 3 * (int64_t)ci.cm[2 * a] + 1);
        ci.rx[a] = __double_as_longlong(x[a]);
        ci.ry[a] = __double_as_longlong(y[a]);
      }
      ci.cc0 = fabs((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0])) *
               (0.5 * (NH == 3 ? 1.0 / 12.0 : 1.0) * (NV == 2 ? 1.0 / 6.0 : 1.0));
    }
    __syncwarp();
    const int nitems = VAR ? __reduce_add_sync(0xffffffffu, my_items) : ncol * layers;
    int cl, l;
    if (VAR) {
      cl = 0;
      l = lane;
      while (cl < ncol && l >= cols[warp][cl].lay) { l -= cols[warp][cl].lay; ++cl; }
    } else {
      cl = lane / layers;
      l = lane - cl * layers;
    }
    for (int base = 0; base < nitems; base += 32) {
      if (base + lane < nitems) {
        const DGPCol &ci = cols[warp][cl];
        double Xl[6][3];
        int ok = 1;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const int64_t cd = (int64_t)ci.cm[q] + (int64_t)l * p.coff[q];
          Xl[q][0] = __ldg(p.X + 3 * cd + 0);
          Xl[q][1] = __ldg(p.X + 3 * cd + 1);
          Xl[q][2] = __ldg(p.X + 3 * cd + 2);
          ok &= (__double_as_longlong(Xl[q][0]) == ci.rx[q >> 1]) & (__double_as_longlong(Xl[q][1]) == ci.ry[q >> 1]);
        }
        ok &= (__double_as_longlong(Xl[0][2]) == __double_as_longlong(Xl[2][2])) &
              (__double_as_longlong(Xl[0][2]) == __double_as_longlong(Xl[4][2])) &
              (__double_as_longlong(Xl[1][2]) == __double_as_longlong(Xl[3][2])) &
              (__double_as_longlong(Xl[1][2]) == __double_as_longlong(Xl[5][2]));
        const int64_t blk = (int64_t)ci.blk + (int64_t)l * K;
        double f[K], b[K];
#pragma unroll
        for (int j = 0; j < K; ++j) f[j] = __ldg(p.f + blk + j);
        const double cc = ci.cc0 * fabs(Xl[1][2] - Xl[0][2]);
        if (ok) {
          if (NH == 1 && NV == 1) {
            b[0] = cc * f[0];
          } else if (NH == 1) {
            const double c2 = cc + cc;
            b[0] = fma(c2, f[0], cc * f[1]);
            b[K - 1] = fma(c2, f[K - 1], cc * f[0]);
          } else if (NV == 1) {
            const double cS = cc * ((f[0] + f[1 % K]) + f[2 % K]);
#pragma unroll
            for (int a = 0; a < K; ++a) b[a] = fma(cc, f[a], cS);
          } else {
            double t[K];
#pragma unroll
            for (int a = 0; a < K / 2; ++a) {
              t[2 * a] = fma(2.0, f[2 * a], f[2 * a + 1]);
              t[2 * a + 1] = fma(2.0, f[2 * a + 1], f[2 * a]);
            }
            const double K0 = cc * ((t[0] + t[2 % K]) + t[4 % K]), K1 = cc * ((t[1 % K] + t[3 % K]) + t[5 % K]);
#pragma unroll
            for (int q = 0; q < K; ++q) b[q] = fma(cc, t[q], (q & 1) ? K1 : K0);
          }
        } else {
          tp_general<NH, NV>(Xl, f, b);
        }
#pragma unroll
        for (int j = 0; j < K; ++j) atomicAdd(p.b + blk + j, b[j]);
      }
      l += 32;
      if (VAR) {
        while (cl < ncol && l >= cols[warp][cl].lay) { l -= cols[warp][cl].lay; ++cl; }
      } else {
        while (l >= layers) { l -= layers; ++cl; }
      }
    }
    __syncwarp();
  }
}

template <int NH, int NV, bool VAR>
cudaError_t launch_dgp(const MassDGPLaunch &p, cudaStream_t s) {
  const double lay = VAR ? p.mean_layers : (double)p.layers;
  int cpw = (int)((EXT_TP_ITEMS + lay - 1.0) / lay);
  if (cpw < 1) cpw = 1;
  if (cpw > kMaxCols) cpw = kMaxCols;
  const int64_t warps = (p.ncells + cpw - 1) / cpw;
  int64_t blocks = (warps + kWarps - 1) / kWarps;
  static int resident = 0, sms = 0;
  if (resident == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_mass_dgp<NH, NV, VAR>, kWarps * 32, 0);
    if (resident < 1) resident = 1;
  }
  if (blocks > (int64_t)resident * sms) blocks = (int64_t)resident * sms;
  k_mass_dgp<NH, NV, VAR><<<(unsigned)blocks, kWarps * 32, 0, s>>>(p, cpw);
  return cudaGetLastError();
}

template <bool VAR>
cudaError_t launch_dgp_kind(const MassDGPLaunch &p, cudaStream_t s) {
  switch (p.kind) {
    case 1: return launch_dgp<1, 1, VAR>(p, s);
    case 2: return launch_dgp<1, 2, VAR>(p, s);
    case 3: return launch_dgp<3, 1, VAR>(p, s);
    case 6: return launch_dgp<3, 2, VAR>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

// CG1 x DG recorded DoFs (the gather path's fix-up): b of vertex a, layer l,
// node beta = the sum over the cells around a of entry (a, beta) of prism
// (c, l)'s element vector by the general 6-point rule, in ascending cell
// order; one warp per 32-DoF record, one lane per DoF.
template <int NV>
__global__ void __launch_bounds__(kWarps * 32) k_cgdg_general(const MassTPLaunch p, const int2 *__restrict__ list,
                                                              const unsigned int *__restrict__ count, unsigned int cap,
                                                              FastDiv dcol, FastDiv col) {
  grid_dep_wait();  // a programmatic dependent of the launch before it
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned int nrec = min(*count, cap);
  for (unsigned int e = blockIdx.x * kWarps + warp; e < nrec; e += gridDim.x * kWarps) {
    const int2 en = list[e];
    if ((((unsigned int)en.y) >> lane & 1u) == 0u) continue;
    const uint32_t d = (uint32_t)en.x + (uint32_t)lane;
    const uint32_t q = fdiv(d, dcol);
    const uint32_t r = d - q * dcol.d;
    const int l = (int)(NV == 2 ? r >> 1 : r), beta = (int)(NV == 2 ? r & 1u : 0u);
    const int32_t v0 = (int32_t)(q * col.d);  // coordinate DoF of vertex q at level 0
    double acc = 0.0;
    for (int32_t t = __ldg(p.vcrow + q); t < __ldg(p.vcrow + q + 1); ++t) {
      const int64_t c = __ldg(p.vcells + t);
      int ia = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (__ldg(p.cmap + c * 6 + 2 * k) == v0) ia = k;
      double Xl[6][3], fl[3 * NV], out[3 * NV];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const int64_t cd = (int64_t)__ldg(p.cmap + c * 6 + i) + (int64_t)l * p.coff[i];
        Xl[i][0] = __ldg(p.X + 3 * cd + 0);
        Xl[i][1] = __ldg(p.X + 3 * cd + 1);
        Xl[i][2] = __ldg(p.X + 3 * cd + 2);
      }
#pragma unroll
      for (int i = 0; i < 3 * NV; ++i) fl[i] = __ldg(p.f + __ldg(p.fmap + c * p.k + p.slot[i]) + (int64_t)l * p.off[i]);
      tp_general<3, NV>(Xl, fl, out);
      acc += out[ia * NV + beta];
    }
    p.b[d] = acc;
  }
}

// In cell-loop mode only: b cleared, then the (unflagged) cell kernel with
// FP64 reductions.
__global__ void __launch_bounds__(256) k_tp_clear_cells(double *__restrict__ b, int64_t n,
                                                        const unsigned int *__restrict__ mode) {
  if ((*mode & 3u) != 3u) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = 0.0;
}

}  // namespace

// The flagged form runs on constant layers when the mesh has base
// coordinates and the launch has a million (column, layer) items or more
// (EXTMESH_TP_FLAGS=1 / 0, read once per process: at any size / never), and
// its scratch (one bit per coordinate DoF and two level tables) can be taken
// from the stream-ordered pool; otherwise every lane loads its coordinates.
cudaError_t launch_mass_tp(const MassTPLaunch &p, cudaStream_t s) {
  if (p.ncells == 0) return cudaSuccess;
  // CG1 x DG0 / CG1 x DG1 with WRITE on constant layers from
  // EXT_GATHER_MIN_LAYERS layers: the gather path (no atomics, no clearing;
  // EXTMESH_TP_CGDG=0, read once per process, keeps the cell kernel)
  static int cgdg_env = -1;
  if (cgdg_env < 0) {
    const char *ev = getenv("EXTMESH_TP_CGDG");
    cgdg_env = (ev && ev[0] == '0') ? 0 : 1;
  }
  if (cgdg_env == 1 && p.overwrite && p.nh == 3 && !p.hown && !p.vcont && !p.cell_layers && p.vrow && p.vnbr &&
      p.vedge && p.vcrow && p.vcells && p.nvent > 0 && p.layers >= EXT_GATHER_MIN_LAYERS &&
      (double)p.nf < 2147483647.0 && (double)p.ncoord < 2147483647.0)
    return launch_mass_cgdg(p, s);
  // DG x CG1 takes the atomic form (FP64 reductions into the shared facet
  // DoFs, b cleared first for WRITE), which measured 5-10 % faster at 10 and
  // 100 layers than the level kernel that merges the shared DoFs in
  // registers; EXTMESH_TP_LEVELS=1 (read once per process) selects the level
  // kernel on constant layers
  static int levels_env = -1;
  if (levels_env < 0) {
    const char *ev = getenv("EXTMESH_TP_LEVELS");
    levels_env = (ev && ev[0] == '1') ? 1 : 0;
  }
  // the forms that add into shared DoFs with atomics (horizontal CG1, variable
  // layers) clear b first for WRITE
  const bool owned = p.hown && !p.cell_layers && (!p.vcont || levels_env == 1);
  static int flags_env = -1;
  if (flags_env < 0) {
    const char *ev = getenv("EXTMESH_TP_FLAGS");
    flags_env = (ev && ev[0] == '1') ? 1 : ((ev && ev[0] == '0') ? 0 : 2);
  }
  const double items = (double)p.ncells * (double)p.layers;
  const bool want = !p.cell_layers && p.base_xy && p.ncoord > 0 && flags_env != 0 && (flags_env == 1 || items >= 1.0e6);
  // the optimistic forms (WRITE, constant layers from EXT_TP_MULTI_LAYERS,
  // 32-bit item and DoF indices; EXTMESH_TP_OPTIMISTIC=0, read once per
  // process, turns them off): DG x DG (every DoF in one cell-layer) up to
  // EXT_TP_DGDG_MAX_LAYERS layers, DG x CG1 (the level-merged form, no
  // clearing of b) up to EXT_TP_DGCG_MAX_LAYERS
  static int opt_env = -1;
  if (opt_env < 0) {
    const char *ev = getenv("EXTMESH_TP_OPTIMISTIC");
    opt_env = (ev && ev[0] == '0') ? 0 : 1;
  }
  const bool opt_common = want && opt_env == 1 && p.overwrite && p.hown && p.layers >= EXT_TP_MULTI_LAYERS &&
                          (double)p.ncells * (double)(p.layers + 1) < 2147483647.0 &&
                          (double)p.ncoord < 2147483647.0 && (double)p.nf < 2147483647.0;
  const bool optimistic = opt_common && !p.vcont && p.layers <= EXT_TP_DGDG_MAX_LAYERS;
  const bool opt_dgcg = opt_common && p.vcont && p.layers <= EXT_TP_DGCG_MAX_LAYERS;
  char *scr = nullptr;
  const size_t fbytes = (sizeof(uint32_t) * (size_t)((p.ncoord + 31) / 32) + 255) & ~(size_t)255;
  const size_t zbytes = (sizeof(double) * (size_t)(p.layers + 1) + 255) & ~(size_t)255;
  const size_t smem = optimistic ? sizeof(double) * (size_t)(2 * p.layers + 1)
                                 : sizeof(double) * 4 * (size_t)(p.layers + 1);  // DG x CG1: z, lo, mid, hi
  int64_t oblocks = 0;
  if (optimistic) {
    if (p.nh == 1 && p.nv == 1) oblocks = dgdg_grid<1, 1>(p, smem);
    else if (p.nh == 1) oblocks = dgdg_grid<1, 2>(p, smem);
    else if (p.nv == 1) oblocks = dgdg_grid<3, 1>(p, smem);
    else oblocks = dgdg_grid<3, 2>(p, smem);
  } else if (opt_dgcg) {
    oblocks = p.nh == 1 ? dgcg_grid<1>(p, smem) : dgcg_grid<3>(p, smem);
  }
  const size_t abytes = (sizeof(double) * (size_t)p.ncells + 255) & ~(size_t)255;
  const size_t sbytes = (optimistic || opt_dgcg)
                            ? ((sizeof(int32_t) * (size_t)oblocks + 255) & ~(size_t)255) + abytes + (opt_dgcg ? 2 * zbytes : 0)
                            : 2 * zbytes;
  if (want && cudaMallocAsync(reinterpret_cast<void **>(&scr), fbytes + sbytes, s) != cudaSuccess) {
    (void)cudaGetLastError();  // not sticky: the plain form needs no scratch
    scr = nullptr;
  }
  if (p.overwrite && !owned && !(scr && opt_dgcg)) {
    const cudaError_t ez = cudaMemsetAsync(p.b, 0, sizeof(double) * (size_t)p.nf, s);
    if (ez != cudaSuccess) {
      if (scr) (void)cudaFreeAsync(scr, s);
      return ez;
    }
  }
  if (p.cell_layers) return launch_tp_pair<true, false>(p, s);
  if (!scr) return owned ? launch_tp_owned<false>(p, s) : launch_tp_pair<false, false>(p, s);
  if (opt_dgcg) {
    MassTPLaunch q = p;
    uint32_t *flags = reinterpret_cast<uint32_t *>(scr);
    double *area2 = reinterpret_cast<double *>(scr + fbytes);
    int32_t *badv = reinterpret_cast<int32_t *>(scr + fbytes + abytes);
    static int sms_c = 0;
    if (sms_c == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms_c, cudaDevAttrMultiProcessorCount, dev);
    }
    int64_t ga = (p.ncells + 255) / 256;
    if (ga > (int64_t)sms_c * 8) ga = (int64_t)sms_c * 8;
    if (ga * 256 < (int64_t)p.layers + 1) ga = ((int64_t)p.layers + 1 + 255) / 256;
    const FastDiv colv = make_fastdiv((uint32_t)(p.layers + 1));
    // |2A| per cell, and the fix-up's level tables in the same launch
    double *ztab = reinterpret_cast<double *>(scr + fbytes + abytes + ((sizeof(int32_t) * (size_t)oblocks + 255) & ~(size_t)255));
    double *hlay = ztab + zbytes / sizeof(double);
    k_tp_area2<<<(unsigned)ga, 256, 0, s>>>(p.cmap, p.base_xy, colv, p.ncells, area2, p.X, p.layers, ztab, hlay);
    cudaError_t e = cudaGetLastError();
    const int64_t nfc = ((p.ncoord + 31) / 32 + 1) / 2;
    const int64_t nic = (p.ncells * ((int64_t)p.layers + 1) + 63) / 64;
    if (e == cudaSuccess)
      e = p.nh == 1 ? launch_dependent(k_dgcg_opt<1>, dim3((unsigned)oblocks), dim3(kWarps * 32), smem, s, q, area2,
                                       flags, badv, colv, nfc, nic)
                    : launch_dependent(k_dgcg_opt<3>, dim3((unsigned)oblocks), dim3(kWarps * 32), smem, s, q, area2,
                                       flags, badv, colv, nfc, nic);
    // the fix-up: the level kernel over the columns not straight at every level
    q.vflags = flags;
    q.hlay = hlay;
    q.badv = badv;
    q.nbadv = (int32_t)oblocks;
    if (e == cudaSuccess)
      e = p.nh == 1 ? launch_tp_levels<1, true, true, true>(q, s) : launch_tp_levels<3, true, true, true>(q, s);
    const cudaError_t ef = cudaFreeAsync(scr, s);
    return e != cudaSuccess ? e : ef;
  }
  MassTPLaunch q = p;
  uint32_t *flags = reinterpret_cast<uint32_t *>(scr);
  q.vflags = flags;
  if (optimistic) {
    double *area2 = reinterpret_cast<double *>(scr + fbytes);
    int32_t *badv = reinterpret_cast<int32_t *>(scr + fbytes + abytes);
    static int sms_a = 0;
    if (sms_a == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms_a, cudaDevAttrMultiProcessorCount, dev);
    }
    int64_t ga = (p.ncells + 255) / 256;
    if (ga > (int64_t)sms_a * 8) ga = (int64_t)sms_a * 8;
    k_tp_area2<<<(unsigned)ga, 256, 0, s>>>(p.cmap, p.base_xy, make_fastdiv((uint32_t)(p.layers + 1)), p.ncells, area2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
      if (p.nh == 1 && p.nv == 1) e = launch_tp_dgdg<1, 1>(q, area2, flags, badv, oblocks, smem, s);
      else if (p.nh == 1) e = launch_tp_dgdg<1, 2>(q, area2, flags, badv, oblocks, smem, s);
      else if (p.nv == 1) e = launch_tp_dgdg<3, 1>(q, area2, flags, badv, oblocks, smem, s);
      else e = launch_tp_dgdg<3, 2>(q, area2, flags, badv, oblocks, smem, s);
    }
    q.badv = badv;
    q.nbadv = (int32_t)oblocks;
    if (e == cudaSuccess) e = launch_tp_kind<false, true, true, true, true>(q, s);
    const cudaError_t ef = cudaFreeAsync(scr, s);
    return e != cudaSuccess ? e : ef;
  }
  double *ztab = reinterpret_cast<double *>(scr + fbytes);
  double *hlay = reinterpret_cast<double *>(scr + fbytes + zbytes);
  q.hlay = hlay;
  static int sms = 0, res_vf = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res_vf, k_tp_vflags, 256, 0);
    if (res_vf < 1) res_vf = 1;
  }
  int64_t gv = ((p.ncoord + 31) / 32 + kWarps - 1) / kWarps;
  if (gv > (int64_t)res_vf * sms) gv = (int64_t)res_vf * sms;
  if (gv < 1) gv = 1;
  k_tp_levels<<<(unsigned)((p.layers + 1 + 255) / 256), 256, 0, s>>>(p.X, p.layers, ztab, hlay);
  k_tp_vflags<<<(unsigned)gv, 256, 0, s>>>(p.X, p.base_xy, ztab, p.ncoord, make_fastdiv((uint32_t)(p.layers + 1)), flags);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = owned ? launch_tp_owned<true>(q, s) : launch_tp_pair<false, true>(q, s);
  const cudaError_t ef = cudaFreeAsync(scr, s);
  return e != cudaSuccess ? e : ef;
}

cudaError_t launch_mass_dgp(const MassDGPLaunch &p, cudaStream_t s) {
  if (p.ncells == 0) return cudaSuccess;
  return p.cell_layers ? launch_dgp_kind<true>(p, s) : launch_dgp_kind<false>(p, s);
}

cudaError_t launch_cgdg_general(const MassTPLaunch &p, const int2 *list, const unsigned int *count, unsigned int cap,
                                cudaStream_t s) {
  static int sms = 0, res[2] = {0, 0};
  const int w = p.nv == 2 ? 1 : 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (res[w] == 0) {
    if (p.nv == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res[w], k_cgdg_general<2>, kWarps * 32, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res[w], k_cgdg_general<1>, kWarps * 32, 0);
    if (res[w] < 1) res[w] = 1;
  }
  const dim3 grid((unsigned)(sms * res[w])), block(kWarps * 32);
  const FastDiv dcol = make_fastdiv((uint32_t)(p.nv * p.layers)), col = make_fastdiv((uint32_t)(p.layers + 1));
  if (p.nv == 2) return launch_dependent(k_cgdg_general<2>, grid, block, 0, s, p, list, count, cap, dcol, col);
  return launch_dependent(k_cgdg_general<1>, grid, block, 0, s, p, list, count, cap, dcol, col);
}

cudaError_t launch_tp_cells_gated(const MassTPLaunch &p, const unsigned int *mode, cudaStream_t s) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  int64_t gb = (p.nf + 255) / 256;
  if (gb > (int64_t)sms * 8) gb = (int64_t)sms * 8;
  k_tp_clear_cells<<<(unsigned)(gb > 0 ? gb : 1), 256, 0, s>>>(p.b, p.nf, mode);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  MassTPLaunch q = p;
  q.mode = mode;
  q.vflags = nullptr;
  return launch_tp_pair<false, false>(q, s);
}

