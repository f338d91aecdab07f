// P1xP1 prism par_loop for b_i += int_cell f_h phi_i dx (the residual I_1 of
// Sec. 4.1.1 with f in V; with f := x it is the mass-matrix action y += M x).
//
// Work decomposition (Algorithm 3, layers innermost).  One warp owns a run of
// whole base columns and walks the flattened items (column, vertex level m),
// m = 0..layers, 32 consecutive items per step, so lanes run along a column
// and every load of a column-contiguous field is coalesced.  Item (c, m)
// produces the full contribution of cell column c to the three P1xP1 DoFs at
// level m: the top rows of layer m-1 plus the bottom rows of layer m.  Values
// of level m are loaded once and handed to the neighbouring levels through
// warp shuffles (vertical reuse: the top DoFs of layer l are the bottom DoFs
// of layer l+1); a one-step lookahead supplies level m+1 to the last lane.
// Increments go to the shared vertex columns with FP64 atomic adds, which
// L2 executes.
//
// Arithmetic.  On a straight prism (vertical edges, flat horizontal faces)
// the P1xP1 mass matrix is (A h / 72)(1 + [a = a'])(1 + [b = b']) with A the
// triangle area and h the layer height, i.e. (Mt (x) Ml) with
// Mt = A/12 (1 + [a=a']) and Ml = h/6 (1 + [b=b']).  With s_l = A h_l / 72
// and sigma_m = 2 (s_{m-1} + s_m), the contribution of a cell column to
// vertex a at level m is 2 c_a + c_b + c_c ({a, b, c} = {0, 1, 2}) with
//   c_a = s_{m-1} f_{m-1,a} + sigma_m f_{m,a} + s_m f_{m+1,a}
// (the horizontal factor 1 + [a = a'] applied to the vertical sums c).  The
// kernel computes the three c_a on the FP64 pipe (13 operations per item: 3
// DMUL + 6 DFMA for c, 4 for the layer factors) and leaves the horizontal
// sum to L2: every vertex receives c_a twice and the two other c once as FP64
// atomic adds.  GB300's FP64 pipe (about 2 DFMA per clock per SM) is the
// scarce unit; its L2 executes FP64 atomic adds at about 0.4 T/s, so moving
// the 9 additions of the horizontal sum there shortens the kernel.  The
// algorithmic count of the item is 18 FP64 operations / 29 flops (the same
// sums done in registers).  The kernel checks straightness exactly (bitwise
// compares of the loaded coordinates against the column's level-0 x, y and of
// the three z values of a level); a warp step touching any other prism
// evaluates the element integrals with the full 6-point rule and the general
// Jacobian instead, so any coordinate field is handled.
#include "ext_internal.cuh"

namespace {

constexpr int kWarps = 8;
constexpr int kMaxCols = 32;  // columns per warp (lane j sets up column j)
constexpr unsigned kFull = 0xffffffffu;

#ifndef EXT_MASS_MINB
#define EXT_MASS_MINB 2  // resident CTAs per SM the register budget must allow
#endif
#ifndef EXT_MASS_ITEMS
#define EXT_MASS_ITEMS 1616  // target items (column levels) per column group
#endif

// a + b on the FP64 pipe; with EXT_MASS_ADD_AS_FMA as fma(a, 1, b), which
// rounds identically
__device__ __forceinline__ double dadd(double a, double b) {
#ifdef EXT_MASS_ADD_AS_FMA
  double r;
  asm("fma.rn.f64 %0, %1, 0d3FF0000000000000, %2;" : "=d"(r) : "d"(a), "d"(b));
  return r;
#else
  return a + b;
#endif
}

struct ColInfo {
  int32_t cbot[3], ctop[3];  // coords DoF: vertex a at level 0, and at level `layers`
  int32_t fbot[3], ftop[3];
  int32_t bbot[3], btop[3];
  double alpha;              // |2 A| / 144, so that s = alpha * |h| = A h / 72
  double alpha2;             // 2 alpha
  long long rx[3], ry[3];    // bit patterns of the level-0 x, y of the vertices
  int lay;                   // layers of this column
};

struct Level {
  double f[3];   // field values of the three vertices
  double z;      // z of vertex 0
  int ok;        // level is horizontal and above the column's base vertices
};

__device__ __forceinline__ int dof_at(int32_t bot, int32_t top, int32_t off, int m, int layers) {
  return m < layers ? bot + m * off : top;
}

// 6-point prism rule, general geometry: out_i = sum_q w_q |det J_q| f(x_q) phi_i(x_q),
// stencil order i = 2a + b (vertex a, bottom/top b).
__device__ void prism_general(const double X[6][3], const double f[6], double out[6]) {
  const double tp[3][2] = {{1.0 / 6.0, 1.0 / 6.0}, {2.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 3.0}};
  const double gz[2] = {0.5 - 0.28867513459481288225, 0.5 + 0.28867513459481288225};
  const double w = 1.0 / 12.0;
  for (int i = 0; i < 6; ++i) out[i] = 0.0;
  for (int t = 0; t < 3; ++t) {
    const double lam[3] = {1.0 - tp[t][0] - tp[t][1], tp[t][0], tp[t][1]};
    const double dlx[3] = {-1.0, 1.0, 0.0}, dly[3] = {-1.0, 0.0, 1.0};
    for (int g = 0; g < 2; ++g) {
      const double psi[2] = {1.0 - gz[g], gz[g]};
      const double dpsi[2] = {-1.0, 1.0};
      double J[3][3] = {{0.0}};
      double phi[6];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 2; ++b) {
          const int i = 2 * a + b;
          phi[i] = lam[a] * psi[b];
          const double gr[3] = {dlx[a] * psi[b], dly[a] * psi[b], lam[a] * dpsi[b]};
          for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) J[r][s] += X[i][r] * gr[s];
        }
      const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                         J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      double fq = 0.0;
      for (int i = 0; i < 6; ++i) fq += phi[i] * f[i];
      const double wq = w * fabs(det) * fq;
      for (int i = 0; i < 6; ++i) out[i] += wq * phi[i];
    }
  }
}

__device__ __forceinline__ bool same_bits(double a, long long b) { return __double_as_longlong(a) == b; }

// VAR: column c has cell_layers[c] layers (its stencil lists are taken at its
// own bottom layer), so a group's item count and the (column, level) walk
// read each column's layer count from shared memory.
template <bool VAR>
__global__ void __launch_bounds__(kWarps * 32, EXT_MASS_MINB) k_mass_p1(const MassP1Launch p, int cpw) {
  __shared__ ColInfo cols[kWarps][kMaxCols];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  // Persistent grid: warps take groups of cpw columns round-robin, so all
  // resident warps advance through the base mesh together and vertex
  // columns shared by nearby cells are reused from L2.
  const int64_t ngroups = (p.ncells + cpw - 1) / cpw;
  const int64_t wstride = (int64_t)gridDim.x * kWarps;
  for (int64_t grp = (int64_t)blockIdx.x * kWarps + warp; grp < ngroups; grp += wstride) {
    const int64_t c0 = grp * cpw;
    const int ncol = (int)(p.ncells - c0 < cpw ? p.ncells - c0 : (int64_t)cpw);
    const int layers = p.layers;
    const int L1 = layers + 1;
    int my_items = 0;

    // ---- per-column set-up: read the three stencil lists once (Algorithm 3's
    // outer loop), the level-0 corner coordinates and the area factor.
    if (lane < ncol) {
      const int64_t c = c0 + lane;
      ColInfo &ci = cols[warp][lane];
      const int lay = VAR ? __ldg(p.cell_layers + c) : layers;
      ci.lay = lay;
      my_items = lay + 1;
      double x[3], y[3];
  #pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int32_t cb = __ldg(p.cmap + c * 6 + 2 * a), ct = __ldg(p.cmap + c * 6 + 2 * a + 1);
        const int32_t fb = __ldg(p.fmap + c * 6 + 2 * a), ft = __ldg(p.fmap + c * 6 + 2 * a + 1);
        const int32_t bb = __ldg(p.bmap + c * 6 + 2 * a), bt = __ldg(p.bmap + c * 6 + 2 * a + 1);
        ci.cbot[a] = cb;
        ci.ctop[a] = ct + (lay - 1) * p.coff[2 * a + 1];
        ci.fbot[a] = fb;
        ci.ftop[a] = ft + (lay - 1) * p.foff[2 * a + 1];
        ci.bbot[a] = bb;
        ci.btop[a] = bt + (lay - 1) * p.boff[2 * a + 1];
        x[a] = __ldg(p.X + 3 * (int64_t)cb + 0);
        y[a] = __ldg(p.X + 3 * (int64_t)cb + 1);
        ci.rx[a] = __double_as_longlong(x[a]);
        ci.ry[a] = __double_as_longlong(y[a]);
      }
      const double det2 = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
      ci.alpha = fabs(det2) * (1.0 / 144.0);
      ci.alpha2 = fabs(det2) * (1.0 / 72.0);
    }
    __syncwarp();

    const int nitems = VAR ? __reduce_add_sync(kFull, my_items) : ncol * L1;
    // lane's item: column cl (local), level m
    int cl, m;
    if (VAR) {
      cl = 0;
      m = lane;
      while (cl < ncol && m > cols[warp][cl].lay) { m -= cols[warp][cl].lay + 1; ++cl; }
    } else {
      cl = lane / L1;
      m = lane - cl * L1;
    }

    auto load_level = [&](int item, int clx, int mx, Level &lv) {
      lv.f[0] = lv.f[1] = lv.f[2] = 0.0;
      lv.z = 0.0;
      lv.ok = 1;
      if (item < nitems) {
        const ColInfo &ci = cols[warp][clx];
        const int lay = VAR ? ci.lay : layers;
        double f[3], zz[3];
        int ok = 1;
  #pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int64_t cd = dof_at(ci.cbot[a], ci.ctop[a], p.coff[2 * a], mx, lay);
          const double xa = __ldg(p.X + 3 * cd + 0);
          const double ya = __ldg(p.X + 3 * cd + 1);
          zz[a] = __ldg(p.X + 3 * cd + 2);
          ok &= same_bits(xa, ci.rx[a]) & same_bits(ya, ci.ry[a]);
          f[a] = __ldg(p.f + dof_at(ci.fbot[a], ci.ftop[a], p.foff[2 * a], mx, lay));
        }
        ok &= (__double_as_longlong(zz[0]) == __double_as_longlong(zz[1])) &
              (__double_as_longlong(zz[1]) == __double_as_longlong(zz[2]));
        lv.f[0] = f[0];
        lv.f[1] = f[1];
        lv.f[2] = f[2];
        lv.z = zz[0];
        lv.ok = ok;
      }
    };

    Level cur, nxt;
    int item = lane;
    load_level(item, cl, m, cur);
    // carry from the previous step's last lane: s_{m-1}, 2 s_{m-1}, f_{m-1}, S_{m-1}
    double carry_s = 0.0, carry_s2 = 0.0, carry_f[3] = {0.0, 0.0, 0.0};
    int carry_ok = 1;

    for (int base = 0; base < nitems; base += 32) {
      // advance (cl, m) by 32 items for the lookahead
      int ncl = cl, nm = m + 32;
      if (VAR) {
        while (ncl < ncol && nm > cols[warp][ncl].lay) { nm -= cols[warp][ncl].lay + 1; ++ncl; }
      } else {
        while (nm >= L1) { nm -= L1; ++ncl; }
      }
      const int nitem = item + 32;
      if (base + 32 < nitems) load_level(nitem, ncl < ncol ? ncl : ncol - 1, nm, nxt);
      else { nxt.f[0] = nxt.f[1] = nxt.f[2] = 0.0; nxt.z = 0.0; nxt.ok = 1; }

      const bool valid = item < nitems;
      const ColInfo &ci = cols[warp][valid ? cl : 0];
      const int lay = VAR ? ci.lay : layers;

      // neighbours: level m+1 (next lane or lookahead), level m-1 (previous lane or carry)
      const bool top = (m == lay);
      const bool bottom = (m == 0);
      double fn[3], zn;
  #pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double dn = __shfl_down_sync(kFull, cur.f[a], 1);
        const double la = __shfl_sync(kFull, nxt.f[a], 0);
        fn[a] = top ? 0.0 : (lane == 31 ? la : dn);
      }
      {
        const double dz = __shfl_down_sync(kFull, cur.z, 1);
        const double lz = __shfl_sync(kFull, nxt.z, 0);
        zn = lane == 31 ? lz : dz;
      }
      const int nxt_ok0 = __shfl_sync(kFull, nxt.ok, 0);
      double s = 0.0, s2 = 0.0;
      if (!top) {
        const double h = fabs(dadd(zn, -cur.z));
        s = ci.alpha * h;
        s2 = ci.alpha2 * h;
      }
      double fp[3], sp, sp2;
  #pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double up = __shfl_up_sync(kFull, cur.f[a], 1);
        fp[a] = bottom ? 0.0 : (lane == 0 ? carry_f[a] : up);
      }
      {
        const double us = __shfl_up_sync(kFull, s, 1);
        const double us2 = __shfl_up_sync(kFull, s2, 1);
        sp = bottom ? 0.0 : (lane == 0 ? carry_s : us);
        sp2 = lane == 0 ? carry_s2 : us2;
      }

      const bool step_ok = __all_sync(kFull, cur.ok) && carry_ok && nxt_ok0;
      double val[3];
      if (step_ok) {
        const double sig = bottom ? s2 : dadd(sp2, s2);
        // c_a = s_{m-1} f_{m-1,a} + sigma f_{m,a} + s_m f_{m+1,a}
  #pragma unroll
        for (int a = 0; a < 3; ++a) val[a] = fma(sp, fp[a], fma(sig, cur.f[a], s * fn[a]));
      } else if (valid) {
        // general geometry: evaluate the two element integrals touching level m
        val[0] = val[1] = val[2] = 0.0;
        for (int half = 0; half < 2; ++half) {
          const int l = half == 0 ? m - 1 : m;  // layer below / above level m
          if (l < 0 || l >= lay) continue;
          double X[6][3], f6[6], out[6];
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 2; ++b) {
              const int lev = l + b;
              const int64_t cd = dof_at(ci.cbot[a], ci.ctop[a], p.coff[2 * a], lev, lay);
              X[2 * a + b][0] = __ldg(p.X + 3 * cd + 0);
              X[2 * a + b][1] = __ldg(p.X + 3 * cd + 1);
              X[2 * a + b][2] = __ldg(p.X + 3 * cd + 2);
              f6[2 * a + b] = __ldg(p.f + dof_at(ci.fbot[a], ci.ftop[a], p.foff[2 * a], lev, lay));
            }
          prism_general(X, f6, out);
          for (int a = 0; a < 3; ++a) val[a] += out[2 * a + (half == 0 ? 1 : 0)];
        }
      }
      if (valid) {
  #pragma unroll
        for (int a = 0; a < 3; ++a) {
          // straight: value_a = 2 c_a + c_b + c_c, the horizontal sum done by L2
          double *dst = p.b + dof_at(ci.bbot[a], ci.btop[a], p.boff[2 * a], m, lay);
          atomicAdd(dst, val[a]);
          if (step_ok) {
            atomicAdd(dst, val[0]);
            atomicAdd(dst, val[1]);
            atomicAdd(dst, val[2]);
          }
        }
      }

      // carry this step's last lane into the next step, shift the lookahead in
      carry_s = __shfl_sync(kFull, s, 31);
      carry_s2 = __shfl_sync(kFull, s2, 31);
  #pragma unroll
      for (int a = 0; a < 3; ++a) carry_f[a] = __shfl_sync(kFull, cur.f[a], 31);
      carry_ok = __shfl_sync(kFull, cur.ok, 31);
      cur = nxt;
      cl = ncl;
      m = nm;
      item = nitem;
    }
    __syncwarp();  // the next group's set-up overwrites cols[warp]
  }
}

}  // namespace

cudaError_t launch_mass_p1(const MassP1Launch &p, cudaStream_t s) {
  if (p.ncells == 0) return cudaSuccess;
  const bool var = p.cell_layers != nullptr;
  // columns per group: about EXT_MASS_ITEMS items (mean items with variable layers)
  const double L1 = var ? p.mean_layers + 1.0 : (double)(p.layers + 1);
  int cpw = (int)((EXT_MASS_ITEMS + L1 - 1.0) / L1);
  if (cpw < 1) cpw = 1;
  if (cpw > kMaxCols) cpw = kMaxCols;
  const int64_t warps = (p.ncells + cpw - 1) / cpw;
  int64_t blocks = (warps + kWarps - 1) / kWarps;
  static int resident[2] = {0, 0}, sms = 0;  // per process: one GPU model
  if (resident[var] == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (var) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident[1], k_mass_p1<true>, kWarps * 32, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident[0], k_mass_p1<false>, kWarps * 32, 0);
    if (resident[var] < 1) resident[var] = 1;
  }
  if (blocks > (int64_t)resident[var] * sms) blocks = (int64_t)resident[var] * sms;
  if (var) k_mass_p1<true><<<(unsigned)blocks, kWarps * 32, 0, s>>>(p, cpw);
  else k_mass_p1<false><<<(unsigned)blocks, kWarps * 32, 0, s>>>(p, cpw);
  return cudaGetLastError();
}
