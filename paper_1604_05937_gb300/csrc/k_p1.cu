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
#include <cstdlib>
#include <cstring>

#include "ext_internal.cuh"
#include "fastdiv.cuh"

namespace {

constexpr int kWarps = 8;
constexpr int kMaxCols = 32;  // columns per warp (lane j sets up column j)
constexpr unsigned kFull = 0xffffffffu;

#ifndef EXT_MASS_MINB
#define EXT_MASS_MINB 2  // resident CTAs per SM the register budget must allow
#endif
#ifndef EXT_CELLS_MINB
#define EXT_CELLS_MINB 5  // resident CTAs per SM of the split form's cell pass (constant layers)
#endif
#ifndef EXT_CELLS_VAR_MINB
#define EXT_CELLS_VAR_MINB 4  // the same with variable layers
#endif
#ifndef EXT_FACTORED_MIN_LAYERS
#define EXT_FACTORED_MIN_LAYERS 3  // constant layers: the factored split form from this many layers
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

// P1xP1 element vector of one prism with the 6-point rule (3-point triangle
// rule x 2-point Gauss rule, weight 1/12 per point), stencil order
// i = 2a + b (vertex a, bottom/top b):
//   out_i = sum_q (1/12) |det J_q| f_h(x_q) phi_i(x_q).
// Nodes X[i] (x, y, z) and values f[i]; rx, ry: bit patterns of the level-0
// x, y of the cell's three vertex columns; k2 = |2A| / 864 and
// k6 = |2A| / 2592 with A the area of the level-0 triangle.
//
// Vertical form: when all six nodes lie on the vertical lines through the
// level-0 vertices (x, y equal to rx, ry bitwise), J has the columns
// (e1, e2, (0, 0, h(t))) with h(t) = sum_a lambda_a(t) h_a the interpolated
// height of the vertical edges h_a = z_a1 - z_a0, so det J = 2A h(t) does not
// depend on the Gauss point.  With lambda_a(t) = 1/6 + [a = t]/2 at the
// triangle points and sum_g psi_b psi_b' = (1 + [b = b']) / 3 over the two
// Gauss points, the rule sums to
//   out_ab = D_a (G_b + 3 g_ab) + G_b (D_0 + D_1 + D_2) / 3 + sum_t D_t g_tb,
//   D_t = |k2 h_t + k6 (h_0 + h_1 + h_2)|,  g_ab = 2 f_ab + f_a(1-b),
//   G_b = g_0b + g_1b + g_2b:
// 42 FP64 operations, all issued as DFMA.
//
// General form (any other prism): per Gauss point height z the horizontal
// tangents e1 = P_1 - P_0, e2 = P_2 - P_0 of the points P_a = (1 - z) X_a0 +
// z X_a1 on the vertical edges, n = e1 x e2, and with the edge vectors
// H_a = X_a1 - X_a0 the determinant at triangle point t is
// det = sum_a lambda_a(t) (H_a . n) (about 130 FP64 operations).
__device__ __forceinline__ void p1_prism(const double X[6][3], const double f[6], const long long rx[3],
                                         const long long ry[3], double k2, double k6, const Fp64Ones &k1,
                                         double out[6]) {
  bool vert = true;
#pragma unroll
  for (int i = 0; i < 6; ++i) vert &= same_bits(X[i][0], rx[i >> 1]) & same_bits(X[i][1], ry[i >> 1]);
  if (vert) {
    double h[3], D[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) h[a] = fsub(X[2 * a + 1][2], X[2 * a][2], k1);
    const double ks = fmul(k6, fadd(h[0], fadd(h[1], h[2], k1), k1), k1);
#pragma unroll
    for (int t = 0; t < 3; ++t) D[t] = fabs(fma(k2, h[t], ks));
    const double Ds = fmul(fadd(D[0], fadd(D[1], D[2], k1), k1), 1.0 / 3.0, k1);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      double g[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) g[a] = fma(2.0, f[2 * a + b], f[2 * a + 1 - b]);
      const double G = fadd(g[0], fadd(g[1], g[2], k1), k1);
      const double Q = fma(D[0], g[0], fma(D[1], g[1], fmul(D[2], g[2], k1)));
      const double C = fma(G, Ds, Q);
#pragma unroll
      for (int a = 0; a < 3; ++a) out[2 * a + b] = fma(D[a], fma(3.0, g[a], G), C);
    }
    return;
  }
  const double zg[2] = {0.5 - 0.28867513459481288225, 0.5 + 0.28867513459481288225};
  double H[3][3], E10[3], E20[3], dE1[3], dE2[3], df[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int a = 0; a < 3; ++a) H[a][r] = fsub(X[2 * a + 1][r], X[2 * a][r], k1);
    E10[r] = fsub(X[2][r], X[0][r], k1);
    E20[r] = fsub(X[4][r], X[0][r], k1);
    dE1[r] = fsub(fsub(X[3][r], X[1][r], k1), E10[r], k1);
    dE2[r] = fsub(fsub(X[5][r], X[1][r], k1), E20[r], k1);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    df[a] = fsub(f[2 * a + 1], f[2 * a], k1);
    out[2 * a] = 0.0;
    out[2 * a + 1] = 0.0;
  }
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const double z = zg[g];
    double e1[3], e2[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      e1[r] = fma(z, dE1[r], E10[r]);
      e2[r] = fma(z, dE2[r], E20[r]);
    }
    const double n[3] = {fma(e1[1], e2[2], -e1[2] * e2[1]), fma(e1[2], e2[0], -e1[0] * e2[2]),
                         fma(e1[0], e2[1], -e1[1] * e2[0])};
    double pa[3], F[3], w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      pa[a] = fma(H[a][0], n[0], fma(H[a][1], n[1], fmul(H[a][2], n[2], k1)));
      F[a] = fma(z, df[a], f[2 * a]);
    }
    const double sp = fmul(fadd(pa[0], fadd(pa[1], pa[2], k1), k1), 1.0 / 72.0, k1);
    const double sf = fmul(fadd(F[0], fadd(F[1], F[2], k1), k1), 1.0 / 6.0, k1);
#pragma unroll
    for (int t = 0; t < 3; ++t) w[t] = fmul(fabs(fma(1.0 / 24.0, pa[t], sp)), fma(0.5, F[t], sf), k1);
    const double sw = fmul(fadd(w[0], fadd(w[1], w[2], k1), k1), 1.0 / 6.0, k1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double R = fma(0.5, w[a], sw);
      out[2 * a] = fma(1.0 - z, R, out[2 * a]);
      out[2 * a + 1] = fma(z, R, out[2 * a + 1]);
    }
  }
}

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

// ---------------------------------------------------------------------------
// Split form.  On a straight column the vertical sums depend only on the
// vertex column: with h_l the layer heights of that column,
//   w_m = h_{m-1} (f_{m-1} + 2 f_m) + h_m (2 f_m + f_{m+1})
// and a straight cell with area factor alpha = |2A| / 144 contributes
// c_a = alpha w_{a,m} at level m, i.e. value_a = alpha (w_a + w_0 + w_1 + w_2).
// Summed over the cells around vertex a this factors into a vertex part and
// a cell part,
//   b_{a,m} += A_a w_{a,m} + sum_{c containing a} alpha_c S_{c,m},
//   A_a = sum_{c containing a} alpha_c,  S_{c,m} = w_0 + w_1 + w_2,
// so with two or more constant layers the launch runs
//   k_area        alpha_c per cell (stored) and A_a (alpha_c added to the
//                 cell's three vertices),
//   k_vsum        per vertex level: w, and b += A_a w (the vertex part),
//   k_mass_cells  per (column, level) item: alpha_c S_c added to the three
//                 vertices (3 FP64 operations and 3 atomic adds per item,
//                 against 13 and 12 when every cell forms its own sums),
//   k_mass_general the warp steps that met a prism which is not straight:
//                 the 6-point rule with the general Jacobian, minus the
//                 alpha_c w_a that the vertex part already added for them.
// Straightness is checked exactly: k_vsum compares every DoF's x, y with its
// column's reference x, y (those alpha was formed from: the mesh's base
// coordinates, or the field's level 0) and stores z next to w (a NaN pattern
// when x, y differ; coordinates are finite), and the cell pass compares the
// three z of each level bitwise.  With one layer the area pass costs more than the
// vertex part saves (a cell has two items to spread it over), and the cell
// pass forms alpha (w_a + S) per item instead (6 FP64 operations).  With
// variable layers a vertex column spans the hull of its cells' ranges, so the
// w of a cell's bottom and top levels may include a layer outside that cell;
// that form keeps the per-item combination with the one-layer halves at the
// cell's ends.

// bit pattern stored in place of z when a DoF's x, y differ from its column's
// level-0 x, y (a NaN, which finite coordinates never produce)
constexpr long long kNotVertical = 0x7ff4000000000badLL;

// A_a over the vertices (constant layers): cell c adds alpha_c = |2A_c| / 144
// to the three vertex columns of its level-0 DoFs (column of DoF d: d / col,
// which is base vertex d / col) and stores alpha_c for the cell and general
// passes.  The reference x, y are the mesh's base coordinates when it has
// them (16 bytes per vertex, which stay in L2 however the cells are ordered),
// else the coordinate field's level 0; the vertex pass checks every level
// against the same reference.
__global__ void __launch_bounds__(256) k_area(const MassP1Launch p, double *__restrict__ A,
                                              double *__restrict__ alpha_out, FastDiv col) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < p.ncells;
       c += (int64_t)gridDim.x * blockDim.x) {
    double x[3], y[3];
    uint32_t v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      v[a] = fdiv((uint32_t)__ldg(p.fmap + c * 6 + 2 * a), col);
      if (p.base_xy) {
        x[a] = __ldg(p.base_xy + 2 * (int64_t)v[a] + 0);
        y[a] = __ldg(p.base_xy + 2 * (int64_t)v[a] + 1);
      } else {
        const int64_t cb = __ldg(p.cmap + c * 6 + 2 * a);
        x[a] = __ldg(p.X + 3 * cb + 0);
        y[a] = __ldg(p.X + 3 * cb + 1);
      }
    }
    const double det2 = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
    const double alpha = fabs(det2) * (1.0 / 144.0);
    alpha_out[c] = alpha;
#pragma unroll
    for (int a = 0; a < 3; ++a) atomicAdd(A + v[a], alpha);
  }
}

// Vertex pass over the DoFs [0, n) of a CG1xCG1 field (the column of a vertex
// is a contiguous run, so level m's neighbours are DoFs d - 1 and d + 1).
// Constant layers (`col` = layers + 1, level m = d mod col, the ends have one
// layer): W holds n pairs (w, z or kNotVertical), and in the factored form
// (FAC) b[d] += A[d / col] w (b[d] = A[d / col] w with `overwrite`).  VAR:
// the ends of vertex columns are never read; W holds 3n values: w, the upper
// half |h_hi| (2 f + f_hi) and the lower half |h_lo| (f_lo + 2 f); A is
// unused.  Without FAC, `overwrite` clears b for the cell pass.
#ifndef EXT_VSUM_MINB
#define EXT_VSUM_MINB 4  // resident 256-thread CTAs per SM the vertex pass's registers must allow
#endif
#ifndef EXT_VSUM_VU
#define EXT_VSUM_VU 2  // 32-DoF chunks per warp step of the vertex pass
#endif

template <bool VAR, bool FAC>
__global__ void __launch_bounds__(256, EXT_VSUM_MINB) k_vsum(const double *__restrict__ X, const double *__restrict__ f,
                                              double *__restrict__ W, int64_t n, FastDiv col,
                                              const double *__restrict__ A, double *__restrict__ b, Fp64Ones k1,
                                              const double *__restrict__ ref_xy, bool overwrite) {
  // A warp takes VU consecutive 32-DoF chunks per step and issues all their
  // loads before any arithmetic (the loop is latency-bound otherwise); the
  // neighbours across chunk edges come from the adjacent chunk's lanes.
  constexpr int VU = EXT_VSUM_VU;
  const int lane = threadIdx.x & 31;
  const int64_t wstride = (int64_t)gridDim.x * 8 * 32 * VU;
  for (int64_t base = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * 32 * VU; base < n; base += wstride) {
    double zc[VU], fc[VU];
    double bc[VU], Ac[VU];   // constant layers: b and A of the DoF's column
    int okv[VU];             // constant layers: x, y equal the column's level-0 x, y
    uint32_t mmv[VU];        // constant layers: level of the DoF
#pragma unroll
    for (int u = 0; u < VU; ++u) {
      const int64_t d = base + u * 32 + lane;
      zc[u] = 0.0;
      fc[u] = 0.0;
      bc[u] = 0.0;
      Ac[u] = 0.0;
      okv[u] = 1;
      mmv[u] = 0;
      if (d < n) {
        zc[u] = __ldg(X + 3 * d + 2);
        fc[u] = __ldg(f + d);
        if (!VAR) {
          const uint32_t q = fdiv((uint32_t)d, col);
          const int64_t d0 = (int64_t)q * col.d;
          mmv[u] = (uint32_t)(d - d0);
          // reference x, y of the column: the base coordinates (factored
          // form, when the mesh has them) or the field's level 0
          const double *r = (FAC && ref_xy) ? ref_xy + 2 * (int64_t)q : X + 3 * d0;
          okv[u] = (__double_as_longlong(__ldg(X + 3 * d + 0)) == __double_as_longlong(__ldg(r + 0))) &
                   (__double_as_longlong(__ldg(X + 3 * d + 1)) == __double_as_longlong(__ldg(r + 1)));
          if (FAC) {
            Ac[u] = __ldg(A + q);
            // b = A w + b, or with overwrite A w + (-0), which is A w exactly
            bc[u] = overwrite ? -0.0 : b[d];
          }
        }
      }
    }
    // the DoF before the first chunk and after the last one
    double zb = 0.0, fb = 0.0, za = 0.0, fa = 0.0;
    if (lane == 0 && base > 0 && base - 1 < n) {
      zb = __ldg(X + 3 * (base - 1) + 2);
      fb = __ldg(f + base - 1);
    }
    if (lane == 31 && base + 32 * VU < n) {
      za = __ldg(X + 3 * (base + 32 * VU) + 2);
      fa = __ldg(f + base + 32 * VU);
    }
    // signed heights of the layer below each DoF, hl = z - z_left (left
    // neighbour: previous lane; for lane 0 the previous chunk's lane 31 or
    // its own load of DoF base - 1; u > 0 is a compile-time condition, so
    // every lane reaches the shuffles), and the left f
    double hl[VU], fl[VU];
#pragma unroll
    for (int u = 0; u < VU; ++u) {
      double zl = __shfl_up_sync(kFull, zc[u], 1);
      fl[u] = __shfl_up_sync(kFull, fc[u], 1);
      double zlp = zb, flp = fb;
      if (u > 0) {
        zlp = __shfl_sync(kFull, zc[u > 0 ? u - 1 : 0], 31);
        flp = __shfl_sync(kFull, fc[u > 0 ? u - 1 : 0], 31);
      }
      if (lane == 0) {
        zl = zlp;
        fl[u] = flp;
      }
      hl[u] = fsub(zc[u], zl, k1);
    }
    // height of the layer above the last chunk's lane 31 (one DFMA per warp
    // step; the value is used by lane 31 only)
    const double ha = fsub(za, zc[VU - 1], k1);
#pragma unroll
    for (int u = 0; u < VU; ++u) {
      const int64_t d = base + u * 32 + lane;
      // height above and right f: next lane; for lane 31 the next chunk's
      // lane 0, or the DoF after the last chunk
      double hh = __shfl_down_sync(kFull, hl[u], 1), fr = __shfl_down_sync(kFull, fc[u], 1);
      double hhn = ha, frn = fa;
      if (u + 1 < VU) {
        hhn = __shfl_sync(kFull, hl[u + 1 < VU ? u + 1 : u], 0);
        frn = __shfl_sync(kFull, fc[u + 1 < VU ? u + 1 : u], 0);
      }
      if (lane == 31) {
        hh = hhn;
        fr = frn;
      }
      bool lo_end, hi_end;
      if (VAR) {
        lo_end = d == 0;
        hi_end = d + 1 >= n;
      } else {
        lo_end = mmv[u] == 0;
        hi_end = mmv[u] + 1 == col.d;
      }
      // w = |hl| (fl + 2 fc) + |hh| (2 fc + fr): four DFMA (the absolute
      // values are operand modifiers).  At a column end the missing layer's
      // f factor is cleared bitwise (an integer AND, off the FP64 pipe); the
      // height read across the column boundary is then multiplied by zero
      // (coordinates are finite).
      const long long kl = lo_end ? 0LL : -1LL, kh = hi_end ? 0LL : -1LL;
      const double al = __longlong_as_double(__double_as_longlong(fma(2.0, fc[u], fl[u])) & kl);
      const double bh = __longlong_as_double(__double_as_longlong(fma(2.0, fc[u], fr)) & kh);
      // overwrite without the factored form: clear b before the cell pass adds
      if (!FAC && overwrite && d < n) b[d] = 0.0;
      if (VAR) {
        // variable layers: also the one-layer halves, which the bottom (upper
        // half) and top (lower half) levels of a cell column use
        const double up = fmul(fabs(hh), bh, k1);
        const double lo = fmul(fabs(hl[u]), al, k1);
        if (d < n) {
          W[d] = fma(fabs(hl[u]), al, up);
          W[n + d] = up;
          W[2 * n + d] = lo;
        }
      } else if (d < n) {
        const double w = fma(fabs(hl[u]), al, fmul(fabs(hh), bh, k1));
        if (FAC) b[d] = fma(w, Ac[u], bc[u]);
        reinterpret_cast<double2 *>(W)[d] =
            make_double2(w, okv[u] ? zc[u] : __longlong_as_double(kNotVertical));
      }
    }
  }
}

// Stencil rows, area factor and level-0 corner bits of column c (Algorithm
// 3's outer loop: the lists are read once per column).  STORED (the
// factored form): the area factor is the one the area pass stored in
// `alpha`, and the corner bits are not needed.
template <bool VAR, bool STORED = false>
__device__ __forceinline__ int setup_column(const MassP1Launch &p, int64_t c, ColInfo &ci,
                                            const double *__restrict__ alpha = nullptr) {
  const int lay = VAR ? __ldg(p.cell_layers + c) : p.layers;
  ci.lay = lay;
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
    if (!STORED) {
      x[a] = __ldg(p.X + 3 * (int64_t)cb + 0);
      y[a] = __ldg(p.X + 3 * (int64_t)cb + 1);
      ci.rx[a] = __double_as_longlong(x[a]);
      ci.ry[a] = __double_as_longlong(y[a]);
    }
  }
  if (STORED) {
    ci.alpha = __ldg(alpha + c);
  } else {
    const double det2 = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
    ci.alpha = fabs(det2) * (1.0 / 144.0);
  }
  ci.alpha2 = 2.0 * ci.alpha;
  return lay + 1;
}

// (column, level) of item `it` of a group: constant layers by division,
// variable layers by walking the columns' layer counts.
template <bool VAR>
__device__ __forceinline__ void item_pos(const ColInfo *cols, int ncol, int L1, int it, int &cl, int &m) {
  if (VAR) {
    cl = 0;
    m = it;
    while (cl < ncol && m > cols[cl].lay) { m -= cols[cl].lay + 1; ++cl; }
  } else {
    cl = it / L1;
    m = it - cl * L1;
  }
}

struct WLevel {
  double w[3];  // vertical sums of the three vertices
  int ok;
};

// A warp step of the cell pass that meets a prism which is not straight is
// recorded as (group, first item) and evaluated by k_mass_general instead.
struct Deferred {
  int2 *list;
  unsigned int *count;
  unsigned int cap;
};

template <bool VAR, bool FAC>
__global__ void __launch_bounds__(kWarps * 32, VAR ? EXT_CELLS_VAR_MINB : EXT_CELLS_MINB) k_mass_cells(const MassP1Launch p,
                                                                            const double *__restrict__ W,
                                                                            Deferred dfr, int cpw, Fp64Ones k1,
                                                                            const double *__restrict__ alpha) {
  __shared__ ColInfo cols[kWarps][kMaxCols];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t ngroups = (p.ncells + cpw - 1) / cpw;
  const int64_t wstride = (int64_t)gridDim.x * kWarps;
  for (int64_t grp = (int64_t)blockIdx.x * kWarps + warp; grp < ngroups; grp += wstride) {
    const int64_t c0 = grp * cpw;
    const int ncol = (int)(p.ncells - c0 < cpw ? p.ncells - c0 : (int64_t)cpw);
    const int layers = p.layers;
    const int L1 = layers + 1;
    int my_items = 0;
    if (lane < ncol) my_items = setup_column<VAR, FAC>(p, c0 + lane, cols[warp][lane], alpha);
    __syncwarp();
    const int nitems = VAR ? __reduce_add_sync(kFull, my_items) : ncol * L1;
    int cl, m;
    item_pos<VAR>(cols[warp], ncol, L1, lane, cl, m);

    auto load_level = [&](int item, int clx, int mx, WLevel &lv) {
      lv.w[0] = lv.w[1] = lv.w[2] = 0.0;
      lv.ok = 1;
      if (item < nitems) {
        const ColInfo &ci = cols[warp][clx];
        const int lay = VAR ? ci.lay : layers;
        if (VAR) {
          double zz[3];
          int ok = 1;
          // variable layers: the bottom and top levels of this cell column
          // take the one-layer half that lies inside the column (the vertex
          // column may extend beyond it)
          const double *src = mx == 0 ? W + p.nf : (mx == lay ? W + 2 * p.nf : W);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const int64_t cd = dof_at(ci.cbot[a], ci.ctop[a], p.coff[2 * a], mx, lay);
            const double xa = __ldg(p.X + 3 * cd + 0);
            const double ya = __ldg(p.X + 3 * cd + 1);
            zz[a] = __ldg(p.X + 3 * cd + 2);
            ok &= same_bits(xa, ci.rx[a]) & same_bits(ya, ci.ry[a]);
            lv.w[a] = __ldg(src + dof_at(ci.fbot[a], ci.ftop[a], p.foff[2 * a], mx, lay));
          }
          ok &= (__double_as_longlong(zz[0]) == __double_as_longlong(zz[1])) &
                (__double_as_longlong(zz[1]) == __double_as_longlong(zz[2]));
          lv.ok = ok;
        } else {
          // constant layers: (w, z) pairs; z equal at the three vertices and
          // none of them marked as off its column's vertical
          long long zb[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const double2 v = __ldg(reinterpret_cast<const double2 *>(W) +
                                    dof_at(ci.fbot[a], ci.ftop[a], p.foff[2 * a], mx, lay));
            lv.w[a] = v.x;
            zb[a] = __double_as_longlong(v.y);
          }
          lv.ok = (zb[0] == zb[1]) & (zb[1] == zb[2]) & (zb[0] != kNotVertical);
        }
      }
    };

    WLevel cur, nxt;
    int item = lane;
    load_level(item, cl, m, cur);
    int carry_ok = 1;

    for (int base = 0; base < nitems; base += 32) {
      int ncl = cl, nm = m + 32;
      if (VAR) {
        while (ncl < ncol && nm > cols[warp][ncl].lay) { nm -= cols[warp][ncl].lay + 1; ++ncl; }
      } else {
        while (nm >= L1) { nm -= L1; ++ncl; }
      }
      const int nitem = item + 32;
      if (base + 32 < nitems) load_level(nitem, ncl < ncol ? ncl : ncol - 1, nm, nxt);
      else { nxt.w[0] = nxt.w[1] = nxt.w[2] = 0.0; nxt.ok = 1; }

      const bool valid = item < nitems;
      const ColInfo &ci = cols[warp][valid ? cl : 0];
      const int lay = VAR ? ci.lay : layers;
      const int nxt_ok0 = __shfl_sync(kFull, nxt.ok, 0);
      const bool step_ok = __all_sync(kFull, cur.ok) && carry_ok && nxt_ok0;
      if (step_ok) {
        // alpha S = alpha (w_0 + w_1 + w_2): three DFMA; unfactored (variable
        // layers, or few layers) value_a = alpha (w_a + S) (three DFMA more);
        // factored, the vertex part alpha w_a is in A_a w_a already
        const double aw = fma(ci.alpha, cur.w[0], fma(ci.alpha, cur.w[1], fmul(ci.alpha, cur.w[2], k1)));
        double val[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) val[a] = FAC ? aw : fma(ci.alpha, cur.w[a], aw);
        if (valid) {
#pragma unroll
          for (int a = 0; a < 3; ++a)
            atomicAdd(p.b + dof_at(ci.bbot[a], ci.btop[a], p.boff[2 * a], m, lay), val[a]);
        }
      } else if (lane == 0) {
        const unsigned int slot = atomicAdd(dfr.count, 1u);
        if (slot < dfr.cap) dfr.list[slot] = make_int2((int)grp, base);
        else atomicOr(p.err, EXT_DERR_BOUNDS);
      }
      carry_ok = __shfl_sync(kFull, cur.ok, 31);
      cur = nxt;
      cl = ncl;
      m = nm;
      item = nitem;
    }
    __syncwarp();
  }
}

// Reference x, y bit patterns of a cell column (its bottom coordinate DoFs)
// and the area constants k2 = |2A| / 864, k6 = |2A| / 2592 of p1_prism.
__device__ __forceinline__ void column_ref(const double *__restrict__ X, const int32_t cb[3], long long rx[3],
                                          long long ry[3], double &k2, double &k6) {
  double x[3], y[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    x[a] = __ldg(X + 3 * (int64_t)cb[a] + 0);
    y[a] = __ldg(X + 3 * (int64_t)cb[a] + 1);
    rx[a] = __double_as_longlong(x[a]);
    ry[a] = __double_as_longlong(y[a]);
  }
  const double det2 = fabs((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]));
  k2 = det2 * (1.0 / 864.0);
  k6 = det2 * (1.0 / 2592.0);
}

// Nodes and values of prism (c, l) of a column set up in `ci` (layers lay).
__device__ __forceinline__ void load_prism(const MassP1Launch &p, const ColInfo &ci, int l, int lay, double X[6][3],
                                           double f[6]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int64_t cd = dof_at(ci.cbot[a], ci.ctop[a], p.coff[2 * a], l + b, lay);
      X[2 * a + b][0] = __ldg(p.X + 3 * cd + 0);
      X[2 * a + b][1] = __ldg(p.X + 3 * cd + 1);
      X[2 * a + b][2] = __ldg(p.X + 3 * cd + 2);
      f[2 * a + b] = __ldg(p.f + dof_at(ci.fbot[a], ci.ftop[a], p.foff[2 * a], l + b, lay));
    }
}

// The deferred warp steps: every item of the step evaluates the two element
// vectors touching its level (p1_prism: the 6-point rule, vertical or
// general form).
template <bool VAR, bool FAC>
__global__ void __launch_bounds__(kWarps * 32) k_mass_general(const MassP1Launch p, const double *__restrict__ W,
                                                              Deferred dfr, int cpw, const double *__restrict__ alpha,
                                                              Fp64Ones k1) {
  __shared__ ColInfo cols[kWarps][kMaxCols];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const unsigned int n = min(*dfr.count, dfr.cap);
  for (unsigned int e = blockIdx.x * kWarps + warp; e < n; e += gridDim.x * kWarps) {
    const int2 en = dfr.list[e];
    const int64_t c0 = (int64_t)en.x * cpw;
    const int ncol = (int)(p.ncells - c0 < cpw ? p.ncells - c0 : (int64_t)cpw);
    int my_items = 0;
    if (lane < ncol) my_items = setup_column<VAR, FAC>(p, c0 + lane, cols[warp][lane], alpha);
    __syncwarp();
    const int nitems = VAR ? __reduce_add_sync(kFull, my_items) : ncol * (p.layers + 1);
    const int it = en.y + lane;
    if (it < nitems) {
      int cl, m;
      item_pos<VAR>(cols[warp], ncol, p.layers + 1, it, cl, m);
      const ColInfo &ci = cols[warp][cl];
      const int lay = VAR ? ci.lay : p.layers;
      long long rx[3], ry[3];
      double k2, k6;
      column_ref(p.X, ci.cbot, rx, ry, k2, k6);
      double val[3] = {0.0, 0.0, 0.0};
      for (int half = 0; half < 2; ++half) {
        const int l = half == 0 ? m - 1 : m;
        if (l < 0 || l >= lay) continue;
        double Xp[6][3], fp[6], out[6];
        load_prism(p, ci, l, lay, Xp, fp);
        p1_prism(Xp, fp, rx, ry, k2, k6, k1, out);
        for (int a = 0; a < 3; ++a) val[a] += out[2 * a + (half == 0 ? 1 : 0)];
      }
      // factored form: the vertex pass added alpha_c w_a for this item too
      if (FAC)
        for (int a = 0; a < 3; ++a)
          val[a] = fma(-ci.alpha,
                       __ldg(reinterpret_cast<const double2 *>(W) + dof_at(ci.fbot[a], ci.ftop[a], p.foff[2 * a], m, lay)).x,
                       val[a]);
      for (int a = 0; a < 3; ++a) atomicAdd(p.b + dof_at(ci.bbot[a], ci.btop[a], p.boff[2 * a], m, lay), val[a]);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Gather form (constant layers, triangle meshes).  A straight extrusion with
// flat levels (every DoF at the x, y of its column's level 0, level m at one
// height z_m in every column) is a tensor product, and the P1xP1 mass matrix
// factors as M = Mh (x) Mv: Mh the P1 mass matrix of the level-0
// triangulation, applied through the mesh's vertex rows (the weight of
// neighbour j of vertex a is the sum of alpha_c = |2 A_c| / 144 over the
// cells holding edge (a, j), the diagonal weight is the sum of the row), and
// Mv the P1 mass matrix of the column,
//   w_m = (Mv f)_m = |h_{m-1}| f_{m-1} + 2 (|h_{m-1}| + |h_m|) f_m + |h_m| f_{m+1}
// (the factor 1/6 of Mv is in alpha).  b = Mh (x) Mv f is then, per level,
// the row sums b_{a,m} = sum_j Mh_{aj} w_{j,m}: 3 FP64 operations per DoF
// for Mv and one per row entry (about 7 per DoF) for Mh.  Every geometric
// quantity comes from the coordinate field of the launch.  The launch runs
//   k_p1_prep           the level table (z_m, |h_{m-1}|, 2 (|h_{m-1}| + |h_m|),
//                       |h_m|) from the column of vertex 0, alpha_c of every
//                       cell from its level-0 nodes, and (automatic form) a
//                       probe of the coordinates of a sample of vertex
//                       columns: any sampled DoF off its column's vertical or
//                       its level's height sets the mode word, and the launch
//                       then runs as the cell loop k_p1_cells instead,
//   k_p1_rowweights     the row weights from alpha,
//   k_vsum_bulk         w per DoF, stored; a NaN pattern instead where the DoF
//                       or a vertical neighbour of it is off its column's
//                       level-0 x, y or its level's height (coordinates and f
//                       staged in shared memory by bulk copies; k_vsum_tab is
//                       the same pass with plain loads, for X or f not 16-byte
//                       aligned),
//   k_vgather           b per DoF: one thread forms the row sum over the
//                       vertex row (no atomics) and overwrites b (WRITE) or
//                       adds to it (INC); a 32-DoF chunk whose sums came out
//                       NaN is recorded with the mask of those DoFs and left
//                       untouched,
//   k_vgather_general   the recorded DoFs: p1_prism over both layers of every
//                       cell around the vertex,
//   k_p1_cells          (cell-loop mode only) Algorithm 3 over the cell
//                       columns with p1_prism per prism.
// A NaN input or a non-straight prism anywhere in a DoF's stencil makes its
// row sum NaN (NaN survives every product and sum), so every DoF is either
// formed by the gather on a verified tensor-product stencil or recomputed in
// full.  In the gather mode every DoF of b is written by one thread, in a
// fixed order of operations: the result does not depend on scheduling.

struct LevelCoef {
  double z, lo, mid, hi;  // z_m, |h_{m-1}|, 2 (|h_{m-1}| + |h_m|), |h_m| (0 beyond the column)
};

// Mode word of the gather form (set by the probe): bit 0 = not a flat
// extrusion, bit 1 = not terrain-following either.  0: flat gather, 1:
// terrain-following gather, 3: cell loop.
constexpr unsigned kNotFlat = 1u, kNotSigma = 2u;
__device__ __forceinline__ bool mode_cells(unsigned m) { return (m & 3u) == 3u; }

// Terrain-following (sigma) levels: z_{q,m} = z_{q,0} + sigma_m D_q in every
// vertex column q, with sigma_m = (z_{0,m} - z_{0,0}) / D_0 from the column
// of vertex 0, D_q = z_{q,layers} - z_{q,0} > 0 and sigma increasing.  A
// DoF's z is accepted only where it provably lies within kSigmaTol D_q min_l (sigma_{l+1} -
// sigma_l) of that model (the probe: within kSigmaTol D_q times the smaller
// of its two adjacent layer spacings): every layer height then differs from
// sigma's by a relative 2 kSigmaTol = 4.5e-13 at most, which bounds the
// relative change of every element contribution.
constexpr double kSigmaTol = 0x1p-42;

__device__ __forceinline__ double sigma_at(const double *__restrict__ X, int layers, int m) {
  return (X[3 * (int64_t)m + 2] - X[2]) / (X[3 * (int64_t)layers + 2] - X[2]);
}

// Level tables (one thread per level, before the probe): tab[m] from the
// heights of column 0, tab[layers + 1 + m] from its sigma; the smallest sigma
// spacing (the complement of the bit pattern of a positive double, atomic max
// from the cleared word, in *minds); bit 1 of
// *mode when sigma does not increase (or D_0 is not positive).
__global__ void __launch_bounds__(256) k_p1_levels(const double *__restrict__ X, int layers,
                                                   LevelCoef *__restrict__ tab, unsigned int *__restrict__ mode,
                                                   unsigned long long *__restrict__ minds) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > layers) return;
  const int64_t col = (int64_t)layers + 1;
  const double z = X[3 * (int64_t)m + 2];
  const double hl = m > 0 ? fabs(z - X[3 * (int64_t)(m - 1) + 2]) : 0.0;
  const double hh = m < layers ? fabs(X[3 * (int64_t)(m + 1) + 2] - z) : 0.0;
  LevelCoef c;
  c.z = z;
  c.lo = hl;
  c.mid = 2.0 * (hl + hh);
  c.hi = hh;
  tab[m] = c;
  const double sg = sigma_at(X, layers, m);
  const double sl = m > 0 ? sg - sigma_at(X, layers, m - 1) : 0.0;
  const double sh = m < layers ? sigma_at(X, layers, m + 1) - sg : 0.0;
  LevelCoef cs;
  cs.z = sg;
  cs.lo = sl;
  cs.mid = 2.0 * (sl + sh);
  cs.hi = sh;
  tab[col + m] = cs;
  if (m < layers) {
    if (!(sh > 0.0)) atomicOr(mode, kNotSigma);  // also catches NaN (D_0 = 0)
    else atomicMax(minds, ~(unsigned long long)__double_as_longlong(sh));
  }
}

// alpha_c per cell, and the sampled probe over the DoFs of vertex columns
// q = s * stride, s < nsamp (all levels): bit 0 of *mode when a DoF is off
// its column's level-0 x, y or off its level's height in column 0, bit 1 when
// it is off its column's vertical or off the terrain-following model by more
// than kSigmaTol D_q times the smaller of its two adjacent sigma spacings (or
// D_q <= 0).  Reads the level tables of k_p1_levels.
__global__ void __launch_bounds__(256) k_p1_prep(const double *__restrict__ X, int layers, const int32_t *__restrict__ cmap,
                                                 int64_t ncells, int64_t nsamp, int64_t stride,
                                                 const LevelCoef *__restrict__ tab, double *__restrict__ alpha,
                                                 unsigned int *__restrict__ mode) {
  grid_dep_wait();  // a programmatic dependent of the launch before it
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  const int64_t col = (int64_t)layers + 1;
  unsigned bad = 0u;
  for (int64_t c = gid; c < ncells; c += gstride) {
    double x[3], y[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int64_t cb = __ldg(cmap + c * 6 + 2 * a);
      x[a] = __ldg(X + 3 * cb + 0);
      y[a] = __ldg(X + 3 * cb + 1);
    }
    alpha[c] = fabs((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0])) * (1.0 / 144.0);
  }
  for (int64_t i = gid; i < nsamp * col; i += gstride) {
    const int64_t s = i / col, m = i - s * col;
    const int64_t d0 = s * stride * col, d = d0 + m;
    const bool vert = (__double_as_longlong(__ldg(X + 3 * d + 0)) == __double_as_longlong(__ldg(X + 3 * d0 + 0))) &
                      (__double_as_longlong(__ldg(X + 3 * d + 1)) == __double_as_longlong(__ldg(X + 3 * d0 + 1)));
    const double z = __ldg(X + 3 * d + 2);
    if (vert && __double_as_longlong(z) == __double_as_longlong(__ldg(&tab[m].z))) continue;
    // not flat; a flat DoF also fits the terrain-following model (its column
    // has column 0's z_0 and D), so only the others need that test
    bad |= kNotFlat;
    const double z0 = __ldg(X + 3 * d0 + 2), D = __ldg(X + 3 * (d0 + layers) + 2) - z0;
    const LevelCoef ts = tab[col + m];
    const double gap = m == 0 ? ts.hi : (m == layers ? ts.lo : fmin(ts.lo, ts.hi));
    if (!vert || !(D > 0.0) || !(fabs(z - fma(ts.z, D, z0)) <= kSigmaTol * D * gap)) bad |= kNotSigma;
  }
  const unsigned wbad = __reduce_or_sync(kFull, bad);
  if (wbad && (threadIdx.x & 31) == 0) atomicOr(mode, wbad);
}

// Terrain-following gather only (mode 1): per vertex column q its D_q, z_q0
// and the acceptance bound B_q = kSigmaTol D_q min(sigma spacing) (-1 when
// D_q <= 0, so that no DoF of the column passes); per cell S_c = the sum of
// D over its three vertex columns.
__global__ void __launch_bounds__(256) k_p1_sigma_prep(const double *__restrict__ X, int layers,
                                                       const int32_t *__restrict__ cmap, int64_t ncells, int64_t nv,
                                                       const unsigned int *__restrict__ mode,
                                                       const unsigned long long *__restrict__ minds,
                                                       double *__restrict__ Dv, double *__restrict__ Z0,
                                                       double *__restrict__ Bv, double *__restrict__ S) {
  grid_dep_wait();  // a programmatic dependent of the launch before it
  if (*mode != kNotFlat) return;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  const int64_t col = (int64_t)layers + 1;
  const double gap = __longlong_as_double((long long)~*minds);
  for (int64_t v = gid; v < nv; v += gstride) {
    const double z0 = __ldg(X + 3 * v * col + 2);
    const double zl = __ldg(X + 3 * (v * col + layers) + 2);
    const double D = zl - z0;
    Dv[v] = D;
    Z0[v] = z0;
    // the bound in units in the last place of the column's largest |z| (a
    // column is monotonic, so its end levels hold that value): any z of the
    // column within kb units of its model, with the same sign, is within
    // kSigmaTol D gap of it
    const double zmax = fmax(fabs(z0), fabs(zl));
    const double ulp = __longlong_as_double(__double_as_longlong(zmax) + 1) - zmax;  // zmax >= 0
    const double kb = D > 0.0 && ulp > 0.0 ? floor(kSigmaTol * D * gap / ulp) : -1.0;
    Bv[v] = __longlong_as_double(kb < 0.0 ? -1LL : (kb > 4.0e18 ? (long long)4e18 : (long long)kb));
  }
  for (int64_t c = gid; c < ncells; c += gstride) {
    double sum = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int64_t cb = __ldg(cmap + c * 6 + 2 * a);
      sum += __ldg(X + 3 * (cb + layers) + 2) - __ldg(X + 3 * cb + 2);
    }
    S[c] = sum;
  }
}

// Row weights (gather modes only), one thread per vertex row.  Flat
// extrusion, Mh: entry (a, j) = the sum of alpha over the one or two cells on
// edge (a, j), ascending; the diagonal, the sum of 2 alpha over the cells
// around a, is formed as the sum of the row's off-diagonal entries.
// Terrain-following levels, Hd: a prism's heights are h_k = (sigma_{l+1} -
// sigma_l) D_k, so its element matrix under the 6-point rule is the column
// factor times (alpha_c / 54) sum_k D_k T_{aa'k}, with T = 54 sum_t lambda_a
// lambda_a' lambda_k over the three triangle points = 66 (a = a' = k), 21 (two
// equal), 12 (all different): entry (a, j) = sum_c alpha_c (9 (D_a + D_j) +
// 12 S_c) / 54 over the cells on the edge, diagonal = sum over the cells
// around a of alpha_c (45 D_a + 21 S_c) / 54, S_c the sum of the cell's D.
// (D = 1 gives Mh.)
__global__ void __launch_bounds__(256) k_p1_rowweights(const int32_t *__restrict__ vrow, const int32_t *__restrict__ vnbr,
                                                       const int2 *__restrict__ vedge, const int32_t *__restrict__ vcrow,
                                                       const int32_t *__restrict__ vcells,
                                                       const double *__restrict__ alpha, const double *__restrict__ Dv,
                                                       const double *__restrict__ S, double *__restrict__ wts,
                                                       int32_t nv, int64_t nent, FastDiv col,
                                                       const unsigned int *__restrict__ mode) {
  grid_dep_wait();  // a programmatic dependent of the launch before it
  const unsigned md = *mode;
  if (mode_cells(md)) return;
  const bool sig = (md & kNotFlat) != 0u;
  // one thread per vertex row; flat: the diagonal is the sum of the row's
  // off-diagonal weights (each cell around a lies on two of a's edges, so
  // that sum is sum_c 2 alpha_c), the row's loads all independent
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nv; a += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t0 = __ldg(vrow + a), t1 = __ldg(vrow + a + 1);
    double diag = 0.0;
    if (!sig) {
#pragma unroll 4
      for (int32_t t = t0 + 1; t < t1; ++t) {
        const int2 e = __ldg(vedge + t);
        const double w = e.y >= 0 ? __ldg(alpha + e.x) + __ldg(alpha + e.y) : __ldg(alpha + e.x);
        wts[t] = w;
        diag += w;
      }
    } else {
      const double Da = __ldg(Dv + a);
      for (int32_t t = t0 + 1; t < t1; ++t) {
        const int2 e = __ldg(vedge + t);
        const double Dj = __ldg(Dv + fdiv((uint32_t)__ldg(vnbr + t), col));
        const double dd = 9.0 * (Da + Dj);
        double w = __ldg(alpha + e.x) * fma(12.0, __ldg(S + e.x), dd);
        if (e.y >= 0) w = fma(__ldg(alpha + e.y), fma(12.0, __ldg(S + e.y), dd), w);
        wts[t] = w * (1.0 / 54.0);
      }
      for (int32_t t = __ldg(vcrow + a); t < __ldg(vcrow + a + 1); ++t) {
        const int32_t c = __ldg(vcells + t);
        diag = fma(__ldg(alpha + c), fma(21.0, __ldg(S + c), 45.0 * Da), diag);
      }
      diag *= 1.0 / 54.0;
    }
    wts[t0] = diag;
  }
}

#ifndef EXT_VTAB_MINB
#define EXT_VTAB_MINB 4  // resident 256-thread CTAs per SM of the table vertex pass
#endif
#ifndef EXT_VGATHER_MINB
#define EXT_VGATHER_MINB 4  // resident 256-thread CTAs per SM of the gather pass
#endif
#ifndef EXT_VT_VU
#define EXT_VT_VU 2  // 32-DoF chunks per warp step of the table vertex pass
#endif
#ifndef EXT_VSUM_BULK
#define EXT_VSUM_BULK 1  // 1: the table vertex pass with bulk copies (k_vsum_bulk); 0: plain loads (k_vsum_tab)
#endif
#ifndef EXT_VG_VU
#define EXT_VG_VU 1  // 32-DoF chunks per warp step of the gather
#endif
#ifndef EXT_VG_UNROLL
#define EXT_VG_UNROLL 4  // unrolling of the gather's row loop
#endif
constexpr int kVGUnroll = EXT_VG_UNROLL;

// Per vertex column arrays of the terrain-following gather (k_p1_sigma_prep).
struct SigmaCols {
  const double *Dv, *Z0, *Bv;
};

// z of a DoF of vertex column q at a level whose table entry holds zt (the
// height in column 0, or sigma): flat mode, bitwise equal; terrain-following
// mode, z and the model z_q0 + sigma D_q (one DFMA) of one sign and at most
// K_q apart as ordered bit patterns (integer ALU; K_q in units in the last
// place of the column's largest |z|, negative when nothing may pass).
__device__ __forceinline__ int z_ok(double z, double zt, bool sig, const SigmaCols &sc, uint32_t q, const Fp64Ones &k1) {
  (void)k1;
  if (!sig) return __double_as_longlong(z) == __double_as_longlong(zt);
  const long long bm = __double_as_longlong(fma(zt, __ldg(sc.Dv + q), __ldg(sc.Z0 + q)));
  const long long bz = __double_as_longlong(z);
  const long long dd = bz > bm ? bz - bm : bm - bz;
  return ((bz ^ bm) >= 0) & (dd <= __double_as_longlong(__ldg(sc.Bv + q)));
}

// DoF d is on its column's vertical (x, y of its level 0, bitwise) and at its
// level (z_ok)
__device__ __forceinline__ int dof_straight(const double *__restrict__ X, const LevelCoef *__restrict__ tab, int64_t d,
                                            FastDiv col, bool sig, const SigmaCols &sc, const Fp64Ones &k1) {
  const uint32_t q = fdiv((uint32_t)d, col);
  const uint32_t m = (uint32_t)d - q * col.d;
  const int64_t d0 = (int64_t)q * col.d;
  return (__double_as_longlong(__ldg(X + 3 * d + 0)) == __double_as_longlong(__ldg(X + 3 * d0 + 0))) &
         (__double_as_longlong(__ldg(X + 3 * d + 1)) == __double_as_longlong(__ldg(X + 3 * d0 + 1))) &
         z_ok(__ldg(X + 3 * d + 2), __ldg(&tab[m].z), sig, sc, q, k1);
}

template <bool SIG>
__global__ void __launch_bounds__(256, EXT_VTAB_MINB) k_vsum_tab(const double *__restrict__ X, const double *__restrict__ f,
                                                                const LevelCoef *__restrict__ tab0,
                                                                double *__restrict__ W, int64_t n, FastDiv col,
                                                                Fp64Ones k1, const unsigned int *__restrict__ mode,
                                                                SigmaCols sc) {
  const unsigned md = *mode;
  if (mode_cells(md) || ((md & kNotFlat) != 0u) != SIG) return;
  const LevelCoef *__restrict__ tab = SIG ? tab0 + col.d : tab0;
  constexpr int VU = EXT_VT_VU;
  const int lane = threadIdx.x & 31;
  const int64_t wstride = (int64_t)gridDim.x * 8 * 32 * VU;
  for (int64_t base = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * 32 * VU; base < n; base += wstride) {
    double fc[VU], clo[VU], cmid[VU], chi[VU];
    int ok[VU];
    uint32_t mm[VU];
#pragma unroll
    for (int u = 0; u < VU; ++u) {
      const int64_t d = base + u * 32 + lane;
      fc[u] = 0.0;
      clo[u] = cmid[u] = chi[u] = 0.0;
      ok[u] = 1;
      mm[u] = 0;
      if (d < n) {
        const uint32_t q = fdiv((uint32_t)d, col);
        mm[u] = (uint32_t)d - q * col.d;
        const double2 t0 = __ldg(reinterpret_cast<const double2 *>(tab + mm[u]));
        const double2 t1 = __ldg(reinterpret_cast<const double2 *>(tab + mm[u]) + 1);
        clo[u] = t0.y;
        cmid[u] = t1.x;
        chi[u] = t1.y;
        const int64_t d0 = (int64_t)q * col.d;
        ok[u] = (__double_as_longlong(__ldg(X + 3 * d + 0)) == __double_as_longlong(__ldg(X + 3 * d0 + 0))) &
                (__double_as_longlong(__ldg(X + 3 * d + 1)) == __double_as_longlong(__ldg(X + 3 * d0 + 1))) &
                z_ok(__ldg(X + 3 * d + 2), t0.x, SIG, sc, q, k1);
        fc[u] = __ldg(f + d);
      }
    }
    // the DoF before the first chunk and after the last one
    double fb = 0.0, fa = 0.0;
    int okb = 1, oka = 1;
    if (lane == 0 && base > 0 && base - 1 < n) {
      fb = __ldg(f + base - 1);
      okb = dof_straight(X, tab, base - 1, col, SIG, sc, k1);
    }
    if (lane == 31 && base + 32 * VU < n) {
      fa = __ldg(f + base + 32 * VU);
      oka = dof_straight(X, tab, base + 32 * VU, col, SIG, sc, k1);
    }
#pragma unroll
    for (int u = 0; u < VU; ++u) {
      const int64_t d = base + u * 32 + lane;
      // left neighbour: previous lane (lane 0: the previous chunk's lane 31,
      // or the DoF before the first chunk); right neighbour likewise
      double fl = __shfl_up_sync(kFull, fc[u], 1), fr = __shfl_down_sync(kFull, fc[u], 1);
      int okl = __shfl_up_sync(kFull, ok[u], 1), okr = __shfl_down_sync(kFull, ok[u], 1);
      double flp = fb, frn = fa;
      int oklp = okb, okrn = oka;
      if (u > 0) {
        flp = __shfl_sync(kFull, fc[u > 0 ? u - 1 : 0], 31);
        oklp = __shfl_sync(kFull, ok[u > 0 ? u - 1 : 0], 31);
      }
      if (u + 1 < VU) {
        frn = __shfl_sync(kFull, fc[u + 1 < VU ? u + 1 : u], 0);
        okrn = __shfl_sync(kFull, ok[u + 1 < VU ? u + 1 : u], 0);
      }
      if (lane == 0) {
        fl = flp;
        okl = oklp;
      }
      if (lane == 31) {
        fr = frn;
        okr = okrn;
      }
      const bool lo_end = mm[u] == 0, hi_end = mm[u] + 1 == col.d;
      // the neighbour across a column end is cleared bitwise (an integer AND)
      fl = __longlong_as_double(__double_as_longlong(fl) & (lo_end ? 0LL : -1LL));
      fr = __longlong_as_double(__double_as_longlong(fr) & (hi_end ? 0LL : -1LL));
      const int good = ok[u] & (lo_end | okl) & (hi_end | okr);
      const double w = fma(clo[u], fl, fma(cmid[u], fc[u], fmul(chi[u], fr, k1)));
      if (d < n) W[d] = good ? w : __longlong_as_double(kNotVertical);
    }
  }
}

// The same vertex pass with bulk copies.  A warp step covers 64 DoFs
// [base, base + 64); the coordinates (24 bytes per DoF) and f (8 bytes) of
// the DoFs base - 2 .. base + 65 are copied into one of the warp's two
// shared-memory stages by the bulk-copy engine (cp.async.bulk, completion
// counted in bytes on an mbarrier), the next step's copy in flight while the
// current step is computed.  A step starts at an even DoF, so with 16-byte
// aligned X and f every copy starts on a 16-byte boundary and has a length
// that is a multiple of 16; a step whose clamped range is odd (the last one,
// when n is odd) is filled by the lanes with plain loads.  A warp issues the
// next step's copy only after the wait for the current one has succeeded, so
// at most one of its copies is unconfirmed at any time.  Every wait is
// bounded: when it runs out the warp sets EXT_DERR_TIMEOUT, waits once more
// (bounded) for that copy and returns.  Test hook: skip_step >= 0 makes lane
// 0 of the warp that owns that step leave its copy out (no arrival on the
// barrier either), so the wait runs out with no copy in flight; wait_limit
// is then small.
constexpr int kBulkDofs = 64;              // DoFs per warp step
constexpr int kBulkSpan = kBulkDofs + 4;   // with two DoFs before and two after
constexpr unsigned kBulkWaitLimit = 1u << 22;  // polls of an mbarrier before giving up

struct __align__(16) BulkStage {
  double X[3 * kBulkSpan];
  double f[kBulkSpan];
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, unsigned limit) {
  for (unsigned i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// DoF range [lo, hi) of the step at `base`, clamped to [0, n), and whether
// bulk copies can fetch it (even length; the start is even by construction)
__device__ __forceinline__ void bulk_range(int64_t base, int64_t n, int64_t &lo, int64_t &hi, bool &bulk, bool aligned) {
  lo = base - 2 > 0 ? base - 2 : 0;
  hi = base + kBulkDofs + 2 < n ? base + kBulkDofs + 2 : n;
  bulk = aligned && ((hi - lo) & 1) == 0;
}

template <bool SIG>
__global__ void __launch_bounds__(256, EXT_VTAB_MINB) k_vsum_bulk(const double *__restrict__ X, const double *__restrict__ f,
                                                                 const LevelCoef *__restrict__ tab0,
                                                                 double *__restrict__ W, int64_t n, FastDiv col,
                                                                 Fp64Ones k1, unsigned int *err,
                                                                 const unsigned int *__restrict__ mode, SigmaCols sc,
                                                                 int64_t skip_step, unsigned wait_limit) {
  grid_dep_wait();  // a programmatic dependent of the launch before it
  // one instantiation per gather mode (flat: SIG = false); the other exits,
  // as both do in cell-loop mode
  const unsigned md = *mode;
  if (mode_cells(md) || ((md & kNotFlat) != 0u) != SIG) return;
  const LevelCoef *__restrict__ tab = SIG ? tab0 + col.d : tab0;
  __shared__ BulkStage stage[8][2];
  __shared__ __align__(8) uint64_t bar[8][2];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const bool aligned = ((((uintptr_t)X) | ((uintptr_t)f)) & 15) == 0;
  if (lane == 0) {
    for (int q = 0; q < 2; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[warp][q])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const int64_t nsteps = (n + kBulkDofs - 1) / kBulkDofs;
  const int64_t wstride = (int64_t)gridDim.x * 8;
  // lane 0 starts the copies of a step into stage q
  auto issue = [&](int64_t stp, int q) {
    int64_t lo, hi;
    bool bulk;
    bulk_range(stp * kBulkDofs, n, lo, hi, bulk, aligned);
    if (bulk && lane == 0 && stp != skip_step) {
      const int64_t off = lo - (stp * kBulkDofs - 2);  // 0, or 2 for the first step
      const unsigned bx = (unsigned)(24 * (hi - lo)), bf = (unsigned)(8 * (hi - lo));
      const uint32_t b = smem_addr(&bar[warp][q]);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bx + bf) : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_addr(&stage[warp][q].X[3 * off])),
                   "l"(X + 3 * lo), "r"(bx), "r"(b)
                   : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_addr(&stage[warp][q].f[off])),
                   "l"(f + lo), "r"(bf), "r"(b)
                   : "memory");
    }
  };
  int64_t stp = (int64_t)blockIdx.x * 8 + warp;
  if (stp < nsteps) issue(stp, 0);
  unsigned use0 = 0u, use1 = 0u;  // completed uses of each stage's barrier (their parity is the phase to wait for)
  for (int it = 0; stp < nsteps; stp += wstride, ++it) {
    const int q = it & 1;
    const int64_t nxt = stp + wstride;
    const int64_t base = stp * kBulkDofs;
    int64_t lo, hi;
    bool bulk;
    bulk_range(base, n, lo, hi, bulk, aligned);
    BulkStage &sg = stage[warp][q];
    if (bulk) {
      const unsigned par = (q ? use1 : use0) & 1u;
      if (!mbar_wait_bounded(&bar[warp][q], par, wait_limit)) {
        // the only unconfirmed copy of this warp is this stage's
        if (lane == 0) atomicOr(err, EXT_DERR_TIMEOUT);
        (void)mbar_wait_bounded(&bar[warp][q], par, wait_limit);
        return;
      }
      if (q) ++use1;
      else ++use0;
    }
    __syncwarp();  // every lane is done with stage q ^ 1 (the previous step)
    if (nxt < nsteps) issue(nxt, q ^ 1);
    if (!bulk) {
      for (int64_t d = lo + lane; d < hi; d += 32) {
        const int64_t r = d - (base - 2);
        sg.X[3 * r + 0] = __ldg(X + 3 * d + 0);
        sg.X[3 * r + 1] = __ldg(X + 3 * d + 1);
        sg.X[3 * r + 2] = __ldg(X + 3 * d + 2);
        sg.f[r] = __ldg(f + d);
      }
      __syncwarp();
    }
    // stage row r holds DoF base - 2 + r
    auto ok_row = [&](int r, int64_t d) {
      const uint32_t qv = fdiv((uint32_t)d, col);
      const uint32_t m = (uint32_t)d - qv * col.d;
      const int64_t d0 = (int64_t)qv * col.d;
      return (__double_as_longlong(sg.X[3 * r + 0]) == __double_as_longlong(__ldg(X + 3 * d0 + 0))) &
             (__double_as_longlong(sg.X[3 * r + 1]) == __double_as_longlong(__ldg(X + 3 * d0 + 1))) &
             z_ok(sg.X[3 * r + 2], __ldg(&tab[m].z), SIG, sc, qv, k1);
    };
    int ok[2];
    uint32_t mm[2];
    double clo[2], cmid[2], chi[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t d = base + 32 * u + lane;
      ok[u] = 1;
      mm[u] = 0;
      clo[u] = cmid[u] = chi[u] = 0.0;
      if (d < n) {
        const uint32_t qv = fdiv((uint32_t)d, col);
        mm[u] = (uint32_t)d - qv * col.d;
        const double2 t0 = __ldg(reinterpret_cast<const double2 *>(tab + mm[u]));
        const double2 t1 = __ldg(reinterpret_cast<const double2 *>(tab + mm[u]) + 1);
        clo[u] = t0.y;
        cmid[u] = t1.x;
        chi[u] = t1.y;
        const int r = 32 * u + lane + 2;
        const int64_t d0 = (int64_t)qv * col.d;
        ok[u] = (__double_as_longlong(sg.X[3 * r + 0]) == __double_as_longlong(__ldg(X + 3 * d0 + 0))) &
                (__double_as_longlong(sg.X[3 * r + 1]) == __double_as_longlong(__ldg(X + 3 * d0 + 1))) &
                z_ok(sg.X[3 * r + 2], t0.x, SIG, sc, qv, k1);
      }
    }
    // straightness of the DoFs just outside the step (lanes 0 and 31 in one pass)
    int okx = 1;
    if ((lane == 0 && base > 0) || (lane == 31 && base + kBulkDofs < n)) {
      const int rx = lane == 0 ? 1 : kBulkDofs + 2;
      const int64_t dx = lane == 0 ? base - 1 : base + kBulkDofs;
      okx = ok_row(rx, dx);
    }
    const int okb = okx, oka = okx;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t d = base + 32 * u + lane;
      const int r = 32 * u + lane + 2;
      int okl = __shfl_up_sync(kFull, ok[u], 1), okr = __shfl_down_sync(kFull, ok[u], 1);
      const int oklp = u > 0 ? __shfl_sync(kFull, ok[0], 31) : okb;
      const int okrn = u == 0 ? __shfl_sync(kFull, ok[1], 0) : oka;
      if (lane == 0) okl = oklp;
      if (lane == 31) okr = okrn;
      const bool lo_end = mm[u] == 0, hi_end = mm[u] + 1 == col.d;
      // neighbours across a column end (or outside the array) are cleared bitwise
      const double fl = __longlong_as_double(__double_as_longlong(sg.f[r - 1]) & (lo_end ? 0LL : -1LL));
      const double fr = __longlong_as_double(__double_as_longlong(sg.f[r + 1]) & (hi_end ? 0LL : -1LL));
      const int good = ok[u] & (lo_end | okl) & (hi_end | okr);
      const double w = fma(clo[u], fl, fma(cmid[u], sg.f[r], fmul(chi[u], fr, k1)));
      if (d < n) W[d] = good ? w : __longlong_as_double(kNotVertical);
    }
  }
}


template <bool INC>
__global__ void __launch_bounds__(256, EXT_VGATHER_MINB) k_vgather(const double *__restrict__ W,
                                                                   const int32_t *__restrict__ vrow,
                                                                   const int32_t *__restrict__ vnbr,
                                                                   const double *__restrict__ wts,
                                                                   double *__restrict__ b, int64_t n, FastDiv col,
                                                                   Deferred dfr, unsigned int *err, Fp64Ones k1,
                                                                   const unsigned int *__restrict__ mode,
                                                                   unsigned skip_modes) {
  grid_dep_wait();  // a programmatic dependent of the launch before it
  constexpr int VU = EXT_VG_VU;
  const int lane = threadIdx.x & 31;
  // bit m of skip_modes: in gather mode m (0 flat, 1 terrain-following) a
  // one-pass kernel (k_vfused, k_p1_opt) formed b
  if (!mode_cells(*mode) && ((skip_modes >> *mode) & 1u)) return;
  if (mode_cells(*mode)) {
    // cell-loop mode: k_p1_cells adds every contribution; WRITE clears b first
    if (!INC)
      for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < n; d += (int64_t)gridDim.x * blockDim.x)
        b[d] = 0.0;
    return;
  }
  const int64_t wstride = (int64_t)gridDim.x * 8 * 32 * VU;
  for (int64_t base = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * 32 * VU; base < n; base += wstride) {
    int r0[VU], deg[VU];
    uint32_t mm[VU];
    double acc[VU];
    int dmx = 0;
#pragma unroll
    for (int u = 0; u < VU; ++u) {
      const int64_t d = base + u * 32 + lane;
      r0[u] = 0;
      deg[u] = 0;
      mm[u] = 0;
      acc[u] = k1.mzero;  // WRITE: the first product is added to -0, which leaves it exact
      if (d < n) {
        const uint32_t q = fdiv((uint32_t)d, col);
        mm[u] = (uint32_t)d - q * col.d;
        r0[u] = __ldg(vrow + q);
        deg[u] = __ldg(vrow + q + 1) - r0[u];
        if (INC) acc[u] = b[d];
      }
      const int dm = __reduce_max_sync(kFull, deg[u]);
      dmx = dm > dmx ? dm : dmx;
    }
    // one product per row entry up to the warp's longest row; past its own
    // row a lane multiplies zeros.  The trip count is the loop bound (no
    // guarded products, which the compiler turns into a product and a select)
#pragma unroll kVGUnroll
    for (int t = 0; t < dmx; ++t) {
      double ev[VU], wv[VU];
#pragma unroll
      for (int u = 0; u < VU; ++u) {
        ev[u] = 0.0;
        wv[u] = 0.0;
        if (t < deg[u]) {
          ev[u] = __ldg(wts + r0[u] + t);
          wv[u] = __ldg(W + (int64_t)__ldg(vnbr + r0[u] + t) + mm[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < VU; ++u) acc[u] = fma(ev[u], wv[u], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < VU; ++u) {
      const int64_t d = base + u * 32 + lane;
      // NaN test on the bit pattern (integer ALU)
      const bool bad = d < n && (__double_as_longlong(acc[u]) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
      if (d < n && !bad) b[d] = acc[u];
      const unsigned int mask = __ballot_sync(kFull, bad);
      if (mask != 0u && lane == 0) {
        const unsigned int slot = atomicAdd(dfr.count, 1u);
        if (slot < dfr.cap) dfr.list[slot] = make_int2((int)(base + u * 32), (int)mask);
        else atomicOr(err, EXT_DERR_BOUNDS);
      }
    }
  }
}

// Flat gather in one pass (flat mode only): b = Mh (x) Mv f evaluated as
// b_{a,m} = lo_m g_{a,m-1} + mid_m g_{a,m} + hi_m g_{a,m+1} with g_{a,m} =
// sum over the vertex row of a of weight x f_{j,m}, so no vertical sums are
// stored and read back.  A warp step covers 32 consecutive DoFs, d = start - 1
// .. start + 30: every lane forms g of its own DoF (one DFMA per row entry),
// and lanes 1..30 take their lower and upper neighbours' g by shuffles and
// write b of DoFs start .. start + 29 (lanes 0 and 31 only supply the halo).
// While it walks the row, each lane checks bitwise that every f_{j,m} it uses
// sits on a straight flat DoF (x, y of column j's level 0, z of level m in
// column 0); a DoF whose own check or a vertical neighbour's fails, or whose
// sum comes out NaN, is recorded for k_vgather_general instead of written.
template <bool INC>
__global__ void __launch_bounds__(256, EXT_VGATHER_MINB) k_vfused(const double *__restrict__ X,
                                                                  const double *__restrict__ f,
                                                                  const int32_t *__restrict__ vrow,
                                                                  const int32_t *__restrict__ vnbr,
                                                                  const double *__restrict__ wts,
                                                                  const LevelCoef *__restrict__ tab,
                                                                  double *__restrict__ b, int64_t n, FastDiv col,
                                                                  Deferred dfr, unsigned int *err, Fp64Ones k1,
                                                                  const unsigned int *__restrict__ mode) {
  grid_dep_wait();  // a programmatic dependent of the launch before it
  if (*mode != 0u) return;  // terrain-following or cell-loop mode
  const int lane = threadIdx.x & 31;
  constexpr int kOut = 30;
  const int64_t nsteps = (n + kOut - 1) / kOut;
  const int64_t wstride = (int64_t)gridDim.x * 8;
  for (int64_t stp = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); stp < nsteps; stp += wstride) {
    const int64_t start = stp * kOut;
    const int64_t d = start - 1 + lane;
    const bool in = d >= 0 && d < n;
    int r0 = 0, deg = 0;
    uint32_t m = 0;
    double acc = k1.mzero, zl = 0.0;
    double2 c01 = make_double2(0.0, 0.0), c23 = make_double2(0.0, 0.0);
    if (in) {
      const uint32_t q = fdiv((uint32_t)d, col);
      m = (uint32_t)d - q * col.d;
      r0 = __ldg(vrow + q);
      deg = __ldg(vrow + q + 1) - r0;
      c01 = __ldg(reinterpret_cast<const double2 *>(tab + m));      // z_m, |h_{m-1}|
      c23 = __ldg(reinterpret_cast<const double2 *>(tab + m) + 1);  // 2 (|h_{m-1}| + |h_m|), |h_m|
      zl = c01.x;
    }
    const long long zbits = __double_as_longlong(zl);
    int ok = 1;
    const int dmx = __reduce_max_sync(kFull, deg);
#pragma unroll 4
    for (int t = 0; t < dmx; ++t) {
      double ev = 0.0, fv = 0.0;
      if (t < deg) {
        const int64_t j0 = __ldg(vnbr + r0 + t);  // first DoF of column j
        const int64_t dj = j0 + m;
        ev = __ldg(wts + r0 + t);
        fv = __ldg(f + dj);
        ok &= (__double_as_longlong(__ldg(X + 3 * dj + 0)) == __double_as_longlong(__ldg(X + 3 * j0 + 0))) &
              (__double_as_longlong(__ldg(X + 3 * dj + 1)) == __double_as_longlong(__ldg(X + 3 * j0 + 1))) &
              (__double_as_longlong(__ldg(X + 3 * dj + 2)) == zbits);
      }
      acc = fma(ev, fv, acc);
    }
    // vertical neighbours (lanes -1 and +1, the same column unless at its end)
    const bool lo_end = m == 0, hi_end = m + 1 == col.d;
    const double gl = __shfl_up_sync(kFull, acc, 1), gr = __shfl_down_sync(kFull, acc, 1);
    const int okl = __shfl_up_sync(kFull, ok, 1), okr = __shfl_down_sync(kFull, ok, 1);
    const double glm = __longlong_as_double(__double_as_longlong(gl) & (lo_end ? 0LL : -1LL));
    const double grm = __longlong_as_double(__double_as_longlong(gr) & (hi_end ? 0LL : -1LL));
    double res = fma(c01.y, glm, fma(c23.x, acc, fmul(c23.y, grm, k1)));
    const bool out = lane >= 1 && lane <= kOut && in;
    const int good = ok & (lo_end | okl) & (hi_end | okr);
    if (INC && out) res = fadd(res, b[d], k1);
    const bool nan = (__double_as_longlong(res) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
    const bool bad = out && (!good || nan);
    if (out && !bad) b[d] = res;
    const unsigned int mask = __ballot_sync(kFull, bad) >> 1;  // bit i: DoF start + i
    if (mask != 0u && lane == 0) {
      const unsigned int slot = atomicAdd(dfr.count, 1u);
      if (slot < dfr.cap) dfr.list[slot] = make_int2((int)start, (int)mask);
      else atomicOr(err, EXT_DERR_BOUNDS);
    }
  }
}

#ifndef EXT_P1OPT_MINB
#define EXT_P1OPT_MINB 4  // resident 256-thread CTAs per SM of the optimistic flat gather
#endif
#ifndef EXT_P1OPT_UF
#define EXT_P1OPT_UF 2  // flag words per lane per flag chunk
#endif
#ifndef EXT_P1OPT_R
#define EXT_P1OPT_R 2  // 32-DoF blocks per gather chunk (it writes 32 R - 2 DoFs; 1M x 100: R = 1, 2, 4, 8 took 1.07, 1.04, 1.21, 1.15 ms)
#endif

// Optimistic flat gather (flat mode, WRITE access).  The one-pass flat
// gather of k_vfused checks, for every row entry it reads, that the DoF sits
// on a straight flat extrusion; here nothing is checked in the gather:
// b = Mh (x) Mv f is formed for every DoF as if the whole mesh were straight
// and flat (g_{a,m} = the row of a against f at level m, then
// b_{a,m} = lo_m g_{a,m-1} + mid_m g_{a,m} + hi_m g_{a,m+1} by warp shuffles,
// each g formed once within a chunk of 32 R DoFs), while the same launch
// sets one straightness bit per coordinate DoF (x, y of its column's level 0
// and z of its level in column 0, bitwise), one bit per vertex column holding
// a DoF that fails, and one word per CTA saying whether it saw such a DoF.
// The warps take flag chunks and gather chunks interleaved in proportion to
// their counts, so
// the HBM-bound flag work runs beside the FP64-bound gather on every SM, and
// the coordinate field is read once.  k_p1_fix then records, for the general
// path, every DoF whose stencil (the vertex row's columns at levels m - 1 ..
// m + 1) holds a DoF that is not straight; it exits at once when no CTA saw
// one.  So each DoF keeps the Kronecker value exactly when its stencil is
// verified straight and flat, as in the split form.  A NaN in f reaches
// exactly the DoFs whose stencil holds it, as it would through the general
// path.
__global__ void __launch_bounds__(256, EXT_P1OPT_MINB)
    k_p1_opt(const double *__restrict__ X, const double *__restrict__ f, const int32_t *__restrict__ vrow,
             const int32_t *__restrict__ vnbr, const double *__restrict__ wts, const LevelCoef *__restrict__ tab,
             double *__restrict__ b, uint32_t n, FastDiv col, uint32_t *__restrict__ flags,
             uint32_t *__restrict__ vbad, int32_t *__restrict__ badv, Fp64Ones k1,
             const unsigned int *__restrict__ mode, SigmaCols sc, int64_t nfc, int64_t ngc) {
  grid_dep_wait();  // a programmatic dependent of the launch before it
  constexpr int UF = EXT_P1OPT_UF, R = EXT_P1OPT_R;
  __shared__ int cta_bad;
  const unsigned md = *mode;
  if (mode_cells(md)) return;  // cell-loop mode (k_p1_fix exits too)
  // terrain-following mode: the depth-weighted rows, the sigma table and the
  // model check of z (z_ok) in place of the flat ones
  const bool sig = (md & kNotFlat) != 0u;
  const LevelCoef *__restrict__ ct = sig ? tab + col.d : tab;
  if (blockIdx.x == 0 && threadIdx.x == 0) flags[(n + 31) / 32] = 0u;  // the zero word past the end
  if (threadIdx.x == 0) cta_bad = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t nwords = (n + 31) / 32;
  const int64_t nch = nfc + ngc;
  const int64_t wstride = (int64_t)gridDim.x * 8;
  bool bad = false;
  // Bresenham's interleave of the nfc flag chunks among the nch chunks, as in
  // the nine-space optimistic form (no division in the loop)
  const int64_t j0 = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
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
      const uint32_t dbase = (uint32_t)fcur * (uint32_t)(UF * 32) + (uint32_t)lane;
      long long x[UF], y[UF], x0[UF], y0[UF];
      double z[UF], zt[UF];
      uint32_t qv[UF];
      bool v[UF];
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const uint32_t d = dbase + (uint32_t)(u * 32);
        v[u] = d < n;
        x[u] = y[u] = x0[u] = y0[u] = 0;
        z[u] = zt[u] = 0.0;
        qv[u] = 0;
        if (v[u]) {
          const uint32_t q = fdiv(d, col);
          const uint32_t m = d - q * col.d;
          const double *xp = X + 3 * (size_t)d;
          const double *x0p = X + 3 * (size_t)(q * col.d);
          qv[u] = q;
          x[u] = __double_as_longlong(__ldg(xp + 0));
          y[u] = __double_as_longlong(__ldg(xp + 1));
          z[u] = __ldg(xp + 2);
          x0[u] = __double_as_longlong(__ldg(x0p + 0));
          y0[u] = __double_as_longlong(__ldg(x0p + 1));
          zt[u] = __ldg(&ct[m].z);
        }
      }
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const uint32_t w = (uint32_t)fcur * (uint32_t)UF + (uint32_t)u;
        const bool ok = v[u] && x[u] == x0[u] && y[u] == y0[u] && z_ok(z[u], zt[u], sig, sc, qv[u], k1);
        const unsigned int word = __ballot_sync(kFull, ok);
        const unsigned int want = __ballot_sync(kFull, v[u]);
        if (w < nwords) {
          if (lane == 0) flags[w] = word;
          bad |= word != want;
        }
        if (v[u] && !ok) atomicOr(vbad + (qv[u] >> 5), 1u << (qv[u] & 31u));
      }
    } else {
      // gather chunk (j - fcur): R blocks of 32 consecutive DoFs d = cs - 1 +
      // 32 t + lane; g of block t and of block t - 1 (kept in gprev) give the
      // output DoF e = d - 1 of every lane: g(e - 1), g(e), g(e + 1) from
      // lanes - 2, - 1 and 0 (the previous block's lanes 30 and 31 below lane
      // 2).  The chunk writes DoFs cs .. cs + 32 R - 3 and forms g of each
      // once, except for the two DoFs it shares with the next chunk.
      const int64_t cs = (j - fcur) * (int64_t)(32 * R - 2);
      double gprev = 0.0;
#pragma unroll 1
      for (int t = 0; t < R; ++t) {
        const int64_t d = cs - 1 + 32 * t + lane;
        int r0 = 0, deg = 0;
        uint32_t m = 0;
        double acc = k1.mzero;
        if (d >= 0 && d < (int64_t)n) {
          const uint32_t q = fdiv((uint32_t)d, col);
          m = (uint32_t)d - q * col.d;
          r0 = __ldg(vrow + q);
          deg = __ldg(vrow + q + 1) - r0;
        }
        const int dmx = __reduce_max_sync(kFull, deg);
#pragma unroll 4
        for (int u = 0; u < dmx; ++u) {
          double ev = 0.0, fv = 0.0;
          if (u < deg) {
            ev = __ldg(wts + r0 + u);
            fv = __ldg(f + (uint32_t)__ldg(vnbr + r0 + u) + m);
          }
          acc = fma(ev, fv, acc);
        }
        const double g1 = __shfl_up_sync(kFull, acc, 1), g2 = __shfl_up_sync(kFull, acc, 2);
        const double p30 = __shfl_sync(kFull, gprev, 30), p31 = __shfl_sync(kFull, gprev, 31);
        gprev = acc;
        const int64_t e = d - 1;
        if (e >= cs && e < (int64_t)n) {
          const uint32_t qe = fdiv((uint32_t)e, col);
          const uint32_t me = (uint32_t)e - qe * col.d;
          const double2 c01 = __ldg(reinterpret_cast<const double2 *>(ct + me));      // z_m, |h_{m-1}|
          const double2 c23 = __ldg(reinterpret_cast<const double2 *>(ct + me) + 1);  // 2 (|h_{m-1}| + |h_m|), |h_m|
          const double gm = lane >= 2 ? g2 : (lane == 1 ? p31 : p30);  // g(e - 1)
          const double g0 = lane >= 1 ? g1 : p31;                      // g(e)
          // vertical neighbours beyond the column's ends are cleared bitwise
          const double gmm = __longlong_as_double(__double_as_longlong(gm) & (me == 0 ? 0LL : -1LL));
          const double gpm = __longlong_as_double(__double_as_longlong(acc) & (me + 1 == col.d ? 0LL : -1LL));
          b[e] = fma(c01.y, gmm, fma(c23.x, g0, fmul(c23.y, gpm, k1)));
        }
      }
    }
  }
  if (bad && lane == 0) cta_bad = 1;
  __syncthreads();
  if (threadIdx.x == 0) badv[blockIdx.x] = cta_bad;
}

// bits pos .. pos + 31 of a bitmap (which holds a zero word past its end)
__device__ __forceinline__ uint32_t bits32(const uint32_t *__restrict__ bm, uint32_t pos) {
  const uint32_t w = pos >> 5, s = pos & 31u;
  const uint32_t lo = __ldg(bm + w) >> s;
  return s ? lo | (__ldg(bm + w + 1) << (32u - s)) : lo;
}

// Fix-up of the optimistic flat gather: returns at once unless a CTA of
// k_p1_opt saw a coordinate DoF that is not straight.  Then one thread per
// vertex column a whose row (a and its neighbours) holds a column with such a
// DoF records, 32 levels at a time, the DoFs b_{a,m} whose stencil (row
// columns at levels m - 1, m, m + 1) holds one, for k_vgather_general.
__global__ void __launch_bounds__(256) k_p1_fix(const int32_t *__restrict__ vrow, const int32_t *__restrict__ vnbr,
                                                const uint32_t *__restrict__ flags, const uint32_t *__restrict__ vbad,
                                                const int32_t *__restrict__ badv, int32_t nbadv, uint32_t nverts,
                                                FastDiv col, Deferred dfr, unsigned int *err,
                                                const unsigned int *__restrict__ mode) {
  grid_dep_wait();  // a programmatic dependent of the launch before it
  if (mode_cells(*mode)) return;
  int any = 0;
  for (int i = threadIdx.x; i < nbadv; i += blockDim.x) any |= __ldg(badv + i);
  if (!__syncthreads_or(any)) return;
  const uint32_t L1 = col.d;
  for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < nverts; a += gridDim.x * blockDim.x) {
    const int32_t r0 = __ldg(vrow + a), r1 = __ldg(vrow + a + 1);
    bool hit = false;
    for (int32_t t = r0; t < r1 && !hit; ++t) {
      const uint32_t jv = fdiv((uint32_t)__ldg(vnbr + t), col);
      hit = (__ldg(vbad + (jv >> 5)) >> (jv & 31u)) & 1u;
    }
    if (!hit) continue;
    for (uint32_t lo = 0; lo < L1; lo += 32) {
      const uint32_t nl = L1 - lo < 32 ? L1 - lo : 32;  // levels lo .. lo + nl - 1 of this word
      const uint32_t valid = nl == 32 ? 0xffffffffu : (1u << nl) - 1u;
      uint32_t B = 0, below = 0, above = 0;  // not straight: at lo + i, at lo - 1, at lo + 32
      for (int32_t t = r0; t < r1; ++t) {
        const uint32_t j0 = (uint32_t)__ldg(vnbr + t);
        B |= ~bits32(flags, j0 + lo) & valid;
        if (lo > 0) below |= ~bits32(flags, j0 + lo - 1) & 1u;
        if (lo + 32 < L1) above |= ~bits32(flags, j0 + lo + 32) & 1u;
      }
      const uint32_t need = (B | (B << 1) | (B >> 1) | below | (above << 31)) & valid;
      if (need) {
        const unsigned int slot = atomicAdd(dfr.count, 1u);
        if (slot < dfr.cap) dfr.list[slot] = make_int2((int)(a * L1 + lo), (int)need);
        else atomicOr(err, EXT_DERR_BOUNDS);
      }
    }
  }
}

// CG1 x DG0 and CG1 x DG1 (horizontal CG1, vertical DG; WRITE access,
// constant layers, the gather modes of the probe).  On a straight extrusion
// with flat (or terrain-following) levels the element matrix of prism (c, l)
// is the base triangle's row block times the vertical DG mass of layer l, so
// M = Hd (x) Mv_DG with Mv_DG block diagonal over the layers: DG0, Delta_l;
// DG1, (Delta_l / 6) [[2, 1], [1, 2]] (Delta_l = |h_l|, or the sigma spacing
// with Hd depth-weighted), and Hd = 6 x the row weights of the P1xP1 gather.
// The DoF of vertex a, layer l, node beta is a NV lambda + NV l + beta
// (Algorithm 1: vertex columns first, NV DoFs per layer), so every neighbour
// column j of a's row is read at the same offset r = NV l + beta:
// g = sum_t w_t f[j_t NV lambda + r]; then b = 6 Delta_l g (DG0) or
// Delta_l (2 g_beta + g_{1-beta}) (DG1: the pair beta, 1 - beta sits in lanes
// d and d ^ 1, one shuffle).  No atomics: every DoF is written once.  The
// straightness flags of the coordinate DoFs are set beside it, in the same
// chunks as k_p1_opt; k_cgdg_fix records the DoFs whose layer's prisms touch
// a coordinate DoF that is not straight, for the general rule.
template <int NV>
__global__ void __launch_bounds__(256, EXT_P1OPT_MINB)
    k_cgdg_opt(const double *__restrict__ X, const double *__restrict__ f, const int32_t *__restrict__ vrow,
               const int32_t *__restrict__ vnbr, const double *__restrict__ wts, const LevelCoef *__restrict__ tab,
               double *__restrict__ b, uint32_t ncoord, uint32_t nf, FastDiv col, FastDiv dcol,
               uint32_t *__restrict__ flags, uint32_t *__restrict__ vbad, int32_t *__restrict__ badv, Fp64Ones k1,
               const unsigned int *__restrict__ mode, SigmaCols sc, int64_t nfc, int64_t ngc) {
  grid_dep_wait();  // a programmatic dependent of the launch before it
  constexpr int UF = EXT_P1OPT_UF, R = EXT_P1OPT_R;
  __shared__ int cta_bad;
  const unsigned md = *mode;
  if (mode_cells(md)) return;  // cell-loop mode: the nine-space cell kernel runs instead
  const bool sig = (md & kNotFlat) != 0u;
  const LevelCoef *__restrict__ ct = sig ? tab + col.d : tab;
  if (blockIdx.x == 0 && threadIdx.x == 0) flags[(ncoord + 31) / 32] = 0u;  // the zero word past the end
  if (threadIdx.x == 0) cta_bad = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t nwords = (ncoord + 31) / 32;
  const int64_t nch = nfc + ngc;
  const int64_t wstride = (int64_t)gridDim.x * 8;
  bool bad = false;
  const int64_t j0 = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
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
      const uint32_t dbase = (uint32_t)fcur * (uint32_t)(UF * 32) + (uint32_t)lane;
      long long x[UF], y[UF], x0[UF], y0[UF];
      double z[UF], zt[UF];
      uint32_t qv[UF];
      bool v[UF];
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const uint32_t d = dbase + (uint32_t)(u * 32);
        v[u] = d < ncoord;
        x[u] = y[u] = x0[u] = y0[u] = 0;
        z[u] = zt[u] = 0.0;
        qv[u] = 0;
        if (v[u]) {
          const uint32_t q = fdiv(d, col);
          const uint32_t m = d - q * col.d;
          const double *xp = X + 3 * (size_t)d;
          const double *x0p = X + 3 * (size_t)(q * col.d);
          qv[u] = q;
          x[u] = __double_as_longlong(__ldg(xp + 0));
          y[u] = __double_as_longlong(__ldg(xp + 1));
          z[u] = __ldg(xp + 2);
          x0[u] = __double_as_longlong(__ldg(x0p + 0));
          y0[u] = __double_as_longlong(__ldg(x0p + 1));
          zt[u] = __ldg(&ct[m].z);
        }
      }
#pragma unroll
      for (int u = 0; u < UF; ++u) {
        const uint32_t w = (uint32_t)fcur * (uint32_t)UF + (uint32_t)u;
        const bool ok = v[u] && x[u] == x0[u] && y[u] == y0[u] && z_ok(z[u], zt[u], sig, sc, qv[u], k1);
        const unsigned int word = __ballot_sync(kFull, ok);
        const unsigned int want = __ballot_sync(kFull, v[u]);
        if (w < nwords) {
          if (lane == 0) flags[w] = word;
          bad |= word != want;
        }
        if (v[u] && !ok) atomicOr(vbad + (qv[u] >> 5), 1u << (qv[u] & 31u));
      }
    } else {
      const int64_t cs = (j - fcur) * (int64_t)(32 * R);
#pragma unroll 1
      for (int t = 0; t < R; ++t) {
        const int64_t d = cs + 32 * t + lane;
        int r0 = 0, deg = 0;
        uint32_t rr = 0;
        if (d < (int64_t)nf) {
          const uint32_t q = fdiv((uint32_t)d, dcol);
          rr = (uint32_t)d - q * dcol.d;
          r0 = __ldg(vrow + q);
          deg = __ldg(vrow + q + 1) - r0;
        }
        double acc = k1.mzero;
        const int dmx = __reduce_max_sync(kFull, deg);
#pragma unroll 4
        for (int u = 0; u < dmx; ++u) {
          double ev = 0.0, fv = 0.0;
          if (u < deg) {
            ev = __ldg(wts + r0 + u);
            fv = __ldg(f + (size_t)fdiv((uint32_t)__ldg(vnbr + r0 + u), col) * dcol.d + rr);
          }
          acc = fma(ev, fv, acc);
        }
        const double other = NV == 2 ? __shfl_xor_sync(kFull, acc, 1) : 0.0;
        if (d < (int64_t)nf) {
          const double hi = __ldg(&ct[NV == 2 ? rr >> 1 : rr].hi);  // Delta_l of layer l
          b[d] = NV == 2 ? fmul(hi, fma(2.0, acc, other), k1) : fmul(fmul(6.0, hi, k1), acc, k1);
        }
      }
    }
  }
  if (bad && lane == 0) cta_bad = 1;
  __syncthreads();
  if (threadIdx.x == 0) badv[blockIdx.x] = cta_bad;
}

// bits 0..15 of m spread to bit pairs (bit i -> bits 2i and 2i + 1)
__device__ __forceinline__ uint32_t spread_pairs(uint32_t m) {
  uint32_t x = m & 0xffffu;
  x = (x | (x << 8)) & 0x00ff00ffu;
  x = (x | (x << 4)) & 0x0f0f0f0fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x | (x << 1);
}

// Fix-up of k_cgdg_opt (the counterpart of k_p1_fix): one thread per vertex
// column a whose row holds a column with a failing coordinate DoF records,
// 32 / NV layers at a time, the DoFs of the layers l whose levels l or l + 1
// hold a failing DoF in a row column.
template <int NV>
__global__ void __launch_bounds__(256) k_cgdg_fix(const int32_t *__restrict__ vrow, const int32_t *__restrict__ vnbr,
                                                  const uint32_t *__restrict__ flags,
                                                  const uint32_t *__restrict__ vbad, const int32_t *__restrict__ badv,
                                                  int32_t nbadv, uint32_t nverts, FastDiv col, int32_t layers,
                                                  Deferred dfr, unsigned int *err,
                                                  const unsigned int *__restrict__ mode) {
  grid_dep_wait();  // a programmatic dependent of the launch before it
  if (mode_cells(*mode)) return;
  int any = 0;
  for (int i = threadIdx.x; i < nbadv; i += blockDim.x) any |= __ldg(badv + i);
  if (!__syncthreads_or(any)) return;
  constexpr uint32_t LW = 32 / NV;  // layers per 32-DoF word
  for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < nverts; a += gridDim.x * blockDim.x) {
    const int32_t r0 = __ldg(vrow + a), r1 = __ldg(vrow + a + 1);
    bool hit = false;
    for (int32_t t = r0; t < r1 && !hit; ++t) {
      const uint32_t jv = fdiv((uint32_t)__ldg(vnbr + t), col);
      hit = (__ldg(vbad + (jv >> 5)) >> (jv & 31u)) & 1u;
    }
    if (!hit) continue;
    for (uint32_t lo = 0; lo < (uint32_t)layers; lo += LW) {
      const uint32_t nl = (uint32_t)layers - lo < LW ? (uint32_t)layers - lo : LW;  // layers lo .. lo + nl - 1
      const uint32_t valid = nl == 32 ? 0xffffffffu : (1u << nl) - 1u;
      uint32_t B = 0, top = 0;  // not straight: level lo + i (i < nl), level lo + nl
      for (int32_t t = r0; t < r1; ++t) {
        const uint32_t j0 = (uint32_t)__ldg(vnbr + t);
        B |= ~bits32(flags, j0 + lo) & valid;
        top |= ~(__ldg(flags + ((j0 + lo + nl) >> 5)) >> ((j0 + lo + nl) & 31u)) & 1u;
      }
      // layer lo + i needs levels lo + i and lo + i + 1
      const uint32_t need = (B | (B >> 1) | (top << (nl - 1))) & valid;
      if (!need) continue;
      // one 32-DoF record: NV DoFs per layer
      const uint32_t start = a * (uint32_t)(NV * layers) + (uint32_t)NV * lo;
      const unsigned int slot = atomicAdd(dfr.count, 1u);
      if (slot < dfr.cap) dfr.list[slot] = make_int2((int)start, (int)(NV == 1 ? need : spread_pairs(need)));
      else atomicOr(err, EXT_DERR_BOUNDS);
    }
  }
}

// The recorded DoFs of the gather: b_{a,m} (+)= the bottom-row entries of the
// prisms (c, m) and the top-row entries of the prisms (c, m - 1) for every
// cell c around vertex a (p1_prism), summed in ascending cell order.  One
// warp per record, one lane per DoF of its 32-DoF chunk.
template <bool INC>
__global__ void __launch_bounds__(kWarps * 32) k_vgather_general(const MassP1Launch p, Deferred dfr, FastDiv col,
                                                                 Fp64Ones k1) {
  grid_dep_wait();  // a programmatic dependent of the launch before it
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const unsigned int n = min(*dfr.count, dfr.cap);
  for (unsigned int e = blockIdx.x * kWarps + warp; e < n; e += gridDim.x * kWarps) {
    const int2 en = dfr.list[e];
    if ((((unsigned int)en.y) >> lane & 1u) == 0u) continue;
    const int64_t d = (int64_t)en.x + lane;
    const uint32_t q = fdiv((uint32_t)d, col);
    const int m = (int)((uint32_t)d - q * col.d);
    const int32_t v0 = (int32_t)(q * col.d);  // DoF of vertex q at level 0
    double acc = INC ? p.b[d] : 0.0;
    for (int32_t t = __ldg(p.vcrow + q); t < __ldg(p.vcrow + q + 1); ++t) {
      const int64_t c = __ldg(p.vcells + t);
      int a = 0;
      int32_t cb[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (__ldg(p.fmap + c * 6 + 2 * k) == v0) a = k;
        cb[k] = __ldg(p.cmap + c * 6 + 2 * k);
      }
      long long rx[3], ry[3];
      double k2, k6;
      column_ref(p.X, cb, rx, ry, k2, k6);
      for (int half = 0; half < 2; ++half) {
        const int l = half == 0 ? m - 1 : m;
        if (l < 0 || l >= p.layers) continue;
        double Xp[6][3], fp[6], out[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          const int64_t cd = __ldg(p.cmap + c * 6 + i) + (int64_t)l * p.coff[i];
          Xp[i][0] = __ldg(p.X + 3 * cd + 0);
          Xp[i][1] = __ldg(p.X + 3 * cd + 1);
          Xp[i][2] = __ldg(p.X + 3 * cd + 2);
          fp[i] = __ldg(p.f + __ldg(p.fmap + c * 6 + i) + (int64_t)l * p.foff[i]);
        }
        p1_prism(Xp, fp, rx, ry, k2, k6, k1, out);
        acc += out[2 * a + (half == 0 ? 1 : 0)];
      }
    }
    p.b[d] = acc;
  }
}

#ifndef EXT_P1C_MINB
#define EXT_P1C_MINB 2  // resident CTAs per SM the cell loop's registers must allow
#endif

// Cell-loop mode (Algorithm 3 on any coordinate field): a warp owns a group
// of cpw whole cell columns and walks its flattened items (column, level m),
// 32 consecutive items per step, lanes along a column's levels.  The lane of
// item (c, m), m < layers, evaluates prism (c, m) once with p1_prism (the
// vertical form on columns with vertical edges, e.g. terrain-following
// levels; the general Jacobian otherwise); its bottom row belongs to level m
// and stays with the lane, its top row belongs to level m + 1 and moves one
// lane up (warp shuffle; the step's last lane hands it to the next step).
// Each item then adds its three values to the vertex DoFs with FP64 atomic
// adds.  mode (if given) is the word the probe sets: a zero word (a flat,
// straight extrusion, which the gather form handles) makes the kernel exit.
__global__ void __launch_bounds__(kWarps * 32, EXT_P1C_MINB) k_p1_cells(const MassP1Launch p, int cpw, Fp64Ones k1,
                                                                       const unsigned int *__restrict__ mode) {
  grid_dep_wait();  // a programmatic dependent of the launch before it
  if (mode && !mode_cells(*mode)) return;  // a gather mode formed b
  __shared__ ColInfo cols[kWarps][kMaxCols];
  __shared__ double kk[kWarps][kMaxCols][2];  // k2, k6 of each column
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t ngroups = (p.ncells + cpw - 1) / cpw;
  const int64_t wstride = (int64_t)gridDim.x * kWarps;
  const int layers = p.layers, L1 = layers + 1;
  for (int64_t grp = (int64_t)blockIdx.x * kWarps + warp; grp < ngroups; grp += wstride) {
    const int64_t c0 = grp * cpw;
    const int ncol = (int)(p.ncells - c0 < cpw ? p.ncells - c0 : (int64_t)cpw);
    if (lane < ncol) {
      ColInfo &ci = cols[warp][lane];
      setup_column<false>(p, c0 + lane, ci);
      const double det2 = ci.alpha * 144.0;  // |2A| of the level-0 triangle
      kk[warp][lane][0] = det2 * (1.0 / 864.0);
      kk[warp][lane][1] = det2 * (1.0 / 2592.0);
    }
    __syncwarp();
    const int nitems = ncol * L1;
    double carry[3] = {0.0, 0.0, 0.0};
    for (int base = 0; base < nitems; base += 32) {
      const int it = base + lane;
      const bool valid = it < nitems;
      const int cl = valid ? it / L1 : 0;
      const int m = valid ? it - cl * L1 : L1;
      const ColInfo &ci = cols[warp][cl];
      double r0[3] = {0.0, 0.0, 0.0}, r1[3] = {0.0, 0.0, 0.0};
      if (m < layers) {
        double Xp[6][3], fp[6], out[6];
        load_prism(p, ci, m, layers, Xp, fp);
        p1_prism(Xp, fp, ci.rx, ci.ry, kk[warp][cl][0], kk[warp][cl][1], k1, out);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          r0[a] = out[2 * a];
          r1[a] = out[2 * a + 1];
        }
      }
      // top rows one lane up: item (c, m) receives prism (c, m - 1)'s top row;
      // at m = 0 the lane below holds the previous column's top level, which
      // has no prism above it and passes zeros
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double up = __shfl_up_sync(kFull, r1[a], 1);
        const double last = __shfl_sync(kFull, r1[a], 31);
        if (lane == 0) up = carry[a];
        carry[a] = last;
        r0[a] = fadd(r0[a], up, k1);
      }
      if (valid) {
#pragma unroll
        for (int a = 0; a < 3; ++a) atomicAdd(p.b + dof_at(ci.bbot[a], ci.btop[a], p.boff[2 * a], m, layers), r0[a]);
      }
    }
    __syncwarp();
  }
}


// Resident CTAs per SM of a kernel (one GPU model per process).
template <typename K>
int resident_ctas(K kernel, int &cache) {
  if (cache == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cache, kernel, kWarps * 32, 0);
    if (cache < 1) cache = 1;
  }
  return cache;
}

}  // namespace

// Forms of the launch (ext_set_option(EXT_OPT_P1_FORM, ...)):
//   EXT_P1_AUTO   under a million (column, level) items the single-pass
//                 kernel; otherwise as EXT_P1_SPLIT;
//   EXT_P1_SPLIT  constant layers on a mesh with vertex rows, from
//                 EXT_GATHER_MIN_LAYERS layers: the probe decides between the
//                 flat gather, the terrain-following gather and the cell
//                 loop; fewer layers, or no vertex rows: the factored form
//                 from EXT_FACTORED_MIN_LAYERS layers, else the unfactored
//                 one; variable layers: the variable-layer split form;
//   EXT_P1_GATHER the gather form without the probe (DoFs next to a prism
//                 that is not straight are recomputed one by one);
//   EXT_P1_FACTORED / EXT_P1_UNFACTORED  the split form with / without the
//                 area pass (Algorithm 3 over cells on vertical sums);
//   EXT_P1_CELLS  the cell loop k_p1_cells;
//   EXT_P1_SINGLE the single-pass kernel.
// Variable layers take the variable-layer split form under every form but
// EXT_P1_SINGLE.  When the scratch cannot be allocated the single-pass
// kernel runs.
cudaError_t launch_mass_p1(const MassP1Launch &p, cudaStream_t s) {
  if (p.ncells == 0) return cudaSuccess;
  const bool var = p.cell_layers != nullptr;
  // columns per group: about EXT_MASS_ITEMS items (mean items with variable layers)
  const double L1 = var ? p.mean_layers + 1.0 : (double)(p.layers + 1);
  int cpw = (int)((EXT_MASS_ITEMS + L1 - 1.0) / L1);
  if (cpw < 1) cpw = 1;
  if (cpw > kMaxCols) cpw = kMaxCols;
  const int64_t warps = (p.ncells + cpw - 1) / cpw;
  const int64_t blocks0 = (warps + kWarps - 1) / kWarps;
  static int sms = 0;
  static int res_cells[3] = {0, 0, 0}, res_fused[2] = {0, 0}, res_p1c = 0, res_vgg[2] = {0, 0};
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  int form = p1_form();
  const double items = L1 * (double)p.ncells;
  // on a small launch the split form's extra passes, scratch allocation and
  // launches (about 25 us together) cost more than they save
  if (form == EXT_P1_AUTO) form = items < 1.0e6 ? EXT_P1_SINGLE : EXT_P1_SPLIT;
  const bool rows = !var && p.vrow && p.vnbr && p.vedge && p.vcrow && p.vcells && p.nvent > 0;
  // below EXT_GATHER_MIN_LAYERS layers the per-launch geometry of the gather
  // forms (areas, one weight per vertex-row entry) costs about as much as the
  // vertical work it serves; the cell pass over vertical sums is faster there
  // on a well-ordered base (15M cells, RCM: 0.85 against 1.08 ms at one layer,
  // 0.25 against 0.27 ms at 20)
  if (!var && form == EXT_P1_SPLIT && p.layers < EXT_GATHER_MIN_LAYERS)
    form = p.layers >= EXT_FACTORED_MIN_LAYERS ? EXT_P1_FACTORED : EXT_P1_UNFACTORED;
  if (!var && !rows && (form == EXT_P1_GATHER || form == EXT_P1_SPLIT))
    form = p.layers >= EXT_FACTORED_MIN_LAYERS ? EXT_P1_FACTORED : EXT_P1_UNFACTORED;
  const bool gather = !var && (form == EXT_P1_SPLIT || form == EXT_P1_GATHER);
  const bool probe = !var && form == EXT_P1_SPLIT;
  const bool cells = !var && form == EXT_P1_CELLS;
  const bool factored = !var && form == EXT_P1_FACTORED;
  const Fp64Ones k1 = {1.0, -1.0, -0.0};
  const int64_t n = p.nf;
  // Scratch from the stream-ordered pool, so launches on different streams
  // never share it: a 256-byte block (the recorded-step counter, then the
  // mode word), the vertical sums W, the vertex area sums A (factored), the
  // level table, alpha per cell and the row weights (gather), alpha per cell
  // (factored), and the list of recorded steps: one per warp step of the
  // cell pass at most, or one per 32-DoF chunk of the gather.
  char *scr = nullptr;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t nn = (size_t)(n > 0 ? n : 1);
  // the optimistic flat gather (WRITE): one straightness bit per coordinate
  // DoF (and a zero word past the end), one per vertex column, one word per
  // CTA of k_p1_opt; its fix-up records up to one 32-level word per vertex
  // column and word of levels
  const bool opt = gather && p.overwrite && p1_flat() == EXT_P1_FLAT_OPTIMISTIC;
  static int res_opt = 0;
  const int64_t go = opt ? (int64_t)resident_ctas(k_p1_opt, res_opt) * sms : 0;
  const int64_t fix_recs = opt ? (int64_t)p.nverts * ((p.layers + 1 + 31) / 32) + 2 : 0;
  int64_t cap64 = gather ? (n + 29) / 30 + 2
                         : (int64_t)(items / 32.0) + (p.ncells + cpw - 1) / cpw + 64 + (var ? p.ncells / 8 : 0);
  if (cap64 < fix_recs) cap64 = fix_recs;
  const unsigned int cap = (unsigned int)(cap64 < 0x7fffffff ? cap64 : 0x7fffffff);
  const size_t wbytes = cells ? 0 : al(sizeof(double) * nn * (var ? 3 : (gather ? 1 : 2)));
  const size_t abytes = factored ? al(sizeof(double) * (size_t)(n / (p.layers + 1))) : 0;
  const size_t tbytes = gather ? al(sizeof(LevelCoef) * 2 * (size_t)(p.layers + 1)) : 0;
  const size_t cbytes = (gather || factored) ? al(sizeof(double) * (size_t)p.ncells) : 0;
  const size_t ebytes = gather ? al(sizeof(double) * (size_t)p.nvent) : 0;
  // terrain-following gather: D, z_0 and the bound per vertex column, S per cell
  const size_t vbytes = gather ? al(sizeof(double) * (size_t)p.nverts) : 0;
  const size_t sbytes = gather ? 3 * vbytes + cbytes : 0;
  const size_t lbytes = cells ? 0 : sizeof(int2) * (size_t)cap;
  const size_t vbbytes = opt ? al(sizeof(uint32_t) * (size_t)((p.nverts + 31) / 32)) : 0;
  const size_t fbytes = opt ? al(sizeof(uint32_t) * (size_t)((n + 31) / 32 + 1)) : 0;
  const size_t bvbytes = opt ? al(sizeof(int32_t) * (size_t)go) : 0;
  if (form != EXT_P1_SINGLE &&
      cudaMallocAsync(reinterpret_cast<void **>(&scr), 256 + vbbytes + wbytes + abytes + tbytes + cbytes + ebytes +
                                                           sbytes + lbytes + fbytes + bvbytes,
                      s) != cudaSuccess) {
    (void)cudaGetLastError();  // not sticky: run the single-pass kernel instead
    scr = nullptr;
  }
  if (!scr) {
    const int res = var ? resident_ctas(k_mass_p1<true>, res_fused[1]) : resident_ctas(k_mass_p1<false>, res_fused[0]);
    const int64_t blocks = blocks0 < (int64_t)res * sms ? blocks0 : (int64_t)res * sms;
    if (p.overwrite) {  // the single pass only adds: clear b first
      const cudaError_t ez = cudaMemsetAsync(p.b, 0, sizeof(double) * (size_t)(p.nf > 0 ? p.nf : 0), s);
      if (ez != cudaSuccess) return ez;
    }
    if (var) k_mass_p1<true><<<(unsigned)blocks, kWarps * 32, 0, s>>>(p, cpw);
    else k_mass_p1<false><<<(unsigned)blocks, kWarps * 32, 0, s>>>(p, cpw);
    return cudaGetLastError();
  }
  unsigned int *count = reinterpret_cast<unsigned int *>(scr);
  unsigned int *mode = count + 1;
  unsigned long long *minds = reinterpret_cast<unsigned long long *>(scr + 8);
  uint32_t *vbad = reinterpret_cast<uint32_t *>(scr + 256);  // cleared with the 256-byte block
  scr += vbbytes;  // the rest of the layout follows the vertex-column bits
  char *const scr0 = scr - vbbytes;
  double *W = reinterpret_cast<double *>(scr + 256);
  double *A = reinterpret_cast<double *>(scr + 256 + wbytes);
  LevelCoef *tab = reinterpret_cast<LevelCoef *>(scr + 256 + wbytes + abytes);
  double *alpha = reinterpret_cast<double *>(scr + 256 + wbytes + abytes + tbytes);
  double *wts = reinterpret_cast<double *>(scr + 256 + wbytes + abytes + tbytes + cbytes);
  char *sg0 = scr + 256 + wbytes + abytes + tbytes + cbytes + ebytes;
  SigmaCols sc;
  sc.Dv = reinterpret_cast<double *>(sg0);
  sc.Z0 = reinterpret_cast<double *>(sg0 + vbytes);
  sc.Bv = reinterpret_cast<double *>(sg0 + 2 * vbytes);
  double *Sc = reinterpret_cast<double *>(sg0 + 3 * vbytes);
  Deferred dfr;
  dfr.count = count;
  dfr.list = reinterpret_cast<int2 *>(sg0 + sbytes);
  dfr.cap = cap;
  uint32_t *oflags = reinterpret_cast<uint32_t *>(sg0 + sbytes + lbytes);
  int32_t *badv = reinterpret_cast<int32_t *>(sg0 + sbytes + lbytes + fbytes);
  // the counter, the mode word and the smallest sigma spacing start at zero,
  // and so do the vertex-column bits of the optimistic gather
  cudaError_t e = cudaMemsetAsync(scr0, 0, 256 + vbbytes, s);
  if (e == cudaSuccess && factored && abytes) e = cudaMemsetAsync(A, 0, abytes, s);
  const FastDiv col = make_fastdiv((uint32_t)(var ? 1 : p.layers + 1));
  const int rc = resident_ctas(k_p1_cells, res_p1c);
  const int64_t gc = blocks0 < (int64_t)rc * sms ? blocks0 : (int64_t)rc * sms;
  if (e == cudaSuccess && cells) {
    if (p.overwrite) e = cudaMemsetAsync(p.b, 0, sizeof(double) * (size_t)n, s);
    if (e == cudaSuccess) {
      k_p1_cells<<<(unsigned)gc, kWarps * 32, 0, s>>>(p, cpw, k1, nullptr);
      e = cudaGetLastError();
    }
  } else if (e == cudaSuccess && gather) {
    // every kernel after the first is a programmatic dependent of the one before it
    auto dep = [&e](cudaError_t r) {
      if (e == cudaSuccess) e = r;
    };
    static int res_vtab = 0, res_vg[2] = {0, 0}, res_vb = 0;
    static int64_t skip_step = -2;
    if (skip_step == -2) {
      // test hook, read once per process: the first bulk-copy vertex pass
      // leaves out the copy of this step (its wait then runs out)
      const char *ev = getenv("EXTMESH_TEST_BULK_SKIP");
      skip_step = ev ? atoll(ev) : -1;
    }
    const int64_t skip = skip_step;
    skip_step = -1;
    const unsigned wait_limit = skip >= 0 ? (1u << 12) : kBulkWaitLimit;
    const int rv = resident_ctas(k_vsum_tab<false>, res_vtab);
    const int rg = p.overwrite ? resident_ctas(k_vgather<false>, res_vg[0]) : resident_ctas(k_vgather<true>, res_vg[1]);
    int64_t gv = ((n + 32 * EXT_VT_VU - 1) / (32 * EXT_VT_VU) + 7) / 8;  // CTAs of 8 warps, one warp step each
    int64_t gg = ((n + 32 * EXT_VG_VU - 1) / (32 * EXT_VG_VU) + 7) / 8;
    if (gv > (int64_t)rv * sms) gv = (int64_t)rv * sms;
    if (gg > (int64_t)rg * sms) gg = (int64_t)rg * sms;
    if (gv < 1) gv = 1;
    if (gg < 1) gg = 1;
    // probe: about 4096 vertex columns, every level
    const int64_t nv = p.nverts;
    const int64_t stride = nv > 4096 ? (nv + 4095) / 4096 : 1;
    const int64_t nsamp = probe ? (nv + stride - 1) / stride : 0;
    int64_t gp = ((int64_t)p.ncells > nsamp * (p.layers + 1) ? (int64_t)p.ncells : nsamp * (p.layers + 1)) / 256 + 1;
    if (gp > (int64_t)sms * 8) gp = (int64_t)sms * 8;
    if (gp * 256 < (int64_t)p.layers + 1) gp = ((int64_t)p.layers + 1 + 255) / 256;
    k_p1_levels<<<(unsigned)((p.layers + 1 + 255) / 256), 256, 0, s>>>(p.X, p.layers, tab, mode, minds);
    dep(launch_dependent(k_p1_prep, dim3((unsigned)gp), dim3(256), 0, s, p.X, p.layers, p.cmap, p.ncells, nsamp,
                         stride, tab, alpha, mode));
    int64_t gs = ((nv > (int64_t)p.ncells ? nv : (int64_t)p.ncells) + 255) / 256;
    if (gs > (int64_t)sms * 8) gs = (int64_t)sms * 8;
    dep(launch_dependent(k_p1_sigma_prep, dim3((unsigned)(gs > 0 ? gs : 1)), dim3(256), 0, s, p.X, p.layers, p.cmap,
                         p.ncells, nv, mode, minds, const_cast<double *>(sc.Dv), const_cast<double *>(sc.Z0),
                         const_cast<double *>(sc.Bv), Sc));
    int64_t gw = (nv + 255) / 256;
    if (gw > (int64_t)sms * 8) gw = (int64_t)sms * 8;
    dep(launch_dependent(k_p1_rowweights, dim3((unsigned)(gw > 0 ? gw : 1)), dim3(256), 0, s, p.vrow, p.vnbr,
                         p.vedge, p.vcrow, p.vcells, alpha, sc.Dv, Sc, wts, (int32_t)nv, p.nvent, col, mode));
    const bool fused = p1_flat() == EXT_P1_FLAT_FUSED;
    if (opt) {
      const int64_t nfc = ((n + 31) / 32 + EXT_P1OPT_UF - 1) / EXT_P1OPT_UF;
      const int64_t ngc = (n + 32 * EXT_P1OPT_R - 3) / (32 * EXT_P1OPT_R - 2);
      int64_t g = (nfc + ngc + 7) / 8;
      if (g > go) g = go;
      if (g < 1) g = 1;
      dep(launch_dependent(k_p1_opt, dim3((unsigned)g), dim3(256), 0, s, p.X, p.f, p.vrow, p.vnbr, wts, tab, p.b,
                           (uint32_t)n, col, oflags, vbad, badv, k1, mode, sc, nfc, ngc));
      int64_t gx = (nv + 255) / 256;
      if (gx > (int64_t)sms * 8) gx = (int64_t)sms * 8;
      dep(launch_dependent(k_p1_fix, dim3((unsigned)(gx > 0 ? gx : 1)), dim3(256), 0, s, p.vrow, p.vnbr, oflags, vbad,
                           badv, (int32_t)g, (uint32_t)nv, col, dfr, p.err, mode));
    } else if (fused) {
      static int res_vf[2] = {0, 0};
      const int rf = p.overwrite ? resident_ctas(k_vfused<false>, res_vf[0]) : resident_ctas(k_vfused<true>, res_vf[1]);
      int64_t gf = ((n + 29) / 30 + 7) / 8;
      if (gf > (int64_t)rf * sms) gf = (int64_t)rf * sms;
      if (gf < 1) gf = 1;
      if (p.overwrite)
        dep(launch_dependent(k_vfused<false>, dim3((unsigned)gf), dim3(256), 0, s, p.X, p.f, p.vrow, p.vnbr, wts, tab,
                             p.b, n, col, dfr, p.err, k1, mode));
      else
        dep(launch_dependent(k_vfused<true>, dim3((unsigned)gf), dim3(256), 0, s, p.X, p.f, p.vrow, p.vnbr, wts, tab,
                             p.b, n, col, dfr, p.err, k1, mode));
    }
    if (EXT_VSUM_BULK) {
      const int rb = resident_ctas(k_vsum_bulk<false>, res_vb);
      int64_t gb = ((n + kBulkDofs - 1) / kBulkDofs + 7) / 8;  // CTAs of 8 warps, one warp step each
      if (gb > (int64_t)rb * sms) gb = (int64_t)rb * sms;
      if (gb < 1) gb = 1;
      if (!fused && !opt)
        dep(launch_dependent(k_vsum_bulk<false>, dim3((unsigned)gb), dim3(256), 0, s, p.X, p.f, tab, W, n, col, k1,
                             p.err, mode, sc, skip, wait_limit));
      if (!opt)
        dep(launch_dependent(k_vsum_bulk<true>, dim3((unsigned)gb), dim3(256), 0, s, p.X, p.f, tab, W, n, col, k1,
                             p.err, mode, sc, skip, wait_limit));
    } else {
      if (!fused && !opt) k_vsum_tab<false><<<(unsigned)gv, 256, 0, s>>>(p.X, p.f, tab, W, n, col, k1, mode, sc);
      if (!opt) k_vsum_tab<true><<<(unsigned)gv, 256, 0, s>>>(p.X, p.f, tab, W, n, col, k1, mode, sc);
    }
    if (p.overwrite) {
      dep(launch_dependent(k_vgather<false>, dim3((unsigned)gg), dim3(256), 0, s, W, p.vrow, p.vnbr, wts, p.b, n, col,
                           dfr, p.err, k1, mode, opt ? 3u : (fused ? 1u : 0u)));
      const int r = resident_ctas(k_vgather_general<false>, res_vgg[0]);
      dep(launch_dependent(k_vgather_general<false>, dim3((unsigned)(sms * r)), dim3(kWarps * 32), 0, s, p, dfr, col,
                           k1));
    } else {
      dep(launch_dependent(k_vgather<true>, dim3((unsigned)gg), dim3(256), 0, s, W, p.vrow, p.vnbr, wts, p.b, n, col,
                           dfr, p.err, k1, mode, fused ? 1u : 0u));
      const int r = resident_ctas(k_vgather_general<true>, res_vgg[1]);
      dep(launch_dependent(k_vgather_general<true>, dim3((unsigned)(sms * r)), dim3(kWarps * 32), 0, s, p, dfr, col,
                           k1));
    }
    if (probe) dep(launch_dependent(k_p1_cells, dim3((unsigned)gc), dim3(kWarps * 32), 0, s, p, cpw, k1, mode));
    dep(cudaGetLastError());
  } else if (e == cudaSuccess) {
    const int res = var ? resident_ctas(k_mass_cells<true, false>, res_cells[1])
                        : (factored ? resident_ctas(k_mass_cells<false, true>, res_cells[0])
                                    : resident_ctas(k_mass_cells<false, false>, res_cells[2]));
    const int64_t blocks = blocks0 < (int64_t)res * sms ? blocks0 : (int64_t)res * sms;
    int64_t vb = (n + 255) / 256;
    if (vb > (int64_t)sms * 8) vb = (int64_t)sms * 8;
    if (vb < 1) vb = 1;
    if (var) {
      k_vsum<true, false><<<(unsigned)vb, 256, 0, s>>>(p.X, p.f, W, n, col, nullptr, p.b, k1, nullptr, p.overwrite);
      k_mass_cells<true, false><<<(unsigned)blocks, kWarps * 32, 0, s>>>(p, W, dfr, cpw, k1, nullptr);
      k_mass_general<true, false><<<(unsigned)sms * 2, kWarps * 32, 0, s>>>(p, W, dfr, cpw, nullptr, k1);
    } else if (factored) {
      int64_t ab = (p.ncells + 255) / 256;
      if (ab > (int64_t)sms * 8) ab = (int64_t)sms * 8;
      k_area<<<(unsigned)ab, 256, 0, s>>>(p, A, alpha, col);
      k_vsum<false, true><<<(unsigned)vb, 256, 0, s>>>(p.X, p.f, W, n, col, A, p.b, k1, p.base_xy, p.overwrite);
      k_mass_cells<false, true><<<(unsigned)blocks, kWarps * 32, 0, s>>>(p, W, dfr, cpw, k1, alpha);
      k_mass_general<false, true><<<(unsigned)sms * 2, kWarps * 32, 0, s>>>(p, W, dfr, cpw, alpha, k1);
    } else {
      k_vsum<false, false><<<(unsigned)vb, 256, 0, s>>>(p.X, p.f, W, n, col, nullptr, p.b, k1, nullptr, p.overwrite);
      k_mass_cells<false, false><<<(unsigned)blocks, kWarps * 32, 0, s>>>(p, W, dfr, cpw, k1, nullptr);
      k_mass_general<false, false><<<(unsigned)sms * 2, kWarps * 32, 0, s>>>(p, W, dfr, cpw, nullptr, k1);
    }
    e = cudaGetLastError();
  }
  const cudaError_t ef = cudaFreeAsync(scr0, s);
  return e != cudaSuccess ? e : ef;
}

// CG1 x DG0 / CG1 x DG1 with WRITE on constant layers (k_tp.cu hands the
// launch over when the mesh has vertex rows and the layers reach
// EXT_GATHER_MIN_LAYERS): the level tables, probe, areas and row weights of
// the P1xP1 gather, then k_cgdg_opt (the gather beside the straightness
// flags) and k_cgdg_fix; the recorded DoFs are recomputed with the general
// element rule (launch_cgdg_general), and in cell-loop mode the nine-space
// cell kernel runs instead (launch_tp_cells_gated: b cleared, FP64 reductions).
cudaError_t launch_mass_cgdg(const MassTPLaunch &p, cudaStream_t s) {
  static int sms = 0, res_o[2] = {0, 0};
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int NV = p.nv;
  const int64_t L1 = (int64_t)p.layers + 1, nv = p.nverts, n = p.nf, nc = p.ncoord;
  const int64_t go = (int64_t)(NV == 2 ? resident_ctas(k_cgdg_opt<2>, res_o[1]) : resident_ctas(k_cgdg_opt<1>, res_o[0])) *
                     sms;
  const int64_t nfc = ((nc + 31) / 32 + EXT_P1OPT_UF - 1) / EXT_P1OPT_UF;
  const int64_t ngc = (n + 32 * EXT_P1OPT_R - 1) / (32 * EXT_P1OPT_R);
  int64_t g = (nfc + ngc + 7) / 8;
  if (g > go) g = go;
  if (g < 1) g = 1;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const int64_t cap64 = nv * ((p.layers * NV + 31) / 32) + 2;
  const unsigned int cap = (unsigned int)(cap64 < 0x7fffffff ? cap64 : 0x7fffffff);
  const size_t vbbytes = al(sizeof(uint32_t) * (size_t)((nv + 31) / 32));
  const size_t tbytes = al(sizeof(LevelCoef) * 2 * (size_t)L1);
  const size_t cbytes = al(sizeof(double) * (size_t)p.ncells);
  const size_t ebytes = al(sizeof(double) * (size_t)p.nvent);
  const size_t vbytes = al(sizeof(double) * (size_t)nv);
  const size_t lbytes = al(sizeof(int2) * (size_t)cap);
  const size_t fbytes = al(sizeof(uint32_t) * (size_t)((nc + 31) / 32 + 1));
  const size_t bvbytes = al(sizeof(int32_t) * (size_t)g);
  char *scr = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scr), 256 + vbbytes + tbytes + 2 * cbytes + ebytes +
                                                                       3 * vbytes + lbytes + fbytes + bvbytes,
                                  s);
  if (e != cudaSuccess) return e;
  unsigned int *count = reinterpret_cast<unsigned int *>(scr);
  unsigned int *mode = count + 1;
  unsigned long long *minds = reinterpret_cast<unsigned long long *>(scr + 8);
  char *q = scr + 256;
  uint32_t *vbad = reinterpret_cast<uint32_t *>(q);
  q += vbbytes;
  LevelCoef *tab = reinterpret_cast<LevelCoef *>(q);
  q += tbytes;
  double *alpha = reinterpret_cast<double *>(q);
  q += cbytes;
  double *Sc = reinterpret_cast<double *>(q);
  q += cbytes;
  double *wts = reinterpret_cast<double *>(q);
  q += ebytes;
  SigmaCols sc;
  sc.Dv = reinterpret_cast<double *>(q);
  sc.Z0 = reinterpret_cast<double *>(q + vbytes);
  sc.Bv = reinterpret_cast<double *>(q + 2 * vbytes);
  q += 3 * vbytes;
  Deferred dfr;
  dfr.count = count;
  dfr.list = reinterpret_cast<int2 *>(q);
  dfr.cap = cap;
  q += lbytes;
  uint32_t *flags = reinterpret_cast<uint32_t *>(q);
  q += fbytes;
  int32_t *badv = reinterpret_cast<int32_t *>(q);
  // the counter, the mode word, the smallest sigma spacing and the vertex-column bits start at zero
  e = cudaMemsetAsync(scr, 0, 256 + vbbytes, s);
  auto dep = [&e](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  const FastDiv col = make_fastdiv((uint32_t)L1);
  const Fp64Ones k1 = {1.0, -1.0, -0.0};
  if (e == cudaSuccess) {
    const int64_t stride = nv > 4096 ? (nv + 4095) / 4096 : 1;
    const int64_t nsamp = (nv + stride - 1) / stride;
    int64_t gp = ((int64_t)p.ncells > nsamp * L1 ? (int64_t)p.ncells : nsamp * L1) / 256 + 1;
    if (gp > (int64_t)sms * 8) gp = (int64_t)sms * 8;
    if (gp * 256 < L1) gp = (L1 + 255) / 256;
    k_p1_levels<<<(unsigned)((L1 + 255) / 256), 256, 0, s>>>(p.X, p.layers, tab, mode, minds);
    dep(cudaGetLastError());
    dep(launch_dependent(k_p1_prep, dim3((unsigned)gp), dim3(256), 0, s, p.X, p.layers, p.cmap, p.ncells, nsamp,
                         stride, tab, alpha, mode));
    int64_t gs = ((nv > (int64_t)p.ncells ? nv : (int64_t)p.ncells) + 255) / 256;
    if (gs > (int64_t)sms * 8) gs = (int64_t)sms * 8;
    dep(launch_dependent(k_p1_sigma_prep, dim3((unsigned)(gs > 0 ? gs : 1)), dim3(256), 0, s, p.X, p.layers, p.cmap,
                         p.ncells, nv, mode, minds, const_cast<double *>(sc.Dv), const_cast<double *>(sc.Z0),
                         const_cast<double *>(sc.Bv), Sc));
    int64_t gw = (nv + 255) / 256;
    if (gw > (int64_t)sms * 8) gw = (int64_t)sms * 8;
    dep(launch_dependent(k_p1_rowweights, dim3((unsigned)(gw > 0 ? gw : 1)), dim3(256), 0, s, p.vrow, p.vnbr,
                         p.vedge, p.vcrow, p.vcells, alpha, sc.Dv, Sc, wts, (int32_t)nv, p.nvent, col, mode));
    const FastDiv dcol = make_fastdiv((uint32_t)(NV * p.layers));
    if (NV == 2)
      dep(launch_dependent(k_cgdg_opt<2>, dim3((unsigned)g), dim3(256), 0, s, p.X, p.f, p.vrow, p.vnbr, wts, tab,
                           p.b, (uint32_t)nc, (uint32_t)n, col, dcol, flags, vbad, badv, k1, mode, sc, nfc, ngc));
    else
      dep(launch_dependent(k_cgdg_opt<1>, dim3((unsigned)g), dim3(256), 0, s, p.X, p.f, p.vrow, p.vnbr, wts, tab,
                           p.b, (uint32_t)nc, (uint32_t)n, col, dcol, flags, vbad, badv, k1, mode, sc, nfc, ngc));
    int64_t gx = (nv + 255) / 256;
    if (gx > (int64_t)sms * 8) gx = (int64_t)sms * 8;
    if (NV == 2)
      dep(launch_dependent(k_cgdg_fix<2>, dim3((unsigned)(gx > 0 ? gx : 1)), dim3(256), 0, s, p.vrow, p.vnbr, flags,
                           vbad, badv, (int32_t)g, (uint32_t)nv, col, p.layers, dfr, p.err, mode));
    else
      dep(launch_dependent(k_cgdg_fix<1>, dim3((unsigned)(gx > 0 ? gx : 1)), dim3(256), 0, s, p.vrow, p.vnbr, flags,
                           vbad, badv, (int32_t)g, (uint32_t)nv, col, p.layers, dfr, p.err, mode));
    if (e == cudaSuccess) e = launch_cgdg_general(p, dfr.list, dfr.count, dfr.cap, s);
    if (e == cudaSuccess) e = launch_tp_cells_gated(p, mode, s);
  }
  const cudaError_t ef = cudaFreeAsync(scr, s);
  return e != cudaSuccess ? e : ef;
}
