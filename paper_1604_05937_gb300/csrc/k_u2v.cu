// par_loops for the nonlinear residual F_i = int u_h^2 phi_i dx and its
// hand-written adjoint g_j = int 2 u_h w_h phi_j dx = ((dF/du)^T w)_j:
//   - P1xP1 prisms (6-point rule), one lane per (column, layer) item;
//   - Q2xP2 (continuous, INC) and DG2 (discontinuous, WRITE) hexahedra with
//     4x4x4 Gauss points, one lane per (column, layer) item.
// Every kernel is bound by the FP64 pipe, so the local kernels are written
// to minimise FP64 operations: sum factorisation, per-column hoisting of the
// horizontal Jacobian on straight columns, and increments handed to L2 as
// FP64 atomic adds instead of being merged in registers; products and sums
// are issued as DFMA with run-time constants (Fp64Ones), which round like
// DMUL and DADD but issue at the higher DFMA rate.
#include "ext_internal.cuh"
#include "prism_u2v.cuh"

namespace {

// ----------------------------------------------------------------------------
// 4-point Gauss-Legendre rule on [0,1] (nodes (1 -+ x)/2 with x the roots of
// P_4, x^2 = 3/7 -+ (2/7) sqrt(6/5); weights (18 +- sqrt 30)/72).
__device__ constexpr double kG[4] = {0.06943184420297371239, 0.33000947820757186760, 0.66999052179242813240,
                          0.93056815579702628761};
__device__ constexpr double kW[4] = {0.17392742256872692869, 0.32607257743127307131, 0.32607257743127307131,
                          0.17392742256872692869};
// 1-D P2 Lagrange basis on nodes (0, 1, 1/2): l0 = (2t-1)(t-1), l1 = t(2t-1), l2 = 4t(1-t)
__host__ __device__ constexpr double l0(double t) { return (2.0 * t - 1.0) * (t - 1.0); }
__host__ __device__ constexpr double l1(double t) { return t * (2.0 * t - 1.0); }
__host__ __device__ constexpr double l2(double t) { return 4.0 * t * (1.0 - t); }
__device__ constexpr double kB0[4] = {l0(kG[0]), l0(kG[1]), l0(kG[2]), l0(kG[3])};
__device__ constexpr double kB1[4] = {l1(kG[0]), l1(kG[1]), l1(kG[2]), l1(kG[3])};
__device__ constexpr double kB2[4] = {l2(kG[0]), l2(kG[1]), l2(kG[2]), l2(kG[3])};
// horizontal node (ix, iy) of stencil entity e = v0..v3, e0..e3, centre;
// 1-D node index 0 -> 0, 1 -> 1, 2 -> 1/2
__device__ constexpr int kIX[9] = {0, 1, 1, 0, 2, 1, 2, 0, 2};
__device__ constexpr int kIY[9] = {0, 0, 1, 1, 0, 2, 1, 2, 2};

__device__ __forceinline__ double B(int k, int g) { return k == 0 ? kB0[g] : (k == 1 ? kB1[g] : kB2[g]); }

struct HexCol {
  double Wc[16];            // |det J_2D| w_g1 w_g2 at the 16 horizontal points
  long long rx[4], ry[4];   // bit patterns of the level-0 x, y
};

// Horizontal weights of a straight hexahedral column from its base quad.
__device__ void hex_col_weights(const double x[4], const double y[4], double Wc[16]) {
  for (int g1 = 0; g1 < 4; ++g1)
    for (int g2 = 0; g2 < 4; ++g2) {
      const double xi = kG[g1], eta = kG[g2];
      const double xx = (x[1] - x[0]) * (1.0 - eta) + (x[2] - x[3]) * eta;
      const double yx = (y[1] - y[0]) * (1.0 - eta) + (y[2] - y[3]) * eta;
      const double xe = (x[3] - x[0]) * (1.0 - xi) + (x[2] - x[1]) * xi;
      const double ye = (y[3] - y[0]) * (1.0 - xi) + (y[2] - y[1]) * xi;
      Wc[g1 * 4 + g2] = fabs(xx * ye - xe * yx) * (kW[g1] * kW[g2]);
    }
}

// |det J| w_g1 w_g2 at the 16 points (g1, g2) of vertical point g3 of a
// general hexahedron; X[2a+b] is vertex a of the base quad at bottom/top b.
__device__ void hex_general_weights(const double X[8][3], int g3, double W[16]) {
  const int vx[4] = {0, 1, 1, 0}, vy[4] = {0, 0, 1, 1};
  const double zeta = kG[g3];
  for (int g1 = 0; g1 < 4; ++g1)
    for (int g2 = 0; g2 < 4; ++g2) {
      const double xi = kG[g1], eta = kG[g2];
      double J[3][3] = {{0.0}};
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 2; ++b) {
          const double nx = vx[a] ? xi : 1.0 - xi, ny = vy[a] ? eta : 1.0 - eta;
          const double nz = b ? zeta : 1.0 - zeta;
          const double dx = vx[a] ? 1.0 : -1.0, dy = vy[a] ? 1.0 : -1.0, dz = b ? 1.0 : -1.0;
          const double gr[3] = {dx * ny * nz, nx * dy * nz, nx * ny * dz};
          for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) J[r][s] += X[2 * a + b][r] * gr[s];
        }
      const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                         J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      W[g1 * 4 + g2] = fabs(det) * (kW[g1] * kW[g2]);
    }
}

// Values at the 4 Gauss points of a 1-D P2 function with nodal values
// (v0, v1, v2), using l2 = 1 - l0 - l1.
__device__ __forceinline__ void interp4(double v0, double v1, double v2, double out[4], const Fp64Ones &k) {
  const double d0 = fsub(v0, v2, k), d1 = fsub(v1, v2, k);
#pragma unroll
  for (int g = 0; g < 4; ++g) out[g] = fma(d1, kB1[g], fma(d0, kB0[g], v2));
}

// For vertical point g3: field values D[g1][g2] at the 16 points from the
// nodal values (diff form: U2[ix][iy] and d0, d1 = U0 - U2, U1 - U2).
__device__ __forceinline__ void hex_eval_slice(const double U2[3][3], const double d0[3][3],
                                               const double d1[3][3], int g3, double D[4][4], const Fp64Ones &k) {
  double A[3][3];
#pragma unroll
  for (int ix = 0; ix < 3; ++ix)
#pragma unroll
    for (int iy = 0; iy < 3; ++iy) A[ix][iy] = fma(d1[ix][iy], kB1[g3], fma(d0[ix][iy], kB0[g3], U2[ix][iy]));
  double C[3][4];
#pragma unroll
  for (int ix = 0; ix < 3; ++ix) interp4(A[ix][0], A[ix][1], A[ix][2], C[ix], k);
#pragma unroll
  for (int g2 = 0; g2 < 4; ++g2) {
    double t[4];
    interp4(C[0][g2], C[1][g2], C[2][g2], t, k);
#pragma unroll
    for (int g1 = 0; g1 < 4; ++g1) D[g1][g2] = t[g1];
  }
}

// Projects point values r[g1][g2] of vertical point g3 back onto the 27
// basis functions, accumulating Facc[ix][iy][v] += sum r B_ix B_iy B_v w_g3.
__device__ __forceinline__ void hex_project_slice(const double r[4][4], int g3, double Facc[3][3][3],
                                                  const Fp64Ones &k) {
  double E1[3][4];
#pragma unroll
  for (int ix = 0; ix < 3; ++ix)
#pragma unroll
    for (int g2 = 0; g2 < 4; ++g2)
      E1[ix][g2] = fma(r[3][g2], B(ix, 3), fma(r[2][g2], B(ix, 2), fma(r[1][g2], B(ix, 1), fmul(r[0][g2], B(ix, 0), k))));
  const double wz = kW[g3];
  const double bw[3] = {fmul(kB0[g3], wz, k), fmul(kB1[g3], wz, k), fmul(kB2[g3], wz, k)};
#pragma unroll
  for (int ix = 0; ix < 3; ++ix)
#pragma unroll
    for (int iy = 0; iy < 3; ++iy) {
      const double e2 =
          fma(E1[ix][3], B(iy, 3), fma(E1[ix][2], B(iy, 2), fma(E1[ix][1], B(iy, 1), fmul(E1[ix][0], B(iy, 0), k))));
#pragma unroll
      for (int v = 0; v < 3; ++v) Facc[ix][iy][v] = fma(e2, bw[v], Facc[ix][iy][v]);
    }
}

template <int MODE, bool DG>
__global__ void __launch_bounds__(128) k_u2v_hex(const U2VLaunch p, int cpw, Fp64Ones k1) {
  constexpr int kWarps = 4;
  __shared__ HexCol cols[kWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = ((int64_t)blockIdx.x * kWarps + warp) * cpw;
  if (c0 >= p.ncells) return;
  const int ncol = (int)(p.ncells - c0 < cpw ? p.ncells - c0 : (int64_t)cpw);
  const int layers = p.layers;

  if (lane < ncol) {
    const int64_t c = c0 + lane;
    double x[4], y[4];
    for (int a = 0; a < 4; ++a) {
      const int64_t cd = __ldg(p.cmap + c * 8 + 2 * a);
      x[a] = __ldg(p.X + 3 * cd + 0);
      y[a] = __ldg(p.X + 3 * cd + 1);
      cols[warp][lane].rx[a] = __double_as_longlong(x[a]);
      cols[warp][lane].ry[a] = __double_as_longlong(y[a]);
    }
    hex_col_weights(x, y, cols[warp][lane].Wc);
  }
  __syncwarp();

  const int nitems = ncol * layers;
  int cl = lane / layers, l = lane - (lane / layers) * layers;
  for (int base = 0; base < nitems; base += 32) {
    if (base + lane < nitems) {
      const int64_t c = c0 + cl;
      const HexCol &hc = cols[warp][cl];
      // gather coordinates (8 corners) and check the column is straight here
      double X[8][3];
      int ok = 1;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int64_t cd = (int64_t)__ldg(p.cmap + c * 8 + i) + (int64_t)l * p.coff[i];
        X[i][0] = __ldg(p.X + 3 * cd + 0);
        X[i][1] = __ldg(p.X + 3 * cd + 1);
        X[i][2] = __ldg(p.X + 3 * cd + 2);
        ok &= (__double_as_longlong(X[i][0]) == hc.rx[i >> 1]) & (__double_as_longlong(X[i][1]) == hc.ry[i >> 1]);
      }
#pragma unroll
      for (int i = 2; i < 8; i += 2) {
        ok &= __double_as_longlong(X[i][2]) == __double_as_longlong(X[0][2]);
        ok &= __double_as_longlong(X[i + 1][2]) == __double_as_longlong(X[1][2]);
      }
      // gather u (and w) into [ix][iy][v] order
      int32_t ud[27];
      double U2[3][3], d0[3][3], d1[3][3], W2[3][3], e0[3][3], e1[3][3];
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        double uv[3], wv[3];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          const int i = 3 * e + v;
          ud[i] = __ldg(p.umap + c * 27 + i) + l * p.uoff[i];
          uv[v] = __ldg(p.u + ud[i]);
          if (MODE & 2) wv[v] = __ldg(p.w + ud[i]);
        }
        U2[kIX[e]][kIY[e]] = uv[2];
        d0[kIX[e]][kIY[e]] = fsub(uv[0], uv[2], k1);
        d1[kIX[e]][kIY[e]] = fsub(uv[1], uv[2], k1);
        if (MODE & 2) {
          W2[kIX[e]][kIY[e]] = wv[2];
          e0[kIX[e]][kIY[e]] = fsub(wv[0], wv[2], k1);
          e1[kIX[e]][kIY[e]] = fsub(wv[1], wv[2], k1);
        }
      }
      double Facc[3][3][3], Gacc[3][3][3];
#pragma unroll
      for (int ix = 0; ix < 3; ++ix)
#pragma unroll
        for (int iy = 0; iy < 3; ++iy)
#pragma unroll
          for (int v = 0; v < 3; ++v) Facc[ix][iy][v] = Gacc[ix][iy][v] = 0.0;
      const double hscale = ok ? fabs(fsub(X[1][2], X[0][2], k1)) : 1.0;
#pragma unroll 1
      for (int g3 = 0; g3 < 4; ++g3) {
        double Wh[16];
        if (ok) {
#pragma unroll
          for (int q = 0; q < 16; ++q) Wh[q] = hc.Wc[q];
        } else {
          hex_general_weights(X, g3, Wh);
        }
        double Du[4][4];
        hex_eval_slice(U2, d0, d1, g3, Du, k1);
        double P[4][4];
#pragma unroll
        for (int g1 = 0; g1 < 4; ++g1)
#pragma unroll
          for (int g2 = 0; g2 < 4; ++g2) P[g1][g2] = fmul(Wh[g1 * 4 + g2], Du[g1][g2], k1);
        if (MODE & 1) {
          double r[4][4];
#pragma unroll
          for (int g1 = 0; g1 < 4; ++g1)
#pragma unroll
            for (int g2 = 0; g2 < 4; ++g2) r[g1][g2] = fmul(P[g1][g2], Du[g1][g2], k1);
          hex_project_slice(r, g3, Facc, k1);
        }
        if (MODE & 2) {
          double Dw[4][4];
          hex_eval_slice(W2, e0, e1, g3, Dw, k1);
          double r[4][4];
#pragma unroll
          for (int g1 = 0; g1 < 4; ++g1)
#pragma unroll
            for (int g2 = 0; g2 < 4; ++g2) r[g1][g2] = fmul(fadd(P[g1][g2], P[g1][g2], k1), Dw[g1][g2], k1);
          hex_project_slice(r, g3, Gacc, k1);
        }
      }
      // scatter: INC (continuous) via L2 atomics, WRITE (DG2) via stores
#pragma unroll
      for (int e = 0; e < 9; ++e)
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          const int i = 3 * e + v;
          if (MODE & 1) {
            const double val = fmul(Facc[kIX[e]][kIY[e]][v], hscale, k1);
            if (DG) p.F[ud[i]] = val;
            else atomicAdd(p.F + ud[i], val);
          }
          if (MODE & 2) {
            const double val = fmul(Gacc[kIX[e]][kIY[e]][v], hscale, k1);
            if (DG) p.g[ud[i]] = val;
            else atomicAdd(p.g + ud[i], val);
          }
        }
    }
    l += 32;
    while (l >= layers) { l -= layers; ++cl; }
  }
}

// Prism (P1xP1) u^2 v: lanes along (column, layer) items of the warp's columns.
template <int MODE>
__global__ void __launch_bounds__(256) k_u2v_prism(const U2VLaunch p, int cpw, Fp64Ones k1) {
  constexpr int kWarps = 8;
  __shared__ prism_u2v::ColGeom cols[kWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = ((int64_t)blockIdx.x * kWarps + warp) * cpw;
  if (c0 >= p.ncells) return;
  const int ncol = (int)(p.ncells - c0 < cpw ? p.ncells - c0 : (int64_t)cpw);
  const int layers = p.layers;
  if (lane < ncol) {
    const int64_t c = c0 + lane;
    double x[3], y[3];
    for (int a = 0; a < 3; ++a) {
      const int64_t cd = __ldg(p.cmap + c * 6 + 2 * a);
      x[a] = __ldg(p.X + 3 * cd + 0);
      y[a] = __ldg(p.X + 3 * cd + 1);
    }
    prism_u2v::col_geom(x, y, cols[warp][lane]);
  }
  __syncwarp();
  int32_t coff[6], uoff[6];
  for (int i = 0; i < 6; ++i) {
    coff[i] = p.coff[i];
    uoff[i] = p.uoff[i];
  }
  const int nitems = ncol * layers;
  int cl = lane / layers, l = lane - (lane / layers) * layers;
  for (int base = 0; base < nitems; base += 32) {
    if (base + lane < nitems) {
      const int64_t c = c0 + cl;
      int32_t crow[6], urow[6];
      for (int i = 0; i < 6; ++i) {
        crow[i] = __ldg(p.cmap + c * 6 + i);
        urow[i] = __ldg(p.umap + c * 6 + i);
      }
      prism_u2v::cell_layer<MODE>(crow, urow, coff, uoff, l, cols[warp][cl], p.X, p.u, p.w, p.F, p.g, k1);
    }
    l += 32;
    while (l >= layers) { l -= layers; ++cl; }
  }
}

int cols_per_warp(int layers, int target) {
  int cpw = (target + layers - 1) / layers;
  if (cpw < 1) cpw = 1;
  if (cpw > 32) cpw = 32;
  return cpw;
}

}  // namespace

cudaError_t launch_u2v(const U2VLaunch &p, cudaStream_t s) {
  if (p.ncells == 0) return cudaSuccess;
  if (p.nvc == 3) {
    int cpw = cols_per_warp(p.layers, 512);
    // a small mesh takes fewer columns per warp, down to a warp's 32 items,
    // until it has 16 warps per SM (64 meshes of 100-2,000 cells x 8-16
    // layers: 5.9 ms for their 64 launches with 512 items per warp, most SMs
    // idle)
    static int sms = 0;
    if (sms == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (sms < 1) sms = 1;
    }
    const int cpw_min = (32 + p.layers - 1) / p.layers;
    while (cpw > cpw_min && (p.ncells + cpw - 1) / cpw < (int64_t)sms * 16) {
      cpw = (cpw + 1) / 2;
      if (cpw < cpw_min) cpw = cpw_min;
    }
    const int64_t warps = (p.ncells + cpw - 1) / cpw;
    const unsigned blocks = (unsigned)((warps + 7) / 8);
    switch (p.mode) {
      case 1: k_u2v_prism<1><<<blocks, 256, 0, s>>>(p, cpw, fp64_ones()); break;
      case 2: k_u2v_prism<2><<<blocks, 256, 0, s>>>(p, cpw, fp64_ones()); break;
      default: k_u2v_prism<3><<<blocks, 256, 0, s>>>(p, cpw, fp64_ones()); break;
    }
  } else {
    const int cpw = 32;  // lane j sets up column j; items per warp = 32 * layers
    const int64_t warps = (p.ncells + cpw - 1) / cpw;
    const unsigned blocks = (unsigned)((warps + 3) / 4);
    if (p.dg) {
      switch (p.mode) {
        case 1: k_u2v_hex<1, true><<<blocks, 128, 0, s>>>(p, cpw, fp64_ones()); break;
        case 2: k_u2v_hex<2, true><<<blocks, 128, 0, s>>>(p, cpw, fp64_ones()); break;
        default: k_u2v_hex<3, true><<<blocks, 128, 0, s>>>(p, cpw, fp64_ones()); break;
      }
    } else {
      switch (p.mode) {
        case 1: k_u2v_hex<1, false><<<blocks, 128, 0, s>>>(p, cpw, fp64_ones()); break;
        case 2: k_u2v_hex<2, false><<<blocks, 128, 0, s>>>(p, cpw, fp64_ones()); break;
        default: k_u2v_hex<3, false><<<blocks, 128, 0, s>>>(p, cpw, fp64_ones()); break;
      }
    }
  }
  return cudaGetLastError();
}
