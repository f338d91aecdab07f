// P1xP1 prism local kernel for F_i += int u_h^2 phi_i dx and its adjoint
// g_j += int 2 u_h w_h phi_j dx (6-point rule: 3-point degree-2 triangle rule
// x 2-point Gauss), shared by the plain and the batched par_loops.
//
// One call handles one cell of one column at layer l (Algorithm 3's inner
// loop body).  With barycentric weights lambda_a(t) = 1/6 + [a = t]/2 at the
// three triangle points and psi = (1 - zeta, zeta) vertically, u at the six
// points is evaluated in factorised form: vertical interpolation per vertex,
// then u_t = S/6 + ubar_t/2; the projection back onto phi_i is the
// transpose.  On a straight prism |det J| = |2A| |h| at every point; other
// prisms use the full Jacobian per point.  Products and sums are issued as
// DFMA (see Fp64Ones): GB300 runs DADD and DMUL at about 5/6 of the DFMA rate.
#pragma once
#include "ext_internal.cuh"

namespace prism_u2v {

// 2-point Gauss-Legendre on [0,1]: zeta = 1/2 -+ 1/(2 sqrt 3), weights 1/2
constexpr double kZ0 = 0.5 - 0.28867513459481288225;
constexpr double kZ1 = 0.5 + 0.28867513459481288225;

struct ColGeom {
  double wdet;         // |2A| / 12: point weight (1/6 * 1/2) times |2A|; times |h| per layer
  long long rx[3], ry[3];
};

__device__ __forceinline__ void col_geom(const double x[3], const double y[3], ColGeom &g) {
  const double det2 = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
  g.wdet = fabs(det2) * (1.0 / 12.0);
  for (int a = 0; a < 3; ++a) {
    g.rx[a] = __double_as_longlong(x[a]);
    g.ry[a] = __double_as_longlong(y[a]);
  }
}

// |det J| w_q at the six points of a general prism, point order (t, g).
__device__ inline void general_weights(const double X[6][3], double W[6]) {
  const double tp[3][2] = {{1.0 / 6.0, 1.0 / 6.0}, {2.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 3.0}};
  const double gz[2] = {kZ0, kZ1};
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
      W[2 * t + g] = fabs(det) * (1.0 / 12.0);
    }
  }
}

// Values at the six points (t, g) of a P1xP1 field with nodal values v[2a+b].
// Every product and sum here is a DFMA (k: run-time 1, -1, -0).
__device__ __forceinline__ void eval6(const double v[6], double q[6], const Fp64Ones &k) {
  double ub[2][3];
  for (int a = 0; a < 3; ++a) {
    const double d = fsub(v[2 * a + 1], v[2 * a], k);
    ub[0][a] = fma(kZ0, d, v[2 * a]);
    ub[1][a] = fma(kZ1, d, v[2 * a]);
  }
  for (int g = 0; g < 2; ++g) {
    const double s6 = fma(ub[g][0], 1.0 / 6.0, fma(ub[g][1], 1.0 / 6.0, fmul(ub[g][2], 1.0 / 6.0, k)));
    for (int t = 0; t < 3; ++t) q[2 * t + g] = fma(0.5, ub[g][t], s6);
  }
}

// out[2a+b] = W sum_{t,g} r[(t,g)] lambda_a(t) psi_b(g), the transpose of
// eval6 times a weight W common to the six points, with c6 = W / 6 and
// c2 = W / 2 (lambda_a(t) = 1/6 + [a = t]/2).
__device__ __forceinline__ void project6_scaled(const double r[6], double c6, double c2, double out[6],
                                                const Fp64Ones &k) {
  double rho[2][3];
  for (int g = 0; g < 2; ++g) {
    const double r6 = fma(r[g], c6, fma(r[2 + g], c6, fmul(r[4 + g], c6, k)));
    for (int a = 0; a < 3; ++a) rho[g][a] = fma(c2, r[2 * a + g], r6);
  }
  for (int a = 0; a < 3; ++a) {
    // psi_0(z0) = z1, psi_0(z1) = z0 (symmetric points)
    out[2 * a] = fma(kZ1, rho[0][a], fmul(kZ0, rho[1][a], k));
    out[2 * a + 1] = fma(kZ0, rho[0][a], fmul(kZ1, rho[1][a], k));
  }
}

// out[2a+b] = sum_{t,g} r[(t,g)] lambda_a(t) psi_b(g)   (transpose of eval6)
__device__ __forceinline__ void project6(const double r[6], double out[6], const Fp64Ones &k) {
  project6_scaled(r, 1.0 / 6.0, 0.5, out, k);
}

// Local kernel on one prism.  W[6] = w_q |det J_q| (general prisms).
// mode bit 0: F contributions, bit 1: adjoint contributions.
template <int MODE>
__device__ __forceinline__ void local(const double u[6], const double w[6], const double W[6],
                                      double Fo[6], double Go[6], const Fp64Ones &k) {
  double uq[6];
  eval6(u, uq, k);
  double P[6];
  for (int q = 0; q < 6; ++q) P[q] = fmul(W[q], uq[q], k);
  if (MODE & 1) {
    double r[6];
    for (int q = 0; q < 6; ++q) r[q] = fmul(P[q], uq[q], k);
    project6(r, Fo, k);
  }
  if (MODE & 2) {
    double wq[6];
    eval6(w, wq, k);
    double r[6];
    for (int q = 0; q < 6; ++q) r[q] = fmul(fadd(P[q], P[q], k), wq[q], k);
    project6(r, Go, k);
  }
}

// Straight prism: one weight Wc = |2A| |h| / 12 for all six points, folded
// into the projection's constants (Wc / 6, Wc / 2; twice those for the
// adjoint's factor 2), so the point values need no weighting.
template <int MODE>
__device__ __forceinline__ void local_straight(const double u[6], const double w[6], double Wc,
                                               double Fo[6], double Go[6], const Fp64Ones &k) {
  double uq[6];
  eval6(u, uq, k);
  const double c6 = fmul(Wc, 1.0 / 6.0, k), c2 = fmul(Wc, 0.5, k);
  if (MODE & 1) {
    double r[6];
    for (int q = 0; q < 6; ++q) r[q] = fmul(uq[q], uq[q], k);
    project6_scaled(r, c6, c2, Fo, k);
  }
  if (MODE & 2) {
    double wq[6];
    eval6(w, wq, k);
    double r[6];
    for (int q = 0; q < 6; ++q) r[q] = fmul(uq[q], wq[q], k);
    project6_scaled(r, fadd(c6, c6, k), Wc, Go, k);
  }
}

// Cell c, layer l of one mesh: gather, compute, scatter-add (INC).
// cmap/umap rows are the column's stencil lists (k = 6).
template <int MODE>
__device__ __forceinline__ void cell_layer(const int32_t *cmap_row, const int32_t *umap_row,
                                           const int32_t coff[6], const int32_t uoff[6], int l,
                                           const ColGeom &cg, const double *X, const double *u,
                                           const double *w, double *F, double *G, const Fp64Ones &k) {
  double uu[6], ww[6], Xl[6][3];
  int32_t ud[6];
  int ok = 1;
  for (int i = 0; i < 6; ++i) {
    const int64_t cd = (int64_t)cmap_row[i] + (int64_t)l * coff[i];
    Xl[i][0] = __ldg(X + 3 * cd + 0);
    Xl[i][1] = __ldg(X + 3 * cd + 1);
    Xl[i][2] = __ldg(X + 3 * cd + 2);
    ok &= (__double_as_longlong(Xl[i][0]) == cg.rx[i >> 1]) & (__double_as_longlong(Xl[i][1]) == cg.ry[i >> 1]);
    ud[i] = umap_row[i] + l * uoff[i];
    uu[i] = __ldg(u + ud[i]);
    if (MODE & 2) ww[i] = __ldg(w + ud[i]);
  }
  ok &= (__double_as_longlong(Xl[0][2]) == __double_as_longlong(Xl[2][2])) &
        (__double_as_longlong(Xl[0][2]) == __double_as_longlong(Xl[4][2])) &
        (__double_as_longlong(Xl[1][2]) == __double_as_longlong(Xl[3][2])) &
        (__double_as_longlong(Xl[1][2]) == __double_as_longlong(Xl[5][2]));
  double Fo[6], Go[6];
  if (ok) {
    const double Wc = fmul(cg.wdet, fabs(fsub(Xl[1][2], Xl[0][2], k)), k);
    local_straight<MODE>(uu, ww, Wc, Fo, Go, k);
  } else {
    double W[6];
    general_weights(Xl, W);
    local<MODE>(uu, ww, W, Fo, Go, k);
  }
  for (int i = 0; i < 6; ++i) {
    if (MODE & 1) atomicAdd(F + ud[i], Fo[i]);
    if (MODE & 2) atomicAdd(G + ud[i], Go[i]);
  }
}

}  // namespace prism_u2v
