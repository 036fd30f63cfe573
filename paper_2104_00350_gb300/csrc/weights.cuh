// Linear-exact averaging weights for the ghost-cell gathers (used by the 2D and 3D
// geometry precompute).
//
// Eq. weright averaged averages the values at the averaging points with normalised weights
// w_i = (1/h_i^2) / q (Shepard's inverse-distance average), which reproduces constants but
// not linear fields unless the stencil is symmetric about the interpolation point.  The
// linear-exact form keeps that weight function and adds a linear basis (moving least
// squares): with d_i the offset of point i from the interpolation point (in cells),
// xb = sum w_i d_i and S = sum w_i (d_i - xb)(d_i - xb)^T,
//   W_i = w_i (1 + (d_i - xb) . S^{-1} (-xb)),
// so that sum W_i = 1 and sum W_i d_i = 0.  It needs points that are affinely independent
// (not all on one line in 2D, not all in one plane in 3D), decided on the integer stencil
// offsets; otherwise the plain weights stay.
#pragma once

namespace ibpf {

// integer offsets (relative to the first) span D dimensions
template <int D>
__device__ __forceinline__ bool stencil_spans(const int (*off)[3], int n) {
  if constexpr (D == 2) {
    for (int p = 1; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const int ax = off[p][0] - off[0][0], ay = off[p][1] - off[0][1];
        const int bx = off[q][0] - off[0][0], by = off[q][1] - off[0][1];
        if (ax * by - ay * bx != 0) return true;
      }
    return false;
  } else {
    for (int p = 1; p < n; ++p)
      for (int q = p + 1; q < n; ++q)
        for (int r = q + 1; r < n; ++r) {
          int a[3], b[3], c[3];
          for (int k = 0; k < 3; ++k) {
            a[k] = off[p][k] - off[0][k];
            b[k] = off[q][k] - off[0][k];
            c[k] = off[r][k] - off[0][k];
          }
          const int det = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                          a[2] * (b[0] * c[1] - b[1] * c[0]);
          if (det != 0) return true;
        }
    return false;
  }
}

// w: n normalised weights (in place); d: offsets from the interpolation point in cells
template <int D>
__device__ __forceinline__ void linear_exact_weights(double* w, const double (*d)[3], int n) {
  double xb[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < D; ++k) xb[k] = xb[k] + w[i] * d[i][k];
  double S[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  for (int i = 0; i < n; ++i) {
    double e[3];
    for (int k = 0; k < D; ++k) e[k] = d[i][k] - xb[k];
    for (int r = 0; r < D; ++r)
      for (int c = 0; c < D; ++c) S[r][c] = S[r][c] + (e[r] * w[i]) * e[c];
  }
  double v[3] = {0.0, 0.0, 0.0};
  if constexpr (D == 2) {
    const double det = S[0][0] * S[1][1] - S[0][1] * S[1][0];
    v[0] = (S[1][1] * (-xb[0]) - S[0][1] * (-xb[1])) / det;
    v[1] = (S[0][0] * (-xb[1]) - S[1][0] * (-xb[0])) / det;
  } else {
    // Cramer's rule with the cofactors of S
    const double c00 = S[1][1] * S[2][2] - S[1][2] * S[2][1];
    const double c01 = S[1][2] * S[2][0] - S[1][0] * S[2][2];
    const double c02 = S[1][0] * S[2][1] - S[1][1] * S[2][0];
    const double det = S[0][0] * c00 + S[0][1] * c01 + S[0][2] * c02;
    const double c10 = S[0][2] * S[2][1] - S[0][1] * S[2][2];
    const double c11 = S[0][0] * S[2][2] - S[0][2] * S[2][0];
    const double c12 = S[0][1] * S[2][0] - S[0][0] * S[2][1];
    const double c20 = S[0][1] * S[1][2] - S[0][2] * S[1][1];
    const double c21 = S[0][2] * S[1][0] - S[0][0] * S[1][2];
    const double c22 = S[0][0] * S[1][1] - S[0][1] * S[1][0];
    const double b0 = -xb[0], b1 = -xb[1], b2 = -xb[2];
    // S^{-1} = adj(S)/det, adj(S)[r][c] = cofactor[c][r]
    v[0] = (c00 * b0 + c10 * b1 + c20 * b2) / det;
    v[1] = (c01 * b0 + c11 * b1 + c21 * b2) / det;
    v[2] = (c02 * b0 + c12 * b1 + c22 * b2) / det;
  }
  for (int i = 0; i < n; ++i) {
    double t = 0.0;
    for (int k = 0; k < D; ++k) t = t + (d[i][k] - xb[k]) * v[k];
    w[i] = w[i] * (1.0 + t);
  }
}

}  // namespace ibpf
