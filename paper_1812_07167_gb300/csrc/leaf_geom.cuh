// Entries of one leaf's collocation system (Sec. 2.1), shared by the leaf
// kernels.  Nodes: the p x p Chebyshev grid of the leaf without its corners,
// n = p^2 - 4 of them in the order [S, E, N, W, interior] (e = p - 2 a side,
// nb = 4e boundary nodes, then the interior ones).
//   B = [ F ; A-hat(I_i, :) ],  F = N + i eta I(I_b, :),
//   A-hat = -D_x^2 - D_y^2 - kappa^2 diag(c),
//   G = N - i eta I(I_b, :),
// N the outward normal derivative at the boundary nodes (each row is the
// 1-D derivative along the grid line through its node).
#pragma once

#include <cuda_runtime.h>

namespace hps {
namespace {

struct LeafGeom {
  const double *D1x, *D1y, *D2x, *D2y;  // p x p, row-major, scaled to the leaf
  const int *grid;                      // node -> (iy << 8) | ix
  const double *cv;                     // c at the interior nodes
  int p, e, nb;
  double kappa2;
  double2 eta;
};

// N(i, node (jx, jy)) for boundary row i < nb
__device__ __forceinline__ double leaf_dn(const LeafGeom &g, int i, int jx, int jy) {
  const int p = g.p, side = i / g.e;
  const int ix = g.grid[i] & 0xff, iy = g.grid[i] >> 8;
  if (side == 0) return (jx == ix) ? -g.D1y[0 * p + jy] : 0.0;       // south: -d/dy
  if (side == 1) return (jy == iy) ? g.D1x[(p - 1) * p + jx] : 0.0;  // east: +d/dx
  if (side == 2) return (jx == ix) ? g.D1y[(p - 1) * p + jy] : 0.0;  // north: +d/dy
  return (jy == iy) ? -g.D1x[0 * p + jx] : 0.0;                      // west: -d/dx
}

// B(i, j)
__device__ __forceinline__ double2 leaf_B(const LeafGeom &g, int i, int j) {
  const int jx = g.grid[j] & 0xff, jy = g.grid[j] >> 8;
  double vx = 0.0, vy = 0.0;
  if (i < g.nb) {
    vx = leaf_dn(g, i, jx, jy);
    if (i == j) {  // + i eta
      vx -= g.eta.y;
      vy += g.eta.x;
    }
  } else {
    const int p = g.p, ix = g.grid[i] & 0xff, iy = g.grid[i] >> 8;
    if (jy == iy) vx -= g.D2x[ix * p + jx];
    if (jx == ix) vx -= g.D2y[iy * p + jy];
    if (i == j) vx -= g.kappa2 * g.cv[i - g.nb];
  }
  return make_double2(vx, vy);
}

// G(r, j) for boundary row r < nb
__device__ __forceinline__ double2 leaf_G(const LeafGeom &g, int r, int j) {
  double vx = leaf_dn(g, r, g.grid[j] & 0xff, g.grid[j] >> 8), vy = 0.0;
  if (r == j) {  // - i eta
    vx += g.eta.y;
    vy -= g.eta.x;
  }
  return make_double2(vx, vy);
}

// Row equilibration: the exact power of two that brings the largest entry of
// row i of B into [1, 2).  Without it the impedance rows (scale 2/h p^2) and
// the interior rows (scale (2/h)^2 p^4) are ~10^5 apart, which costs
// complex64 most of its digits.
__device__ __forceinline__ double leaf_row_scale(const LeafGeom &g, int i) {
  const int p = g.p, ix = g.grid[i] & 0xff, iy = g.grid[i] >> 8;
  double mx = 0.0;
  if (i < g.nb) {
    const int side = i / g.e;
    const double sgn = (side == 0 || side == 3) ? -1.0 : 1.0;
    for (int t = 0; t < p; t++) {
      const double v = sgn * ((side == 0) ? g.D1y[0 * p + t] : (side == 1) ? g.D1x[(p - 1) * p + t]
                              : (side == 2) ? g.D1y[(p - 1) * p + t] : g.D1x[0 * p + t]);
      const bool diag = (side == 0 || side == 2) ? (t == iy) : (t == ix);
      // at the node itself the entry is the derivative weight + i eta
      mx = fmax(mx, diag ? fmax(fabs(v - g.eta.y), fabs(g.eta.x)) : fabs(v));
    }
  } else {
    for (int t = 0; t < p; t++) {
      if (t != ix) mx = fmax(mx, fabs(g.D2x[ix * p + t]));
      if (t != iy) mx = fmax(mx, fabs(g.D2y[iy * p + t]));
    }
    mx = fmax(mx, fabs(g.D2x[ix * p + ix] + g.D2y[iy * p + iy] + g.kappa2 * g.cv[i - g.nb]));
  }
  int ex = 0;
  frexp(mx > 0.0 ? mx : 1.0, &ex);
  return ldexp(1.0, 1 - ex);
}

}  // namespace
}  // namespace hps
