/*
 * hps_oracle.c -- plain, slow FP64 complex CPU reference for the HPS direct
 * solver of the 2-D variable-coefficient Helmholtz impedance problem
 * (Beams, Gillman, Hewett, "A parallel shared-memory implementation of a
 * high-order accurate solution technique for variable coefficient Helmholtz
 * problems", arXiv:1812.07167).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference legs may load this code.  It shares no code,
 * header, table or helper with the CUDA library and never calls it.
 *
 * What it computes, and where each step comes from:
 *   - Chebyshev nodes and the spectral differentiation matrix (Sec. 2.1, the
 *     classic collocation of Trefethen's "Spectral methods in MATLAB").
 *   - Leaf operators: A-hat, N, F, G, B, Psi, Y, R = G Psi, Gamma = G Y
 *     (Sec. 2.1, Eqs. for A-hat, N, F, G; Sec. 2.1.1 and 2.1.2).
 *   - Merge of two siblings: I1/I2/I3 split, W = I - R33b R33a, Phi_a,
 *     Upsilon_a, Phi_b, Upsilon_b, R^tau (Sec. 2.2, Eqs. (talpha), (tbeta),
 *     (out), (flux_part)); stored operators as in Sec. 2.4; and, as a
 *     diagnostic, ||W||_1 ||W^{-1}||_1 of every merge (the conditioning that
 *     bounds how far two correct FP64 builds can drift apart).
 *   - Build: Algorithm 1 (boxes processed from the largest index down to the
 *     root); the optional thread team processes one level at a time as in
 *     Algorithm 3, which changes no arithmetic.
 *   - Solve: Algorithm 2 (upward pass, then downward pass).
 *   - Brute force: the single global collocation system whose solution the
 *     HPS build+solve reproduces exactly up to rounding: every leaf's interior
 *     collocation rows, the impedance rows F u = t on the outer boundary and,
 *     for each pair of coincident nodes on a shared edge, the two conditions
 *     t3a = -g3b and g3a = -t3b of Sec. 2.2, solved by dense LU.
 *   - Gauss-Legendre interfaces (gauss_q = q > 0), the variant of the earlier
 *     ItI work the paper cites in Sec. 1 (boundary operators represented on
 *     edges through interpolation): every leaf edge carries its boundary data
 *     on q Gauss-Legendre nodes; incoming data t_G enter the leaf as Qm t_G
 *     on its corner-free Chebyshev edge nodes, outgoing data leave as Pm g
 *     (Qm, Pm: Lagrange interpolation between the two node sets), so the leaf
 *     operators become Psi Qh, Ph R Qh, Ph Gamma (Qh, Ph block-diagonal over
 *     the four edges), and the merges and Algorithm 2 run unchanged on the
 *     Gauss nodes.  Its brute force is the global system of that
 *     discretisation (unknowns: nodal values and incoming Gauss data of every
 *     leaf).  For q >= p-2 the solution equals the Chebyshev-edge one (the
 *     data stay polynomials of degree p-3 per edge); for q < p-2 it is a
 *     coarser interface space.  The Gauss nodes are the roots of P_q found by
 *     bisection between sign changes on a fine grid.
 *
 * Readings of the paper taken here (the paper is silent or garbled there):
 *   - Chebyshev nodes increase: x_j = -cos(j pi/(p-1)) mapped to the leaf
 *     interval; D from the closed-form off-diagonal entries, diagonal by the
 *     negative-sum rule.
 *   - Outward normal derivatives with x horizontal: south -D_y, east +D_x,
 *     north +D_y, west -D_x (the printed N block has the axes mixed up).
 *   - The particular-solution system uses the same B as the homogeneous one.
 *   - R^tau uses the block-diagonal diag(R13a, R23b) (Sec. 2.2), not the
 *     stacked column printed in Algorithm 1.
 *   - LU pivots on max |Re|+|Im|, lowest row index on ties.
 *   - Tree: heap numbering (root 1, children 2 tau, 2 tau + 1, parent <
 *     child); leaves in Morton order.  By default the leaf level pairs
 *     west/east neighbours (alpha west); the option first_vertical pairs
 *     south/north first.  alpha is always the child 2 tau.
 *   - I1, I2, I3 are found geometrically: I3 are the boundary nodes of alpha
 *     that coincide with a boundary node of beta; the parent boundary is
 *     [I1, I2] in the children's own orders, exactly as in Sec. 2.2.
 *
 * Layouts shared with the caller (row-major, complex = (re, im) pairs):
 *   leaf index: bit k of the index belongs to merge k counted from the
 *   leaves (merges alternate west/east and south/north, starting west/east;
 *   see merge_dirs): for a square grid this is the Morton order with bit 2i
 *   of the index bit i of the leaf's column and bit 2i+1 bit i of its row.
 *   Per leaf, nodes are ordered [south, east, north, west, interior]; each
 *   edge runs in increasing coordinate and excludes the corners; the
 *   interior is row by row, x fastest.  Outer boundary data t: [south, east,
 *   north, west] sides, each running in increasing coordinate over mx*(p-2)
 *   (south, north) or my*(p-2) (east, west) nodes.
 */
#include <complex.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
  double x0, x1, y0, y1; /* the rectangle Omega */
  int mx, my;            /* leaves along x and along y, powers of two */
  int p;                 /* Chebyshev nodes per leaf side (n_c) */
  double kappa;          /* wave number */
  double eta_re, eta_im; /* impedance parameter eta, Re(eta) != 0 */
  int first_vertical;    /* 0: first merge joins west/east leaves */
  int gauss_q;           /* 0: boundary data on the p-2 corner-free Chebyshev
                            nodes of every leaf edge (the paper's scheme);
                            q > 0: on q Gauss-Legendre nodes per leaf edge,
                            reached by polynomial interpolation (the
                            interface of the earlier ItI work the paper cites) */
} ora_desc;

/* ------------------------------------------------------------------ */
/* small dense helpers (row-major)                                      */
/* ------------------------------------------------------------------ */

static void *xmalloc(size_t n) {
  void *q = calloc(n ? n : 1, 1);
  if (!q) {
    fprintf(stderr, "hps_oracle: out of memory (%zu bytes)\n", n);
    abort();
  }
  return q;
}

/* C (r x c) = A (r x k) * B (k x c) */
static void matmul(int r, int k, int c, const cplx *A, const cplx *B, cplx *C) {
  for (int i = 0; i < r; i++)
    for (int j = 0; j < c; j++) {
      cplx acc = 0;
      for (int l = 0; l < k; l++) acc += A[(size_t)i * k + l] * B[(size_t)l * c + j];
      C[(size_t)i * c + j] = acc;
    }
}

static double cabs1(cplx z) { return fabs(creal(z)) + fabs(cimag(z)); }

/* 1-norm of an n x n matrix: the largest column sum of moduli */
static double norm1(int n, const cplx *A) {
  double best = 0.0;
  for (int j = 0; j < n; j++) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += cabs(A[(size_t)i * n + j]);
    if (s > best) best = s;
  }
  return best;
}

/* LU factorisation with partial pivoting, in place (the zgetrf step).
 * Returns 0, or 1 + the column of the first exactly zero pivot. */
static int lu_factor(int n, cplx *A, int *piv) {
  int bad = 0;
  for (int k = 0; k < n; k++) {
    int r = k;
    double best = cabs1(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; i++) {
      double v = cabs1(A[(size_t)i * n + k]);
      if (v > best) {
        best = v;
        r = i;
      }
    }
    piv[k] = r;
    if (r != k)
      for (int j = 0; j < n; j++) {
        cplx tmp = A[(size_t)k * n + j];
        A[(size_t)k * n + j] = A[(size_t)r * n + j];
        A[(size_t)r * n + j] = tmp;
      }
    cplx d = A[(size_t)k * n + k];
    if (d == 0) {
      if (!bad) bad = k + 1;
      continue;
    }
    for (int i = k + 1; i < n; i++) {
      cplx f = A[(size_t)i * n + k] / d;
      A[(size_t)i * n + k] = f;
      for (int j = k + 1; j < n; j++) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
    }
  }
  return bad;
}

/* Solve A x = b in place with the factors from lu_factor. */
static void lu_solve(int n, const cplx *LU, const int *piv, cplx *b) {
  for (int k = 0; k < n; k++)
    if (piv[k] != k) {
      cplx tmp = b[k];
      b[k] = b[piv[k]];
      b[piv[k]] = tmp;
    }
  for (int i = 0; i < n; i++) {
    cplx acc = b[i];
    for (int j = 0; j < i; j++) acc -= LU[(size_t)i * n + j] * b[j];
    b[i] = acc;
  }
  for (int i = n - 1; i >= 0; i--) {
    cplx acc = b[i];
    for (int j = i + 1; j < n; j++) acc -= LU[(size_t)i * n + j] * b[j];
    b[i] = acc / LU[(size_t)i * n + i];
  }
}

/* X (n x c) = A^{-1} Rhs (n x c) via LU with partial pivoting; A is copied. */
static int lu_solve_many(int n, const cplx *A, int c, const cplx *Rhs, cplx *X) {
  cplx *LU = xmalloc(sizeof(cplx) * (size_t)n * n);
  int *piv = xmalloc(sizeof(int) * (size_t)n);
  cplx *col = xmalloc(sizeof(cplx) * (size_t)n);
  memcpy(LU, A, sizeof(cplx) * (size_t)n * n);
  int bad = lu_factor(n, LU, piv);
  for (int j = 0; j < c; j++) {
    for (int i = 0; i < n; i++) col[i] = Rhs[(size_t)i * c + j];
    lu_solve(n, LU, piv, col);
    for (int i = 0; i < n; i++) X[(size_t)i * c + j] = col[i];
  }
  free(LU);
  free(piv);
  free(col);
  return bad;
}

/* ------------------------------------------------------------------ */
/* Chebyshev collocation (Sec. 2.1)                                     */
/* ------------------------------------------------------------------ */

/* p Chebyshev points of the second kind on [a, b], increasing, and the
 * p x p differentiation matrix D (row-major) on that interval. */
int ora_cheb(int p, double a, double b, double *x, double *D) {
  if (p < 2) return 1;
  int N = p - 1;
  double *xr = xmalloc(sizeof(double) * p);
  for (int j = 0; j < p; j++) {
    /* -cos(j pi / N) written as a sine so the points are symmetric */
    xr[j] = sin(M_PI * (2.0 * j - N) / (2.0 * N));
    x[j] = a + 0.5 * (b - a) * (xr[j] + 1.0);
  }
  for (int i = 0; i < p; i++) {
    double ci = (i == 0 || i == N) ? 2.0 : 1.0;
    double rowsum = 0.0;
    for (int j = 0; j < p; j++) {
      if (i == j) continue;
      double cj = (j == 0 || j == N) ? 2.0 : 1.0;
      double sgn = ((i + j) % 2 == 0) ? 1.0 : -1.0;
      double v = (ci / cj) * sgn / (xr[i] - xr[j]);
      D[i * p + j] = v;
      rowsum += v;
    }
    D[i * p + i] = -rowsum;
  }
  double s = 2.0 / (b - a);
  for (int i = 0; i < p * p; i++) D[i] *= s;
  free(xr);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Gauss-Legendre interface nodes and interpolation (gauss_q > 0)       */
/* ------------------------------------------------------------------ */

/* Legendre polynomial P_q(z) by the three-term recurrence
 * k P_k = (2k - 1) z P_{k-1} - (k - 1) P_{k-2}, P_0 = 1, P_1 = z. */
static double legendre(int q, double z) {
  double a = 1.0, b = z;
  if (q == 0) return a;
  for (int k = 2; k <= q; k++) {
    double c = ((2.0 * k - 1.0) * z * b - (k - 1.0) * a) / k;
    a = b;
    b = c;
  }
  return b;
}

/* The q Gauss-Legendre nodes on [-1, 1] (the roots of P_q), increasing: every
 * sign change of P_q on a fine grid, then bisection to the last bit. */
int ora_gauss_nodes(int q, double *z) {
  if (q < 1) return 1;
  int found = 0, steps = 64 * q;
  double x0 = -1.0, f0 = legendre(q, x0);
  for (int k = 1; k <= steps && found < q; k++) {
    double x1 = -cos(M_PI * k / steps), f1 = legendre(q, x1);
    if (f0 == 0.0) {
      z[found++] = x0;
    } else if (f0 * f1 < 0.0) {
      double lo = x0, hi = x1, flo = f0;
      for (int it = 0; it < 200 && hi - lo > 0.0; it++) {
        double mid = 0.5 * (lo + hi), fm = legendre(q, mid);
        if (mid <= lo || mid >= hi) break;
        if ((fm < 0.0) == (flo < 0.0)) {
          lo = mid;
          flo = fm;
        } else {
          hi = mid;
        }
      }
      z[found++] = 0.5 * (lo + hi);
    }
    x0 = x1;
    f0 = f1;
  }
  return found == q ? 0 : 1;
}

/* Lagrange basis polynomial j of the m nodes xs, evaluated at x. */
static double lagrange(int m, const double *xs, int j, double x) {
  double v = 1.0;
  for (int k = 0; k < m; k++)
    if (k != j) v *= (x - xs[k]) / (xs[j] - xs[k]);
  return v;
}

/* Interpolation between the e = p-2 corner-free Chebyshev nodes of an edge
 * and its q Gauss-Legendre nodes (both on the reference edge [-1, 1]; the
 * matrices do not depend on the edge's position or length):
 *   Pm (q x e): the Chebyshev-node interpolant (degree e-1) at the Gauss nodes
 *   Qm (e x q): the Gauss-node interpolant (degree q-1) at the Chebyshev nodes
 * Outgoing data g (Chebyshev) becomes Pm g on the Gauss nodes; incoming Gauss
 * data t_G becomes Qm t_G on the Chebyshev nodes. */
static void edge_interp(int p, int q, double *Pm, double *Qm) {
  int e = p - 2;
  double *xc = xmalloc(sizeof(double) * p), *D = xmalloc(sizeof(double) * p * p);
  double *zg = xmalloc(sizeof(double) * q);
  ora_cheb(p, -1.0, 1.0, xc, D);
  ora_gauss_nodes(q, zg);
  const double *ce = xc + 1; /* the corner-free nodes x_1 .. x_{p-2} */
  for (int a = 0; a < q; a++)
    for (int j = 0; j < e; j++) Pm[a * e + j] = lagrange(e, ce, j, zg[a]);
  for (int j = 0; j < e; j++)
    for (int a = 0; a < q; a++) Qm[j * q + a] = lagrange(q, zg, a, ce[j]);
  free(xc);
  free(D);
  free(zg);
}

/* Public for tests: Pm (q x e) and Qm (e x q) of edge_interp. */
int ora_edge_interp(int p, int q, double *Pm, double *Qm) {
  if (p < 4 || q < 1) return 1;
  edge_interp(p, q, Pm, Qm);
  return 0;
}

/* ------------------------------------------------------------------ */
/* leaf geometry and ordering                                            */
/* ------------------------------------------------------------------ */

/* tensor-grid coordinates (ix, iy) of local node k in [S, E, N, W, interior] */
static void local_to_grid(int p, int k, int *ix, int *iy) {
  int e = p - 2;
  if (k < e) { *ix = 1 + k; *iy = 0; return; }                 /* south */
  k -= e;
  if (k < e) { *ix = p - 1; *iy = 1 + k; return; }             /* east */
  k -= e;
  if (k < e) { *ix = 1 + k; *iy = p - 1; return; }             /* north */
  k -= e;
  if (k < e) { *ix = 0; *iy = 1 + k; return; }                 /* west */
  k -= e;
  *ix = 1 + k % e;                                             /* interior */
  *iy = 1 + k / e;
}

/* Directions of the merges of an mx x my leaf grid (mx = 2^A, my = 2^B),
 * counted from the leaves: 0 joins west/east neighbours (halves the boxes'
 * count along x), 1 joins south/north neighbours.  The two alternate,
 * starting with west/east (south/north when first_vertical); once one axis
 * has no halvings left, the other takes the remaining merges.  Returns the
 * number of merges, A + B. */
static int merge_dirs(int A, int B, int first_vertical, int *dir) {
  int a = A, b = B, k = 0, want = first_vertical ? 1 : 0;
  while (a + b > 0) {
    int d = want;
    if (d == 0 && a == 0) d = 1;
    if (d == 1 && b == 0) d = 0;
    dir[k++] = d;
    if (d == 0) a--; else b--;
    want = 1 - d;
  }
  return k;
}

/* A leaf index whose bit k belongs to merge k: the bits of west/east merges
 * form the leaf's column, the others its row (lowest merge, lowest bit).
 * For a square grid starting west/east this is the Morton order with the x
 * bit lowest. */
static void leaf_decode(int idx, const int *dir, int L, int *col, int *row) {
  int c = 0, r = 0, bc = 0, br = 0;
  for (int k = 0; k < L; k++) {
    int bit = (idx >> k) & 1;
    if (dir[k] == 0) c |= bit << bc++;
    else r |= bit << br++;
  }
  *col = c;
  *row = r;
}

static int leaf_encode(int col, int row, const int *dir, int L) {
  int idx = 0, bc = 0, br = 0;
  for (int k = 0; k < L; k++) {
    int bit = dir[k] == 0 ? (col >> bc++) & 1 : (row >> br++) & 1;
    idx |= bit << k;
  }
  return idx;
}

static int log2i(int m) {
  int k = 0;
  while ((1 << k) < m) k++;
  return k;
}

static int check_desc(const ora_desc *d) {
  if (d->gauss_q < 0 || d->gauss_q > 64) return 1;
  if (d->mx < 1 || (d->mx & (d->mx - 1))) return 1;
  if (d->my < 1 || (d->my & (d->my - 1))) return 1;
  if (d->p < 4) return 1;
  if (!(d->x1 > d->x0) || !(d->y1 > d->y0)) return 1;
  if (d->eta_re == 0.0) return 1;
  return 0;
}

/* boundary-data points per leaf edge: p-2 Chebyshev nodes, or gauss_q */
static int edge_pts(const ora_desc *d) { return d->gauss_q ? d->gauss_q : d->p - 2; }

/* Coordinates of every leaf node ([leaves][p*p-4][2], public leaf order) and
 * of the outer boundary nodes ([2 (mx + my) q][2], q = edge_pts: sides S, E,
 * N, W, each in increasing coordinate). */
int ora_nodes(const ora_desc *d, double *leaf_xy, double *bdry_xy) {
  if (check_desc(d)) return 1;
  int p = d->p, e = p - 2, n = p * p - 4;
  int dir[64], L = merge_dirs(log2i(d->mx), log2i(d->my), 0, dir);
  double hx = (d->x1 - d->x0) / d->mx, hy = (d->y1 - d->y0) / d->my;
  double *xs = xmalloc(sizeof(double) * p), *ys = xmalloc(sizeof(double) * p);
  double *D = xmalloc(sizeof(double) * p * p);
  if (leaf_xy) {
    for (int l = 0; l < d->mx * d->my; l++) {
      int c, r;
      leaf_decode(l, dir, L, &c, &r);
      ora_cheb(p, d->x0 + c * hx, d->x0 + (c + 1) * hx, xs, D);
      ora_cheb(p, d->y0 + r * hy, d->y0 + (r + 1) * hy, ys, D);
      for (int k = 0; k < n; k++) {
        int ix, iy;
        local_to_grid(p, k, &ix, &iy);
        leaf_xy[((size_t)l * n + k) * 2 + 0] = xs[ix];
        leaf_xy[((size_t)l * n + k) * 2 + 1] = ys[iy];
      }
    }
  }
  if (bdry_xy) {
    int q = 0, gq = d->gauss_q;
    double *zg = xmalloc(sizeof(double) * (gq ? gq : 1));
    if (gq) ora_gauss_nodes(gq, zg);
    for (int side = 0; side < 4; side++) {
      int horizontal = (side == 0 || side == 2);
      for (int c = 0; c < (horizontal ? d->mx : d->my); c++) {
        double lo = horizontal ? d->x0 + c * hx : d->y0 + c * hy;
        double len = horizontal ? hx : hy;
        if (horizontal)
          ora_cheb(p, d->x0 + c * hx, d->x0 + (c + 1) * hx, xs, D);
        else
          ora_cheb(p, d->y0 + c * hy, d->y0 + (c + 1) * hy, ys, D);
        for (int k = 1; k <= (gq ? gq : e); k++, q++) {
          /* the k-th node of this leaf edge along the side: Chebyshev node k,
           * or Gauss node k-1 mapped from [-1, 1] */
          double along = gq ? lo + 0.5 * (zg[k - 1] + 1.0) * len : (horizontal ? xs[k] : ys[k]);
          double x, y;
          if (side == 0) { x = along; y = d->y0; }
          else if (side == 1) { x = d->x1; y = along; }
          else if (side == 2) { x = along; y = d->y1; }
          else { x = d->x0; y = along; }
          bdry_xy[2 * q] = x;
          bdry_xy[2 * q + 1] = y;
        }
      }
    }
    free(zg);
  }
  free(xs);
  free(ys);
  free(D);
  return 0;
}

/* Gauss nodes zg (q of them, on [-1, 1]) of the four edges [S, E, N, W] of
 * the leaf in column col, row row, each edge in increasing coordinate:
 * xy [4 q][2]. */
static void leaf_gauss_xy(const ora_desc *d, int col, int row, int q, const double *zg, double *xy) {
  double hx = (d->x1 - d->x0) / d->mx, hy = (d->y1 - d->y0) / d->my;
  double xl = d->x0 + col * hx, yl = d->y0 + row * hy;
  for (int side = 0; side < 4; side++)
    for (int a = 0; a < q; a++) {
      double *pt = &xy[2 * (side * q + a)];
      double sx = xl + 0.5 * (zg[a] + 1.0) * hx, sy = yl + 0.5 * (zg[a] + 1.0) * hy;
      if (side == 0) { pt[0] = sx; pt[1] = yl; }
      else if (side == 1) { pt[0] = xl + hx; pt[1] = sy; }
      else if (side == 2) { pt[0] = sx; pt[1] = yl + hy; }
      else { pt[0] = xl; pt[1] = sy; }
    }
}

/* ------------------------------------------------------------------ */
/* leaf computation (Sec. 2.1)                                          */
/* ------------------------------------------------------------------ */

typedef struct {
  int p, e, n, nb, ni;
  double hx, hy;
  double *Dx2d, *Dy2d;   /* D_x, D_y on the full p^2 tensor grid */
  double *Lap;           /* D_x^2 + D_y^2 on the full grid */
  int *loc2grid;         /* local node -> tensor grid index iy*p+ix */
} leaf_geom;

static void leaf_geom_init(leaf_geom *g, int p, double hx, double hy) {
  g->p = p;
  g->e = p - 2;
  g->n = p * p - 4;
  g->nb = 4 * (p - 2);
  g->ni = (p - 2) * (p - 2);
  g->hx = hx;
  g->hy = hy;
  int P = p * p;
  double *x = xmalloc(sizeof(double) * p);
  double *Dx = xmalloc(sizeof(double) * p * p), *Dy = xmalloc(sizeof(double) * p * p);
  ora_cheb(p, 0.0, hx, x, Dx);
  ora_cheb(p, 0.0, hy, x, Dy);
  g->Dx2d = xmalloc(sizeof(double) * P * P);
  g->Dy2d = xmalloc(sizeof(double) * P * P);
  g->Lap = xmalloc(sizeof(double) * P * P);
  /* D_x acts along x (grid index ix), D_y along y, on the tensor grid */
  for (int iy = 0; iy < p; iy++)
    for (int ix = 0; ix < p; ix++)
      for (int jy = 0; jy < p; jy++)
        for (int jx = 0; jx < p; jx++) {
          int r = iy * p + ix, c = jy * p + jx;
          g->Dx2d[(size_t)r * P + c] = (iy == jy) ? Dx[ix * p + jx] : 0.0;
          g->Dy2d[(size_t)r * P + c] = (ix == jx) ? Dy[iy * p + jy] : 0.0;
        }
  /* D_x^2 + D_y^2 by plain products on the full grid */
  for (int r = 0; r < P; r++)
    for (int c = 0; c < P; c++) {
      double acc = 0.0;
      for (int k = 0; k < P; k++)
        acc += g->Dx2d[(size_t)r * P + k] * g->Dx2d[(size_t)k * P + c] +
               g->Dy2d[(size_t)r * P + k] * g->Dy2d[(size_t)k * P + c];
      g->Lap[(size_t)r * P + c] = acc;
    }
  g->loc2grid = xmalloc(sizeof(int) * g->n);
  for (int k = 0; k < g->n; k++) {
    int ix, iy;
    local_to_grid(p, k, &ix, &iy);
    g->loc2grid[k] = iy * p + ix;
  }
  free(x);
  free(Dx);
  free(Dy);
}

static void leaf_geom_free(leaf_geom *g) {
  free(g->Dx2d);
  free(g->Dy2d);
  free(g->Lap);
  free(g->loc2grid);
}

/* Leaf operators for one leaf: Psi (n x nb), Y (n x ni), R (nb x nb),
 * Gam (nb x ni).  c holds kappa-independent c(x) at the ni interior nodes.
 * Optionally returns B (n x n), F and G (nb x n).  Returns the LU status. */
static int leaf_ops(const leaf_geom *g, double kappa, cplx eta, const double *c, cplx *Psi,
                    cplx *Y, cplx *R, cplx *Gam, cplx *Bout, cplx *Fout, cplx *Gout) {
  int n = g->n, nb = g->nb, ni = g->ni, P = g->p * g->p;
  cplx *F = xmalloc(sizeof(cplx) * (size_t)nb * n);
  cplx *G = xmalloc(sizeof(cplx) * (size_t)nb * n);
  cplx *B = xmalloc(sizeof(cplx) * (size_t)n * n);
  /* N: outward normal derivative rows, restricted to the corner-free nodes */
  for (int k = 0; k < nb; k++) {
    int side = k / g->e;
    int rg = g->loc2grid[k];
    const double *Dm = (side == 0 || side == 2) ? g->Dy2d : g->Dx2d;
    double sgn = (side == 0 || side == 3) ? -1.0 : 1.0;
    for (int j = 0; j < n; j++) {
      int cg = g->loc2grid[j];
      cplx v = sgn * Dm[(size_t)rg * P + cg];
      cplx idn = (j == k) ? 1.0 : 0.0;
      F[(size_t)k * n + j] = v + I * eta * idn;
      G[(size_t)k * n + j] = v - I * eta * idn;
    }
  }
  /* B = [F ; A-hat(I_i, I^tau)] with A-hat = -D_x^2 - D_y^2 - kappa^2 diag(c) */
  for (int k = 0; k < nb; k++)
    for (int j = 0; j < n; j++) B[(size_t)k * n + j] = F[(size_t)k * n + j];
  for (int q = 0; q < ni; q++) {
    int k = nb + q, rg = g->loc2grid[k];
    for (int j = 0; j < n; j++) {
      int cg = g->loc2grid[j];
      double v = -g->Lap[(size_t)rg * P + cg];
      if (j == k) v -= kappa * kappa * c[q];
      B[(size_t)k * n + j] = v;
    }
  }
  /* B Psi = [I; 0] and B Y = [0; I] (Eqs. hmgsolnopdef, prtsolnopdef) */
  cplx *E = xmalloc(sizeof(cplx) * (size_t)n * n);
  for (int i = 0; i < n; i++) E[(size_t)i * n + i] = 1.0;
  cplx *X = xmalloc(sizeof(cplx) * (size_t)n * n);
  int bad = lu_solve_many(n, B, n, E, X);
  for (int i = 0; i < n; i++) {
    for (int j = 0; j < nb; j++) Psi[(size_t)i * nb + j] = X[(size_t)i * n + j];
    for (int j = 0; j < ni; j++) Y[(size_t)i * ni + j] = X[(size_t)i * n + nb + j];
  }
  /* R = G Psi, Gamma = G Y */
  matmul(nb, n, nb, G, Psi, R);
  matmul(nb, n, ni, G, Y, Gam);
  if (Bout) memcpy(Bout, B, sizeof(cplx) * (size_t)n * n);
  if (Fout) memcpy(Fout, F, sizeof(cplx) * (size_t)nb * n);
  if (Gout) memcpy(Gout, G, sizeof(cplx) * (size_t)nb * n);
  free(F);
  free(G);
  free(B);
  free(E);
  free(X);
  return bad;
}

/* Public single-leaf entry: the operators of a leaf of the descriptor's size
 * with coefficient samples c (they depend on nothing else).  Any of B, F, G
 * may be NULL. */
int ora_leaf(const ora_desc *d, const double *c, cplx *Psi, cplx *Y, cplx *R, cplx *Gam, cplx *B,
             cplx *F, cplx *G) {
  if (check_desc(d)) return -1;
  leaf_geom g;
  leaf_geom_init(&g, d->p, (d->x1 - d->x0) / d->mx, (d->y1 - d->y0) / d->my);
  int bad = leaf_ops(&g, d->kappa, d->eta_re + I * d->eta_im, c, Psi, Y, R, Gam, B, F, G);
  leaf_geom_free(&g);
  return bad;
}

/* ------------------------------------------------------------------ */
/* tree, build (Algorithm 1) and solve (Algorithm 2)                    */
/* ------------------------------------------------------------------ */

typedef struct {
  int is_leaf;
  int pub;             /* public leaf index (leaves only) */
  int nb;              /* boundary length */
  double *bxy;         /* boundary coordinates [nb][2] in this box's order */
  cplx *R;             /* ItI operator nb x nb (freed after the parent merge) */
  /* leaf operators */
  cplx *Psi, *Y, *Gam;
  /* merge operators (this box is the parent tau) */
  int n1, n2, n3;
  int *I1, *I2, *I3a, *I3b;
  cplx *Winv, *R33a, *R33b, *R13a, *R23b, *Phia, *Phib;
  double condW;        /* ||W||_1 ||W^{-1}||_1 of this merge */
} ora_box;

typedef struct {
  ora_desc d;
  int L;          /* leaf level */
  int nboxes;     /* 2^(L+1) - 1, boxes numbered 1..nboxes */
  ora_box *box;   /* box[tau], tau = 1..nboxes */
  int e, n, nb, ni;  /* nb: boundary-data points of a leaf (4 edge_pts) */
  double *Pm, *Qm;   /* gauss_q > 0: edge interpolation (edge_interp) */
  int status;
  int dir[64];      /* merge directions of this tree, from the leaves */
  int pub_dir[64];  /* those of the public leaf order */
} ora_tree;

static int tree_leaf_public(const ora_tree *T, int slot) {
  /* slot: position of the leaf in the tree's order (its merge directions);
   * the public order follows the directions that start west/east */
  int c, r;
  leaf_decode(slot, T->dir, T->L, &c, &r);
  return leaf_encode(c, r, T->pub_dir, T->L);
}

static int same_point(const double *a, const double *b, double tol) {
  return fabs(a[0] - b[0]) <= tol && fabs(a[1] - b[1]) <= tol;
}

/* Merge of box tau from children alpha = 2 tau and beta = 2 tau + 1. */
static void merge_box(ora_tree *T, int tau) {
  ora_box *P = &T->box[tau], *A = &T->box[2 * tau], *Bb = &T->box[2 * tau + 1];
  double tol = 1e-10 * fmax(T->d.x1 - T->d.x0, T->d.y1 - T->d.y0);
  int na = A->nb, nbb = Bb->nb;
  int *inA = xmalloc(sizeof(int) * na), *inB = xmalloc(sizeof(int) * nbb);
  for (int i = 0; i < na; i++) inA[i] = -1;
  for (int j = 0; j < nbb; j++) inB[j] = -1;
  /* I3: nodes on the boundary of both children, ordered as in alpha */
  int n3 = 0;
  int *I3a = xmalloc(sizeof(int) * na), *I3b = xmalloc(sizeof(int) * na);
  for (int i = 0; i < na; i++)
    for (int j = 0; j < nbb; j++)
      if (same_point(&A->bxy[2 * i], &Bb->bxy[2 * j], tol)) {
        I3a[n3] = i;
        I3b[n3] = j;
        inA[i] = n3;
        inB[j] = n3;
        n3++;
        break;
      }
  int n1 = na - n3, n2 = nbb - n3;
  int *I1 = xmalloc(sizeof(int) * (n1 ? n1 : 1)), *I2 = xmalloc(sizeof(int) * (n2 ? n2 : 1));
  for (int i = 0, q = 0; i < na; i++)
    if (inA[i] < 0) I1[q++] = i;
  for (int j = 0, q = 0; j < nbb; j++)
    if (inB[j] < 0) I2[q++] = j;
  int nt = n1 + n2;
  /* sub-blocks of the children's ItI operators (Eqs. ItIalp, ItIbet) */
  cplx *R11a = xmalloc(sizeof(cplx) * n1 * n1), *R13a = xmalloc(sizeof(cplx) * n1 * n3);
  cplx *R31a = xmalloc(sizeof(cplx) * n3 * n1), *R33a = xmalloc(sizeof(cplx) * n3 * n3);
  cplx *R22b = xmalloc(sizeof(cplx) * n2 * n2), *R23b = xmalloc(sizeof(cplx) * n2 * n3);
  cplx *R32b = xmalloc(sizeof(cplx) * n3 * n2), *R33b = xmalloc(sizeof(cplx) * n3 * n3);
  for (int i = 0; i < n1; i++) {
    for (int j = 0; j < n1; j++) R11a[i * n1 + j] = A->R[(size_t)I1[i] * na + I1[j]];
    for (int j = 0; j < n3; j++) R13a[i * n3 + j] = A->R[(size_t)I1[i] * na + I3a[j]];
  }
  for (int i = 0; i < n3; i++) {
    for (int j = 0; j < n1; j++) R31a[i * n1 + j] = A->R[(size_t)I3a[i] * na + I1[j]];
    for (int j = 0; j < n3; j++) R33a[i * n3 + j] = A->R[(size_t)I3a[i] * na + I3a[j]];
  }
  for (int i = 0; i < n2; i++) {
    for (int j = 0; j < n2; j++) R22b[i * n2 + j] = Bb->R[(size_t)I2[i] * nbb + I2[j]];
    for (int j = 0; j < n3; j++) R23b[i * n3 + j] = Bb->R[(size_t)I2[i] * nbb + I3b[j]];
  }
  for (int i = 0; i < n3; i++) {
    for (int j = 0; j < n2; j++) R32b[i * n2 + j] = Bb->R[(size_t)I3b[i] * nbb + I2[j]];
    for (int j = 0; j < n3; j++) R33b[i * n3 + j] = Bb->R[(size_t)I3b[i] * nbb + I3b[j]];
  }
  /* W = I - R33b R33a and its inverse (LU with partial pivoting) */
  cplx *W = xmalloc(sizeof(cplx) * n3 * n3), *Winv = xmalloc(sizeof(cplx) * n3 * n3);
  cplx *Id = xmalloc(sizeof(cplx) * n3 * n3);
  matmul(n3, n3, n3, R33b, R33a, W);
  for (int i = 0; i < n3 * n3; i++) W[i] = -W[i];
  for (int i = 0; i < n3; i++) {
    W[i * n3 + i] += 1.0;
    Id[i * n3 + i] = 1.0;
  }
  int bad = lu_solve_many(n3, W, n3, Id, Winv);
  if (bad && !T->status) T->status = 2;
  P->condW = norm1(n3, W) * norm1(n3, Winv);
  /* Phi_a = W^{-1} [R33b R31a | -R32b] */
  cplx *T1 = xmalloc(sizeof(cplx) * n3 * n1), *Q = xmalloc(sizeof(cplx) * n3 * nt);
  matmul(n3, n3, n1, R33b, R31a, T1);
  for (int i = 0; i < n3; i++) {
    for (int j = 0; j < n1; j++) Q[i * nt + j] = T1[i * n1 + j];
    for (int j = 0; j < n2; j++) Q[i * nt + n1 + j] = -R32b[i * n2 + j];
  }
  cplx *Phia = xmalloc(sizeof(cplx) * n3 * nt);
  matmul(n3, n3, nt, Winv, Q, Phia);
  /* Phi_b = [-R31a - R33a W^{-1} R33b R31a | R33a W^{-1} R32b]  (Eq. for Phi^beta) */
  cplx *S1 = xmalloc(sizeof(cplx) * n3 * n3), *S2 = xmalloc(sizeof(cplx) * n3 * n1);
  cplx *S3 = xmalloc(sizeof(cplx) * n3 * n2);
  matmul(n3, n3, n3, R33a, Winv, S1);    /* R33a W^{-1} */
  matmul(n3, n3, n1, S1, T1, S2);        /* R33a W^{-1} R33b R31a */
  matmul(n3, n3, n2, S1, R32b, S3);      /* R33a W^{-1} R32b */
  cplx *Phib = xmalloc(sizeof(cplx) * n3 * nt);
  for (int i = 0; i < n3; i++) {
    for (int j = 0; j < n1; j++) Phib[i * nt + j] = -R31a[i * n1 + j] - S2[i * n1 + j];
    for (int j = 0; j < n2; j++) Phib[i * nt + n1 + j] = S3[i * n2 + j];
  }
  /* R^tau = diag(R11a, R22b) + diag(R13a, R23b) [Phi_a; Phi_b] */
  cplx *Rt = xmalloc(sizeof(cplx) * (size_t)nt * nt);
  cplx *U1 = xmalloc(sizeof(cplx) * n1 * nt), *U2 = xmalloc(sizeof(cplx) * n2 * nt);
  matmul(n1, n3, nt, R13a, Phia, U1);
  matmul(n2, n3, nt, R23b, Phib, U2);
  for (int i = 0; i < n1; i++)
    for (int j = 0; j < nt; j++)
      Rt[(size_t)i * nt + j] = U1[i * nt + j] + ((j < n1) ? R11a[i * n1 + j] : 0.0);
  for (int i = 0; i < n2; i++)
    for (int j = 0; j < nt; j++)
      Rt[(size_t)(n1 + i) * nt + j] = U2[i * nt + j] + ((j >= n1) ? R22b[i * n2 + (j - n1)] : 0.0);
  /* parent boundary = [I1, I2] */
  P->is_leaf = 0;
  P->nb = nt;
  P->bxy = xmalloc(sizeof(double) * 2 * nt);
  for (int i = 0; i < n1; i++) {
    P->bxy[2 * i] = A->bxy[2 * I1[i]];
    P->bxy[2 * i + 1] = A->bxy[2 * I1[i] + 1];
  }
  for (int i = 0; i < n2; i++) {
    P->bxy[2 * (n1 + i)] = Bb->bxy[2 * I2[i]];
    P->bxy[2 * (n1 + i) + 1] = Bb->bxy[2 * I2[i] + 1];
  }
  P->R = Rt;
  P->n1 = n1;
  P->n2 = n2;
  P->n3 = n3;
  P->I1 = I1;
  P->I2 = I2;
  P->I3a = I3a;
  P->I3b = I3b;
  /* stored operators (Sec. 2.4) */
  P->Winv = Winv;
  P->R33a = R33a;
  P->R33b = R33b;
  P->R13a = R13a;
  P->R23b = R23b;
  P->Phia = Phia;
  P->Phib = Phib;
  /* delete the children's ItI operators */
  free(A->R);
  A->R = NULL;
  free(Bb->R);
  Bb->R = NULL;
  free(R11a);
  free(R31a);
  free(R22b);
  free(R32b);
  free(W);
  free(Id);
  free(T1);
  free(Q);
  free(S1);
  free(S2);
  free(S3);
  free(U1);
  free(U2);
  free(inA);
  free(inB);
}

static void leaf_box(ora_tree *T, const leaf_geom *g, int tau, const double *c) {
  ora_box *b = &T->box[tau];
  int slot = tau - (1 << T->L);
  int pub = tree_leaf_public(T, slot);
  int n = T->n, nb = T->nb, ni = T->ni, nbc = g->nb; /* nbc: Chebyshev edge nodes of a leaf */
  b->is_leaf = 1;
  b->pub = pub;
  b->nb = nb;
  b->Psi = xmalloc(sizeof(cplx) * (size_t)n * nbc);
  b->Y = xmalloc(sizeof(cplx) * (size_t)n * ni);
  b->Gam = xmalloc(sizeof(cplx) * (size_t)nbc * ni);
  b->R = xmalloc(sizeof(cplx) * (size_t)nbc * nbc);
  int bad = leaf_ops(g, T->d.kappa, T->d.eta_re + I * T->d.eta_im, c + (size_t)pub * ni, b->Psi,
                     b->Y, b->R, b->Gam, NULL, NULL, NULL);
  if (bad && !T->status) T->status = 1;
  if (T->d.gauss_q) {
    /* boundary data on the Gauss nodes: incoming t_G enters as Qh t_G on the
     * Chebyshev edge nodes, outgoing data leaves as Ph g; so Psi_G = Psi Qh,
     * R_G = Ph R Qh, Gamma_G = Ph Gamma with Ph = diag(Pm, Pm, Pm, Pm) and
     * Qh = diag(Qm, Qm, Qm, Qm) over the edges [S, E, N, W] */
    int q = T->d.gauss_q, e = T->e;
    cplx *Ph = xmalloc(sizeof(cplx) * (size_t)nb * nbc), *Qh = xmalloc(sizeof(cplx) * (size_t)nbc * nb);
    for (int side = 0; side < 4; side++) {
      for (int a = 0; a < q; a++)
        for (int j = 0; j < e; j++) Ph[(size_t)(side * q + a) * nbc + side * e + j] = T->Pm[a * e + j];
      for (int j = 0; j < e; j++)
        for (int a = 0; a < q; a++) Qh[(size_t)(side * e + j) * nb + side * q + a] = T->Qm[j * q + a];
    }
    cplx *Psi = xmalloc(sizeof(cplx) * (size_t)n * nb), *Gam = xmalloc(sizeof(cplx) * (size_t)nb * ni);
    cplx *RQ = xmalloc(sizeof(cplx) * (size_t)nbc * nb), *R = xmalloc(sizeof(cplx) * (size_t)nb * nb);
    matmul(n, nbc, nb, b->Psi, Qh, Psi);
    matmul(nbc, nbc, nb, b->R, Qh, RQ);
    matmul(nb, nbc, nb, Ph, RQ, R);
    matmul(nb, nbc, ni, Ph, b->Gam, Gam);
    free(b->Psi);
    free(b->R);
    free(b->Gam);
    b->Psi = Psi;
    b->R = R;
    b->Gam = Gam;
    free(Ph);
    free(Qh);
    free(RQ);
  }
  /* boundary coordinates of this leaf, in its local order */
  int p = T->d.p, col, row;
  leaf_decode(pub, T->pub_dir, T->L, &col, &row);
  double hx = (T->d.x1 - T->d.x0) / T->d.mx, hy = (T->d.y1 - T->d.y0) / T->d.my;
  double *xs = xmalloc(sizeof(double) * p), *ys = xmalloc(sizeof(double) * p);
  double *D = xmalloc(sizeof(double) * p * p);
  ora_cheb(p, T->d.x0 + col * hx, T->d.x0 + (col + 1) * hx, xs, D);
  ora_cheb(p, T->d.y0 + row * hy, T->d.y0 + (row + 1) * hy, ys, D);
  b->bxy = xmalloc(sizeof(double) * 2 * nb);
  if (!T->d.gauss_q) {
    for (int k = 0; k < nb; k++) {
      int ix, iy;
      local_to_grid(p, k, &ix, &iy);
      b->bxy[2 * k] = xs[ix];
      b->bxy[2 * k + 1] = ys[iy];
    }
  } else {
    /* the Gauss nodes of the edges [S, E, N, W], each in increasing coordinate */
    int q = T->d.gauss_q;
    double *zg = xmalloc(sizeof(double) * q);
    ora_gauss_nodes(q, zg);
    leaf_gauss_xy(&T->d, col, row, q, zg, b->bxy);
    free(zg);
  }
  free(xs);
  free(ys);
  free(D);
}

/* Algorithm 1 (with the level-by-level grouping of Algorithm 3 when
 * nthreads > 1).  c: [leaves][(p-2)^2] at the interior nodes, public order. */
void *ora_build(const ora_desc *d, const double *c, int nthreads) {
  if (check_desc(d)) return NULL;
  ora_tree *T = xmalloc(sizeof(ora_tree));
  T->d = *d;
  T->L = merge_dirs(log2i(d->mx), log2i(d->my), d->first_vertical, T->dir);
  merge_dirs(log2i(d->mx), log2i(d->my), 0, T->pub_dir);
  T->nboxes = (1 << (T->L + 1)) - 1;
  T->box = xmalloc(sizeof(ora_box) * (size_t)(T->nboxes + 1));
  T->e = d->p - 2;
  T->n = d->p * d->p - 4;
  T->nb = 4 * edge_pts(d);
  T->ni = T->e * T->e;
  T->Pm = T->Qm = NULL;
  if (d->gauss_q) {
    T->Pm = xmalloc(sizeof(double) * d->gauss_q * T->e);
    T->Qm = xmalloc(sizeof(double) * d->gauss_q * T->e);
    edge_interp(d->p, d->gauss_q, T->Pm, T->Qm);
  }
  leaf_geom g;
  leaf_geom_init(&g, d->p, (d->x1 - d->x0) / d->mx, (d->y1 - d->y0) / d->my);
  if (nthreads < 1) nthreads = 1;
  for (int lev = T->L; lev >= 0; lev--) {
    int lo = 1 << lev, hi = (1 << (lev + 1)) - 1;
    /* boxes of one level in decreasing index, as Algorithm 1 visits them */
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) if (nthreads > 1)
    for (int tau = hi; tau >= lo; tau--) {
      if (lev == T->L)
        leaf_box(T, &g, tau, c);
      else
        merge_box(T, tau);
    }
  }
  leaf_geom_free(&g);
  return T;
}

int ora_status(void *h) { return ((ora_tree *)h)->status; }

/* root ItI operator reordered to the public [S, E, N, W] boundary order */
static int *root_order(ora_tree *T) {
  int nbr = 2 * (T->d.mx + T->d.my) * edge_pts(&T->d);
  double *bxy = xmalloc(sizeof(double) * 2 * nbr);
  ora_nodes(&T->d, NULL, bxy);
  double tol = 1e-10 * fmax(T->d.x1 - T->d.x0, T->d.y1 - T->d.y0);
  int *perm = xmalloc(sizeof(int) * nbr); /* perm[public] = root position */
  ora_box *r = &T->box[1];
  for (int q = 0; q < nbr; q++) {
    perm[q] = -1;
    for (int j = 0; j < r->nb; j++)
      if (same_point(&bxy[2 * q], &r->bxy[2 * j], tol)) {
        perm[q] = j;
        break;
      }
  }
  free(bxy);
  return perm;
}

int ora_root_R(void *h, cplx *Rout) {
  ora_tree *T = h;
  ora_box *r = &T->box[1];
  if (!r->R) return 1;
  int nbr = r->nb;
  int *perm = root_order(T);
  for (int i = 0; i < nbr; i++)
    for (int j = 0; j < nbr; j++) Rout[(size_t)i * nbr + j] = r->R[(size_t)perm[i] * nbr + perm[j]];
  free(perm);
  return 0;
}

/* The largest 1-norm condition number ||W||_1 ||W^{-1}||_1 of the interface
 * matrices W = I - R33b R33a (Sec. 2.2) over the merges whose parent lies on
 * tree level lev (0: the root's merge); -1 for a level without merges. */
double ora_cond_W(void *h, int lev) {
  ora_tree *T = h;
  if (lev < 0 || lev >= T->L) return -1.0;
  double best = 0.0;
  for (int tau = 1 << lev; tau < (1 << (lev + 1)); tau++)
    if (T->box[tau].condW > best) best = T->box[tau].condW;
  return best;
}

/* Leaf operators as stored by the build, for the leaf with public index pub. */
int ora_tree_leaf(void *h, int pub, cplx *Psi, cplx *Y, cplx *Gam) {
  ora_tree *T = h;
  for (int tau = 1 << T->L; tau < (1 << (T->L + 1)); tau++)
    if (T->box[tau].pub == pub) {
      ora_box *b = &T->box[tau];
      memcpy(Psi, b->Psi, sizeof(cplx) * (size_t)T->n * T->nb);
      memcpy(Y, b->Y, sizeof(cplx) * (size_t)T->n * T->ni);
      memcpy(Gam, b->Gam, sizeof(cplx) * (size_t)T->nb * T->ni);
      return 0;
    }
  return 1;
}

/* Algorithm 2 for nrhs right-hand sides.
 * s: [nrhs][leaves][(p-2)^2], t: [nrhs][2 (mx + my) q] (q = edge_pts),
 * u: [nrhs][leaves][p^2-4]. */
int ora_solve(void *h, const cplx *s, const cplx *t, cplx *u, int nrhs, int nthreads) {
  ora_tree *T = h;
  int L = T->L, nl = 1 << L, n = T->n, nb = T->nb, ni = T->ni;
  int nbr = 2 * (T->d.mx + T->d.my) * edge_pts(&T->d);
  int *perm = root_order(T);
  if (nthreads < 1) nthreads = 1;
  cplx **hv = xmalloc(sizeof(cplx *) * (size_t)(T->nboxes + 1));
  cplx **tv = xmalloc(sizeof(cplx *) * (size_t)(T->nboxes + 1));
  cplx **tta = xmalloc(sizeof(cplx *) * (size_t)(T->nboxes + 1)); /* t~3a per merge */
  cplx **ttb = xmalloc(sizeof(cplx *) * (size_t)(T->nboxes + 1)); /* t~3b per merge */
  cplx **ut = xmalloc(sizeof(cplx *) * (size_t)(T->nboxes + 1));  /* u~ per leaf */
  for (int r = 0; r < nrhs; r++) {
    const cplx *sr = s + (size_t)r * nl * ni;
    /* upward pass */
    for (int lev = L; lev >= 0; lev--) {
      int lo = 1 << lev, hi = (1 << (lev + 1)) - 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) if (nthreads > 1)
      for (int tau = hi; tau >= lo; tau--) {
        ora_box *b = &T->box[tau];
        hv[tau] = xmalloc(sizeof(cplx) * b->nb);
        if (b->is_leaf) {
          const cplx *sl = sr + (size_t)b->pub * ni;
          ut[tau] = xmalloc(sizeof(cplx) * n);
          matmul(n, ni, 1, b->Y, sl, ut[tau]);
          matmul(nb, ni, 1, b->Gam, sl, hv[tau]);
        } else {
          int n1 = b->n1, n2 = b->n2, n3 = b->n3;
          cplx *ha = hv[2 * tau], *hb = hv[2 * tau + 1];
          cplx *h3a = xmalloc(sizeof(cplx) * n3), *h3b = xmalloc(sizeof(cplx) * n3);
          for (int i = 0; i < n3; i++) {
            h3a[i] = ha[b->I3a[i]];
            h3b[i] = hb[b->I3b[i]];
          }
          /* t~3a = Upsilon_a [h3a; h3b] = W^{-1} R33b h3a - W^{-1} h3b */
          cplx *v1 = xmalloc(sizeof(cplx) * n3), *v2 = xmalloc(sizeof(cplx) * n3);
          cplx *v3 = xmalloc(sizeof(cplx) * n3), *v4 = xmalloc(sizeof(cplx) * n3);
          matmul(n3, n3, 1, b->R33b, h3a, v1);
          matmul(n3, n3, 1, b->Winv, v1, v2); /* W^{-1} R33b h3a */
          matmul(n3, n3, 1, b->Winv, h3b, v3); /* W^{-1} h3b */
          tta[tau] = xmalloc(sizeof(cplx) * n3);
          for (int i = 0; i < n3; i++) tta[tau][i] = v2[i] - v3[i];
          /* t~3b = Upsilon_b [h3a; h3b]
           *      = -(I + R33a W^{-1} R33b) h3a + R33a W^{-1} h3b */
          cplx *w1 = xmalloc(sizeof(cplx) * n3), *w2 = xmalloc(sizeof(cplx) * n3);
          matmul(n3, n3, 1, b->R33a, v2, w1);
          matmul(n3, n3, 1, b->R33a, v3, w2);
          ttb[tau] = xmalloc(sizeof(cplx) * n3);
          for (int i = 0; i < n3; i++) ttb[tau][i] = -(h3a[i] + w1[i]) + w2[i];
          /* h^tau = [h1a; h2b] + diag(R13a, R23b) [t~3a; t~3b]  (Eq. flux_part) */
          cplx *x1 = xmalloc(sizeof(cplx) * (n1 ? n1 : 1)), *x2 = xmalloc(sizeof(cplx) * (n2 ? n2 : 1));
          matmul(n1, n3, 1, b->R13a, tta[tau], x1);
          matmul(n2, n3, 1, b->R23b, ttb[tau], x2);
          for (int i = 0; i < n1; i++) hv[tau][i] = ha[b->I1[i]] + x1[i];
          for (int i = 0; i < n2; i++) hv[tau][n1 + i] = hb[b->I2[i]] + x2[i];
          free(h3a);
          free(h3b);
          free(v1);
          free(v2);
          free(v3);
          free(v4);
          free(w1);
          free(w2);
          free(x1);
          free(x2);
        }
      }
    }
    /* downward pass: the root takes the given boundary data */
    tv[1] = xmalloc(sizeof(cplx) * nbr);
    for (int q = 0; q < nbr; q++) tv[1][perm[q]] = t[(size_t)r * nbr + q];
    for (int lev = 0; lev <= L; lev++) {
      int lo = 1 << lev, hi = (1 << (lev + 1)) - 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) if (nthreads > 1)
      for (int tau = lo; tau <= hi; tau++) {
        ora_box *b = &T->box[tau];
        if (b->is_leaf) {
          cplx *ul = u + ((size_t)r * nl + b->pub) * n;
          matmul(n, nb, 1, b->Psi, tv[tau], ul);
          for (int i = 0; i < n; i++) ul[i] += ut[tau][i];
        } else {
          int n1 = b->n1, n2 = b->n2, n3 = b->n3, nt = n1 + n2;
          cplx *t3a = xmalloc(sizeof(cplx) * n3), *t3b = xmalloc(sizeof(cplx) * n3);
          matmul(n3, nt, 1, b->Phia, tv[tau], t3a);
          matmul(n3, nt, 1, b->Phib, tv[tau], t3b);
          ora_box *A = &T->box[2 * tau], *Bb = &T->box[2 * tau + 1];
          tv[2 * tau] = xmalloc(sizeof(cplx) * A->nb);
          tv[2 * tau + 1] = xmalloc(sizeof(cplx) * Bb->nb);
          for (int i = 0; i < n1; i++) tv[2 * tau][b->I1[i]] = tv[tau][i];
          for (int i = 0; i < n2; i++) tv[2 * tau + 1][b->I2[i]] = tv[tau][n1 + i];
          for (int i = 0; i < n3; i++) {
            tv[2 * tau][b->I3a[i]] = t3a[i] + tta[tau][i];
            tv[2 * tau + 1][b->I3b[i]] = t3b[i] + ttb[tau][i];
          }
          free(t3a);
          free(t3b);
        }
      }
    }
    for (int tau = 1; tau <= T->nboxes; tau++) {
      free(hv[tau]);
      free(tv[tau]);
      hv[tau] = tv[tau] = NULL;
      if (T->box[tau].is_leaf) {
        free(ut[tau]);
        ut[tau] = NULL;
      } else {
        free(tta[tau]);
        free(ttb[tau]);
        tta[tau] = ttb[tau] = NULL;
      }
    }
  }
  free(hv);
  free(tv);
  free(tta);
  free(ttb);
  free(ut);
  free(perm);
  return 0;
}

void ora_free(void *h) {
  ora_tree *T = h;
  if (!T) return;
  for (int tau = 1; tau <= T->nboxes; tau++) {
    ora_box *b = &T->box[tau];
    free(b->bxy);
    free(b->R);
    free(b->Psi);
    free(b->Y);
    free(b->Gam);
    free(b->I1);
    free(b->I2);
    free(b->I3a);
    free(b->I3b);
    free(b->Winv);
    free(b->R33a);
    free(b->R33b);
    free(b->R13a);
    free(b->R23b);
    free(b->Phia);
    free(b->Phib);
  }
  free(T->box);
  free(T->Pm);
  free(T->Qm);
  free(T);
}

/* ------------------------------------------------------------------ */
/* brute force: the global collocation system, dense LU                */
/* ------------------------------------------------------------------ */

/* The global system with boundary data on q Gauss nodes per leaf edge.
 * Unknowns per leaf: its nodal values u (p^2-4) and its incoming data t_G on
 * the Gauss nodes of its edges (4 q).  Equations per leaf: the impedance rows
 * F u = Qh t_G on its Chebyshev edge nodes, its interior collocation rows,
 * and per Gauss node either t_G = t (outer boundary) or, with the coincident
 * Gauss node of the neighbouring leaf, t_G(here) = -(Ph G u)(there), the
 * condition t3a = -g3b / t3b = -g3a of Sec. 2.2 on the Gauss nodes. */
static int brute_gauss(const ora_desc *d, const double *c, const cplx *s, const cplx *t, cplx *u) {
  int p = d->p, e = p - 2, n = p * p - 4, nbc = 4 * e, ni = e * e, q = d->gauss_q, nbq = 4 * q;
  int nl = d->mx * d->my, nu = n + nbq, N = nl * nu, nbr = 2 * (d->mx + d->my) * q;
  double tol = 1e-10 * fmax(d->x1 - d->x0, d->y1 - d->y0);
  leaf_geom g;
  leaf_geom_init(&g, p, (d->x1 - d->x0) / d->mx, (d->y1 - d->y0) / d->my);
  cplx eta = d->eta_re + I * d->eta_im;
  double *Pm = xmalloc(sizeof(double) * q * e), *Qm = xmalloc(sizeof(double) * e * q);
  edge_interp(p, q, Pm, Qm);
  double *zg = xmalloc(sizeof(double) * q);
  ora_gauss_nodes(q, zg);
  double *bxy = xmalloc(sizeof(double) * 2 * nbr);
  ora_nodes(d, NULL, bxy);
  double *gxy = xmalloc(sizeof(double) * 2 * (size_t)nl * nbq); /* Gauss nodes of every leaf */
  int dir[64], L = merge_dirs(log2i(d->mx), log2i(d->my), 0, dir);
  for (int l = 0; l < nl; l++) {
    int col, row;
    leaf_decode(l, dir, L, &col, &row);
    leaf_gauss_xy(d, col, row, q, zg, gxy + 2 * (size_t)l * nbq);
  }
  cplx *Bl = xmalloc(sizeof(cplx) * (size_t)nl * n * n);
  cplx *Fl = xmalloc(sizeof(cplx) * (size_t)nl * nbc * n);
  cplx *Gl = xmalloc(sizeof(cplx) * (size_t)nl * nbc * n);
  cplx *Psi = xmalloc(sizeof(cplx) * (size_t)n * nbc), *Y = xmalloc(sizeof(cplx) * (size_t)n * ni);
  cplx *R = xmalloc(sizeof(cplx) * (size_t)nbc * nbc), *Gam = xmalloc(sizeof(cplx) * (size_t)nbc * ni);
  for (int l = 0; l < nl; l++)
    leaf_ops(&g, d->kappa, eta, c + (size_t)l * ni, Psi, Y, R, Gam, Bl + (size_t)l * n * n,
             Fl + (size_t)l * nbc * n, Gl + (size_t)l * nbc * n);
  cplx *A = xmalloc(sizeof(cplx) * (size_t)N * N);
  cplx *rhs = xmalloc(sizeof(cplx) * (size_t)N);
  for (int l = 0; l < nl; l++) {
    size_t base = (size_t)l * nu, tbase = base + n;
    const cplx *F = Fl + (size_t)l * nbc * n, *B = Bl + (size_t)l * n * n;
    /* F u - Qh t_G = 0 on the Chebyshev edge nodes */
    for (int k = 0; k < nbc; k++) {
      size_t row = base + k;
      int side = k / e, j = k % e;
      for (int jj = 0; jj < n; jj++) A[row * N + base + jj] = F[(size_t)k * n + jj];
      for (int a = 0; a < q; a++) A[row * N + tbase + side * q + a] = -Qm[j * q + a];
      rhs[row] = 0.0;
    }
    /* interior collocation rows */
    for (int i = 0; i < ni; i++) {
      size_t row = base + nbc + i;
      for (int jj = 0; jj < n; jj++) A[row * N + base + jj] = B[(size_t)(nbc + i) * n + jj];
      rhs[row] = s[(size_t)l * ni + i];
    }
    /* one row per Gauss node of this leaf */
    for (int k = 0; k < nbq; k++) {
      size_t row = tbase + k;
      const double *pt = &gxy[2 * ((size_t)l * nbq + k)];
      A[row * N + tbase + k] = 1.0;
      int outer = -1;
      for (int qb = 0; qb < nbr; qb++)
        if (same_point(pt, &bxy[2 * qb], tol)) {
          outer = qb;
          break;
        }
      if (outer >= 0) {
        rhs[row] = t[outer];
        continue;
      }
      int found = 0;
      for (int l2 = 0; l2 < nl && !found; l2++) {
        if (l2 == l) continue;
        for (int k2 = 0; k2 < nbq; k2++)
          if (same_point(pt, &gxy[2 * ((size_t)l2 * nbq + k2)], tol)) {
            /* + (Ph G u)(k2) of the neighbour: row k2 of Ph is Pm's row a2 on side2 */
            int side2 = k2 / q, a2 = k2 % q;
            const cplx *G2 = Gl + (size_t)l2 * nbc * n;
            for (int j = 0; j < e; j++) {
              double w = Pm[a2 * e + j];
              for (int jj = 0; jj < n; jj++)
                A[row * N + (size_t)l2 * nu + jj] += w * G2[(size_t)(side2 * e + j) * n + jj];
            }
            found = 1;
            break;
          }
      }
      rhs[row] = 0.0;
      if (!found) {
        fprintf(stderr, "hps_oracle: unmatched Gauss node\n");
        abort();
      }
    }
  }
  int *piv = xmalloc(sizeof(int) * (size_t)N);
  int bad = lu_factor(N, A, piv);
  if (!bad) lu_solve(N, A, piv, rhs);
  for (int l = 0; l < nl; l++) memcpy(u + (size_t)l * n, rhs + (size_t)l * nu, sizeof(cplx) * n);
  free(piv);
  free(A);
  free(rhs);
  free(Bl);
  free(Fl);
  free(Gl);
  free(Psi);
  free(Y);
  free(R);
  free(Gam);
  free(Pm);
  free(Qm);
  free(zg);
  free(bxy);
  free(gxy);
  leaf_geom_free(&g);
  return bad;
}

/* u: [leaves][p^2-4] for one right-hand side (s: [leaves][(p-2)^2],
 * t: [2 (mx + my) q], q = edge_pts).  Returns 0, or nonzero when the system
 * is singular. */
int ora_brute(const ora_desc *d, const double *c, const cplx *s, const cplx *t, cplx *u) {
  if (check_desc(d)) return -1;
  if (d->gauss_q) return brute_gauss(d, c, s, t, u);
  int p = d->p, e = p - 2, n = p * p - 4, nb = 4 * e, ni = e * e;
  int nl = d->mx * d->my, N = nl * n, nbr = 2 * (d->mx + d->my) * e;
  double tol = 1e-10 * fmax(d->x1 - d->x0, d->y1 - d->y0);
  leaf_geom g;
  leaf_geom_init(&g, p, (d->x1 - d->x0) / d->mx, (d->y1 - d->y0) / d->my);
  cplx eta = d->eta_re + I * d->eta_im;
  double *xy = xmalloc(sizeof(double) * 2 * (size_t)nl * n);
  double *bxy = xmalloc(sizeof(double) * 2 * nbr);
  ora_nodes(d, xy, bxy);
  cplx *Bl = xmalloc(sizeof(cplx) * (size_t)nl * n * n); /* B of every leaf */
  cplx *Fl = xmalloc(sizeof(cplx) * (size_t)nl * nb * n);
  cplx *Gl = xmalloc(sizeof(cplx) * (size_t)nl * nb * n);
  cplx *Psi = xmalloc(sizeof(cplx) * (size_t)n * nb), *Y = xmalloc(sizeof(cplx) * (size_t)n * ni);
  cplx *R = xmalloc(sizeof(cplx) * (size_t)nb * nb), *Gam = xmalloc(sizeof(cplx) * (size_t)nb * ni);
  for (int l = 0; l < nl; l++)
    leaf_ops(&g, d->kappa, eta, c + (size_t)l * ni, Psi, Y, R, Gam, Bl + (size_t)l * n * n,
             Fl + (size_t)l * nb * n, Gl + (size_t)l * nb * n);
  cplx *A = xmalloc(sizeof(cplx) * (size_t)N * N);
  cplx *rhs = xmalloc(sizeof(cplx) * (size_t)N);
  for (int l = 0; l < nl; l++) {
    size_t base = (size_t)l * n;
    /* interior collocation rows of this leaf */
    for (int q = 0; q < ni; q++) {
      size_t row = base + nb + q;
      for (int j = 0; j < n; j++) A[row * N + base + j] = Bl[(size_t)l * n * n + (size_t)(nb + q) * n + j];
      rhs[row] = s[(size_t)l * ni + q];
    }
    /* one row per boundary node of this leaf */
    for (int k = 0; k < nb; k++) {
      size_t row = base + k;
      const double *pt = &xy[2 * (base + k)];
      for (int j = 0; j < n; j++) A[row * N + base + j] = Fl[(size_t)l * nb * n + (size_t)k * n + j];
      int outer = -1;
      for (int qb = 0; qb < nbr; qb++)
        if (same_point(pt, &bxy[2 * qb], tol)) {
          outer = qb;
          break;
        }
      if (outer >= 0) {
        rhs[row] = t[outer]; /* F u = t on the outer boundary */
        continue;
      }
      /* the coincident node of the neighbouring leaf: F u (here) + G u (there) = 0 */
      int found = 0;
      for (int l2 = 0; l2 < nl && !found; l2++) {
        if (l2 == l) continue;
        for (int k2 = 0; k2 < nb; k2++)
          if (same_point(pt, &xy[2 * ((size_t)l2 * n + k2)], tol)) {
            for (int j = 0; j < n; j++)
              A[row * N + (size_t)l2 * n + j] += Gl[(size_t)l2 * nb * n + (size_t)k2 * n + j];
            found = 1;
            break;
          }
      }
      rhs[row] = 0.0;
      if (!found) {
        fprintf(stderr, "hps_oracle: unmatched edge node\n");
        abort();
      }
    }
  }
  int *piv = xmalloc(sizeof(int) * (size_t)N);
  int bad = lu_factor(N, A, piv);
  if (!bad) lu_solve(N, A, piv, rhs);
  memcpy(u, rhs, sizeof(cplx) * (size_t)N);
  free(piv);
  free(A);
  free(rhs);
  free(Bl);
  free(Fl);
  free(Gl);
  free(Psi);
  free(Y);
  free(R);
  free(Gam);
  free(xy);
  free(bxy);
  leaf_geom_free(&g);
  return bad;
}

/* Threads available to the oracle's optional level-parallel loops. */
int ora_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
