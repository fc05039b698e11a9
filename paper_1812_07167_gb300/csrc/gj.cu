// Leaf kernel and interface-inverse kernel: blocked in-place Gauss-Jordan
// inversion with partial pivoting, one matrix per thread-block cluster.
//
// Leaf (Sec. 2.1): for every leaf the kernel assembles
//     B = [ F ; A-hat(I_i, I^tau) ],  F = N + i eta I(I_b, :),
//     A-hat = -D_x^2 - D_y^2 - kappa^2 diag(c),
// inverts it, and writes X = B^{-1} = [Psi | Y] (Eqs. hmgsolnopdef and
// prtsolnopdef: B Psi = [I; 0], B Y = [0; I]) together with
// G X = [R | Gamma] (R = G Psi, Gamma = G Y), G = N - i eta I(I_b, :).
// Interface (Sec. 2.2): W^{-1} for every merge of a level.
//
// Algorithm.  Gauss-Jordan elimination with row pivoting, in place on a
// scratch copy of the matrix in global memory (it stays in L2), the columns
// split over the `cs` CTAs of a cluster in slabs of cw columns (cw a multiple
// of the panel width KB).  The steps are taken KB at a time:
//   * the CTA owning panel p = [k0, k0+KB) eliminates it alone, in shared
//     memory: for each k it picks the pivot row (largest max(|Re|,|Im|) at or
//     below row k, lowest row on ties), swaps it into row k and applies the
//     Gauss-Jordan step to the panel's columns.  The resulting panel columns T
//     are the panel's columns of the accumulated elimination matrix; the row
//     swaps are summarised as a short list of row moves.
//   * every CTA then applies the panel to each of its other columns a: the
//     row moves, then a <- a + (T - I[:, P]) a[P], a rank-KB update.
//   * the row swaps become a column permutation of the inverse, applied when
//     the result is written out.
// Look-ahead: the owner of panel p+1 updates those columns first, eliminates
// that panel and publishes it (cluster barrier arrive) before it updates its
// remaining columns, so a panel's elimination overlaps the other CTAs'
// updates.  One cluster barrier (hardware barrier.cluster, split into arrive
// and wait) per panel; no kernel here spins on a flag.
#include <cooperative_groups.h>

#include "hps_internal.h"

namespace cg = cooperative_groups;

namespace hps {

namespace {

constexpr int kThreads = 256;
constexpr int KB = 8;           // panel width
constexpr int kMoves = 2 * KB;  // row moves of one panel, at most
constexpr int kMoveInts = 1 + 2 * kMoves;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ double2 crecip(double2 z) {
  // 1 / z with Smith's scaling (Smith, CACM 1962)
  if (fabs(z.x) >= fabs(z.y)) {
    double r = z.y / z.x, d = z.x + z.y * r;
    return make_double2(1.0 / d, -r / d);
  } else {
    double r = z.x / z.y, d = z.x * r + z.y;
    return make_double2(r / d, -1.0 / d);
  }
}

// max(|Re|, |Im|) as the integer image of its IEEE-754 bits (for
// non-negative doubles integer order is numeric order): the pivot search
// compares integers instead of spending FP64 instructions.
__device__ __forceinline__ unsigned long long mag_key(double2 z) {
  unsigned long long a = (unsigned long long)__double_as_longlong(z.x) & 0x7fffffffffffffffull;
  unsigned long long b = (unsigned long long)__double_as_longlong(z.y) & 0x7fffffffffffffffull;
  return a > b ? a : b;
}

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline int npanels(int n) { return (n + KB - 1) / KB; }
// ints of per-matrix bookkeeping: pivot rows, then the row moves of each panel
__host__ __device__ inline int meta_ints(int n) { return n + npanels(n) * kMoveInts; }

struct SmemPlan {
  size_t T, F, x, mvbuf, col, prow, mv, rows, srcs, scal, pinv, perm, dtab, grid, loc, cv, total;
};

__host__ __device__ inline SmemPlan plan_smem(int n, int cw, bool leaf, int p) {
  SmemPlan s;
  size_t o = 0;
  s.T = o;    o = align16(o + sizeof(double2) * (size_t)KB * n);
  s.F = o;    o = align16(o + sizeof(double2) * (size_t)KB * n);
  s.x = o;    o = align16(o + sizeof(double2) * (size_t)KB * cw);
  s.mvbuf = o; o = align16(o + sizeof(double2) * (size_t)kMoves * cw);
  s.col = o;  o = align16(o + sizeof(double2) * (size_t)n);
  s.prow = o; o = align16(o + sizeof(double2) * KB);
  s.mv = o;   o = align16(o + sizeof(int) * kMoveInts);
  s.rows = o; o = align16(o + sizeof(int) * 2 * KB);
  s.srcs = o; o = align16(o + sizeof(int) * 2 * KB);
  s.scal = o; o = align16(o + sizeof(int) * 4);
  s.pinv = o; o = align16(o + sizeof(double2));
  s.perm = o; o = align16(o + sizeof(int) * (size_t)n);
  if (leaf) {
    int ni = (p - 2) * (p - 2);
    s.dtab = o; o = align16(o + sizeof(double) * 4 * (size_t)p * p);
    s.grid = o; o = align16(o + sizeof(int) * (size_t)n);
    s.loc = o;  o = align16(o + sizeof(int) * (size_t)p * p);
    s.cv = o;   o = align16(o + sizeof(double) * (size_t)ni);
  } else {
    s.dtab = s.grid = s.loc = s.cv = o;
  }
  s.total = o;
  return s;
}

struct Shared {
  double2 *T;     // [KB][n] panel being applied (column-major)
  double2 *F;     // [KB][n] panel being eliminated (owner only)
  double2 *x;     // [KB][cw] panel rows of the own columns, after the moves
  double2 *mvbuf; // [cw][kMoves] values in flight during the row moves
  double2 *col;   // [n] pivot column of the current elimination step
  double2 *prow;  // [KB] scaled pivot row within the panel
  int *mv;        // [kMoveInts] row moves of the panel being applied
  int *rows;      // [2 KB] scratch for building a move list
  int *srcs;      // [2 KB]
  int *scal;      // [4] pivot row, zero flag
  double2 *pinv;  // [1] reciprocal of the pivot
  int *perm;      // [n] pivot rows, for the final column permutation
  int n, cw;
};

__device__ Shared bind(unsigned char *smem, const SmemPlan &sp, int n, int cw) {
  Shared s;
  s.T = (double2 *)(smem + sp.T);
  s.F = (double2 *)(smem + sp.F);
  s.x = (double2 *)(smem + sp.x);
  s.mvbuf = (double2 *)(smem + sp.mvbuf);
  s.col = (double2 *)(smem + sp.col);
  s.prow = (double2 *)(smem + sp.prow);
  s.mv = (int *)(smem + sp.mv);
  s.rows = (int *)(smem + sp.rows);
  s.srcs = (int *)(smem + sp.srcs);
  s.scal = (int *)(smem + sp.scal);
  s.pinv = (double2 *)(smem + sp.pinv);
  s.perm = (int *)(smem + sp.perm);
  s.n = n;
  s.cw = cw;
  return s;
}

// Eliminate panel [k0, k0 + kbp) of S (column-major, ld n) in shared memory
// and write it back; record its pivot rows and row moves in `meta`.
// Returns true if a zero pivot was met.
__device__ bool eliminate_panel(const Shared &s, double2 *S, int *meta, int k0, int kbp) {
  const int tid = threadIdx.x, nthr = blockDim.x, n = s.n;
  bool zero = false;
  for (int e = tid; e < kbp * n; e += nthr) {
    const int q = e / n, i = e % n;
    s.F[q * n + i] = S[(size_t)(k0 + q) * n + i];
  }
  __syncthreads();
  for (int q = 0; q < kbp; q++) {
    const int k = k0 + q;
    const double2 *Fk = s.F + q * n;
    if (tid < 32) {
      unsigned long long best = 0;
      int bi = n;
      for (int i = k + tid; i < n; i += 32) {
        unsigned long long key = mag_key(Fk[i]);
        if (bi == n || key > best) {
          best = key;
          bi = i;
        }
      }
      for (int off = 16; off; off >>= 1) {
        unsigned long long ov = __shfl_down_sync(0xffffffffu, best, off);
        int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (oi < n && (bi == n || ov > best || (ov == best && oi < bi))) {
          best = ov;
          bi = oi;
        }
      }
      if (tid == 0) {
        const int r = (bi < n) ? bi : k;
        const double2 pv = Fk[r];
        const bool z = (mag_key(pv) == 0ull);
        s.scal[0] = r;
        s.scal[1] = z ? 1 : 0;
        s.pinv[0] = z ? make_double2(0.0, 0.0) : crecip(pv);
        meta[k] = r;
      }
    }
    __syncthreads();
    const int r = s.scal[0];
    if (s.scal[1]) zero = true;
    const double2 pinv = s.pinv[0];
    // swap rows k and r inside the panel
    if (r != k)
      for (int qq = tid; qq < kbp; qq += nthr) {
        double2 t = s.F[qq * n + k];
        s.F[qq * n + k] = s.F[qq * n + r];
        s.F[qq * n + r] = t;
      }
    __syncthreads();
    // pivot column with its pivot entry zeroed, and the scaled pivot row
    for (int i = tid; i < n; i += nthr) s.col[i] = (i == k) ? make_double2(0.0, 0.0) : Fk[i];
    for (int qq = tid; qq < kbp; qq += nthr) s.prow[qq] = cmul(s.F[qq * n + k], pinv);
    __syncthreads();
    for (int e = tid; e < kbp * n; e += nthr) {
      const int qq = e / n, i = e % n;
      double2 *a = &s.F[qq * n + i];
      if (qq == q) {
        // the eliminated column becomes -col / pivot, 1 / pivot at the pivot
        if (i == k) {
          *a = pinv;
        } else {
          double2 f = cmul(s.col[i], pinv);
          *a = make_double2(-f.x, -f.y);
        }
      } else if (i == k) {
        *a = s.prow[qq];
      } else {
        double2 f = s.col[i], pr = s.prow[qq], v = *a;
        v.x = fma(-f.x, pr.x, v.x);
        v.x = fma(f.y, pr.y, v.x);
        v.y = fma(-f.x, pr.y, v.y);
        v.y = fma(-f.y, pr.x, v.y);
        *a = v;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < kbp * n; e += nthr) {
    const int q = e / n, i = e % n;
    S[(size_t)(k0 + q) * n + i] = s.F[q * n + i];
  }
  if (tid == 0) {
    // net row moves of the panel's swaps: after the swaps (k, piv[k]) in
    // order, row rows[t] holds what row srcs[t] held before
    int na = 0;
    for (int q = 0; q < kbp; q++) {
      const int k = k0 + q, r = meta[k];
      if (r == k) continue;
      int ia = -1, ib = -1;
      for (int t = 0; t < na; t++) {
        if (s.rows[t] == k) ia = t;
        if (s.rows[t] == r) ib = t;
      }
      if (ia < 0) {
        ia = na;
        s.rows[na] = k;
        s.srcs[na] = k;
        na++;
      }
      if (ib < 0) {
        ib = na;
        s.rows[na] = r;
        s.srcs[na] = r;
        na++;
      }
      int t = s.srcs[ia];
      s.srcs[ia] = s.srcs[ib];
      s.srcs[ib] = t;
    }
    int *m = meta + n + (k0 / KB) * kMoveInts;
    int cnt = 0;
    for (int t = 0; t < na; t++)
      if (s.rows[t] != s.srcs[t]) {
        m[1 + 2 * cnt] = s.rows[t];
        m[2 + 2 * cnt] = s.srcs[t];
        cnt++;
      }
    m[0] = cnt;
  }
  __syncthreads();
  return zero;
}

__device__ __forceinline__ bool skipped(int j, int a0, int a1, int b0, int b1) {
  return (j >= a0 && j < a1) || (j >= b0 && j < b1);
}

// Apply the panel [k0, k0+kbp) held in s.T / s.mv to the own columns
// j = c0 + jj, jj in [ja, jb), except those in [a0, a1) and [b0, b1).
__device__ void apply_panel(const Shared &s, double2 *S, int c0, int ja, int jb, int a0, int a1,
                            int b0, int b1, int k0, int kbp) {
  const int tid = threadIdx.x, nthr = blockDim.x, n = s.n, cw = s.cw;
  const int nm = s.mv[0];
  // 1) row moves (all loads, then all stores, staged in shared memory), then
  //    the panel rows x of each column
  const int nj = jb - ja;
  for (int e = tid; e < nm * nj; e += nthr) {
    const int t = e % nm, jj = ja + e / nm, j = c0 + jj;
    if (!skipped(j, a0, a1, b0, b1)) s.mvbuf[(jj - ja) * kMoves + t] = S[(size_t)j * n + s.mv[2 + 2 * t]];
  }
  __syncthreads();
  for (int e = tid; e < nm * nj; e += nthr) {
    const int t = e % nm, jj = ja + e / nm, j = c0 + jj;
    if (!skipped(j, a0, a1, b0, b1)) S[(size_t)j * n + s.mv[1 + 2 * t]] = s.mvbuf[(jj - ja) * kMoves + t];
  }
  __syncthreads();
  for (int e = tid; e < kbp * nj; e += nthr) {
    const int q = e % kbp, jj = ja + e / kbp, j = c0 + jj;
    if (!skipped(j, a0, a1, b0, b1)) s.x[q * cw + jj] = S[(size_t)j * n + k0 + q];
  }
  __syncthreads();
  // 2) a <- a + (T - I[:, P]) x: rows P get T x, the other rows add T x
  const int cl = tid >> 6, rl = tid & 63;
  for (int jj = ja + cl; jj < jb; jj += (nthr >> 6)) {
    const int j = c0 + jj;
    if (skipped(j, a0, a1, b0, b1)) continue;
    double2 *Sj = S + (size_t)j * n;
    for (int base = 0; base < n; base += 256) {
      double2 v[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int i = base + rl + 64 * u;
        v[u] = (i < n && (i < k0 || i >= k0 + kbp)) ? Sj[i] : make_double2(0.0, 0.0);
      }
      for (int q = 0; q < kbp; q++) {
        const double2 xv = s.x[q * cw + jj];
        const double2 *Tq = s.T + q * n + base + rl;
#pragma unroll
        for (int u = 0; u < 4; u++) {
          if (base + rl + 64 * u < n) {
            const double2 t = Tq[64 * u];
            v[u].x = fma(t.x, xv.x, v[u].x);
            v[u].x = fma(-t.y, xv.y, v[u].x);
            v[u].y = fma(t.x, xv.y, v[u].y);
            v[u].y = fma(t.y, xv.x, v[u].y);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int i = base + rl + 64 * u;
        if (i < n) Sj[i] = v[u];
      }
    }
  }
  __syncthreads();
}

// The blocked Gauss-Jordan sweep over the matrix S of this cluster.
__device__ bool gj_blocked(const Shared &s, double2 *S, int *meta, int rank) {
  const int n = s.n, cw = s.cw, c0 = rank * cw;
  const int ncols = max(0, min(cw, n - c0));
  const int np = npanels(n);
  bool zero = false;
  // prologue: the owner of panel 0 eliminates it
  if (0 >= c0 && 0 < c0 + ncols) zero |= eliminate_panel(s, S, meta, 0, min(KB, n));
  __threadfence();
  cluster_arrive();
  cluster_wait();
  for (int p = 0; p < np; p++) {
    const int k0 = p * KB, kbp = min(KB, n - k0);
    for (int e = threadIdx.x; e < kbp * n; e += blockDim.x) {
      const int q = e / n, i = e % n;
      s.T[q * n + i] = S[(size_t)(k0 + q) * n + i];
    }
    for (int t = threadIdx.x; t < kMoveInts; t += blockDim.x) s.mv[t] = meta[n + p * kMoveInts + t];
    __syncthreads();
    const int kn0 = (p + 1) * KB, kbn = (p + 1 < np) ? min(KB, n - kn0) : 0;
    const bool next_mine = (kbn > 0) && kn0 >= c0 && kn0 < c0 + ncols;
    if (next_mine) {
      // the next panel's columns first, then eliminate it and publish
      apply_panel(s, S, c0, kn0 - c0, kn0 - c0 + kbn, k0, k0 + kbp, 0, 0, k0, kbp);
      zero |= eliminate_panel(s, S, meta, kn0, kbn);
      __threadfence();
      cluster_arrive();
      apply_panel(s, S, c0, 0, ncols, k0, k0 + kbp, kn0, kn0 + kbn, k0, kbp);
      cluster_wait();
    } else {
      apply_panel(s, S, c0, 0, ncols, k0, k0 + kbp, 0, 0, k0, kbp);
      cluster_arrive();
      cluster_wait();
    }
  }
  // pivot rows for the final column permutation
  for (int t = threadIdx.x; t < n; t += blockDim.x) s.perm[t] = meta[t];
  __syncthreads();
  return zero;
}

// Destination column of column j of the in-place result: the row swaps
// (k, perm[k]) become column swaps applied in reverse step order.
__device__ __forceinline__ int dest_col(const int *perm, int n, int j) {
  int loc = j;
  for (int k = n - 1; k >= 0; k--) {
    const int pk = perm[k];
    if (loc == k)
      loc = pk;
    else if (loc == pk)
      loc = k;
  }
  return loc;
}

__device__ __forceinline__ void record_status(unsigned int *status, unsigned int code, int level,
                                              int box) {
  unsigned int w = (code << 28) | ((unsigned)(level & 0xff) << 20) | ((unsigned)box & 0xfffffu);
  atomicCAS(status, 0u, w);
}

struct LeafArgs {
  LeafTables lt;
  const double *tab;  // D1x, D1y, D2x, D2y (p*p each), then int grid[n]
  const double *c;    // [leaves][ni]
  double2 *X;         // [leaf][n][n] column-major
  double2 *GX;        // [leaf][n][nb] column-major
  double2 *S;         // [chunk][n][n] scratch
  int *meta;          // [chunk][meta_ints(n)]
  int leaf0;          // first leaf of this chunk
  unsigned int *status;
  int level;
  int cw;
};

__global__ void __launch_bounds__(kThreads, 2) leaf_kernel(const __grid_constant__ LeafArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int slot = blockIdx.x / cs;
  const int leaf = a.leaf0 + slot;
  const int p = a.lt.p, e = a.lt.e, n = a.lt.n, nb = a.lt.nb, ni = a.lt.ni;
  const int cw = a.cw, c0 = rank * cw;
  const int ncols = max(0, min(cw, n - c0));
  const SmemPlan sp = plan_smem(n, cw, true, p);
  const Shared s = bind(smem, sp, n, cw);
  double *D1x = (double *)(smem + sp.dtab);
  double *D1y = D1x + p * p, *D2x = D1y + p * p, *D2y = D2x + p * p;
  int *grid = (int *)(smem + sp.grid);
  int *loc = (int *)(smem + sp.loc);
  double *cv = (double *)(smem + sp.cv);
  const int tid = threadIdx.x, nthr = blockDim.x;
  double2 *S = a.S + (size_t)slot * n * n;
  int *meta = a.meta + (size_t)slot * meta_ints(n);

  for (int i = tid; i < 4 * p * p; i += nthr) D1x[i] = a.tab[i];
  const int *gsrc = (const int *)(a.tab + 4 * p * p);
  for (int i = tid; i < n; i += nthr) grid[i] = gsrc[i];
  for (int i = tid; i < p * p; i += nthr) loc[i] = -1;
  for (int i = tid; i < ni; i += nthr) cv[i] = a.c[(size_t)leaf * ni + i];
  __syncthreads();
  for (int i = tid; i < n; i += nthr) loc[(grid[i] >> 8) * p + (grid[i] & 0xff)] = i;
  __syncthreads();

  // assemble the own columns of B
  const double2 eta = a.lt.eta;
  for (int idx = tid; idx < n * ncols; idx += nthr) {
    const int i = idx % n, jj = idx / n, j = c0 + jj;
    const int ix = grid[i] & 0xff, iy = grid[i] >> 8;
    const int jx = grid[j] & 0xff, jy = grid[j] >> 8;
    double2 v = make_double2(0.0, 0.0);
    if (i < nb) {
      const int side = i / e;
      if (side == 0) {
        if (jx == ix) v.x = -D1y[0 * p + jy];  // south: -d/dy
      } else if (side == 1) {
        if (jy == iy) v.x = D1x[(p - 1) * p + jx];  // east: +d/dx
      } else if (side == 2) {
        if (jx == ix) v.x = D1y[(p - 1) * p + jy];  // north: +d/dy
      } else {
        if (jy == iy) v.x = -D1x[0 * p + jx];  // west: -d/dx
      }
      if (i == j) {  // + i eta
        v.x -= eta.y;
        v.y += eta.x;
      }
    } else {
      if (jy == iy) v.x -= D2x[ix * p + jx];
      if (jx == ix) v.x -= D2y[iy * p + jy];
      if (i == j) v.x -= a.lt.kappa2 * cv[i - nb];
    }
    S[(size_t)j * n + i] = v;
  }
  __syncthreads();

  const bool zero = gj_blocked(s, S, meta, rank);
  if (zero && tid == 0) record_status(a.status, 1u, a.level, leaf);

  // X = B^{-1}: own columns to their destination columns
  double2 *Xl = a.X + (size_t)leaf * n * n;
  for (int idx = tid; idx < n * ncols; idx += nthr) {
    const int i = idx % n, jj = idx / n, j = c0 + jj;
    Xl[(size_t)dest_col(s.perm, n, j) * n + i] = S[(size_t)j * n + i];
  }
  // G X for the own columns: row r of G is the outward normal derivative
  // along the line through boundary node r, minus i eta at r itself
  double2 *GXl = a.GX + (size_t)leaf * n * nb;
  for (int idx = tid; idx < nb * ncols; idx += nthr) {
    const int r = idx % nb, jj = idx / nb, j = c0 + jj;
    const double2 *Sj = S + (size_t)j * n;
    const int side = r / e;
    const int ix = grid[r] & 0xff, iy = grid[r] >> 8;
    double2 acc = make_double2(0.0, 0.0);
    for (int t = 0; t < p; t++) {
      double w;
      int q;
      if (side == 0) {
        w = -D1y[0 * p + t];
        q = loc[t * p + ix];
      } else if (side == 1) {
        w = D1x[(p - 1) * p + t];
        q = loc[iy * p + t];
      } else if (side == 2) {
        w = D1y[(p - 1) * p + t];
        q = loc[t * p + ix];
      } else {
        w = -D1x[0 * p + t];
        q = loc[iy * p + t];
      }
      double2 x = Sj[q];
      acc.x = fma(w, x.x, acc.x);
      acc.y = fma(w, x.y, acc.y);
    }
    double2 ie = cmul(make_double2(-eta.y, eta.x), Sj[r]);  // - i eta x_r
    acc.x -= ie.x;
    acc.y -= ie.y;
    GXl[(size_t)dest_col(s.perm, n, j) * nb + r] = acc;
  }
}

struct GJArgs {
  double2 *S;     // [batch][n][n] column-major input, destroyed
  double2 *out;   // [batch][n][n] column-major inverse
  int *meta;      // [batch][meta_ints(n)]
  int n;
  int cw;
  unsigned int *status;
  int level;
};

__global__ void __launch_bounds__(kThreads, 2) gj_kernel(const __grid_constant__ GJArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int mat = blockIdx.x / cs;
  const int n = a.n, cw = a.cw, c0 = rank * cw;
  const int ncols = max(0, min(cw, n - c0));
  const SmemPlan sp = plan_smem(n, cw, false, 0);
  const Shared s = bind(smem, sp, n, cw);
  double2 *S = a.S + (size_t)mat * n * n;
  int *meta = a.meta + (size_t)mat * meta_ints(n);
  const bool zero = gj_blocked(s, S, meta, rank);
  if (zero && threadIdx.x == 0) record_status(a.status, 2u, a.level, mat);
  double2 *O = a.out + (size_t)mat * n * n;
  for (int idx = threadIdx.x; idx < n * ncols; idx += blockDim.x) {
    const int i = idx % n, jj = idx / n, j = c0 + jj;
    O[(size_t)dest_col(s.perm, n, j) * n + i] = S[(size_t)j * n + i];
  }
}

template <typename Kern, typename Args>
cudaError_t launch_cluster(Kern kern, const Args &args, int blocks, int cs, size_t smem,
                           cudaStream_t st) {
  cudaError_t err;
  if (cs > 8) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (err != cudaSuccess) return err;
  }
  err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks * cs, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args);
}

}  // namespace

int gj_max_cluster() { return 16; }

int gj_slab(int n, int cs) {
  int cw = (n + cs - 1) / cs;
  return ((cw + KB - 1) / KB) * KB;
}

size_t gj_smem_bytes(int n, int cs, bool leaf, int p) {
  return plan_smem(n, gj_slab(n, cs), leaf, p).total;
}

size_t gj_meta_ints(int n) { return (size_t)meta_ints(n); }

cudaError_t launch_leaf(const LeafTables &lt, const void *tab_dev, const double *c, int leaf0,
                        int count, double2 *X, double2 *GX, double2 *S, int *meta,
                        unsigned int *status, int level, int cs, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  LeafArgs a;
  a.lt = lt;
  a.tab = (const double *)tab_dev;
  a.c = c;
  a.X = X;
  a.GX = GX;
  a.S = S;
  a.meta = meta;
  a.leaf0 = leaf0;
  a.status = status;
  a.level = level;
  a.cw = gj_slab(lt.n, cs);
  size_t smem = plan_smem(lt.n, a.cw, true, lt.p).total;
  return launch_cluster(leaf_kernel, a, count, cs, smem, st);
}

cudaError_t launch_gj_inverse(double2 *S, double2 *out, int n, int batch, int *meta,
                              unsigned int *status, int level, int cs, cudaStream_t st) {
  if (batch <= 0 || n <= 0) return cudaSuccess;
  GJArgs a;
  a.S = S;
  a.out = out;
  a.meta = meta;
  a.n = n;
  a.cw = gj_slab(n, cs);
  a.status = status;
  a.level = level;
  size_t smem = plan_smem(n, a.cw, false, 0).total;
  return launch_cluster(gj_kernel, a, batch, cs, smem, st);
}

}  // namespace hps
