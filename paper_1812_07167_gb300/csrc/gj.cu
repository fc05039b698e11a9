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

#include <algorithm>

#include "cx.cuh"
#include "hps_internal.h"
#include "leaf_geom.cuh"

namespace cg = cooperative_groups;

namespace hps {

namespace {

constexpr int kThreads = 256;
// The panel width KB is a template parameter: 8 where the elimination is
// FP64-throughput-bound (the leaf, levels with many matrices), 4 where the
// serial panel chain is the critical path (few, large interface matrices:
// half the FP64 work a panel on the owning CTA, twice the barriers).  A
// panel's swaps make at most 2 KB row moves, listed in 1 + 2 (2 KB) ints.
template <int KB>
struct Pn {
  static constexpr int kMoves = 2 * KB;
  static constexpr int kMoveInts = 1 + 2 * kMoves;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
template <int KB>
__host__ __device__ inline int npanels(int n) { return (n + KB - 1) / KB; }
// ints of per-matrix bookkeeping: pivot rows, then the row moves of each panel
template <int KB>
__host__ __device__ inline int meta_ints(int n) { return n + npanels<KB>(n) * Pn<KB>::kMoveInts; }

struct SmemPlan {
  size_t T, F, x, mvbuf, col, prow, krow, red, mv, rows, srcs, scal, pinv, perm, dcol, dtab, grid, loc, cv, rsc,
      total;
};

// Panel placement: 0 = the panel being applied (T) and the one being
// eliminated (F) both in shared memory, 1 = both read in place from the
// global scratch, 2 = T in place and F in shared memory.
template <int KB>
__host__ __device__ inline SmemPlan plan_smem(int n, int cw, bool leaf, int p, int tmode = 0,
                                               size_t esz = 16) {
  constexpr int kMoves = Pn<KB>::kMoves, kMoveInts = Pn<KB>::kMoveInts;
  SmemPlan s;
  size_t o = 0;
  s.T = o;    if (tmode == 0) o = align16(o + esz * (size_t)KB * n);
  s.F = o;    if (tmode != 1) o = align16(o + esz * (size_t)KB * n);
  s.x = o;    o = align16(o + esz * (size_t)KB * cw);
  s.mvbuf = o; o = align16(o + esz * (size_t)kMoves * cw);
  s.col = o;  o = align16(o + esz * (size_t)n);
  s.prow = o; o = align16(o + esz * KB);
  s.krow = o; o = align16(o + esz * KB);
  s.red = o;  o = align16(o + 16 * (kThreads / 32));
  s.mv = o;   o = align16(o + sizeof(int) * kMoveInts);
  s.rows = o; o = align16(o + sizeof(int) * 2 * KB);
  s.srcs = o; o = align16(o + sizeof(int) * 2 * KB);
  s.scal = o; o = align16(o + sizeof(int) * 4);
  s.pinv = o; o = align16(o + esz);
  s.perm = o; o = align16(o + sizeof(int) * (size_t)n);
  s.dcol = o; o = align16(o + sizeof(int) * (size_t)cw);
  if (leaf) {
    int ni = (p - 2) * (p - 2);
    s.dtab = o; o = align16(o + sizeof(double) * 4 * (size_t)p * p);
    s.grid = o; o = align16(o + sizeof(int) * (size_t)n);
    s.loc = o;  o = align16(o + sizeof(int) * (size_t)p * p);
    s.cv = o;   o = align16(o + sizeof(double) * (size_t)ni);
    s.rsc = o;  o = align16(o + sizeof(double) * (size_t)n);
  } else {
    s.dtab = s.grid = s.loc = s.cv = s.rsc = o;
  }
  s.total = o;
  return s;
}

template <class C>
struct Shared {
  C *T;     // [KB][n] panel being applied (column-major), or null: read in place
  C *F;     // [KB][n] panel being eliminated (owner only), or null: in place
  C *x;     // [KB][cw] panel rows of the own columns, after the moves
  C *mvbuf; // [cw][kMoves] values in flight during the row moves
  C *col;   // [n] pivot column of the current elimination step
  C *prow;  // [KB] scaled pivot row within the panel
  C *krow;  // [KB] row k of the panel before the step's swap
  unsigned long long *rkey;  // [warps] pivot search: best key of each warp
  int *ridx;                 // [warps] and its row
  int *mv;        // [kMoveInts] row moves of the panel being applied
  int *rows;      // [2 KB] scratch for building a move list
  int *srcs;      // [2 KB]
  int *scal;      // [4] pivot row, zero flag
  C *pinv;  // [1] reciprocal of the pivot
  int *perm;      // [n] pivot rows, for the final column permutation
  int *dcol;      // [cw] destination column of each own column
  int n, cw;
};

template <class C>
__device__ Shared<C> bind(unsigned char *smem, const SmemPlan &sp, int n, int cw) {
  Shared<C> s;
  s.T = (sp.F > sp.T) ? (C *)(smem + sp.T) : nullptr;
  s.F = (sp.x > sp.F) ? (C *)(smem + sp.F) : nullptr;
  s.x = (C *)(smem + sp.x);
  s.mvbuf = (C *)(smem + sp.mvbuf);
  s.col = (C *)(smem + sp.col);
  s.prow = (C *)(smem + sp.prow);
  s.krow = (C *)(smem + sp.krow);
  s.rkey = (unsigned long long *)(smem + sp.red);
  s.ridx = (int *)(smem + sp.red + 8 * (kThreads / 32));
  s.mv = (int *)(smem + sp.mv);
  s.rows = (int *)(smem + sp.rows);
  s.srcs = (int *)(smem + sp.srcs);
  s.scal = (int *)(smem + sp.scal);
  s.pinv = (C *)(smem + sp.pinv);
  s.perm = (int *)(smem + sp.perm);
  s.dcol = (int *)(smem + sp.dcol);
  s.n = n;
  s.cw = cw;
  return s;
}

// Eliminate panel [k0, k0 + kbp) of S (column-major, ld n) in shared memory
// and write it back; record its pivot rows and row moves in `meta`.
// Returns true if a zero pivot was met.  For short columns one warp finds
// each pivot; with kLong (long columns) every warp searches a share of the
// rows and the pivot row is staged beside the pivot column (four barriers
// a step either way).
template <class C, int KB, bool kLong = false>
__device__ bool eliminate_panel(const Shared<C> &s, C *S, int *meta, int k0, int kbp) {
  constexpr int kMoveInts = Pn<KB>::kMoveInts;
  const int tid = threadIdx.x, nthr = blockDim.x, n = s.n;
  bool zero = false;
  // work on a shared-memory copy of the panel, or in place in S when the
  // panel does not fit next to the other buffers
  C *F = s.F ? s.F : S + (size_t)k0 * n;
  if (s.F)
    for (int q = 0; q < kbp; q++)
      for (int i = tid; i < n; i += nthr) F[q * n + i] = S[(size_t)(k0 + q) * n + i];
  __syncthreads();
  if (!kLong) {
    for (int q = 0; q < kbp; q++) {
      const int k = k0 + q;
      const C *Fk = F + q * n;
      if (tid < 32) {
        unsigned long long best = 0;
        int bi = n;
        for (int i = k + tid; i < n; i += 32) {
          unsigned long long key = CX<C>::key(Fk[i]);
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
          const C pv = Fk[r];
          const bool z = (CX<C>::key(pv) == 0ull);
          s.scal[0] = r;
          s.scal[1] = z ? 1 : 0;
          s.pinv[0] = z ? CX<C>::make(0.0, 0.0) : crecip(pv);
          meta[k] = r;
        }
      }
      __syncthreads();
      const int r = s.scal[0];
      if (s.scal[1]) zero = true;
      const C pinv = s.pinv[0];
      // swap rows k and r inside the panel
      if (r != k)
        for (int qq = tid; qq < kbp; qq += nthr) {
          C t = F[qq * n + k];
          F[qq * n + k] = F[qq * n + r];
          F[qq * n + r] = t;
        }
      __syncthreads();
      // pivot column with its pivot entry zeroed, and the scaled pivot row
      for (int i = tid; i < n; i += nthr) s.col[i] = (i == k) ? CX<C>::make(0.0, 0.0) : Fk[i];
      for (int qq = tid; qq < kbp; qq += nthr) s.prow[qq] = cmul(F[qq * n + k], pinv);
      __syncthreads();
      for (int e = tid; e < kbp * n; e += nthr) {
        const int qq = e / n, i = e % n;
        C *a = &F[qq * n + i];
        if (qq == q) {
          // the eliminated column becomes -col / pivot, 1 / pivot at the pivot
          if (i == k) {
            *a = pinv;
          } else {
            C f = cmul(s.col[i], pinv);
            *a = CX<C>::make(-f.x, -f.y);
          }
        } else if (i == k) {
          *a = s.prow[qq];
        } else {
          C f = s.col[i], pr = s.prow[qq], v = *a;
          v.x = CX<C>::fmad(-f.x, pr.x, v.x);
          v.x = CX<C>::fmad(f.y, pr.y, v.x);
          v.y = CX<C>::fmad(-f.x, pr.y, v.y);
          v.y = CX<C>::fmad(-f.y, pr.x, v.y);
          *a = v;
        }
      }
      __syncthreads();
    }
  } else {
    const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
    for (int q = 0; q < kbp; q++) {
      const int k = k0 + q;
      C *Fk = F + q * n;
      // pivot: largest max(|Re|, |Im|) at or below row k, lowest row on ties
      unsigned long long best = 0;
      int bi = n;
      for (int i = k + tid; i < n; i += nthr) {
        const unsigned long long key = CX<C>::key(Fk[i]);
        if (bi == n || key > best) {
          best = key;
          bi = i;
        }
      }
      for (int off = 16; off; off >>= 1) {
        const unsigned long long ov = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (oi < n && (bi == n || ov > best || (ov == best && oi < bi))) {
          best = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        s.rkey[wid] = best;
        s.ridx[wid] = bi;
      }
      __syncthreads();
      best = 0;
      bi = n;
      for (int w = 0; w < nw; w++) {
        const unsigned long long ov = s.rkey[w];
        const int oi = s.ridx[w];
        if (oi < n && (bi == n || ov > best || (ov == best && oi < bi))) {
          best = ov;
          bi = oi;
        }
      }
      const int r = (bi < n) ? bi : k;
      const C pv = Fk[r];
      const bool zpiv = CX<C>::key(pv) == 0ull;
      if (zpiv) zero = true;
      if (tid == 0) {
        meta[k] = r;
        s.pinv[0] = zpiv ? CX<C>::make(0.0, 0.0) : crecip(pv);
      }
      __syncthreads();
      const C pinv = s.pinv[0];
      // the pivot column after the swap of rows k and r (zero at k), the
      // scaled pivot row (old row r) and old row k
      for (int i = tid; i < n; i += nthr) s.col[i] = (i == k) ? CX<C>::make(0.0, 0.0) : Fk[i == r ? k : i];
      if (tid < kbp) {
        s.prow[tid] = cmul(F[tid * n + r], pinv);
        s.krow[tid] = F[tid * n + k];
      }
      __syncthreads();
      for (int qq = 0; qq < kbp; qq++) {
        C *Fq = F + qq * n;
        const C pr = s.prow[qq], kr = s.krow[qq];
        for (int i = tid; i < n; i += nthr) {
          C v;
          if (qq == q) {
            // the eliminated column becomes -col / pivot, 1 / pivot at the pivot
            if (i == k) {
              v = pinv;
            } else {
              const C f = cmul(s.col[i], pinv);
              v = CX<C>::make(-f.x, -f.y);
            }
          } else if (i == k) {
            v = pr;
          } else {
            const C f = s.col[i];
            v = (i == r) ? kr : Fq[i];
            v.x = CX<C>::fmad(-f.x, pr.x, v.x);
            v.x = CX<C>::fmad(f.y, pr.y, v.x);
            v.y = CX<C>::fmad(-f.x, pr.y, v.y);
            v.y = CX<C>::fmad(-f.y, pr.x, v.y);
          }
          Fq[i] = v;
        }
      }
      __syncthreads();
    }
  }
  if (s.F)
    for (int q = 0; q < kbp; q++)
      for (int i = tid; i < n; i += nthr) S[(size_t)(k0 + q) * n + i] = F[q * n + i];
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
// CU columns go through the update together (more loads in flight; the
// panel values are read once for all of them): 4 for complex64, whose
// update is short and latency-bound, 1 for complex128.
template <class C, int KB, int CU = (sizeof(C) == 8 ? 4 : 1)>
__device__ void apply_panel(const Shared<C> &s, const C *T, C *S, int c0, int ja, int jb,
                            int a0, int a1, int b0, int b1, int k0, int kbp) {
  constexpr int kMoves = Pn<KB>::kMoves;
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
  if (CU == 1) {
    const int cl = tid >> 6, rl = tid & 63;
    for (int jj = ja + cl; jj < jb; jj += (nthr >> 6)) {
      const int j = c0 + jj;
      if (skipped(j, a0, a1, b0, b1)) continue;
      C *Sj = S + (size_t)j * n;
      for (int base = 0; base < n; base += 256) {
        C v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int i = base + rl + 64 * u;
          v[u] = (i < n && (i < k0 || i >= k0 + kbp)) ? Sj[i] : CX<C>::make(0.0, 0.0);
        }
        for (int q = 0; q < kbp; q++) {
          const C xv = s.x[q * cw + jj];
          const C *Tq = T + q * n + base + rl;
#pragma unroll
          for (int u = 0; u < 4; u++) {
            if (base + rl + 64 * u < n) {
              const C t = Tq[64 * u];
              v[u].x = CX<C>::fmad(t.x, xv.x, v[u].x);
              v[u].x = CX<C>::fmad(-t.y, xv.y, v[u].x);
              v[u].y = CX<C>::fmad(t.x, xv.y, v[u].y);
              v[u].y = CX<C>::fmad(t.y, xv.x, v[u].y);
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
  } else {
    const int cl = tid >> 6, rl = tid & 63, lanes = nthr >> 6;
    for (int j0 = cl; j0 < nj; j0 += lanes * CU) {
      int jjs[CU];
      bool ok[CU];
#pragma unroll
      for (int u = 0; u < CU; u++) {
        jjs[u] = ja + j0 + lanes * u;
        ok[u] = (j0 + lanes * u < nj) && !skipped(c0 + jjs[u], a0, a1, b0, b1);
      }
      for (int base = 0; base < n; base += 256) {
        C v[CU][4];
#pragma unroll
        for (int u = 0; u < CU; u++)
#pragma unroll
          for (int r = 0; r < 4; r++) {
            const int i = base + rl + 64 * r;
            v[u][r] = (ok[u] && i < n && (i < k0 || i >= k0 + kbp)) ? S[(size_t)(c0 + jjs[u]) * n + i]
                                                                   : CX<C>::make(0.0, 0.0);
          }
        for (int q = 0; q < kbp; q++) {
          const C *Tq = T + q * n + base + rl;
          C t[4];
#pragma unroll
          for (int r = 0; r < 4; r++) t[r] = (base + rl + 64 * r < n) ? Tq[64 * r] : CX<C>::make(0.0, 0.0);
#pragma unroll
          for (int u = 0; u < CU; u++) {
            const C xv = ok[u] ? s.x[q * cw + jjs[u]] : CX<C>::make(0.0, 0.0);
#pragma unroll
            for (int r = 0; r < 4; r++) {
              v[u][r].x = CX<C>::fmad(t[r].x, xv.x, v[u][r].x);
              v[u][r].x = CX<C>::fmad(-t[r].y, xv.y, v[u][r].x);
              v[u][r].y = CX<C>::fmad(t[r].x, xv.y, v[u][r].y);
              v[u][r].y = CX<C>::fmad(t[r].y, xv.x, v[u][r].y);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < CU; u++)
#pragma unroll
          for (int r = 0; r < 4; r++) {
            const int i = base + rl + 64 * r;
            if (ok[u] && i < n) S[(size_t)(c0 + jjs[u]) * n + i] = v[u][r];
          }
      }
    }
  }
  __syncthreads();
}

// The blocked Gauss-Jordan sweep over the matrix S of this cluster.
template <class C, int KB>
__device__ bool gj_blocked(const Shared<C> &s, C *S, int *meta, int rank) {
  constexpr int kMoveInts = Pn<KB>::kMoveInts;
  const int n = s.n, cw = s.cw, c0 = rank * cw;
  const int ncols = max(0, min(cw, n - c0));
  const int np = npanels<KB>(n);
  bool zero = false;
  // prologue: the owner of panel 0 eliminates it
  if (0 >= c0 && 0 < c0 + ncols) zero |= eliminate_panel<C, KB>(s, S, meta, 0, min(KB, n));
  __threadfence();
  cluster_arrive();
  cluster_wait();
  for (int p = 0; p < np; p++) {
    const int k0 = p * KB, kbp = min(KB, n - k0);
    const C *T = s.T ? s.T : S + (size_t)k0 * n;
    if (s.T)
      for (int q = 0; q < kbp; q++)
        for (int i = threadIdx.x; i < n; i += blockDim.x) s.T[q * n + i] = S[(size_t)(k0 + q) * n + i];
    for (int t = threadIdx.x; t < kMoveInts; t += blockDim.x) s.mv[t] = meta[n + p * kMoveInts + t];
    __syncthreads();
    const int kn0 = (p + 1) * KB, kbn = (p + 1 < np) ? min(KB, n - kn0) : 0;
    const bool next_mine = (kbn > 0) && kn0 >= c0 && kn0 < c0 + ncols;
    if (next_mine) {
      // the next panel's columns first, then eliminate it and publish
      apply_panel<C, KB>(s, T, S, c0, kn0 - c0, kn0 - c0 + kbn, k0, k0 + kbp, 0, 0, k0, kbp);
      zero |= eliminate_panel<C, KB>(s, S, meta, kn0, kbn);
      __threadfence();
      cluster_arrive();
      apply_panel<C, KB>(s, T, S, c0, 0, ncols, k0, k0 + kbp, kn0, kn0 + kbn, k0, kbp);
      cluster_wait();
    } else {
      apply_panel<C, KB>(s, T, S, c0, 0, ncols, k0, k0 + kbp, 0, 0, k0, kbp);
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

// s.dcol[jj] = destination of column c0 + jj, jj < ncols (s.perm filled);
// one O(n) walk a column instead of one an element.
template <class C>
__device__ void fill_dcol(const Shared<C> &s, int c0, int ncols) {
  for (int jj = threadIdx.x; jj < ncols; jj += blockDim.x) s.dcol[jj] = dest_col(s.perm, s.n, c0 + jj);
  __syncthreads();
}

constexpr int kLeafKB = 8;  // the leaf elimination is FP64-throughput-bound

struct LeafArgs {
  LeafTables lt;
  const LeafProb *probs;  // per-problem tables, c, kappa^2, eta (device)
  int nprob;
  void *X;            // [leaf][n][n] column-major (element type C)
  void *GX;           // [leaf][n][nb] column-major
  void *S;            // [chunk][n][n] scratch
  int *meta;          // [chunk][meta_ints(n)]
  long long leaf0;    // first leaf of this chunk
  unsigned int *status;
  int level;
  int cw;
};

template <class C>
__global__ void __launch_bounds__(kThreads, 2) leaf_kernel(const __grid_constant__ LeafArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  using R = typename CX<C>::R;
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int slot = blockIdx.x / cs;
  const long long leaf = a.leaf0 + slot;
  // the problem this leaf belongs to: the last one starting at or before it
  int pk = 0;
  for (int lo = 0, hi = a.nprob - 1; lo <= hi;) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(&a.probs[mid].leaf0) <= leaf) {
      pk = mid;
      lo = mid + 1;
    } else {
      hi = mid - 1;
    }
  }
  const LeafProb &pb = a.probs[pk];
  const double *tab = pb.tab;
  const double kappa2 = pb.kappa2;
  const double2 eta = pb.eta;
  const double *cleaf = pb.c + (size_t)(leaf - pb.leaf0) * a.lt.ni;
  const int p = a.lt.p, e = a.lt.e, n = a.lt.n, nb = a.lt.nb, ni = a.lt.ni;
  const int cw = a.cw, c0 = rank * cw;
  const int ncols = max(0, min(cw, n - c0));
  const SmemPlan sp = plan_smem<kLeafKB>(n, cw, true, p, false, sizeof(C));
  const Shared<C> s = bind<C>(smem, sp, n, cw);
  double *D1x = (double *)(smem + sp.dtab);
  double *D1y = D1x + p * p, *D2x = D1y + p * p, *D2y = D2x + p * p;
  int *grid = (int *)(smem + sp.grid);
  int *loc = (int *)(smem + sp.loc);
  double *cv = (double *)(smem + sp.cv);
  const int tid = threadIdx.x, nthr = blockDim.x;
  C *S = (C *)a.S + (size_t)slot * n * n;
  int *meta = a.meta + (size_t)slot * meta_ints<kLeafKB>(n);

  for (int i = tid; i < 4 * p * p; i += nthr) D1x[i] = tab[i];
  const int *gsrc = (const int *)(tab + 4 * p * p);
  for (int i = tid; i < n; i += nthr) grid[i] = gsrc[i];
  for (int i = tid; i < p * p; i += nthr) loc[i] = -1;
  for (int i = tid; i < ni; i += nthr) cv[i] = cleaf[i];
  __syncthreads();
  for (int i = tid; i < n; i += nthr) loc[(grid[i] >> 8) * p + (grid[i] & 0xff)] = i;
  __syncthreads();

  LeafGeom geo;
  geo.D1x = D1x;
  geo.D1y = D1y;
  geo.D2x = D2x;
  geo.D2y = D2y;
  geo.grid = grid;
  geo.cv = cv;
  geo.p = p;
  geo.e = e;
  geo.nb = nb;
  geo.kappa2 = kappa2;
  geo.eta = eta;
  // Row equilibration: row i of B is scaled by an exact power of two d_i;
  // the elimination inverts D B and X = (D B)^{-1} D, i.e. column j of the
  // result is scaled by d_j.
  double *rsc = (double *)(smem + sp.rsc);
  for (int i = tid; i < n; i += nthr) rsc[i] = leaf_row_scale(geo, i);
  __syncthreads();

  // assemble the own columns of D B (entries computed in FP64, stored as C)
  for (int idx = tid; idx < n * ncols; idx += nthr) {
    const int i = idx % n, jj = idx / n, j = c0 + jj;
    const double2 v = leaf_B(geo, i, j);
    S[(size_t)j * n + i] = CX<C>::make(rsc[i] * v.x, rsc[i] * v.y);
  }
  __syncthreads();

  const bool zero = gj_blocked<C, kLeafKB>(s, S, meta, rank);
  if (zero && tid == 0) record_status(a.status, 1u, a.level, (int)leaf);
  fill_dcol(s, c0, ncols);

  // X = (D B)^{-1} D: own columns to their destination columns, scaled
  C *Xl = (C *)a.X + (size_t)leaf * n * n;
  for (int idx = tid; idx < n * ncols; idx += nthr) {
    const int i = idx % n, jj = idx / n, j = c0 + jj;
    const int dc = s.dcol[jj];
    const R d = (R)rsc[dc];
    const C v = S[(size_t)j * n + i];
    Xl[(size_t)dc * n + i] = CX<C>::make(d * v.x, d * v.y);
  }
  // G X for the own columns: row r of G is the outward normal derivative
  // along the line through boundary node r, minus i eta at r itself
  C *GXl = (C *)a.GX + (size_t)leaf * n * nb;
  const C ieta = CX<C>::make(-eta.y, eta.x);
  for (int idx = tid; idx < nb * ncols; idx += nthr) {
    const int r = idx % nb, jj = idx / nb, j = c0 + jj;
    const C *Sj = S + (size_t)j * n;
    const int side = r / e;
    const int ix = grid[r] & 0xff, iy = grid[r] >> 8;
    C acc = CX<C>::make(0.0, 0.0);
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
      const C x = Sj[q];
      acc.x = CX<C>::fmad((R)w, x.x, acc.x);
      acc.y = CX<C>::fmad((R)w, x.y, acc.y);
    }
    const C ie = cmul(ieta, Sj[r]);  // - i eta x_r
    acc.x -= ie.x;
    acc.y -= ie.y;
    const int dc = s.dcol[jj];
    const R d = (R)rsc[dc];
    GXl[(size_t)dc * nb + r] = CX<C>::make(d * acc.x, d * acc.y);
  }
}

struct GJArgs {
  int tglobal;    // panel placement (plan_smem's tmode): 0 shared memory, 1 in place
  void *S;        // [batch][n][n] column-major input, destroyed (element type C)
  void *out;      // [batch][n][n] column-major inverse
  int *meta;      // [batch][meta_ints(n)]
  int n;
  int cw;
  unsigned int *status;
  int level;
};

template <class C, int KB>
__global__ void __launch_bounds__(kThreads, 2) gj_kernel(const __grid_constant__ GJArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int mat = blockIdx.x / cs;
  const int n = a.n, cw = a.cw, c0 = rank * cw;
  const int ncols = max(0, min(cw, n - c0));
  const SmemPlan sp = plan_smem<KB>(n, cw, false, 0, a.tglobal, sizeof(C));
  const Shared<C> s = bind<C>(smem, sp, n, cw);
  C *S = (C *)a.S + (size_t)mat * n * n;
  int *meta = a.meta + (size_t)mat * meta_ints<KB>(n);
  const bool zero = gj_blocked<C, KB>(s, S, meta, rank);
  if (zero && threadIdx.x == 0) record_status(a.status, 2u, a.level, mat);
  fill_dcol(s, c0, ncols);
  C *O = (C *)a.out + (size_t)mat * n * n;
  for (int idx = threadIdx.x; idx < n * ncols; idx += blockDim.x) {
    const int i = idx % n, jj = idx / n, j = c0 + jj;
    O[(size_t)s.dcol[jj] * n + i] = S[(size_t)j * n + i];
  }
}

// ---- wide variant: one launch per panel, a matrix spread over G CTAs ----
// For levels with few matrices (the top of the tree) a cluster's 16 SMs at
// most are too few.  Here every panel round is its own launch over the whole
// chip: CTA 0 of each matrix applies panel p to the columns of panel p+1 and
// eliminates that panel (the look-ahead of the cluster kernel); CTAs 1..G-1
// apply panel p to their slabs of the remaining columns.  Launch order on the
// stream is the barrier between rounds.  Phase -1 eliminates panel 0 only;
// phase np writes the inverse out with the column permutation.
struct WideArgs {
  int tglobal;  // panel placement (plan_smem's tmode)
  void *S;      // [batch][n][n] column-major input, destroyed
  void *out;    // [batch][n][n] column-major inverse
  int *meta;    // [batch][meta_ints(n)]
  int n, G, slab;
  unsigned int *status;
  int level;
};

template <class C, int KB>
__global__ void __launch_bounds__(kThreads, 2) gj_wide_kernel(const __grid_constant__ WideArgs a, int phase) {
  constexpr int kMoveInts = Pn<KB>::kMoveInts;
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, G = a.G;
  const int mat = blockIdx.x / G, g = blockIdx.x % G;
  const int cwmax = a.slab > KB ? a.slab : KB;
  const SmemPlan sp = plan_smem<KB>(n, cwmax, false, 0, a.tglobal, sizeof(C));
  const Shared<C> s = bind<C>(smem, sp, n, cwmax);
  C *S = (C *)a.S + (size_t)mat * n * n;
  int *meta = a.meta + (size_t)mat * meta_ints<KB>(n);
  const int np = npanels<KB>(n);
  // slab of CTA g >= 1: columns [c0, c0 + slab) of the matrix
  const int c0 = (g - 1) * a.slab;
  const int nc = (g >= 1) ? max(0, min(a.slab, n - c0)) : 0;
  if (phase < 0) {
    if (g == 0) {
      const bool z = (n > 512) ? eliminate_panel<C, KB, true>(s, S, meta, 0, min(KB, n))
                               : eliminate_panel<C, KB, false>(s, S, meta, 0, min(KB, n));
      if (z && threadIdx.x == 0) record_status(a.status, 2u, a.level, mat);
    }
    return;
  }
  if (phase >= np) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) s.perm[t] = meta[t];
    __syncthreads();
    fill_dcol(s, c0, nc);
    C *O = (C *)a.out + (size_t)mat * n * n;
    for (int idx = threadIdx.x; idx < n * nc; idx += blockDim.x) {
      const int i = idx % n, jj = idx / n, j = c0 + jj;
      O[(size_t)s.dcol[jj] * n + i] = S[(size_t)j * n + i];
    }
    return;
  }
  const int k0 = phase * KB, kbp = min(KB, n - k0);
  const int kn0 = (phase + 1) * KB, kbn = (phase + 1 < np) ? min(KB, n - kn0) : 0;
  const C *T = s.T ? s.T : S + (size_t)k0 * n;
  if (s.T)
    for (int q = 0; q < kbp; q++)
      for (int i = threadIdx.x; i < n; i += blockDim.x) s.T[q * n + i] = S[(size_t)(k0 + q) * n + i];
  for (int t = threadIdx.x; t < kMoveInts; t += blockDim.x) s.mv[t] = meta[n + phase * kMoveInts + t];
  __syncthreads();
  if (g == 0) {
    if (kbn > 0) {
      apply_panel<C, KB>(s, T, S, kn0, 0, kbn, k0, k0 + kbp, 0, 0, k0, kbp);
      const bool z = (n > 512) ? eliminate_panel<C, KB, true>(s, S, meta, kn0, kbn)
                               : eliminate_panel<C, KB, false>(s, S, meta, kn0, kbn);
      if (z && threadIdx.x == 0) record_status(a.status, 2u, a.level, mat);
    }
  } else if (nc > 0) {
    apply_panel<C, KB>(s, T, S, c0, 0, nc, k0, k0 + kbp, kn0, kn0 + kbn, k0, kbp);
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

int gj_slab(int n, int cs, int kb) {
  int cw = (n + cs - 1) / cs;
  return ((cw + kb - 1) / kb) * kb;
}

namespace {
template <int KB>
size_t plan_total(int n, int cw, bool leaf, int p, int tmode, size_t esz) {
  return plan_smem<KB>(n, cw, leaf, p, tmode, esz).total;
}
size_t plan_total_kb(int kb, int n, int cw, bool leaf, int p, int tmode, size_t esz) {
  return kb == 4 ? plan_total<4>(n, cw, leaf, p, tmode, esz) : plan_total<8>(n, cw, leaf, p, tmode, esz);
}

template <int KB>
cudaError_t run_gj_wide(WideArgs a, int batch, int G, bool f32, cudaStream_t st) {
  // Panel placement: both panels in shared memory when they fit; else the
  // eliminated one (the serial part) there and the applied one read in
  // place; else both in place.  Every CTA of a panel launch should be
  // resident at once (one wave): fewer CTAs per matrix when the shared
  // memory allows less than two per SM.
  const int n = a.n;
  const size_t esz = f32 ? 8 : 16;
  size_t smem = 0;
  for (int it = 0; it < 3; it++) {
    a.G = G;
    a.slab = (n + G - 2) / (G - 1);
    const int cwmax = a.slab > KB ? a.slab : KB;
    a.tglobal = 0;
    if (plan_total<KB>(n, cwmax, false, 0, 0, esz) > 200 * 1024)
      a.tglobal = plan_total<KB>(n, cwmax, false, 0, 2, esz) <= 200 * 1024 ? 2 : 1;
    smem = plan_total<KB>(n, cwmax, false, 0, a.tglobal, esz);
    const long long per_sm = std::max<long long>(1, std::min<long long>(2, (227 * 1024) / (long long)smem));
    if ((long long)batch * G <= 152LL * per_sm) break;
    const int G2 = (int)std::max<long long>(2, 152LL * per_sm / batch);
    if (G2 == G) break;
    G = G2;
  }
  cudaError_t err = f32 ? cudaFuncSetAttribute(gj_wide_kernel<float2, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                        : cudaFuncSetAttribute(gj_wide_kernel<double2, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int np = npanels<KB>(n);
  for (int phase = -1; phase <= np; phase++) {
    if (f32)
      gj_wide_kernel<float2, KB><<<batch * G, kThreads, smem, st>>>(a, phase);
    else
      gj_wide_kernel<double2, KB><<<batch * G, kThreads, smem, st>>>(a, phase);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}
}  // namespace

size_t gj_smem_bytes(int n, int cs, bool leaf, int p, bool tglobal, bool f32, int kb) {
  if (leaf) kb = kLeafKB;
  return plan_total_kb(kb, n, gj_slab(n, cs, kb), leaf, p, tglobal ? 1 : 0, f32 ? 8 : 16);
}

size_t gj_meta_ints(int n) { return (size_t)std::max(meta_ints<4>(n), meta_ints<8>(n)); }

size_t gj_wide_smem_bytes(int n, int slab, bool f32, bool tglobal, int kb) {
  return plan_total_kb(kb, n, slab > kb ? slab : kb, false, 0, tglobal ? 1 : 0, f32 ? 8 : 16);
}

int gj_wide_launches(int n, int kb) { return (n + kb - 1) / kb + 2; }

cudaError_t launch_gj_wide(void *S, void *out, int n, int batch, int G, int *meta,
                           unsigned int *status, int level, bool f32, cudaStream_t st, int kb) {
  if (batch <= 0 || n <= 0) return cudaSuccess;
  if (G < 2) G = 2;
  WideArgs a;
  a.S = S;
  a.out = out;
  a.meta = meta;
  a.n = n;
  a.status = status;
  a.level = level;
  return kb == 4 ? run_gj_wide<4>(a, batch, G, f32, st) : run_gj_wide<8>(a, batch, G, f32, st);
}

cudaError_t launch_leaf(const LeafTables &lt, const LeafProb *probs, int nprob, long long leaf0,
                        int count, void *X, void *GX, void *S, int *meta, unsigned int *status,
                        int level, int cs, bool f32, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  LeafArgs a;
  a.lt = lt;
  a.probs = probs;
  a.nprob = nprob;
  a.X = X;
  a.GX = GX;
  a.S = S;
  a.meta = meta;
  a.leaf0 = leaf0;
  a.status = status;
  a.level = level;
  a.cw = gj_slab(lt.n, cs, kLeafKB);
  size_t smem = plan_total<kLeafKB>(lt.n, a.cw, true, lt.p, 0, f32 ? 8 : 16);
  return f32 ? launch_cluster(leaf_kernel<float2>, a, count, cs, smem, st)
             : launch_cluster(leaf_kernel<double2>, a, count, cs, smem, st);
}

cudaError_t launch_gj_inverse(void *S, void *out, int n, int batch, int *meta, unsigned int *status,
                              int level, int cs, bool tglobal, bool f32, cudaStream_t st, int kb) {
  if (batch <= 0 || n <= 0) return cudaSuccess;
  GJArgs a;
  a.tglobal = tglobal ? 1 : 0;
  a.S = S;
  a.out = out;
  a.meta = meta;
  a.n = n;
  a.cw = gj_slab(n, cs, kb);
  a.status = status;
  a.level = level;
  const size_t smem = plan_total_kb(kb, n, a.cw, false, 0, tglobal ? 1 : 0, f32 ? 8 : 16);
  if (kb == 4)
    return f32 ? launch_cluster(gj_kernel<float2, 4>, a, batch, cs, smem, st)
               : launch_cluster(gj_kernel<double2, 4>, a, batch, cs, smem, st);
  return f32 ? launch_cluster(gj_kernel<float2, 8>, a, batch, cs, smem, st)
             : launch_cluster(gj_kernel<double2, 8>, a, batch, cs, smem, st);
}

}  // namespace hps
