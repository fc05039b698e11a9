// Leaf step in factored form (Sec. 2.1); the solve's leaf action from these
// factors is in lu_solve.cu.
//
// The leaf system is B u = [t; s] (B = [F; A-hat(I_i, :)], the impedance rows
// first).  Algorithm 2 needs u = B^{-1} [t; s] on the way down and the build
// needs G B^{-1} = [R | Gamma] (R = G Psi, Gamma = G Y).  Instead of forming
// B^{-1} (n^3 complex multiply-adds by Gauss-Jordan) this kernel factors
//     P D B = L U          (D an exact power-of-two row scaling, P the row
//                           pivoting, L unit lower and U upper triangular)
// in n^3/3, carrying the nb rows of G along as rows that are eliminated but
// never chosen as pivots, which leaves W = G U^{-1} in them (n^2 nb / 2), and
// then solves Z L = W row by row (another n^2 nb / 2), so that
//     G B^{-1} = Z P D,  i.e.  column pi(k) of G B^{-1} is d_pi(k) Z[:, k],
// where row k of P D B is row pi(k) of B.  About 0.55 of the Gauss-Jordan
// flops at p = 16.  The solve then applies B^{-1} = U^{-1} L^{-1} P D with two
// triangular sweeps (lu_solve.cu) instead of one product with B^{-1}.
//
// Layout per leaf: X [n][n] column-major holds L (unit diagonal implied) and
// U in place; GX [n][nb] holds G B^{-1}; perm[n] = pi; dsc[n] = d_pi(k).
//
// Factorisation: right-looking, panels of KB = 8 columns dealt out to the
// cs CTAs of a cluster round-robin (panel P to CTA P mod cs, so that every
// CTA keeps trailing work to the end).  Per panel: its owner factors it in
// shared memory (pivot: largest max(|Re|, |Im|) at or below the diagonal,
// lowest row on ties); every CTA then applies the panel's row swaps to its
// own columns, solves the panel's unit lower block for their U rows and
// updates their trailing rows, G rows included.  Look-ahead: the owner of
// panel P+1 updates and factors it first and publishes it (cluster barrier
// arrive) before it updates the rest of its columns.  The working matrix
// lives in X and GX themselves (in L2 while a launch's leaves fit there; the
// trailing updates stream through HBM beyond that).  One hardware cluster
// barrier per panel; no kernel here spins on a flag.
#include <cooperative_groups.h>

#include <algorithm>

#include "cx.cuh"
#include "hps_internal.h"
#include "leaf_geom.cuh"

namespace cg = cooperative_groups;

namespace hps {

namespace {

constexpr int kThreads = 256;
constexpr int KB = 8;           // panel width
constexpr int kMoves = 2 * KB;  // row moves of one panel, at most
constexpr int kMoveInts = 1 + 2 * kMoves;

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline int lu_np(int n) { return (n + KB - 1) / KB; }
// panels CTA `rank` of `cs` owns: rank, rank + cs, ...
__host__ __device__ inline int lu_own(int n, int cs, int rank) {
  const int np = lu_np(n);
  return rank < np ? (np - rank + cs - 1) / cs : 0;
}
// ints of bookkeeping per leaf: pivot rows, then the row moves of each panel
__host__ __device__ inline int lu_meta(int n) { return n + lu_np(n) * kMoveInts; }

struct LuSmem {
  size_t T, F, x, prow, krow, red, pinv, mv, rows, srcs, ld, perm, dtab, grid, cv, rsc, total;
};

__host__ __device__ inline LuSmem lu_smem(int n, int nb, int cs, int p, size_t esz) {
  LuSmem s;
  size_t o = 0;
  const size_t rows = (size_t)n + nb;
  s.T = o;    o = al16(o + esz * KB * rows);
  s.F = o;    o = al16(o + esz * KB * rows);
  s.x = o;    o = al16(o + esz * KB * KB * (size_t)lu_own(n, cs, 0));
  s.prow = o; o = al16(o + esz * KB);
  s.krow = o; o = al16(o + esz * KB);
  s.red = o;  o = al16(o + 16 * (kThreads / 32));
  s.pinv = o; o = al16(o + esz);
  s.mv = o;   o = al16(o + sizeof(int) * kMoveInts);
  s.rows = o; o = al16(o + sizeof(int) * 2 * KB);
  s.srcs = o; o = al16(o + sizeof(int) * 2 * KB);
  s.ld = o;   o = al16(o + esz * KB * KB);
  s.perm = o; o = al16(o + sizeof(int) * (size_t)n);
  const int ni = (p - 2) * (p - 2);
  s.dtab = o; o = al16(o + sizeof(double) * 4 * (size_t)p * p);
  s.grid = o; o = al16(o + sizeof(int) * (size_t)n);
  s.cv = o;   o = al16(o + sizeof(double) * (size_t)ni);
  s.rsc = o;  o = al16(o + sizeof(double) * (size_t)n);
  s.total = o;
  return s;
}

// Element (a, j) of the working matrix [D B; G]: rows a < n in X (ld n), the
// G rows a = n + r in GX (ld nb).
template <class C>
struct Work {
  C *X, *G;
  int n, nb;
  __device__ __forceinline__ C *at(int a, int j) const {
    return a < n ? X + (size_t)j * n + a : G + (size_t)j * nb + (a - n);
  }
};

struct LuShared {
  unsigned char *base;
  LuSmem sp;
};

// Factor panel [k0, k0 + kbp) (already updated by every earlier panel) in
// shared memory and write it back; record its pivot rows and net row moves
// in `meta`.  Returns true if a zero pivot was met.
template <class C>
__device__ bool lu_factor_panel(const Work<C> &w, const LuShared &sh, int *meta, int k0, int kbp) {
  const int tid = threadIdx.x, nthr = blockDim.x, n = w.n, rows = w.n + w.nb;
  const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
  C *F = (C *)(sh.base + sh.sp.F);
  C *prow = (C *)(sh.base + sh.sp.prow);
  C *krow = (C *)(sh.base + sh.sp.krow);
  C *pinv_s = (C *)(sh.base + sh.sp.pinv);
  unsigned long long *rkey = (unsigned long long *)(sh.base + sh.sp.red);
  int *ridx = (int *)(sh.base + sh.sp.red + 8 * (kThreads / 32));
  bool zero = false;
  for (int q = 0; q < kbp; q++)
    for (int a = k0 + tid; a < rows; a += nthr) F[q * rows + a] = *w.at(a, k0 + q);
  __syncthreads();
  for (int q = 0; q < kbp; q++) {
    const int k = k0 + q;
    C *Fq = F + q * rows;
    unsigned long long best = 0;
    int bi = n;
    for (int a = k + tid; a < n; a += nthr) {
      const unsigned long long key = CX<C>::key(Fq[a]);
      if (bi == n || key > best) {
        best = key;
        bi = a;
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
      rkey[wid] = best;
      ridx[wid] = bi;
    }
    __syncthreads();
    best = 0;
    bi = n;
    for (int v = 0; v < nw; v++) {
      const unsigned long long ov = rkey[v];
      const int oi = ridx[v];
      if (oi < n && (bi == n || ov > best || (ov == best && oi < bi))) {
        best = ov;
        bi = oi;
      }
    }
    const int r = (bi < n) ? bi : k;
    const bool zpiv = CX<C>::key(Fq[r]) == 0ull;
    if (zpiv) zero = true;
    if (tid < kbp) {
      prow[tid] = F[tid * rows + r];  // the new row k (U row of the panel)
      krow[tid] = F[tid * rows + k];  // old row k, which moves to row r
    }
    if (tid == 0) {
      meta[k] = r;
      pinv_s[0] = zpiv ? CX<C>::make(0.0, 0.0) : crecip(Fq[r]);
    }
    __syncthreads();
    const C pinv = pinv_s[0];
    for (int a = k + tid; a < rows; a += nthr) {
      if (a == k) {
        for (int qq = 0; qq < kbp; qq++) F[qq * rows + k] = prow[qq];
        continue;
      }
      const bool isr = (a == r);
      const C vq = isr ? krow[q] : Fq[a];
      const C l = cmul(vq, pinv);
      Fq[a] = l;
      if (isr)  // the L entries of the earlier panel columns move with the row
        for (int qq = 0; qq < q; qq++) F[qq * rows + a] = krow[qq];
      for (int qq = q + 1; qq < kbp; qq++) {
        const C v = isr ? krow[qq] : F[qq * rows + a];
        F[qq * rows + a] = cfms(v, l, prow[qq]);
      }
    }
    __syncthreads();
  }
  for (int q = 0; q < kbp; q++)
    for (int a = k0 + tid; a < rows; a += nthr) *w.at(a, k0 + q) = F[q * rows + a];
  if (tid == 0) {
    // net row moves of the panel's swaps: after the swaps (k, piv[k]) in
    // order, row rws[t] holds what row src[t] held before
    int *rws = (int *)(sh.base + sh.sp.rows);
    int *src = (int *)(sh.base + sh.sp.srcs);
    int na = 0;
    for (int q = 0; q < kbp; q++) {
      const int k = k0 + q, r = meta[k];
      if (r == k) continue;
      int ia = -1, ib = -1;
      for (int t = 0; t < na; t++) {
        if (rws[t] == k) ia = t;
        if (rws[t] == r) ib = t;
      }
      if (ia < 0) {
        ia = na;
        rws[na] = k;
        src[na] = k;
        na++;
      }
      if (ib < 0) {
        ib = na;
        rws[na] = r;
        src[na] = r;
        na++;
      }
      const int t = src[ia];
      src[ia] = src[ib];
      src[ib] = t;
    }
    int *m = meta + n + (k0 / KB) * kMoveInts;
    int cnt = 0;
    for (int t = 0; t < na; t++)
      if (rws[t] != src[t]) {
        m[1 + 2 * cnt] = rws[t];
        m[2 + 2 * cnt] = src[t];
        cnt++;
      }
    m[0] = cnt;
  }
  __syncthreads();
  return zero;
}

// Apply panel P (its columns in T, absolute rows, G row r at n + r; its row
// moves in mv) to the own columns: the local panels [ma, mb) get the row
// moves only (L columns left of P; the one that is P itself is skipped), the
// local panels [ta, tb) the moves, the unit lower solve for their U rows and
// the trailing update of rows [k0 + kbp, n + nb).  Every phase runs over all
// the columns at once, so their memory accesses overlap; the update runs
// over a flat (column, row) index, so a short trailing block costs only the
// multiply-adds it needs (on this part the FP64 pipe is the bound).
template <class C, int RPL = (sizeof(C) == 8 ? 8 : 2)>
__device__ void lu_apply(const Work<C> &w, const LuShared &sh, int rank, int cs, int P, int k0, int kbp,
                         int ma, int mb, int ta, int tb) {
  const int tid = threadIdx.x, nthr = blockDim.x, n = w.n, rows = w.n + w.nb;
  const C *T = (const C *)(sh.base + sh.sp.T);
  C *xs = (C *)(sh.base + sh.sp.x);
  const int *mv = (const int *)(sh.base + sh.sp.mv);
  const int nm = mv[0];
  const int np = lu_np(n);
  const int cwl = KB * lu_own(n, cs, 0);
  // column lists: moves-only slots [0, nmv), then trailing slots; the
  // columns past n of the last (partial) panel are left out
  auto cut = [&](int a, int b) {
    int c = (b - a) * KB;
    if (b > a && rank + cs * (b - 1) == np - 1) c -= np * KB - n;
    return c;
  };
  const int nmv = cut(ma, mb), ntr = cut(ta, tb);
  // slot -> global column j and local column index jl
  auto col = [&](int c, int &j, int &jl) {
    const int lp = c < nmv ? ma + c / KB : ta + (c - nmv) / KB;
    const int cc = c < nmv ? c % KB : (c - nmv) % KB;
    j = (rank + cs * lp) * KB + cc;
    jl = lp * KB + cc;
  };
  // 1) row moves: every source of a column is read before any of its
  //    destinations is written (kPer moves a thread per round)
  if (nm > 0) {
    constexpr int kPer = 4;
    const int cpr = max(1, (nthr * kPer) / nm);
    for (int cr = 0; cr < nmv + ntr; cr += cpr) {
      const int items = (min(nmv + ntr, cr + cpr) - cr) * nm;
      C val[kPer];
#pragma unroll
      for (int u = 0; u < kPer; u++) {
        const int it = tid + u * nthr;
        if (it < items) {
          int j, jl;
          col(cr + it / nm, j, jl);
          if (j / KB != P) val[u] = *w.at(mv[2 + 2 * (it % nm)], j);
        }
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < kPer; u++) {
        const int it = tid + u * nthr;
        if (it < items) {
          int j, jl;
          col(cr + it / nm, j, jl);
          if (j / KB != P) *w.at(mv[1 + 2 * (it % nm)], j) = val[u];
        }
      }
      __syncthreads();
    }
  }
  if (ntr == 0) return;
  // 2) panel rows of the trailing columns, then x = L_PP^{-1} a[P] (one
  //    thread a column), written back as their U rows
  for (int it = tid; it < ntr * kbp; it += nthr) {
    int j, jl;
    col(nmv + it / kbp, j, jl);
    const int q = it % kbp;
    xs[q * cwl + jl] = *w.at(k0 + q, j);
  }
  __syncthreads();
  for (int c = tid; c < ntr; c += nthr) {
    int j, jl;
    col(nmv + c, j, jl);
    C x[KB];
#pragma unroll
    for (int q = 0; q < KB; q++) x[q] = (q < kbp) ? xs[q * cwl + jl] : CX<C>::make(0.0, 0.0);
#pragma unroll
    for (int q = 1; q < KB; q++)
#pragma unroll
      for (int qq = 0; qq < q; qq++)
        if (q < kbp) x[q] = cfms(x[q], T[qq * rows + k0 + q], x[qq]);
#pragma unroll
    for (int q = 0; q < KB; q++)
      if (q < kbp) {
        xs[q * cwl + jl] = x[q];
        *w.at(k0 + q, j) = x[q];
      }
  }
  __syncthreads();
  // 3) a[i] -= sum_q L[i, k0 + q] x_q for the rows below the panel
  const int r0 = k0 + kbp, R = rows - r0;
  const int total = ntr * R;
  for (int e0 = tid; e0 < total; e0 += nthr * RPL) {
    int ra[RPL], xi[RPL];
    C *dst[RPL];
    C v[RPL];
#pragma unroll
    for (int u = 0; u < RPL; u++) {
      const int e = e0 + u * nthr;
      const bool ok = e < total;
      const int c = ok ? e / R : 0, rr = ok ? e - c * R : 0;
      int j, jl;
      col(nmv + c, j, jl);
      ra[u] = r0 + rr;
      xi[u] = ok ? jl : -1;
      dst[u] = w.at(r0 + rr, j);
      v[u] = ok ? *dst[u] : CX<C>::make(0.0, 0.0);
    }
    for (int q = 0; q < kbp; q++) {
#pragma unroll
      for (int u = 0; u < RPL; u++) {
        if (xi[u] < 0) continue;
        v[u] = cfms(v[u], T[q * rows + ra[u]], xs[q * cwl + xi[u]]);
      }
    }
#pragma unroll
    for (int u = 0; u < RPL; u++)
      if (xi[u] >= 0) *dst[u] = v[u];
  }
  __syncthreads();
}

struct LuLeafArgs {
  LeafTables lt;
  const LeafProb *probs;  // per-problem tables, c, kappa^2, eta (device)
  int nprob;
  void *X;           // [leaf][n][n]: L and U
  void *GX;          // [leaf][n][nb]: G B^{-1}
  int *perm;         // [leaf][n]
  double *dsc;       // [leaf][n]
  int *meta;         // [slot][lu_meta(n)]
  long long leaf0;   // first leaf of this launch
  unsigned int *status;
  int level;
};

template <class C>
__global__ void __launch_bounds__(kThreads, 2) lu_leaf_kernel(const __grid_constant__ LuLeafArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int slot = blockIdx.x / cs;
  const long long leaf = a.leaf0 + slot;
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
  const int p = a.lt.p, n = a.lt.n, nb = a.lt.nb, ni = a.lt.ni;
  const int rows = n + nb, np = lu_np(n);
  const int tid = threadIdx.x, nthr = blockDim.x;
  LuShared sh;
  sh.base = smem;
  sh.sp = lu_smem(n, nb, cs, p, sizeof(C));
  double *D1x = (double *)(smem + sh.sp.dtab);
  int *grid = (int *)(smem + sh.sp.grid);
  double *cv = (double *)(smem + sh.sp.cv);
  double *rsc = (double *)(smem + sh.sp.rsc);
  int *perm = (int *)(smem + sh.sp.perm);
  int *mv = (int *)(smem + sh.sp.mv);
  C *T = (C *)(smem + sh.sp.T);
  Work<C> w;
  w.X = (C *)a.X + (size_t)leaf * n * n;
  w.G = (C *)a.GX + (size_t)leaf * n * nb;
  w.n = n;
  w.nb = nb;
  int *meta = a.meta + (size_t)slot * lu_meta(n);
  const double *cleaf = pb.c + (size_t)(leaf - pb.leaf0) * ni;

  for (int i = tid; i < 4 * p * p; i += nthr) D1x[i] = tab[i];
  const int *gsrc = (const int *)(tab + 4 * p * p);
  for (int i = tid; i < n; i += nthr) grid[i] = gsrc[i];
  for (int i = tid; i < ni; i += nthr) cv[i] = cleaf[i];
  __syncthreads();
  LeafGeom geo;
  geo.D1x = D1x;
  geo.D1y = D1x + p * p;
  geo.D2x = D1x + 2 * p * p;
  geo.D2y = D1x + 3 * p * p;
  geo.grid = grid;
  geo.cv = cv;
  geo.p = p;
  geo.e = a.lt.e;
  geo.nb = nb;
  geo.kappa2 = pb.kappa2;
  geo.eta = pb.eta;
  for (int i = tid; i < n; i += nthr) rsc[i] = leaf_row_scale(geo, i);
  __syncthreads();

  // own columns of [D B; G] (entries computed in FP64, stored as C)
  const int own = lu_own(n, cs, rank);
  for (int idx = tid; idx < rows * own * KB; idx += nthr) {
    const int r = idx % rows, c = idx / rows;
    const int j = (rank + cs * (c / KB)) * KB + c % KB;
    if (j >= n) continue;
    double2 v;
    if (r < n) {
      v = leaf_B(geo, r, j);
      v.x *= rsc[r];
      v.y *= rsc[r];
    } else {
      v = leaf_G(geo, r - n, j);
    }
    *w.at(r, j) = CX<C>::make(v.x, v.y);
  }
  __syncthreads();

  bool zero = false;
  if (rank == 0) zero |= lu_factor_panel(w, sh, meta, 0, min(KB, n));
  __threadfence();
  cluster_arrive();
  cluster_wait();
  // Data another CTA of the cluster wrote (its panels, pivots, moves) is
  // read with __ldcg (from L2, past this SM's L1) after the cluster barrier.
  for (int P = 0; P < np; P++) {
    const int k0 = P * KB, kbp = min(KB, n - k0);
    for (int q = 0; q < kbp; q++)
      for (int r = k0 + tid; r < rows; r += nthr) T[q * rows + r] = __ldcg(w.at(r, k0 + q));
    for (int t = tid; t < kMoveInts; t += nthr) mv[t] = __ldcg(&meta[n + P * kMoveInts + t]);
    __syncthreads();
    // local panels left of P (moves only) and right of it (full update)
    const int lp0 = (P >= rank) ? (P - rank) / cs + 1 : 0;
    const int Pn = P + 1;
    const bool next_mine = Pn < np && (Pn % cs) == rank;
    if (next_mine) {
      lu_apply(w, sh, rank, cs, P, k0, kbp, 0, 0, lp0, lp0 + 1);
      zero |= lu_factor_panel(w, sh, meta, Pn * KB, min(KB, n - Pn * KB));
      __threadfence();
      cluster_arrive();
      lu_apply(w, sh, rank, cs, P, k0, kbp, 0, lp0, lp0 + 1, own);
      cluster_wait();
    } else {
      lu_apply(w, sh, rank, cs, P, k0, kbp, 0, lp0, lp0, own);
      __threadfence();
      cluster_arrive();
      cluster_wait();
    }
  }
  if (zero && tid == 0) record_status(a.status, 1u, a.level, (int)leaf);

  // pi: row k of P D B is row perm[k] of B
  if (tid == 0) {
    for (int i = 0; i < n; i++) perm[i] = i;
    for (int k = 0; k < n; k++) {
      const int r = __ldcg(&meta[k]);
      const int t = perm[k];
      perm[k] = perm[r];
      perm[r] = t;
    }
  }
  __syncthreads();
  if (rank == 0)
    for (int k = tid; k < n; k += nthr) {
      a.perm[(size_t)leaf * n + k] = perm[k];
      a.dsc[(size_t)leaf * n + k] = rsc[perm[k]];
    }

  // G B^{-1}: this CTA's G rows [g0, g1), in chunks of rw rows held in
  // shared memory as Ws[j][rr]; solve z L = w from the last panel back
  const int per = (nb + cs - 1) / cs;
  const int g0 = min(nb, rank * per), g1 = min(nb, g0 + per);
  const int rwmax = (int)((sh.sp.prow - sh.sp.T) / (sizeof(C) * (size_t)n));
  C *Ws = (C *)(smem + sh.sp.T);
  C *Ld = (C *)(smem + sh.sp.ld);
  for (int c0 = g0; c0 < g1; c0 += rwmax) {
    const int rw = min(rwmax, g1 - c0);
    for (int idx = tid; idx < n * rw; idx += nthr) {
      const int j = idx / rw, rr = idx % rw;
      Ws[idx] = __ldcg(&w.G[(size_t)j * nb + c0 + rr]);
    }
    __syncthreads();
    for (int J = np - 1; J >= 0; J--) {
      const int j0 = J * KB, jb = min(KB, n - j0);
      // Ld[j][i] = L[j0 + i, j0 + j]
      for (int t = tid; t < jb * jb; t += nthr) Ld[t] = __ldcg(&w.X[(size_t)(j0 + t / jb) * n + j0 + t % jb]);
      __syncthreads();
      if (tid < rw)
        for (int j = jb - 1; j >= 0; j--) {
          C acc = Ws[(j0 + j) * rw + tid];
          for (int i = j + 1; i < jb; i++) acc = cfms(acc, Ws[(j0 + i) * rw + tid], Ld[j * jb + i]);
          Ws[(j0 + j) * rw + tid] = acc;
        }
      __syncthreads();
      // w_j -= sum_{i in J} z_i L[j0 + i, j] for the columns j < j0; rows
      // split into ng groups when there are few columns
      if (j0 > 0) {
        const int ng = max(1, min(rw, nthr / j0));
        for (int it = tid; it < j0 * ng; it += nthr) {
          const int j = it % j0, gq = it / j0;
          const int ra = gq * rw / ng, rb = (gq + 1) * rw / ng;
          C lv[KB];
#pragma unroll
          for (int i = 0; i < KB; i++)
            lv[i] = (i < jb) ? __ldcg(&w.X[(size_t)j * n + j0 + i]) : CX<C>::make(0.0, 0.0);
          for (int rr = ra; rr < rb; rr++) {
            C acc = Ws[j * rw + rr];
#pragma unroll
            for (int i = 0; i < KB; i++)
              if (i < jb) acc = cfms(acc, Ws[(j0 + i) * rw + rr], lv[i]);
            Ws[j * rw + rr] = acc;
          }
        }
      }
      __syncthreads();
    }
    // column pi(k) of G B^{-1} = d_pi(k) z_k
    for (int idx = tid; idx < n * rw; idx += nthr) {
      const int k = idx / rw, rr = idx % rw;
      const int pk2 = perm[k];
      const C z = Ws[idx];
      const typename CX<C>::R d = (typename CX<C>::R)rsc[pk2];
      w.G[(size_t)pk2 * nb + c0 + rr] = CX<C>::make(d * z.x, d * z.y);
    }
    __syncthreads();
  }
}

template <typename Kern, typename Args>
cudaError_t launch_cluster_lu(Kern kern, const Args &args, int blocks, int cs, size_t smem, cudaStream_t st) {
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

size_t lu_meta_ints(int n) { return (size_t)lu_meta(n); }

size_t lu_leaf_smem_bytes(int n, int nb, int p, int cs, bool f32) {
  return lu_smem(n, nb, cs, p, f32 ? 8 : 16).total;
}

cudaError_t launch_leaf_lu(const LeafTables &lt, const LeafProb *probs, int nprob, long long leaf0,
                           int count, void *X, void *GX, int *perm, double *dsc, int *meta,
                           unsigned int *status, int level, int cs, bool f32, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  LuLeafArgs a;
  a.lt = lt;
  a.probs = probs;
  a.nprob = nprob;
  a.X = X;
  a.GX = GX;
  a.perm = perm;
  a.dsc = dsc;
  a.meta = meta;
  a.leaf0 = leaf0;
  a.status = status;
  a.level = level;
  const size_t smem = lu_smem(lt.n, lt.nb, cs, lt.p, f32 ? 8 : 16).total;
  return f32 ? launch_cluster_lu(lu_leaf_kernel<float2>, a, count, cs, smem, st)
             : launch_cluster_lu(lu_leaf_kernel<double2>, a, count, cs, smem, st);
}

}  // namespace hps
