// Complex64 inverse of the leaf matrices (Sec. 2.1) for the refined leaf
// step: X0 = B^{-1} in complex64, one CTA a leaf.
//
// B = [F ; A-hat(I_i, :)] is assembled in FP64, row-equilibrated by exact
// powers of two (D B) and stored in complex64 in a global scratch matrix S
// (column-major; the working set of the resident leaves stays in L2).  S is
// inverted in place by Gauss-Jordan elimination with row pivoting, taken in
// panels of KB = 32 columns:
//   * the panel is eliminated with each thread holding one of its rows in
//     registers (n <= 256; larger leaves in shared memory, a row a thread at
//     a time): for each column the pivot row is the largest max(|Re|, |Im|)
//     at or below the diagonal, lowest row on ties; rows k and r change
//     places and the Gauss-Jordan step is applied to the panel's columns
//     (two barriers a column).  The result T goes to shared memory and back
//     to S in place, and the panel's row swaps are folded into one row
//     permutation src (row i of a column after the swaps is its row src[i]
//     before them);
//   * every other column a then takes the panel's swaps and rank-KB update
//         a <- a[src] + (T - I[:, P]) a[src][P],   P = the panel's rows,
//     in blocks of 2 CU columns: each thread holds RT rows x CU columns of the
//     block in registers and accumulates sum_q T[i][q] x_q with T and x from
//     shared memory (RT CU complex multiply-adds per RT + CU shared loads);
//     the CTA's two halves take alternate blocks with their own barriers, so
//     that the loads of one overlap the multiply-adds of the other.
// A panel of 32 columns makes n / 32 passes over S (the 8-column panels of
// the cluster kernel make four times as many, each reading and writing the
// whole matrix), and puts 32 multiply-adds behind every element read.
// The row swaps become a column permutation of the inverse, applied with
// the row equilibration (X0 = (D B)^{-1} D) when X0 is written out.
// Only __syncthreads barriers; no spin waits.
#include "cx.cuh"
#include "hps_internal.h"
#include "leaf_geom.cuh"

namespace hps {

namespace {

constexpr int kGjPanel = 32;   // panel width KB
constexpr int kGjThreads = 256;

struct Gj32Plan {
  size_t F, xs, src, piv, dcol, col, prow, kbuf, red, scal, tabs, cv, rsc, grid, loc, total;
  int cb;   // columns of a group's update block (2 CU)
  int xld;  // row stride of xs (cb + 1: the panel rows' stores fall in different banks)
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline Gj32Plan gj32_plan(int n, int p, int ni, int cb) {
  Gj32Plan s;
  size_t o = 0;
  s.cb = cb;
  s.xld = cb + 1;
  s.F = o;    o = al16(o + sizeof(float2) * (size_t)kGjPanel * n);
  s.xs = o;   o = al16(o + sizeof(float2) * 2 * (size_t)kGjPanel * s.xld);
  s.src = o;  o = al16(o + sizeof(int) * (size_t)n);
  s.piv = o;  o = al16(o + sizeof(int) * (size_t)n);
  s.dcol = o; o = al16(o + sizeof(int) * (size_t)n);
  s.col = o;  o = al16(o + sizeof(float2) * (size_t)n);
  s.prow = o; o = al16(o + sizeof(float2) * kGjPanel);
  s.kbuf = o; o = al16(o + sizeof(float2) * kGjPanel);
  s.red = o;  o = al16(o + 24 * (kGjThreads / 32));
  s.scal = o; o = al16(o + 16);
  s.tabs = o; o = al16(o + sizeof(double) * 4 * (size_t)p * p);
  s.cv = o;   o = al16(o + sizeof(double) * (size_t)ni);
  s.rsc = o;  o = al16(o + sizeof(double) * (size_t)n);
  s.grid = o; o = al16(o + sizeof(int) * (size_t)n);
  s.loc = o;  o = al16(o + sizeof(int) * (size_t)p * p);
  s.total = o;
  return s;
}

struct Gj32Args {
  LeafTables lt;
  const LeafProb *probs;
  int nprob;
  long long leaf0;    // first leaf of the launch
  float2 *X0;         // [leaf][n][n] column-major, indexed by the absolute leaf number
  float2 *GX;         // [leaf][n][nb] column-major (G X0), or null
  float2 *S;          // [launch slot][n][n] scratch
  unsigned *status;
  int level;
};

// the problem of leaf `leaf`: the last one starting at or before it
__device__ __forceinline__ int gj32_problem(const LeafProb *probs, int nprob, long long leaf) {
  int pk = 0;
  for (int lo = 0, hi = nprob - 1; lo <= hi;) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(&probs[mid].leaf0) <= leaf) {
      pk = mid;
      lo = mid + 1;
    } else {
      hi = mid - 1;
    }
  }
  return pk;
}

// Barrier of one 128-thread group (named barriers 1 and 2; 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, 128;\n" ::"r"(1 + g) : "memory");
}

// The pivot of one elimination step from every warp's candidate (largest
// key, lowest row on ties): rkey/ridx/rval hold one candidate a warp.
__device__ __forceinline__ void gj32_pick(const unsigned long long *rkey, const int *ridx, const float2 *rval, int n,
                                          unsigned long long &best, int &r, float2 &pv) {
  best = 0;
  r = n;
  pv = make_float2(0.f, 0.f);
#pragma unroll
  for (int w = 0; w < kGjThreads / 32; w++) {
    const unsigned long long ov = rkey[w];
    const int oi = ridx[w];
    if (oi < n && (r == n || ov > best || (ov == best && oi < r))) {
      best = ov;
      r = oi;
      pv = rval[w];
    }
  }
}

// A warp's candidate: the largest key among its lanes' (key, row, value).
__device__ __forceinline__ void gj32_warp_best(unsigned long long &key, int &bi, float2 &bv, int n) {
  for (int off = 16; off; off >>= 1) {
    const unsigned long long ov = __shfl_down_sync(0xffffffffu, key, off);
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    const float ox = __shfl_down_sync(0xffffffffu, bv.x, off);
    const float oy = __shfl_down_sync(0xffffffffu, bv.y, off);
    if (oi < n && (bi == n || ov > key || (ov == key && oi < bi))) {
      key = ov;
      bi = oi;
      bv = make_float2(ox, oy);
    }
  }
}

// Eliminate the panel of kbp columns starting at column k0 of S with one row
// a thread in registers (n <= kGjThreads): T into F (shared, column-major)
// and back into S; pivot rows to piv[k].  Returns true on a zero pivot.
__device__ bool gj32_eliminate_reg(float2 *S, float2 *F, int n, int k0, int kbp, int *piv, float2 *prow,
                                   float2 *kbuf, unsigned long long *rkey, int *ridx, float2 *rval) {
  const int i = threadIdx.x, lane = i & 31, wid = i >> 5;
  float2 f[kGjPanel];
#pragma unroll
  for (int qq = 0; qq < kGjPanel; qq++)
    f[qq] = (i < n && qq < kbp) ? S[(size_t)(k0 + qq) * n + i] : make_float2(0.f, 0.f);
  bool zero = false;
#pragma unroll 1
  for (int q = 0; q < kbp; q++) {
    {
      const int k = k0 + q;
      // f[q] by selection (the register array is indexed by constants only)
      float2 fq = f[0];
#pragma unroll
      for (int qq = 1; qq < kGjPanel; qq++)
        if (qq == q) fq = f[qq];
      const bool cand = i >= k && i < n;
      unsigned long long key = cand ? CX<float2>::key(fq) : 0ull;
      int bi = cand ? i : n;
      float2 bv = fq;
      gj32_warp_best(key, bi, bv, n);
      if (lane == 0) {
        rkey[wid] = key;
        ridx[wid] = bi;
        rval[wid] = bv;
      }
      __syncthreads();
      unsigned long long best;
      int r;
      float2 pv;
      gj32_pick(rkey, ridx, rval, n, best, r, pv);
      const bool z = best == 0ull;
      zero |= z;
      const float2 pinv = z ? make_float2(0.f, 0.f) : crecip(pv);
      if (i == 0) piv[k] = r;
      // rows k and r change places; the new row k, scaled, is the pivot row
      if (i == r) {
#pragma unroll
        for (int qq = 0; qq < kGjPanel; qq++) prow[qq] = cmul(f[qq], pinv);
      }
      if (i == k && r != k) {
#pragma unroll
        for (int qq = 0; qq < kGjPanel; qq++) kbuf[qq] = f[qq];
      }
      __syncthreads();
      if (i == r && r != k) {
        fq = kbuf[q];
#pragma unroll
        for (int qq = 0; qq < kGjPanel; qq++) f[qq] = kbuf[qq];
      }
      if (i == k) {
#pragma unroll
        for (int qq = 0; qq < kGjPanel; qq++) f[qq] = (qq == q) ? pinv : prow[qq];
      } else {
        const float2 c = fq;
        const float2 t = cmul(c, pinv);
        const float2 mt = make_float2(-t.x, -t.y);
#pragma unroll
        for (int qq = 0; qq < kGjPanel; qq++) f[qq] = (qq == q) ? mt : cfms(f[qq], c, prow[qq]);
      }
    }
  }
  if (i < n)
#pragma unroll
    for (int qq = 0; qq < kGjPanel; qq++)
      if (qq < kbp) {
        F[(size_t)qq * n + i] = f[qq];
        S[(size_t)(k0 + qq) * n + i] = f[qq];
      }
  return zero;
}

// The same with the panel in shared memory (any n): F holds the kbp
// columns (column-major) on entry and T on return; a thread takes rows i,
// i + kGjThreads, ... of every column.
__device__ bool gj32_eliminate_smem(float2 *F, int n, int k0, int kbp, int *piv, float2 *col, float2 *prow,
                                    unsigned long long *rkey, int *ridx, float2 *rval) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  bool zero = false;
  for (int q = 0; q < kbp; q++) {
    const int k = k0 + q;
    const float2 *Fq = F + (size_t)q * n;
    unsigned long long key = 0;
    int bi = n;
    float2 bv = make_float2(0.f, 0.f);
    for (int i = k + tid; i < n; i += kGjThreads) {
      const unsigned long long kk = CX<float2>::key(Fq[i]);
      if (bi == n || kk > key) {
        key = kk;
        bi = i;
        bv = Fq[i];
      }
    }
    gj32_warp_best(key, bi, bv, n);
    if (lane == 0) {
      rkey[wid] = key;
      ridx[wid] = bi;
      rval[wid] = bv;
    }
    __syncthreads();
    unsigned long long best;
    int r;
    float2 pv;
    gj32_pick(rkey, ridx, rval, n, best, r, pv);
    if (r == n) r = k;
    const bool z = best == 0ull;
    zero |= z;
    const float2 pinv = z ? make_float2(0.f, 0.f) : crecip(pv);
    if (tid == 0) piv[k] = r;
    // swap rows k and r of the panel; the pivot column and scaled pivot row
    if (tid < kbp) {
      float2 *Fc = F + (size_t)tid * n;
      const float2 a = Fc[k], b = Fc[r];
      Fc[k] = b;
      Fc[r] = a;
      prow[tid] = cmul(b, pinv);
    }
    __syncthreads();
    for (int i = tid; i < n; i += kGjThreads) col[i] = (i == k) ? make_float2(0.f, 0.f) : Fq[i];
    __syncthreads();
    for (int i = tid; i < n; i += kGjThreads) {
      const float2 c = col[i];
      for (int qq = 0; qq < kbp; qq++) {
        float2 *a = &F[(size_t)qq * n + i];
        if (qq == q) {
          if (i == k) {
            *a = pinv;
          } else {
            const float2 t = cmul(c, pinv);
            *a = make_float2(-t.x, -t.y);
          }
        } else if (i == k) {
          *a = prow[qq];
        } else {
          *a = cfms(*a, c, prow[qq]);
        }
      }
    }
    __syncthreads();
  }
  return zero;
}

template <int RT, int CU>
__global__ void __launch_bounds__(kGjThreads, 2) gj32_leaf_kernel(const __grid_constant__ Gj32Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int CB = 2 * CU;  // columns of a group's update block
  const int tid = threadIdx.x;
  const long long leaf = a.leaf0 + blockIdx.x;
  const LeafProb &pb = a.probs[gj32_problem(a.probs, a.nprob, leaf)];
  const int p = a.lt.p, n = a.lt.n, ni = a.lt.ni;
  const Gj32Plan sp = gj32_plan(n, p, ni, CB);  // (x buffers: two groups x KB rows x (CB + 1))
  float2 *F = (float2 *)(smem + sp.F);
  float2 *xs = (float2 *)(smem + sp.xs);
  int *src = (int *)(smem + sp.src);
  int *piv = (int *)(smem + sp.piv);
  int *dcol = (int *)(smem + sp.dcol);
  float2 *col = (float2 *)(smem + sp.col);
  float2 *prow = (float2 *)(smem + sp.prow);
  float2 *kbuf = (float2 *)(smem + sp.kbuf);
  unsigned long long *rkey = (unsigned long long *)(smem + sp.red);
  int *ridx = (int *)(smem + sp.red + 8 * (kGjThreads / 32));
  float2 *rval = (float2 *)(smem + sp.red + 16 * (kGjThreads / 32));
  const int XL = sp.xld;
  double *D1x = (double *)(smem + sp.tabs);
  double *cv = (double *)(smem + sp.cv);
  double *rsc = (double *)(smem + sp.rsc);
  int *grid = (int *)(smem + sp.grid);
  int *loc = (int *)(smem + sp.loc);

  // the leaf's tables
  for (int i = tid; i < 4 * p * p; i += kGjThreads) D1x[i] = pb.tab[i];
  const int *gsrc = (const int *)(pb.tab + 4 * p * p);
  for (int i = tid; i < n; i += kGjThreads) grid[i] = gsrc[i];
  const double *cl = pb.c + (size_t)(leaf - pb.leaf0) * ni;
  for (int i = tid; i < ni; i += kGjThreads) cv[i] = cl[i];
  for (int i = tid; i < p * p; i += kGjThreads) loc[i] = -1;
  __syncthreads();
  for (int i = tid; i < n; i += kGjThreads) loc[(grid[i] >> 8) * p + (grid[i] & 0xff)] = i;
  LeafGeom geo;
  geo.D1x = D1x;
  geo.D1y = D1x + p * p;
  geo.D2x = D1x + 2 * p * p;
  geo.D2y = D1x + 3 * p * p;
  geo.grid = grid;
  geo.cv = cv;
  geo.p = p;
  geo.e = a.lt.e;
  geo.nb = a.lt.nb;
  geo.kappa2 = pb.kappa2;
  geo.eta = pb.eta;
  for (int i = tid; i < n; i += kGjThreads) rsc[i] = leaf_row_scale(geo, i);
  __syncthreads();

  // S = D B in complex64 (entries formed in FP64)
  float2 *S = a.S + (size_t)blockIdx.x * n * n;
  for (int idx = tid; idx < n * n; idx += kGjThreads) {
    const int i = idx % n, j = idx / n;
    const double2 v = leaf_B(geo, i, j);
    S[idx] = make_float2((float)(rsc[i] * v.x), (float)(rsc[i] * v.y));
  }
  __syncthreads();

  bool zero = false;
  for (int k0 = 0; k0 < n; k0 += kGjPanel) {
    const int kbp = min(kGjPanel, n - k0);
    // ---- the panel: eliminate, T to F and back to S; its row permutation ----
    for (int i = tid; i < n; i += kGjThreads) src[i] = i;
    if constexpr (RT == 4) {
      zero |= gj32_eliminate_reg(S, F, n, k0, kbp, piv, prow, kbuf, rkey, ridx, rval);
    } else {
      for (int e = tid; e < kbp * n; e += kGjThreads) F[e] = S[(size_t)k0 * n + e];
      __syncthreads();
      zero |= gj32_eliminate_smem(F, n, k0, kbp, piv, col, prow, rkey, ridx, rval);
      for (int e = tid; e < kbp * n; e += kGjThreads) S[(size_t)k0 * n + e] = F[e];
    }
    __syncthreads();
    if (tid == 0)
      for (int q = 0; q < kbp; q++) {
        const int k = k0 + q, r = piv[k];
        const int t = src[k];
        src[k] = src[r];
        src[r] = t;
      }
    __syncthreads();
    // ---- every other column: a <- a[src] + (T - I[:, P]) a[src][P] ----
    // Two groups of four warps take alternate blocks of CB columns, each
    // with its own barrier and x buffer, so that one group's loads overlap
    // the other's multiply-adds.
    {
      const int g = tid >> 7, gt = tid & 127, rl = gt & 63, cgl = gt >> 6;
      float2 *xg = xs + (size_t)g * kGjPanel * XL;
      for (int jb = g * CB; jb < n; jb += 2 * CB) {
        float2 acc[RT][CU];
        int rows[RT];
#pragma unroll
        for (int t = 0; t < RT; t++) rows[t] = rl + 64 * t;
#pragma unroll
        for (int u = 0; u < CU; u++) {
          const int j = jb + cgl + 2 * u;
          const bool live = j < n && (j < k0 || j >= k0 + kbp);
#pragma unroll
          for (int t = 0; t < RT; t++) {
            const int i = rows[t];
            float2 v = make_float2(0.f, 0.f);
            if (live && i < n) v = S[(size_t)j * n + src[i]];
            acc[t][u] = v;
          }
        }
#pragma unroll
        for (int t = 0; t < RT; t++)
          if (rows[t] >= k0 && rows[t] < k0 + kbp) {
#pragma unroll
            for (int u = 0; u < CU; u++) {
              xg[(rows[t] - k0) * XL + cgl + 2 * u] = acc[t][u];
              acc[t][u] = make_float2(0.f, 0.f);
            }
          }
        group_sync(g);
#pragma unroll 2
        for (int q = 0; q < kbp; q++) {
          float2 tq[RT], xq[CU];
#pragma unroll
          for (int t = 0; t < RT; t++) tq[t] = rows[t] < n ? F[(size_t)q * n + rows[t]] : make_float2(0.f, 0.f);
#pragma unroll
          for (int u = 0; u < CU; u++) xq[u] = xg[q * XL + cgl + 2 * u];
#pragma unroll
          for (int t = 0; t < RT; t++)
#pragma unroll
            for (int u = 0; u < CU; u++) {
              acc[t][u].x = fmaf(tq[t].x, xq[u].x, acc[t][u].x);
              acc[t][u].x = fmaf(-tq[t].y, xq[u].y, acc[t][u].x);
              acc[t][u].y = fmaf(tq[t].x, xq[u].y, acc[t][u].y);
              acc[t][u].y = fmaf(tq[t].y, xq[u].x, acc[t][u].y);
            }
        }
#pragma unroll
        for (int u = 0; u < CU; u++) {
          const int j = jb + cgl + 2 * u;
          if (j < n && (j < k0 || j >= k0 + kbp))
#pragma unroll
            for (int t = 0; t < RT; t++)
              if (rows[t] < n) S[(size_t)j * n + rows[t]] = acc[t][u];
        }
        group_sync(g);  // before this group's next x buffer
      }
    }
    __syncthreads();
  }
  if (zero && tid == 0) record_status(a.status, 1u, a.level, (int)leaf);

  // destination column of column j: the row swaps (k, piv[k]) as column
  // swaps in reverse step order
  for (int j = tid; j < n; j += kGjThreads) {
    int d = j;
    for (int k = n - 1; k >= 0; k--) {
      const int pk = piv[k];
      if (d == k)
        d = pk;
      else if (d == pk)
        d = k;
    }
    dcol[j] = d;
  }
  __syncthreads();
  // X0 = (D B)^{-1} D
  float2 *Xl = a.X0 + (size_t)leaf * n * n;
  for (int idx = tid; idx < n * n; idx += kGjThreads) {
    const int i = idx % n, j = idx / n;
    const int dc = dcol[j];
    const float d = (float)rsc[dc];
    const float2 v = S[idx];
    Xl[(size_t)dc * n + i] = make_float2(d * v.x, d * v.y);
  }
  if (!a.GX) return;
  // G X0: row r of G is the outward normal derivative along the grid line
  // through boundary node r (p entries), minus i eta at r itself
  const int e = a.lt.e, nb = a.lt.nb;
  const double *D1y = D1x + p * p;
  float2 *GXl = a.GX + (size_t)leaf * n * nb;
  const float2 ieta = make_float2((float)-pb.eta.y, (float)pb.eta.x);
  for (int idx = tid; idx < nb * n; idx += kGjThreads) {
    const int r = idx % nb, j = idx / nb;
    const float2 *Sj = S + (size_t)j * n;
    const int side = r / e, ix = grid[r] & 0xff, iy = grid[r] >> 8;
    float2 acc = make_float2(0.f, 0.f);
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
      if (q < 0) continue;
      const float2 x = Sj[q];
      acc.x = fmaf((float)w, x.x, acc.x);
      acc.y = fmaf((float)w, x.y, acc.y);
    }
    const float2 ie = cmul(ieta, Sj[r]);  // - i eta x_r
    acc.x -= ie.x;
    acc.y -= ie.y;
    const int dc = dcol[j];
    const float d = (float)rsc[dc];
    GXl[(size_t)dc * nb + r] = make_float2(d * acc.x, d * acc.y);
  }
}

template <int RT, int CU>
cudaError_t run_gj32(const Gj32Args &a, int count, size_t smem, cudaStream_t st) {
  cudaError_t err = cudaFuncSetAttribute(gj32_leaf_kernel<RT, CU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  gj32_leaf_kernel<RT, CU><<<count, kGjThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t gj32_smem_bytes(const LeafTables &lt) {
  return gj32_plan(lt.n, lt.p, lt.ni, lt.n <= 256 ? 16 : 8).total;
}

bool gj32_supported(const LeafTables &lt) { return lt.n <= 384 && gj32_smem_bytes(lt) <= 227 * 1024; }

cudaError_t launch_leaf_gj32(const LeafTables &lt, const LeafProb *probs, int nprob, long long leaf0, int count,
                             void *X0, void *GX, void *S, unsigned int *status, int level, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  if (!gj32_supported(lt)) return cudaErrorInvalidValue;
  Gj32Args a;
  a.lt = lt;
  a.probs = probs;
  a.nprob = nprob;
  a.leaf0 = leaf0;
  a.X0 = (float2 *)X0;
  a.GX = (float2 *)GX;
  a.S = (float2 *)S;
  a.status = status;
  a.level = level;
  const size_t smem = gj32_smem_bytes(lt);
  return lt.n <= 256 ? run_gj32<4, 8>(a, count, smem, st) : run_gj32<6, 4>(a, count, smem, st);
}

}  // namespace hps
