// Leaf kernel and interface-inverse kernel: in-place Gauss-Jordan inversion
// with partial pivoting, the matrix spread over a thread-block cluster.
//
// Leaf (Sec. 2.1): for every leaf the kernel assembles
//     B = [ F ; A-hat(I_i, I^tau) ],  F = N + i eta I(I_b, :),
//     A-hat = -D_x^2 - D_y^2 - kappa^2 diag(c),
// inverts it, and writes X = B^{-1} = [Psi | Y] (Eqs. hmgsolnopdef and
// prtsolnopdef: B Psi = [I; 0], B Y = [0; I]) together with
// G X = [R | Gamma] (R = G Psi, Gamma = G Y), G = N - i eta I(I_b, :).
// Interface (Sec. 2.2): W^{-1} for every merge of a level, in place.
//
// Layout: a cluster of `cs` CTAs holds one n x n matrix in shared memory,
// CTA r owning columns [r*cw, r*cw + cw).  At step k the owner of column k
// picks the pivot (max |Re|+|Im| over rows >= k, lowest row on ties), swaps it
// into its broadcast buffer, and every CTA reads that column through
// distributed shared memory and applies the rank-1 Gauss-Jordan update to its
// own columns.  One cluster barrier per step; the broadcast buffers are double
// buffered so a CTA reading step k's column never races the owner of step
// k+2.  Row swaps are undone at the end as a column permutation of the
// result, applied while writing to global memory.
//
// The cluster barrier is the hardware barrier.cluster, whose participants are
// co-scheduled by construction; no kernel here spins on a flag.
#include <cooperative_groups.h>

#include "hps_internal.h"

namespace cg = cooperative_groups;

namespace hps {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double cabs1(double2 z) { return fabs(z.x) + fabs(z.y); }

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

struct GJShared {
  double2 *A;     // [n][lda] row-major local columns
  int lda;
  double2 *bcast; // [2][n] this CTA's broadcast buffers
  int *bpiv;      // [2] pivot rows matching bcast
  double2 *col;   // [n] local copy of the pivot column
  double2 *prow;  // [cw] scaled pivot row (own columns)
  int *perm;      // [n] pivot row chosen at each step
  int *dest;      // [cw] destination column of each own column
};

// Gauss-Jordan inversion of the n x n matrix whose columns [c0, c0 + ncols)
// sit in this CTA's shared memory.  Returns true if an exactly zero pivot was
// met (the step then divides by nothing and the result is not an inverse).
__device__ bool gj_core(cg::cluster_group &cl, const GJShared &s, int n, int c0, int cw,
                        int ncols) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int rank = (int)cl.block_rank();
  int cwt = 32;
  while (cwt > 1 && cwt / 2 >= ncols) cwt /= 2;
  const int rt = nthr / cwt;
  const int jj0 = tid % cwt, i0 = tid / cwt;
  bool singular = false;

  for (int k = 0; k < n; k++) {
    const int owner = k / cw, buf = k & 1;
    if (rank == owner) {
      const int kk = k - c0;
      if (tid < 32) {
        double best = -1.0;
        int bi = n;
        for (int i = k + tid; i < n; i += 32) {
          double v = cabs1(s.A[i * s.lda + kk]);
          if (v > best) {
            best = v;
            bi = i;
          }
        }
        for (int off = 16; off; off >>= 1) {
          double ov = __shfl_down_sync(0xffffffffu, best, off);
          int oi = __shfl_down_sync(0xffffffffu, bi, off);
          if (ov > best || (ov == best && oi < bi)) {
            best = ov;
            bi = oi;
          }
        }
        if (tid == 0) s.bpiv[buf] = (bi < n) ? bi : k;
      }
      __syncthreads();
      const int r = s.bpiv[buf];
      for (int i = tid; i < n; i += nthr) {
        int src = (i == k) ? r : ((i == r) ? k : i);
        s.bcast[buf * n + i] = s.A[src * s.lda + kk];
      }
    }
    cl.sync();
    const double2 *rb = cl.map_shared_rank(s.bcast + buf * n, owner);
    const int *rp = cl.map_shared_rank(s.bpiv + buf, owner);
    const int r = *rp;
    for (int i = tid; i < n; i += nthr) s.col[i] = rb[i];
    if (tid == 0) s.perm[k] = r;
    __syncthreads();
    double2 piv = s.col[k];
    double2 pinv;
    if (piv.x == 0.0 && piv.y == 0.0) {
      singular = true;
      pinv = make_double2(0.0, 0.0);
    } else {
      pinv = crecip(piv);
    }
    // swap rows k and r in the own columns; scale the pivot row
    for (int jj = tid; jj < ncols; jj += nthr) {
      double2 ak = s.A[k * s.lda + jj];
      if (r != k) {
        double2 ar = s.A[r * s.lda + jj];
        s.A[r * s.lda + jj] = ak;
        ak = ar;
      }
      s.prow[jj] = cmul(ak, pinv);
    }
    __syncthreads();
    // rank-1 update of the own columns
    for (int jj = jj0; jj < ncols; jj += cwt) {
      const double2 pr = s.prow[jj];
      const bool colk = (c0 + jj == k);
      for (int i = i0; i < n; i += rt) {
        double2 *a = &s.A[i * s.lda + jj];
        if (colk) {
          if (i == k) {
            *a = pinv;
          } else {
            double2 f = cmul(s.col[i], pinv);
            *a = make_double2(-f.x, -f.y);
          }
        } else if (i == k) {
          *a = pr;
        } else {
          double2 f = s.col[i];
          double2 v = *a;
          v.x = fma(-f.x, pr.x, v.x);
          v.x = fma(f.y, pr.y, v.x);
          v.y = fma(-f.x, pr.y, v.y);
          v.y = fma(-f.y, pr.x, v.y);
          *a = v;
        }
      }
    }
    __syncthreads();
  }
  // every CTA is done reading the others' broadcast buffers
  cl.sync();
  // the row swaps become a column permutation of the inverse, applied to the
  // columns in reverse step order
  for (int jj = tid; jj < ncols; jj += nthr) {
    int loc = c0 + jj;
    for (int k = n - 1; k >= 0; k--) {
      int pk = s.perm[k];
      if (loc == k)
        loc = pk;
      else if (loc == pk)
        loc = k;
    }
    s.dest[jj] = loc;
  }
  __syncthreads();
  return singular;
}

__device__ __forceinline__ void record_status(unsigned int *status, unsigned int code, int level,
                                              int box) {
  unsigned int w = (code << 28) | ((unsigned)(level & 0xff) << 20) | ((unsigned)box & 0xfffffu);
  atomicCAS(status, 0u, w);
}

struct SmemPlan {
  size_t A, bcast, col, prow, perm, dest, bpiv, dtab, grid, loc, cv, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline SmemPlan plan_smem(int n, int cw, bool leaf, int p) {
  SmemPlan s;
  size_t o = 0;
  int lda = cw + 1;
  s.A = o;
  o = align16(o + sizeof(double2) * (size_t)n * lda);
  s.bcast = o;
  o = align16(o + sizeof(double2) * 2 * (size_t)n);
  s.col = o;
  o = align16(o + sizeof(double2) * (size_t)n);
  s.prow = o;
  o = align16(o + sizeof(double2) * (size_t)cw);
  s.perm = o;
  o = align16(o + sizeof(int) * (size_t)n);
  s.dest = o;
  o = align16(o + sizeof(int) * (size_t)cw);
  s.bpiv = o;
  o = align16(o + sizeof(int) * 2);
  if (leaf) {
    int ni = (p - 2) * (p - 2);
    s.dtab = o;
    o = align16(o + sizeof(double) * 4 * (size_t)p * p);
    s.grid = o;
    o = align16(o + sizeof(int) * (size_t)n);
    s.loc = o;
    o = align16(o + sizeof(int) * (size_t)p * p);
    s.cv = o;
    o = align16(o + sizeof(double) * (size_t)ni);
  } else {
    s.dtab = s.grid = s.loc = s.cv = o;
  }
  s.total = o;
  return s;
}

struct LeafArgs {
  LeafTables lt;
  const double *tab;  // D1x, D1y, D2x, D2y (p*p each), then int grid[n]
  const double *c;    // [leaves][ni]
  double2 *X;         // [leaf][n][n] column-major
  double2 *GX;        // [leaf][n][nb] column-major
  unsigned int *status;
  int level;
  int cw;
};

__global__ void __launch_bounds__(kThreads, 1) leaf_kernel(const __grid_constant__ LeafArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int leaf = blockIdx.x / cs;
  const int p = a.lt.p, e = a.lt.e, n = a.lt.n, nb = a.lt.nb, ni = a.lt.ni;
  const int cw = a.cw, c0 = rank * cw;
  const int ncols = max(0, min(cw, n - c0));
  const SmemPlan sp = plan_smem(n, cw, true, p);
  GJShared s;
  s.A = (double2 *)(smem + sp.A);
  s.lda = cw + 1;
  s.bcast = (double2 *)(smem + sp.bcast);
  s.col = (double2 *)(smem + sp.col);
  s.prow = (double2 *)(smem + sp.prow);
  s.perm = (int *)(smem + sp.perm);
  s.dest = (int *)(smem + sp.dest);
  s.bpiv = (int *)(smem + sp.bpiv);
  double *D1x = (double *)(smem + sp.dtab);
  double *D1y = D1x + p * p, *D2x = D1y + p * p, *D2y = D2x + p * p;
  int *grid = (int *)(smem + sp.grid);
  int *loc = (int *)(smem + sp.loc);
  double *cv = (double *)(smem + sp.cv);
  const int tid = threadIdx.x, nthr = blockDim.x;

  // tables and this leaf's coefficient samples
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
    const int i = idx / ncols, jj = idx % ncols, j = c0 + jj;
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
    s.A[i * s.lda + jj] = v;
  }
  __syncthreads();

  const bool singular = gj_core(cl, s, n, c0, cw, ncols);
  if (singular && tid == 0 && rank == 0) record_status(a.status, 1u, a.level, leaf);

  // X = B^{-1}: own columns to their destination columns
  double2 *Xl = a.X + (size_t)leaf * n * n;
  for (int idx = tid; idx < n * ncols; idx += nthr) {
    const int jj = idx / n, i = idx % n;
    Xl[(size_t)s.dest[jj] * n + i] = s.A[i * s.lda + jj];
  }
  // G X for the own columns: row r of G is the outward normal derivative
  // along the line through boundary node r, minus i eta at r itself
  double2 *GXl = a.GX + (size_t)leaf * n * nb;
  for (int idx = tid; idx < nb * ncols; idx += nthr) {
    const int jj = idx / nb, r = idx % nb;
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
      double2 x = s.A[q * s.lda + jj];
      acc.x = fma(w, x.x, acc.x);
      acc.y = fma(w, x.y, acc.y);
    }
    double2 xr = s.A[r * s.lda + jj];  // - i eta x_r
    double2 ie = cmul(make_double2(-eta.y, eta.x), xr);
    acc.x -= ie.x;
    acc.y -= ie.y;
    GXl[(size_t)s.dest[jj] * nb + r] = acc;
  }
}

struct GJArgs {
  double2 *A;  // [batch][n][n] column-major, inverted in place
  int n;
  int cw;
  unsigned int *status;
  int level;
};

__global__ void __launch_bounds__(kThreads) gj_kernel(const __grid_constant__ GJArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int mat = blockIdx.x / cs;
  const int n = a.n, cw = a.cw, c0 = rank * cw;
  const int ncols = max(0, min(cw, n - c0));
  const SmemPlan sp = plan_smem(n, cw, false, 0);
  GJShared s;
  s.A = (double2 *)(smem + sp.A);
  s.lda = cw + 1;
  s.bcast = (double2 *)(smem + sp.bcast);
  s.col = (double2 *)(smem + sp.col);
  s.prow = (double2 *)(smem + sp.prow);
  s.perm = (int *)(smem + sp.perm);
  s.dest = (int *)(smem + sp.dest);
  s.bpiv = (int *)(smem + sp.bpiv);
  const int tid = threadIdx.x, nthr = blockDim.x;
  double2 *Ag = a.A + (size_t)mat * n * n;
  for (int idx = tid; idx < n * ncols; idx += nthr) {
    const int jj = idx / n, i = idx % n;
    s.A[i * s.lda + jj] = Ag[(size_t)(c0 + jj) * n + i];
  }
  __syncthreads();
  const bool singular = gj_core(cl, s, n, c0, cw, ncols);
  if (singular && tid == 0 && rank == 0) record_status(a.status, 2u, a.level, mat);
  // every CTA has loaded its columns (gj_core's barriers), so the in-place
  // write cannot clobber a column another CTA still has to read
  for (int idx = tid; idx < n * ncols; idx += nthr) {
    const int jj = idx / n, i = idx % n;
    Ag[(size_t)s.dest[jj] * n + i] = s.A[i * s.lda + jj];
  }
}

template <typename Kern, typename Args>
cudaError_t launch_cluster(Kern kern, const Args &args, int blocks, int cs, int threads,
                           size_t smem, cudaStream_t st) {
  cudaError_t err;
  if (cs > 8) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (err != cudaSuccess) return err;
  }
  err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks * cs, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
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

size_t gj_smem_bytes(int n, int cs, bool leaf, int p) {
  int cw = (n + cs - 1) / cs;
  return plan_smem(n, cw, leaf, p).total;
}

cudaError_t launch_leaf(const LeafTables &lt, const void *tab_dev, const double *c, int leaves,
                        double2 *X, double2 *GX, unsigned int *status, int level, int cs,
                        cudaStream_t st) {
  if (leaves <= 0) return cudaSuccess;
  LeafArgs a;
  a.lt = lt;
  a.tab = (const double *)tab_dev;
  a.c = c;
  a.X = X;
  a.GX = GX;
  a.status = status;
  a.level = level;
  a.cw = (lt.n + cs - 1) / cs;
  size_t smem = plan_smem(lt.n, a.cw, true, lt.p).total;
  return launch_cluster(leaf_kernel, a, leaves, cs, kThreads, smem, st);
}

cudaError_t launch_gj_inverse(double2 *A, int n, int batch, unsigned int *status, int level,
                              int cs, cudaStream_t st) {
  if (batch <= 0 || n <= 0) return cudaSuccess;
  GJArgs a;
  a.A = A;
  a.n = n;
  a.cw = (n + cs - 1) / cs;
  a.status = status;
  a.level = level;
  size_t smem = plan_smem(n, a.cw, false, 0).total;
  int threads = (n * a.cw <= 2048) ? 64 : ((n * a.cw <= 8192) ? 128 : kThreads);
  return launch_cluster(gj_kernel, a, batch, cs, threads, smem, st);
}

}  // namespace hps
