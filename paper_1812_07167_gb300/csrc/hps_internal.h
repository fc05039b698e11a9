// Internal declarations shared by the CUDA translation units of libhps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hps {

// Element (i, j) of batch b of a strided, optionally index-mapped complex
// matrix:  ptr[b * stride + (rmap ? rmap[i] : i) + (cmap ? cmap[j] : j) * ld]
// (column-major storage, leading dimension ld, complex128 as double2).
struct Mat {
  const double2 *ptr;
  long long ld;
  long long stride;
  const int *rmap;
  const int *cmap;
};

// One batched GEMM:  C = alpha * A * B  + beta * D  (+ I if addI)
// A: M x K, B: K x N (rows k >= ksplit read from B2, row k - ksplit),
// C, D: M x N.  D.ptr may be NULL (then beta is ignored); D may alias C
// element for element.
struct GemmDesc {
  int M, N, K, batch;
  Mat A, B, B2;
  int ksplit;
  Mat C, D;
  double2 alpha, beta;
  int addI;
};

// One batched mapped copy:  dst(i, j) = alpha * src(i, j) for i < M, j < N
// (src(j, i) when trans), or a fill with zeros when src.ptr is NULL.
struct CopyDesc {
  int M, N, batch;
  Mat src, dst;
  double2 alpha;
  int trans;
};

constexpr int kMaxCopies = 12;
struct CopyBatch {
  int count;
  CopyDesc d[kMaxCopies];
};

// Tables every leaf kernel reads (built on the host per handle).
// Local node order [S, E, N, W, interior].
struct LeafTables {
  int p, e, n, nb, ni;
  double2 eta;       // impedance parameter
  double kappa2;     // kappa^2
};

// Device-side status word: 0 = fine; otherwise (code << 28) | (level << 20) | box.
struct DevStatus {
  unsigned int word;
};

// ---- launchers (return cudaError_t of the launch) ----
cudaError_t launch_gemm(const GemmDesc *descs, int ndesc, cudaStream_t st);
cudaError_t launch_copy(const CopyBatch &cb, cudaStream_t st);

// Leaf step (Sec. 2.1) for leaves [leaf0, leaf0 + count): assemble B, invert
// it by blocked Gauss-Jordan with partial pivoting across a cluster of `cs`
// CTAs, write X = B^{-1} = [Psi | Y] ([leaf][n][n] column-major) and
// GX = G X ([leaf][n][nb] column-major: R = GX[:, :nb], Gamma = GX[:, nb:]).
//   tab_dev: device tables: double D1x[p*p], D1y[p*p], D2x[p*p], D2y[p*p]
//            (row-major, scaled to the leaf), then int grid[n] (ix | iy << 8)
//   S, meta: scratch for `count` matrices: count * n * n complex and
//            count * gj_meta_ints(n) ints
cudaError_t launch_leaf(const LeafTables &lt, const void *tab_dev, const double *c, int leaf0,
                        int count, double2 *X, double2 *GX, double2 *S, int *meta,
                        unsigned int *status, int level, int cs, cudaStream_t st);

// Inverse of `batch` n x n column-major matrices (leading dim n, batch stride
// n*n) by blocked Gauss-Jordan with partial pivoting across clusters of `cs`
// CTAs.  S holds the matrices and is destroyed; the inverses go to out.
cudaError_t launch_gj_inverse(double2 *S, double2 *out, int n, int batch, int *meta,
                              unsigned int *status, int level, int cs, cudaStream_t st);

// Cluster limits and scratch / shared-memory sizes of the Gauss-Jordan kernels.
int gj_max_cluster();
int gj_slab(int n, int cs);
size_t gj_smem_bytes(int n, int cs, bool leaf, int p);
size_t gj_meta_ints(int n);

}  // namespace hps
