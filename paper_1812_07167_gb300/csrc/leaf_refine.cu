// Leaf step (Sec. 2.1) in complex128 by a refined inverse: the leaf matrix
// B is inverted in complex64 (blocked Gauss-Jordan with 32-column panels,
// leaf_gj32.cu: X0 ~ B^-1 to ~1e-5 for the row-equilibrated leaf matrices,
// whose condition numbers are ~5e2), and X0 is refined to complex128
// accuracy by steps of
//     E = I - B X      (complex128-accurate: the Ozaki product on the tensor
//                       cores, B assembled exactly in FP64; E is then
//                       rounded to complex64, which costs the correction
//                       nothing: it is formed in complex64 anyway)
//     X = X + X0 E     (the correction product in complex64 arithmetic, added
//                       in FP64 in the product's epilogue)
// Each step multiplies the residual norm by ~||I - B X0|| (~1e-5), and the
// complex64 rounding of the correction is ~1e-7 of a term of that size, so
// two steps reach the complex128 rounding level.  Then G X = [R | Gamma] in
// FP64 with the sparse G.  The result is the inverse form of the leaf
// operators (X = B^-1 = [Psi | Y], GX), to the accuracy of a complex128
// inversion, with most of the work off this part's FP64 pipes.
#include <algorithm>
#include <cstring>
#include <map>

#include "cx.cuh"
#include "hps_internal.h"
#include "leaf_geom.cuh"

namespace hps {

namespace {

// the problem of leaf `leaf`: the last one starting at or before it
__device__ __forceinline__ int leaf_problem(const LeafProb *probs, int nprob, long long leaf) {
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

// The leaf's tables in shared memory: D1x, D1y, D2x, D2y (p x p), the node
// grid, the grid -> node map, c at the interior nodes.
struct LeafSmem {
  double *D1x, *D1y, *D2x, *D2y, *cv;
  int *grid, *loc;
};

__device__ LeafSmem load_leaf_tables(unsigned char *smem, const LeafTables &lt, const LeafProb &pb,
                                     long long leaf) {
  const int p = lt.p, n = lt.n, ni = lt.ni;
  LeafSmem t;
  t.D1x = (double *)smem;
  t.D1y = t.D1x + p * p;
  t.D2x = t.D1y + p * p;
  t.D2y = t.D2x + p * p;
  t.cv = t.D2y + p * p;
  t.grid = (int *)(t.cv + ni);
  t.loc = t.grid + n;
  const double *cl = pb.c + (size_t)(leaf - pb.leaf0) * ni;
  for (int i = threadIdx.x; i < 4 * p * p; i += blockDim.x) t.D1x[i] = pb.tab[i];
  const int *gsrc = (const int *)(pb.tab + 4 * p * p);
  for (int i = threadIdx.x; i < n; i += blockDim.x) t.grid[i] = gsrc[i];
  for (int i = threadIdx.x; i < p * p; i += blockDim.x) t.loc[i] = -1;
  for (int i = threadIdx.x; i < ni; i += blockDim.x) t.cv[i] = cl[i];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) t.loc[(t.grid[i] >> 8) * p + (t.grid[i] & 0xff)] = i;
  __syncthreads();
  return t;
}

size_t leaf_tables_smem(const LeafTables &lt) {
  return sizeof(double) * (4 * lt.p * lt.p + lt.ni) + sizeof(int) * (lt.n + lt.p * lt.p);
}

__device__ LeafGeom make_geom(const LeafSmem &t, const LeafTables &lt, const LeafProb &pb) {
  LeafGeom g;
  g.D1x = t.D1x;
  g.D1y = t.D1y;
  g.D2x = t.D2x;
  g.D2y = t.D2y;
  g.grid = t.grid;
  g.cv = t.cv;
  g.p = lt.p;
  g.e = lt.e;
  g.nb = lt.nb;
  g.kappa2 = pb.kappa2;
  g.eta = pb.eta;
  return g;
}

// B of leaves [leaf0, leaf0 + gridDim.x) in FP64, column-major n x n each
// (entry (i, j) at j n + i; neighbouring threads on neighbouring rows).
__global__ void __launch_bounds__(256) leaf_B_kernel(LeafTables lt, const LeafProb *probs, int nprob,
                                                     long long leaf0, double2 *B) {
  extern __shared__ __align__(16) unsigned char lsm[];
  const long long leaf = leaf0 + blockIdx.x;
  const LeafProb &pb = probs[leaf_problem(probs, nprob, leaf)];
  const LeafSmem t = load_leaf_tables(lsm, lt, pb, leaf);
  const LeafGeom g = make_geom(t, lt, pb);
  const int n = lt.n;
  double2 *Bl = B + (size_t)blockIdx.x * n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) Bl[idx] = leaf_B(g, idx % n, idx / n);
}

// GX = G X for leaves [leaf0, leaf0 + gridDim.x): X n x n, GX nb x n,
// column-major.  Row r of G is the outward normal derivative along the grid
// line through boundary node r (p entries), minus i eta at r itself.
__global__ void __launch_bounds__(256) leaf_GX_kernel(LeafTables lt, const LeafProb *probs, int nprob,
                                                      long long leaf0, const double2 *X, double2 *GX) {
  extern __shared__ __align__(16) unsigned char lsm[];
  const long long leaf = leaf0 + blockIdx.x;
  const LeafProb &pb = probs[leaf_problem(probs, nprob, leaf)];
  const LeafSmem t = load_leaf_tables(lsm, lt, pb, leaf);
  const int p = lt.p, e = lt.e, n = lt.n, nb = lt.nb;
  const double2 *Xl = X + (size_t)blockIdx.x * n * n;
  double2 *GXl = GX + (size_t)blockIdx.x * n * nb;
  const double2 ieta = make_double2(-pb.eta.y, pb.eta.x);
  for (int idx = threadIdx.x; idx < nb * n; idx += blockDim.x) {
    const int r = idx % nb, j = idx / nb;
    const double2 *Xj = Xl + (size_t)j * n;
    const int side = r / e, ix = t.grid[r] & 0xff, iy = t.grid[r] >> 8;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < p; k++) {
      double w;
      int q;
      if (side == 0) {
        w = -t.D1y[0 * p + k];
        q = t.loc[k * p + ix];
      } else if (side == 1) {
        w = t.D1x[(p - 1) * p + k];
        q = t.loc[iy * p + k];
      } else if (side == 2) {
        w = t.D1y[(p - 1) * p + k];
        q = t.loc[k * p + ix];
      } else {
        w = -t.D1x[0 * p + k];
        q = t.loc[iy * p + k];
      }
      if (q < 0) continue;  // (lines through non-corner edge nodes hold no corner; a guard)
      const double2 x = Xj[q];
      acc.x = fma(w, x.x, acc.x);
      acc.y = fma(w, x.y, acc.y);
    }
    const double2 ie = cmul(ieta, Xj[r]);  // - i eta x_r
    acc.x -= ie.x;
    acc.y -= ie.y;
    GXl[(size_t)j * nb + r] = acc;
  }
}

struct RefineLayout {
  size_t x0, gx0, s, meta, b, e, oz, total;
};

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

GemmDesc plain_gemm(int M, int N, int K, int batch, const void *A, int af32, const void *B, int bf32, void *C) {
  GemmDesc g;
  memset(&g, 0, sizeof(g));
  g.M = M;
  g.N = N;
  g.K = K;
  g.batch = batch;
  g.A.ptr = A;
  g.A.ld = M;
  g.A.stride = (long long)M * K;
  g.A.f32 = af32;
  g.B.ptr = B;
  g.B.ld = K;
  g.B.stride = (long long)K * N;
  g.B.f32 = bf32;
  g.ksplit = K;
  g.C.ptr = C;
  g.C.ld = M;
  g.C.stride = (long long)M * N;
  g.alpha = make_double2(1.0, 0.0);
  return g;
}

RefineLayout refine_layout(const LeafTables &lt, int count) {
  const size_t n = lt.n, nb = lt.nb, c = (size_t)count;
  RefineLayout L;
  size_t o = 0;
  L.x0 = o;
  o = al256(o + 8 * c * n * n);
  L.gx0 = o;
  o = al256(o + 8 * c * n * nb);
  L.s = o;
  o = al256(o + 8 * c * n * n);
  L.meta = o;
  o = al256(o + sizeof(int) * c * gj_meta_ints((int)n));
  L.b = o;
  o = al256(o + 16 * c * n * n);
  L.e = o;  // the residual E, stored in complex64 (an operand of the complex64 correction only)
  o = al256(o + 8 * c * n * n);
  L.oz = o;
  GemmDesc g = plain_gemm((int)n, (int)n, (int)n, count, nullptr, 0, nullptr, 1, nullptr);
  o = al256(o + oz_workspace_bytes(g));
  L.total = o;
  return L;
}

}  // namespace

// A second stream of the same device and priority as st for work that can
// run beside st's (one a host thread and priority, created once).
cudaStream_t side_stream(cudaStream_t st) {
  int prio = 0, dev = 0;
  if (cudaStreamGetPriority(st, &prio) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  thread_local std::map<std::pair<int, int>, cudaStream_t> streams;
  auto it = streams.find({dev, prio});
  if (it != streams.end()) return it->second;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio) != cudaSuccess) {
    cudaGetLastError();
    s = nullptr;
  }
  streams[{dev, prio}] = s;
  return s;
}

size_t leaf_refined_scratch_bytes(const LeafTables &lt, int count) { return refine_layout(lt, count).total; }

int leaf_refined_launches(const LeafTables &lt, int count, int steps) {
  GemmDesc g = plain_gemm(lt.n, lt.n, lt.n, count, nullptr, 0, nullptr, 1, nullptr);
  int n = 3;  // X0, B, G X
  for (int it = 0; it < steps; it++) n += oz_launches(g, it > 0) + 1;  // residual, correction
  return n;
}

cudaError_t launch_leaf_refined(const LeafTables &lt, const LeafProb *probs, int nprob, long long leaf0, int count,
                                void *X, void *GX, void *scr, size_t scr_bytes, unsigned int *status, int level,
                                int cs32, int steps, cudaStream_t st, int *launches) {
  if (count <= 0) return cudaSuccess;
  const RefineLayout L = refine_layout(lt, count);
  if (!scr || scr_bytes < L.total) return cudaErrorInvalidValue;
  char *w = (char *)scr;
  const int n = lt.n, nb = lt.nb;
  void *X0 = w + L.x0;
  double2 *Bm = (double2 *)(w + L.b);
  float2 *E = (float2 *)(w + L.e);
  double2 *Xl = (double2 *)X + (size_t)leaf0 * n * n;
  double2 *GXl = (double2 *)GX + (size_t)leaf0 * n * nb;
  int nl = 0;
  // B in FP64 and its digit split (the residuals' first operand) do not
  // depend on X0: they run on a side stream while the complex64 inverse
  // (whose 256 CTAs leave a third of the SMs half empty) runs on st
  const size_t tsm = leaf_tables_smem(lt);
  GemmDesc g0 = plain_gemm(n, n, n, count, Bm, 0, X0, 1, E);
  cudaStream_t side = side_stream(st);
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaError_t err = cudaSuccess;
  if (side && (err = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming)) == cudaSuccess &&
      (err = cudaEventCreateWithFlags(&join, cudaEventDisableTiming)) == cudaSuccess &&
      (err = cudaEventRecord(fork, st)) == cudaSuccess && (err = cudaStreamWaitEvent(side, fork, 0)) == cudaSuccess) {
    leaf_B_kernel<<<count, 256, tsm, side>>>(lt, probs, nprob, leaf0, Bm);
    if ((err = cudaGetLastError()) == cudaSuccess) err = launch_oz_split_a(g0, w + L.oz, L.total - L.oz, side);
    if (err == cudaSuccess) err = cudaEventRecord(join, side);
  } else {
    cudaGetLastError();
    side = nullptr;
  }
  if (err != cudaSuccess) {
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    return err;
  }
  nl += 3;  // B, A's exponents and digits
  // X0: the complex64 inverse (32-column panels, one CTA a leaf; the
  // cluster kernel where the panel does not fit; its G X0 is not used)
  err =
      gj32_supported(lt)
          ? launch_leaf_gj32(lt, probs, nprob, leaf0, count, (float2 *)X0 - (size_t)leaf0 * n * n, nullptr, w + L.s,
                             status, level, st)
          : launch_leaf(lt, probs, nprob, leaf0, count, (float2 *)X0 - (size_t)leaf0 * n * n,
                        (float2 *)(w + L.gx0) - (size_t)leaf0 * n * nb, w + L.s, (int *)(w + L.meta), status, level,
                        cs32, true, st);
  if (err == cudaSuccess) nl++;
  if (side) {
    // (without a side stream: B and its split here, in order)
    if (err == cudaSuccess) err = cudaStreamWaitEvent(st, join, 0);
    cudaEventDestroy(fork);
    cudaEventDestroy(join);
  } else if (err == cudaSuccess) {
    leaf_B_kernel<<<count, 256, tsm, st>>>(lt, probs, nprob, leaf0, Bm);
    if ((err = cudaGetLastError()) == cudaSuccess) err = launch_oz_split_a(g0, w + L.oz, L.total - L.oz, st);
  }
  if (err != cudaSuccess) return err;
  for (int it = 0; it < steps; it++) {
    // E = I - B X, complex128-accurate on the tensor cores (X = X0 in the
    // first step, read in complex64)
    GemmDesc g = it == 0 ? plain_gemm(n, n, n, count, Bm, 0, X0, 1, E) : plain_gemm(n, n, n, count, Bm, 0, Xl, 0, E);
    g.C.f32 = 1;  // (accurate to complex128 rounding, then rounded to complex64)
    g.alpha = make_double2(-1.0, 0.0);
    g.addI = 1;
    // (B's digits are the same in every step: split once)
    // (B's digits are in the workspace already: split once, above)
    if ((err = launch_gemm_oz(g, w + L.oz, L.total - L.oz, st, status, true)) != cudaSuccess) return err;
    nl += oz_launches(g, true);
    // X += X0 E: the product in complex64 arithmetic, the addition in FP64
    // (the error of this product is amplified by cond(B) in the next
    // residual, so it stays in elementwise complex64 arithmetic: a 4-slice
    // tensor-core product, accurate relative to row and column maxima only,
    // left 3e-8 in u)
    // (first step: X = X0 + X0 E, the widening of X0 folded into the epilogue)
    GemmDesc c = plain_gemm(n, n, n, count, X0, 1, E, 1, Xl);
    c.cf32 = 1;
    c.wide_epilogue = 1;
    c.D = c.C;
    if (it == 0) c.D = c.A;
    c.beta = make_double2(1.0, 0.0);
    if ((err = launch_gemm(&c, 1, st)) != cudaSuccess) return err;
    nl++;
  }
  // G X = [R | Gamma]
  leaf_GX_kernel<<<count, 256, tsm, st>>>(lt, probs, nprob, leaf0, Xl, GXl);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  nl++;
  if (launches) *launches += nl;
  return cudaSuccess;
}

}  // namespace hps
