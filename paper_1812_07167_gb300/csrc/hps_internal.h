// Internal declarations shared by the CUDA translation units of libhps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace hps {

// Element (i, j) of batch b of a strided, optionally index-mapped complex
// matrix:  ptr[b * stride + (rmap ? rmap[i] : i) + (cmap ? cmap[j] : j) * ld]
// (column-major storage, leading dimension ld).  Elements are complex128
// (double2) or, with f32 set, complex64 (float2).
struct Mat {
  const void *ptr;
  long long ld;
  long long stride;
  const int *rmap;
  const int *cmap;
  int f32;
};

// One batched GEMM:  C = alpha * A * B  + beta * D  (+ I if addI)
// A: M x K, B: K x N (rows k >= ksplit read from B2, row k - ksplit),
// C, D: M x N.  D.ptr may be NULL (then beta is ignored); D may alias C
// element for element.  Operands may be complex128 or complex64 each; the
// arithmetic is complex64 when cf32 is set, complex128 otherwise.
struct GemmDesc {
  int M, N, K, batch;
  Mat A, B, B2;
  int ksplit;
  Mat C, D;
  double2 alpha, beta;
  int addI;
  int cf32;
  // with cf32: alpha AB + beta D (+ I) formed in FP64 from the complex64
  // product (a complex64 correction added to a complex128 matrix)
  int wide_epilogue;
  int cfg;  // tile configuration for N > 8: 0 = by rule, 1..4 = 64x64, 32x32, 16x16, 64x16,
           // 6, 7 = 128x128, 128x64 (complex64 products without index maps)
  // N <= 16: scratch that lets the skinny kernel split K over several CTAs
  // (without it, products with 9 .. 16 columns take the tiled kernel)
  // (partial sums of up to kGemvBlocks row blocks x 16 splits x 32 rows x N,
  // and kGemvBlocks counters that must be zero; the kernel leaves them zero)
  void *part;
  unsigned *cnt;
};
constexpr int kGemvBlocks = 1024;  // row blocks a skinny launch may split (per descriptor)
constexpr int kGemvSlots = 608;    // (row block, split) pairs a split launch has at most (< 4 x 152)
// bytes of the skinny kernel's scratch (two descriptors a launch): counters,
// then partial sums for up to N (rounded up to 1, 2, 4, 8, 16) right-hand sides
inline size_t gemv_scratch_counters() { return 2 * kGemvBlocks * sizeof(unsigned); }
inline int gemv_nn(int N) { return N <= 1 ? 1 : N <= 2 ? 2 : N <= 4 ? 4 : N <= 8 ? 8 : 16; }
inline size_t gemv_part_bytes(int N) { return 2ull * kGemvSlots * 32 * gemv_nn(N) * 16; }

// One batched mapped copy:  dst(i, j) = alpha * src(i, j) for i < M, j < N
// (src(j, i) when trans; += with accumulate), or a fill with zeros when
// src.ptr is NULL.  The
// element types of src and dst may differ (a precision conversion).
struct CopyDesc {
  int M, N, batch;
  Mat src, dst;
  double2 alpha;
  int trans;
  int accumulate;  // dst(i, j) += alpha * src(i, j) instead of =
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
};

// Per-problem data of a leaf launch that covers the leaves of several
// problems (same p; leaves numbered problem after problem).
struct LeafProb {
  const double *tab;  // D1x, D1y, D2x, D2y (p*p each, scaled to the leaf), then int grid[n]
  const double *c;    // [leaves of this problem][ni]
  long long leaf0;    // first leaf of this problem in the launch's numbering
  double2 eta;        // impedance parameter
  double kappa2;      // kappa^2
};

// Device-side status word: 0 = fine; otherwise (code << 28) | (level << 20) | box.
struct DevStatus {
  unsigned int word;
};

// Chained launches: while a LaunchChain is alive on a thread, the GEMM,
// skinny-product, copy and LU-sweep launchers of that thread launch with
// programmatic stream serialization, so a kernel's CTAs may be scheduled
// while the previous kernel on the stream drains; every such kernel waits
// (griddepcontrol.wait) for the previous one to finish before it reads
// anything, so results are unchanged.  Used for the solve's chain of small
// dependent launches.
struct LaunchChain {
  LaunchChain();
  ~LaunchChain();
  bool prev;
};
bool launch_chained();
// launch kern<<<grid, block, smem, st>>>(args...), chained if a LaunchChain is alive
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (launch_chained()) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

#ifdef __CUDACC__
// Start of a kernel that may run chained after the previous one on its
// stream (LaunchChain): wait until that kernel has finished and its writes
// are visible, then let the next kernel be scheduled.  No-ops for a kernel
// launched the ordinary way.
__device__ __forceinline__ void chain_enter() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
#endif

// ---- launchers (return cudaError_t of the launch) ----
cudaError_t launch_gemm(const GemmDesc *descs, int ndesc, cudaStream_t st);

// Complex GEMM emulated on the bf16 tensor cores (Ozaki scheme, slices of 6
// bits per operand: 9 with cf32 == 0, accuracy ~2^-54 max|A_i.| max|B_.j|
// per term; 5 with cf32 set, ~5 2^-29, the accuracy of complex64 arithmetic),
// the slice products by tcgen05.mma from TMA-staged tiles.  Same semantics
// as launch_gemm for one descriptor (the epilogue is always formed in FP64,
// as with wide_epilogue); needs a 256-byte aligned device workspace of
// oz_workspace_bytes(g).  oz_launches(g) launches (4, or
// 5 when the slice pairs are split over several CTAs a tile).  A pipeline
// wait that gives up (2 s) records code 3 in *status (if given) and leaves C
// unspecified.  reuse_a: the workspace already holds A's digits from the
// previous call with the same A and shape (that call's A split is reused;
// 2 launches fewer).
// Per-launch CUDA events around the product kernel (oz_tc_kernel) of the
// tensor-core products launched by this host thread while a timer is set:
// product k records ev[2k] before and ev[2k + 1] after its product kernel on
// the product's stream, and flops[k] = its bf16 slice flops (8 pairs M N K
// batch: 360 M N K batch for 9 slices, 120 for 5).
struct OzTimer {
  cudaEvent_t *ev;  // 2 cap events, created on first use (null until then)
  double *flops;
  int cap, n;
};
void oz_set_timer(OzTimer *t);  // nullptr: stop timing
bool oz_eligible(const GemmDesc &g);
int oz_launches(const GemmDesc &g, bool reuse_a = false);
size_t oz_workspace_bytes(const GemmDesc &g);
cudaError_t launch_gemm_oz(const GemmDesc &g, void *ws, size_t ws_bytes, cudaStream_t st,
                           unsigned *status = nullptr, bool reuse_a = false);
// A's exponents and digits alone (2 launches), for a later launch_gemm_oz
// with reuse_a on the same workspace (the split can then run ahead, on
// another stream, while what B depends on is still being computed).
cudaError_t launch_oz_split_a(const GemmDesc &g, void *ws, size_t ws_bytes, cudaStream_t st);
// One thread runs the products' bounded mbarrier wait on a barrier that
// nothing completes, with a limit of limit_ms: it gives up, records code 3 in
// *status and returns (a check of the failure reporting).
cudaError_t launch_wait_check(unsigned *status, int limit_ms, cudaStream_t st);
cudaError_t launch_copy(const CopyBatch &cb, cudaStream_t st);

// ---- one-launch solves (solve_engine.cu) ----
// An operand of a solve step: element (i, c) of batch entry b is
//   ((char *)base[base] + off)[b stride + c ld + (rmap ? rmap[i] : i)]
// (complex128, or complex64 with f32), base[0] = null (off is the address),
// base[1..4] = the solve's s, t, u and workspace; base = -1: no operand.
struct EnMat {
  long long off, ld, stride;
  const int *rmap;
  int base, f32;
};
// A step: kind 0, y = alpha A x (+ beta D) with A M x K per batch entry
// (column-major, ld A.ld, no maps; rows k >= ksplit of x come from x2), R <= 2
// columns, accumulated in complex64 with cf32; kind 1, y = alpha x (+ y if
// accumulate), M x R per batch entry.  A phase is a run of independent steps
// closed by phase_end; units: the work units of the step (unit0: the first
// within its phase).  Products in nkc > 1 K chunks of kc keep partial sums at
// part_off (complex) and arrival counters at cnt_off.
struct EnOp {
  int kind, M, K, batch, R, ksplit, cf32, accumulate;
  int nrb, nkc, kc, units, unit0, phase_end;
  long long part_off, cnt_off;
  EnMat A, x, x2, y, D;
  double2 alpha, beta;
};
struct EnArgs {
  const EnOp *ops;  // device program
  int nops;
  const void *base[5];
  double2 *part;    // partial sums of split products
  unsigned *cnt;    // their arrival counters (zero on entry, left zero)
  unsigned *bar;    // grid barrier: count, generation, abort (zero on entry)
  unsigned *status;
};
// CTAs of an engine launch (every one resident; 0 if the device cannot run
// it), rows of a product unit, its longest K chunk, elements of a copy unit.
int engine_grid();
int engine_unit_rows();
int engine_max_kc();
int engine_copy_unit();
cudaError_t launch_solve_engine(const EnArgs &a, cudaStream_t st);

// Leaf step (Sec. 2.1) for leaves [leaf0, leaf0 + count): assemble B, invert
// it by blocked Gauss-Jordan with partial pivoting across a cluster of `cs`
// CTAs, write X = B^{-1} = [Psi | Y] ([leaf][n][n] column-major) and
// GX = G X ([leaf][n][nb] column-major: R = GX[:, :nb], Gamma = GX[:, nb:]).
// The arithmetic and X, GX, S are complex64 when f32, complex128 otherwise.
//   probs: device array of nprob problems, ordered by leaf0 (probs[0].leaf0
//          = 0); leaf l belongs to the last problem whose leaf0 <= l
//   S, meta: scratch for `count` matrices: count * n * n complex and
//            count * gj_meta_ints(n) ints
cudaError_t launch_leaf(const LeafTables &lt, const LeafProb *probs, int nprob, long long leaf0,
                        int count, void *X, void *GX, void *S, int *meta, unsigned int *status,
                        int level, int cs, bool f32, cudaStream_t st);

// Leaf step in factored form for leaves [leaf0, leaf0 + count): assemble
// [D B; G], factor P D B = L U by blocked right-looking LU with partial
// pivoting across a cluster of `cs` CTAs (the G rows eliminated along, never
// pivots), then G B^{-1} by a triangular solve of the G rows.  Writes
// X = L \ U ([leaf][n][n] column-major, unit diagonal of L implied),
// GX = G B^{-1} ([leaf][n][nb] column-major), perm ([leaf][n]: row k of P D B
// is row perm[k] of B) and dsc ([leaf][n]: d of row perm[k]).  X, GX and the
// arithmetic are complex64 when f32.  meta: count * lu_meta_ints(n) ints.
cudaError_t launch_leaf_lu(const LeafTables &lt, const LeafProb *probs, int nprob, long long leaf0,
                           int count, void *X, void *GX, int *perm, double *dsc, int *meta,
                           unsigned int *status, int level, int cs, bool f32, cudaStream_t st);
size_t lu_meta_ints(int n);

// Leaf step in inverse form for complex128 leaves by refinement of a
// complex64 inverse (leaf_refine.cu): X0 = B^-1 in complex64 (launch_leaf
// with cluster size cs32), then `steps` times E = I - B X (Ozaki product on
// the tensor cores) and X += X0 E, then GX = G X.  Writes X and GX of leaves
// [leaf0, leaf0 + count) ([leaf][n][n], [leaf][n][nb] column-major, indexed
// by the absolute leaf number, like launch_leaf).  scr: 256-byte aligned
// device scratch of leaf_refined_scratch_bytes(lt, count).  *launches is
// increased by the kernels launched, leaf_refined_launches(lt, count, steps).
// Complex64 inverse of the leaf matrices, one CTA a leaf, 32-column panels
// (leaf_gj32.cu): X0 = (D B)^{-1} D of leaves [leaf0, leaf0 + count) into X0
// ([leaf][n][n] complex64 column-major, by absolute leaf number) and, if GX
// is not null, G X0 into GX ([leaf][n][nb]), with the scratch S
// ([count][n][n] complex64).  For n <= 384 (gj32_supported); a zero pivot
// records code 1 in *status.
bool gj32_supported(const LeafTables &lt);
size_t gj32_smem_bytes(const LeafTables &lt);
cudaError_t launch_leaf_gj32(const LeafTables &lt, const LeafProb *probs, int nprob, long long leaf0, int count,
                             void *X0, void *GX, void *S, unsigned int *status, int level, cudaStream_t st);
size_t leaf_refined_scratch_bytes(const LeafTables &lt, int count);
// A second stream of st's device and priority, for work that can run beside
// st's (one a host thread, device and priority; null if it cannot be made).
cudaStream_t side_stream(cudaStream_t st);
int leaf_refined_launches(const LeafTables &lt, int count, int steps);
cudaError_t launch_leaf_refined(const LeafTables &lt, const LeafProb *probs, int nprob, long long leaf0, int count,
                                void *X, void *GX, void *scr, size_t scr_bytes, unsigned int *status, int level,
                                int cs32, int steps, cudaStream_t st, int *launches);
size_t lu_leaf_smem_bytes(int n, int nb, int p, int cs, bool f32);

// u = B^{-1} [t; s] for `leaves` leaves from their factors (launch_leaf_lu)
// and R right-hand sides: element i < nb of the right-hand side c of leaf l
// is t[c t_ld + l t_stride + i], element i >= nb is s[c s_ld + l s_stride +
// i - nb]; u[c u_ld + l u_stride + i] receives the solution.  Vectors are
// complex128; the sweeps run in the factors' precision.
cudaError_t launch_lu_solve(const void *LU, const int *perm, const double *dsc, long long leaves, int n,
                            int nb, int R, const double2 *t, long long t_ld, long long t_stride,
                            const double2 *s, long long s_ld, long long s_stride, double2 *u,
                            long long u_ld, long long u_stride, bool f32, cudaStream_t st);
// One stage of a blocked solve on the rows [r0, r1) of every leaf: with
// gather, u = P D [t; s] on all n rows first (rows outside the range straight
// to u), else the rows [r0, r1) are read from u; then the forward (L) and/or
// backward (U) sweep with the diagonal block of those rows only, written
// back to u.  The products with the off-diagonal blocks are the caller's.
cudaError_t launch_lu_solve_part(const void *LU, const int *perm, const double *dsc, long long leaves, int n,
                                 int nb, int R, const double2 *t, long long t_ld, long long t_stride,
                                 const double2 *s, long long s_ld, long long s_stride, double2 *u,
                                 long long u_ld, long long u_stride, bool f32, int r0, int r1, bool gather,
                                 bool fwd, bool bwd, cudaStream_t st);

// Inverse of `batch` n x n column-major matrices (leading dim n, batch stride
// n*n) by blocked Gauss-Jordan with partial pivoting across clusters of `cs`
// CTAs.  S holds the matrices and is destroyed; the inverses go to out.  With
// tglobal the panels are read in place from S (large n) instead of being
// staged in shared memory; with f32 everything is complex64.
// kb: panel width, 8 or 4 (4 halves the serial FP64 work a panel on the
// owning CTA, for few large matrices).
cudaError_t launch_gj_inverse(void *S, void *out, int n, int batch, int *meta, unsigned int *status,
                              int level, int cs, bool tglobal, bool f32, cudaStream_t st, int kb = 8);

// ---- complex128 residual of the global collocation system (refinement) ----
constexpr int kMaxLevels = 24;
struct ResidualLevel {
  const int *pairs;  // [n3][4]: (leaf in parent, node) of the alpha end, then beta's
  int n3, lpp;       // pairs per parent, leaves per parent
  long long off;     // offset of the level's pairs in the flat jump arrays
};
struct ResidualSetup {
  const double *tab;  // leaf tables: D1x, D1y, D2x, D2y, grid[n], loc[p*p]
  const double *c;    // [leaves][ni]
  int p, e, n, nb, ni, leaves, nbdry;
  double2 eta;
  double kappa2;
  const int *outer;   // public boundary index -> leaf * nb + node
  long long total_pairs;
  int nlev;
  ResidualLevel lev[kMaxLevels];
};
// For R right-hand sides: sd = s - A u on every leaf's interior rows; Fu, Gu
// = F u, G u at every leaf's boundary nodes; td = t - F u on the outer
// boundary; JA = -(F^a u^a + G^b u^b), JB = -(G^a u^a + F^b u^b) at every I3
// pair (Sec. 2.2's t3a = -g3b, g3a = -t3b).
cudaError_t launch_residual(const ResidualSetup &rs, const double2 *u, const double2 *s,
                            const double2 *t, double2 *sd, double2 *td, double2 *Fu, double2 *Gu,
                            double2 *JA, double2 *JB, int R, cudaStream_t st);

// The same inverse for few, larger matrices: one launch per 8-column panel
// over batch * G CTAs (CTA 0 of a matrix eliminates the next panel, the
// others update slabs of columns), so a single matrix uses the whole chip.
cudaError_t launch_gj_wide(void *S, void *out, int n, int batch, int G, int *meta,
                           unsigned int *status, int level, bool f32, cudaStream_t st, int kb = 8);
size_t gj_wide_smem_bytes(int n, int slab, bool f32, bool tglobal, int kb = 8);
int gj_wide_launches(int n, int kb);

// Cluster limits and scratch / shared-memory sizes of the Gauss-Jordan kernels.
int gj_max_cluster();
int gj_slab(int n, int cs, int kb = 8);
size_t gj_smem_bytes(int n, int cs, bool leaf, int p, bool tglobal = false, bool f32 = false, int kb = 8);
size_t gj_meta_ints(int n);  // enough for either panel width

}  // namespace hps
