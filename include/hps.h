/*
 * hps.h -- C ABI of the GB300 HPS direct solver for the 2-D variable
 * coefficient Helmholtz impedance problem
 *
 *     -Lap u(x) - kappa^2 c(x) u(x) = s(x)    x in Omega = [x0,x1] x [y0,y1]
 *     du/dnu + i eta u = t(x)                 x on the boundary of Omega
 *
 * (arXiv:1812.07167, Eq. (1); Re(eta) != 0).  The method is the
 * Hierarchical Poincare-Steklov (HPS) scheme of that paper: per-leaf
 * corner-free Chebyshev collocation (Sec. 2.1), level-by-level merges of
 * impedance-to-impedance (ItI) operators (Sec. 2.2, Algorithm 1), and a
 * solve made of an upward and a downward sweep (Algorithm 2), with the
 * operators stored as in Sec. 2.4.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Complex numbers are interleaved (re, im) pairs of doubles (C99
 * double complex / CUDA double2 layout).  Arrays are dense and C-ordered as
 * written ([a][b] means index b runs fastest).
 *
 * Leaves: the domain is cut into mx x my equal rectangles (powers of two).
 * The merges of the tree alternate, from the leaves up, between joining
 * west/east neighbours and joining south/north neighbours, starting west/east;
 * once one axis has no halvings left the other takes the remaining merges.
 * Bit k of a leaf index belongs to merge k: the bits of west/east merges form
 * the leaf's column (x), the others its row (y).  For mx == my this is the
 * Morton order: bit 2i of the leaf index is bit i of the column, bit 2i+1
 * bit i of the row.
 *
 * Nodes: each leaf carries the p x p Chebyshev tensor grid with its four
 * corners dropped (p^2 - 4 nodes, Sec. 2.1), ordered
 *     [south edge, east edge, north edge, west edge, interior]
 * where each edge holds the p-2 non-corner nodes in increasing coordinate and
 * the (p-2)^2 interior nodes run row by row, x fastest.  Nodes on an edge
 * shared by two leaves appear once per leaf.
 *
 * Outer boundary: 2 (mx + my) qe nodes ordered [south, east, north, west]
 * (mx, my, mx, my leaf edges), each side in increasing coordinate (the
 * concatenation of the leaves' edges); qe = p-2 corner-free Chebyshev nodes
 * per leaf edge, or q Gauss-Legendre nodes (see hps_desc.q).
 *
 * Memory: every array argument may be host or device memory; the library
 * asks the CUDA runtime which.  Device arrays are used in place; host arrays
 * are staged through device buffers owned by the handle.  The caller keeps
 * ownership of every array it passes; the handle owns all operators.
 *
 * Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 * Work is enqueued on it in stream order.  Calls whose outputs are host
 * memory return after the outputs are written; calls with device outputs
 * return once the work is enqueued.  A handle must not be used from two
 * host threads at the same time.
 *
 * Devices: a handle's operators live on the device that was current when it
 * was built; hps_solve, hps_solve_batch, hps_solve_noalloc and hps_reserve
 * return HPS_EINVAL when another device is current.
 *
 * Errors: every call returns one of the HPS_* codes below; nothing aborts
 * and no kernel traps.  Numerical failures found on the device (an exactly
 * zero pivot) are recorded in the handle and reported by hps_status().
 */
#ifndef HPS_H
#define HPS_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  HPS_OK = 0,
  HPS_EINVAL = 1,    /* an argument is out of range (see each call) */
  HPS_ENOMEM = 2,    /* a device allocation failed or the handle's memory cap was hit */
  HPS_ESINGULAR = 3, /* a leaf matrix B or an interface matrix W had a zero pivot */
  HPS_ETIMEOUT = 4,  /* a bounded device wait gave up (the tensor-core product's
                        pipeline waits, 2 s each; reported by hps_status) */
  HPS_ECUDA = 5,     /* a CUDA runtime call failed (no device, launch error, ...) */
  HPS_ENOTSUP = 6,   /* a valid request the kernels cannot run (sizes; see each call) */
  HPS_ETOOBIG = 7    /* the request needs more than the fixed no-allocation workspace */
};

enum { HPS_FP64 = 0, HPS_MIXED = 1 };
enum { HPS_LEAF_LU = 0, HPS_LEAF_INVERSE = 1 };

typedef struct {
  double x0, x1, y0, y1; /* the rectangle Omega, x1 > x0, y1 > y0 */
  int mx, my;            /* leaves along x and along y: powers of two, 1 .. 1024,
                            mx my <= 2^20 */
  int p;                 /* Chebyshev nodes per leaf side (the paper's n_c), 4 .. 32 */
  int q;                 /* points per leaf edge for boundary data.  0 or p-2: the
                            corner-free Chebyshev edge nodes of Sec. 2.1 (the paper's
                            scheme).  1 .. 64 otherwise: q Gauss-Legendre nodes per
                            leaf edge, the interface of the earlier ItI work the paper
                            cites in Sec. 1: each leaf's incoming data reach its
                            Chebyshev edge nodes through the degree q-1 interpolant
                            of the Gauss values, and its outgoing data leave as the
                            Chebyshev interpolant evaluated at the Gauss nodes, so
                            the merges and the solve run on the Gauss nodes.  For
                            q > p-2 the solution is the Chebyshev scheme's (the data
                            stay polynomials of degree p-3 per edge); for q < p-2 the
                            interface space is coarser.  Then t and the root R are on
                            the Gauss nodes (hps_nodes lists them), HPS_MIXED is
                            HPS_ENOTSUP and a batch shares one q.  Other values:
                            HPS_EINVAL. */
  double kappa;          /* wave number, > 0 */
  double eta_re, eta_im; /* impedance parameter eta, Re(eta) != 0 */
  int precision;         /* HPS_FP64: complex128 throughout.
                            HPS_MIXED: leaves and the merge levels below the top
                            fp64_levels in complex64, the top levels (their
                            interface inverses W^{-1}, whose conditioning grows
                            with kappa) in complex128; every solve is refined in
                            complex128 against the residual of the global
                            collocation system (see hps_solve). */
  int fp64_levels;       /* HPS_MIXED: merge levels kept in complex128, counted
                            from the root; 0 = 4 (clamped to the tree depth) */
  int refine_steps;      /* HPS_MIXED: refinement steps per solve; 0 = 2, < 0 = none */
  int fp64_native;       /* 0: complex128 merge products large enough to pay for it
                            (K >= 64, M, N >= 32, M N K batch >= 2^26) are done by
                            the Ozaki scheme on the bf16 tensor cores (9 slices of 6
                            bits per operand, exact FP32 accumulation of the slice products,
                            complex128 sums: error ~2^-54 max|A_i.| max|B_.j| per
                            term); 1: every complex128 product on the FP64 pipes */
  int leaf_form;         /* how the leaf solution operator [Psi | Y] = B^{-1} of Sec. 2.1 is
                            stored (both give the same operators up to rounding):
                            HPS_LEAF_LU: the factors P D B = L U (row pivoting P, a
                            power-of-two row scaling D), about 0.55 of the leaf
                            flops; a solve applies them by two triangular sweeps.
                            HPS_LEAF_INVERSE: B^{-1} itself (Gauss-Jordan); a solve
                            applies it as a product, which runs on the tensor cores
                            for 32+ right-hand sides unless fp64_native. */
} hps_desc;

typedef struct hps_handle hps_handle;

typedef struct {
  int leaves;               /* mx * my */
  int levels;               /* merge levels (log2 mx + log2 my) */
  int n_leaf;               /* p^2 - 4 nodes per leaf */
  int n_bdry;               /* 2 (mx + my) (p-2) outer boundary nodes */
  long long dof;            /* leaves * (p^2 - 4) */
  long long operator_bytes; /* device bytes of stored operators (Sec. 2.4) */
  long long build_flops;    /* real floating-point operations of one build */
  long long solve_flops;    /* real floating-point operations of one solve, per RHS */
  long long solve_bytes;    /* operator bytes one solve reads */
  int build_launches;       /* kernels one hps_build launches */
  int solve_launches;       /* kernels one hps_solve launches */
  long long build_scratch_bytes; /* transient device memory a build needs on top of
                                    operator_bytes (released when it finishes) */
  long long solve_ws_bytes_per_rhs; /* solve workspace per right-hand side */
} hps_info_t;

/* Node coordinates (host helper, no device work; Sec. 2.1 grid).
 *   leaf_xy: [leaves][p^2-4][2] (x, y) of every leaf node, or NULL
 *   bdry_xy: [2 (mx + my) qe][2] outer boundary nodes (see hps_desc.q), or NULL
 * Both are host memory.  Returns HPS_EINVAL for an invalid descriptor. */
int hps_nodes(const hps_desc *desc, double *leaf_xy, double *bdry_xy);

/* Build the direct solver (Algorithm 1 with the leaf step of Sec. 2.1 and the
 * merge of Sec. 2.2): leaf operators Psi, Y, Gamma for every leaf, then per
 * merge level W^{-1}, R33a, R33b, R13a, R23b, Phi_a, Phi_b, up to the root
 * ItI operator.
 *   c:    [leaves][(p-2)^2] real c(x) at each leaf's interior nodes (the
 *         boundary rows of the leaf system do not involve c), finite; a
 *         host array with a NaN or infinity is HPS_EINVAL (device arrays
 *         are not scanned: non-finite values there give non-finite operators)
 *   out:  receives the new handle; unchanged on failure
 * Device memory for all operators is allocated here and owned by the handle.
 * Returns HPS_EINVAL (bad descriptor, NULL c/out), HPS_ENOMEM, HPS_ECUDA, or
 * HPS_ENOTSUP when a leaf matrix or an interface of the tree is too large
 * for the kernels' shared memory (p > 25; more than 512 leaves a side at
 * p = 16, more than 256 at p = 24), before any device work. */
int hps_build(const hps_desc *desc, const double *c, void *stream, hps_handle **out);

/* Build nprob independent solvers together (a ragged batch): Algorithm 1
 * for every problem, with the leaves of all problems in one leaf launch and
 * each merge level done once for every problem that has it.  The merge
 * sizes of level j (counted from the leaves) depend on j and p only, so the
 * problems' parents on that level form one batch of equal-size merges.
 *   descs[k], c[k]: problem k as for hps_build.  Every desc must have the
 *     same p, precision, fp64_levels, fp64_native and leaf_form (HPS_EINVAL otherwise); m, the
 *     domain, kappa and eta may differ.
 *   out[k] receives problem k's handle.  The handles share one device
 *     allocation, released with the last of them; hps_free each one.
 * A merge level runs as one launch per kernel over its problems, or as up
 * to three where its problems differ in precision (HPS_MIXED) or some of
 * them end at that level (their roots).  hps_status on any handle of the
 * batch reports the batch's first failure; hps_build_times reports the
 * batch's phases.  Results equal those of separate hps_build calls up to the
 * summation order of the kernel shapes chosen for the batch.  Same errors as
 * hps_build; on error no handle is returned. */
int hps_build_batch(int nprob, const hps_desc *descs, const double *const *c, void *stream,
                    hps_handle **out);

/* Rebuild for new coefficients: recompute every operator of a build (all nh
 * handles one hps_build or hps_build_batch returned, in any order) from new
 * samples c[k] of problem k's c, with the same geometry, p, kappa, eta and
 * precision (Algorithm 1 again, into the same device memory).  The build's
 * launch sequence is captured into a CUDA graph by the first call and
 * replayed by every later one, so a rebuild costs one graph launch on top of
 * the copies of c.
 *   c[k]: [leaves][(p-2)^2] of hs[k], device or host memory (finite, as for
 *         hps_build).
 * Work that used the old operators must be ordered before the call (same
 * stream, or events).  hps_build_times keeps the first build's phases.
 * Returns HPS_EINVAL (not exactly the build's handles, a handle of the build
 * already freed, NULL arrays), HPS_ECUDA. */
int hps_rebuild(int nh, hps_handle *const *hs, const double *const *c, void *stream);

/* Solve for nrhs right-hand sides (Algorithm 2: upward then downward pass).
 * For an HPS_MIXED handle the solve is iterative refinement: u = S(s, t), then
 * refine_steps times: the residual of the global collocation system (every
 * leaf's interior rows, the impedance rows F u = t on the outer boundary and,
 * at every pair of coincident nodes on a shared edge, the two conditions
 * t3a = -g3b, g3a = -t3b of Sec. 2.2) is formed in complex128 and the
 * correction S(residual) added, where S is Algorithm 2 on the mixed
 * operators with the interface residuals injected into h3 at the merge whose
 * interface holds them.
 *   s: [nrhs][leaves][(p-2)^2] complex body load at the interior nodes
 *   t: [nrhs][2 (mx + my) qe] complex impedance data du/dnu + i eta u on the
 *      outer boundary
 *   u: [nrhs][leaves][p^2-4] complex solution at every leaf node (written)
 * nrhs == 0 does nothing and returns HPS_OK.  With the environment variable
 * HPS_SOLVE_ENGINE=1, a solve with 1 or 2 right-hand sides runs as one
 * persistent cooperative launch over a program recorded for the handle at
 * the first such call (kept until hps_free; a pipeline wait that gives up
 * after 2 s reports HPS_ETIMEOUT through hps_status); by default the steps
 * are separate launches, which measured faster.  Returns HPS_EINVAL (NULL
 * handle or array, nrhs < 0), HPS_ENOMEM (workspace), HPS_ECUDA. */
int hps_solve(hps_handle *h, const double *s, const double *t, double *u, int nrhs, void *stream);

/* Several independent solve requests against one handle, done as ONE pass
 * of Algorithm 2 whose right-hand sides are the requests' side by side
 * (R = nrhs[0] + ... + nrhs[nreq-1] columns): the operators are read once for
 * the whole batch.  This is the continuous-batching step of a request loop.
 *   s[k], t[k], u[k]: request k's arrays in the layouts of hps_solve with
 *     nrhs[k] right-hand sides; device or host memory, in any mix.  They are
 *     gathered into the handle's staging buffer by copies on `stream`, and
 *     each u[k] is written back from it.
 *   nrhs[k] >= 0; requests with nrhs[k] == 0 are skipped.
 * Column r of request k gives the same u as solving request k alone, up to
 * the summation order of the kernels chosen for the batch width.  Every call
 * on one handle must be ordered with the others (one stream per handle, or
 * events): the staging and workspace belong to the handle.  When every
 * pointer is device memory the call only enqueues; otherwise it waits for the
 * stream before returning.  Returns HPS_EINVAL (NULL handle or array for a
 * request with nrhs[k] > 0, nreq < 0, nrhs[k] < 0), HPS_ENOMEM, HPS_ECUDA. */
int hps_solve_batch(hps_handle *h, int nreq, const double *const *s, const double *const *t,
                    double *const *u, const int *nrhs, void *stream);

/* Allocate now the handle's solve workspace and staging for calls of up to
 * nrhs right-hand sides in total, so that such later hps_solve and
 * hps_solve_batch calls allocate nothing (cudaMalloc/cudaFree synchronize the
 * device, which stalls other streams' work).  Returns HPS_EINVAL for nrhs < 0,
 * HPS_ENOMEM. */
int hps_reserve(hps_handle *h, int nrhs);

/* Size of the fixed device workspace behind hps_solve_noalloc (16 MiB).  It
 * is part of the library's device image, so every GPU that loads the library
 * holds it until the process exits. */
#define HPS_NOALLOC_WORKSPACE_BYTES (16u << 20)

/* The same solve as hps_solve, for callers that cannot allocate device
 * memory at solve time: code whose device memory is already handed out to a
 * pool or framework allocator up front, and latency-bound request loops where
 * a cudaMalloc (which may synchronize the device, and may fail at run time)
 * is not acceptable.  It allocates nothing: the solve's scratch vectors live
 * in a fixed file-scope device array of HPS_NOALLOC_WORKSPACE_BYTES.
 * The paper has no counterpart; this is a deployment variant of Algorithm 2.
 *   s, t, u: as for hps_solve, but all three must be device memory (host
 *            arrays would need staging buffers): HPS_EINVAL otherwise.
 * HPS_MIXED handles are refused (HPS_ENOTSUP): their refinement needs more
 * workspace than the array holds.
 * Returns HPS_ETOOBIG when nrhs right-hand sides of this handle's tree need
 * more workspace than the array holds (about 1.8 MB per right-hand side for
 * 16 x 16 leaves with p = 16, plus 0.6 to 10 MB for the partial sums of the
 * skinny products of up to 16 right-hand sides), HPS_EINVAL for bad
 * arguments, HPS_ECUDA if the
 * workspace address cannot be obtained.  nrhs == 0 returns HPS_OK.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the one array, which keeps what the last call
 * left in it: calls whose work overlaps on the GPU (different streams, or
 * different handles, without ordering between them) race on it and must be
 * serialized by the caller; such a race gives wrong solutions for the calls
 * involved.  The solve vectors in the array are written before they are
 * read; the arrival counters of the split skinny products at its head must
 * start at zero, and every call clears them (a cudaMemsetAsync on `stream`,
 * which allocates nothing) before its first launch, so a race does not
 * carry over into later, ordered calls.
 * Returns HPS_EINVAL when the current device is not the one the handle was
 * built on. */
int hps_solve_noalloc(hps_handle *h, const double *s, const double *t, double *u, int nrhs,
                      void *stream);

/* The root ItI operator R (Definition of the ItI map; R f = g on the outer
 * boundary) in the outer-boundary order above.  With Gauss-Legendre boundary
 * data (hps_desc.q != p-2) R is on those nodes and gauss_basis must be 1
 * (0 is HPS_EINVAL).
 *   R: [nb][nb] complex with nb = 2 (mx + my) (p-2), row-major (R[i][j] maps incoming data
 *      at node j to outgoing data at node i); host or device memory
 *   gauss_basis: 0 = R on the corner-free Chebyshev edge nodes (the basis the
 *      solver works in); 1 = R_G = diag(P) R diag(P)^-1 on q = p-2 Gauss-Legendre
 *      nodes per edge, P the polynomial interpolation from an edge's Chebyshev
 *      nodes to its Gauss-Legendre nodes (an exact change of basis, since both
 *      sets have p-2 points; the Gauss nodes of an edge run in increasing
 *      coordinate like its Chebyshev nodes).  The change of basis runs on the
 *      device in two batched products and takes a temporary of nb^2 complex.
 * The root R is the last merge's product; the build keeps it.  Returns
 * HPS_EINVAL (null h or R, gauss_basis not 0 or 1), HPS_ENOMEM or HPS_ECUDA. */
int hps_root_R(hps_handle *h, double *R, int gauss_basis, void *stream);

/* Operators of one leaf (Sec. 2.1.1, 2.1.2, 2.4), for inspection.
 *   Psi: [p^2-4][4(p-2)], Y: [p^2-4][(p-2)^2], Gam: [4(p-2)][(p-2)^2], each
 *   complex row-major; any may be NULL; host or device memory.
 * In HPS_LEAF_LU form Psi and Y (the columns of B^{-1}) are not stored: they
 * are formed here by solving with the leaf's factors for every unit vector
 * (in the leaves' precision), with a temporary device allocation of
 * 3 (p^2-4)^2 complex values.  Synchronizes the stream.
 * Returns HPS_EINVAL for a leaf index out of range, HPS_ECUDA. */
int hps_leaf_ops(hps_handle *h, int leaf, double *Psi, double *Y, double *Gam, void *stream);

/* Batched complex GEMM C = A B with the library's product kernels (a
 * diagnostic of them): batch matrices, column-major and densely strided
 * (A: M x K, B: K x N, C: M x N; batch strides M K, K N, M N elements).
 * emulated = 0: complex128 on the FP64 pipes; 1: the Ozaki scheme on the
 * bf16 tensor cores, as the build runs its large complex128 merge products
 * (9 slices of 6 bits an operand, error ~2^-54 max|A_i.| max|B_.j| a term);
 * 2: the same with 5 slices, as the build runs its complex64 products (the
 * mixed path's lower levels): error ~5 2^-29 max|A_i.| max|B_.j| a term, the
 * accuracy of complex64 arithmetic; 3: complex64 arithmetic on the FP32
 * pipes (operands rounded to complex64, results widened), the kernel the
 * refinement corrections take (any size is accepted here).  Device arrays
 * only; enqueued on `stream`.
 * Returns HPS_EINVAL (sizes < 1, NULL or host arrays, emulated not 0 .. 3),
 * HPS_ENOMEM (workspace), HPS_ECUDA. */
int hps_zgemm(int M, int N, int K, int batch, const double *A, const double *B, double *C, int emulated,
              void *stream);

/* Batched inverse of complex128 matrices with the library's interface-inverse
 * kernels (Sec. 2.2's W^{-1}: Gauss-Jordan elimination with partial pivoting
 * in panels of 8 (or 4) columns, one CTA or thread-block cluster a matrix, or,
 * when the batch is too small to fill the device, one launch a panel over
 * CTAs that share each matrix).  A: batch n x n matrices, column-major,
 * complex128 interleaved (re, im), batch stride n^2 complex, device memory,
 * read only (a copy is eliminated); Ainv: the same layout, device memory,
 * written (it may be A itself).
 * mode = 0: the elimination in complex128.  mode = 1: the regime a build takes
 * for this (n, batch): where the elimination would be a chain of per-panel
 * launches, a complex64 inverse refined by two complex128 residual steps
 * (E = I - A X on the tensor cores or the FP64 pipes, X += X0 E), which
 * reaches complex128 accuracy for matrices whose entries complex64 represents
 * and whose condition number is far below 1e7 (the interface matrices: < 100).
 * Returns HPS_OK; HPS_ESINGULAR when an elimination met an exactly zero pivot
 * column (*bad, when not NULL, receives the index of the matrix the device
 * recorded first; that matrix's Ainv is unspecified, the others are valid);
 * HPS_EINVAL (n < 2, batch < 1 or > 2^20, mode not 0 or 1, NULL or host
 * arrays, or no regime of the kernels fits this n); HPS_ENOMEM (scratch of
 * about 16 n^2 batch bytes, three times that with mode 1); HPS_ETIMEOUT (a wait
 * of the tensor-core residual gave up); HPS_ECUDA.  Synchronizes the stream
 * (it reads the device status word).  *bad = -1 unless HPS_ESINGULAR. */
int hps_zinv(int n, int batch, const double *A, double *Ainv, int mode, int *bad, void *stream);

/* A check of the device-side failure reporting that needs no failing
 * computation: one thread of one CTA runs the tensor-core product's bounded
 * pipeline wait (the mbarrier wait with a time limit) on a barrier that
 * nothing completes, with a limit of limit_ms milliseconds instead of the
 * products' 2 s.  The wait gives up, records a timeout in a status word and
 * the kernel returns, leaving the context usable.  Returns HPS_ETIMEOUT (the
 * expected result), HPS_OK only if the wait completed, HPS_EINVAL (limit_ms
 * not in 1 .. 2000), HPS_ENOMEM, HPS_ECUDA.  Synchronizes the stream. */
int hps_check_wait(int limit_ms, void *stream);

/* The FP64 fused multiply-add rate of the current device, measured: a
 * kernel of independent FMA chains on every SM, timed with CUDA events on
 * `stream` (best of 3 after a warm-up, about 20 ms each).  *tflops receives
 * TFLOP/s (2 flop an FMA).  A diagnostic beside the solver, for the roofline
 * of its complex128 kernels on the FMA pipes; the paper has no counterpart.
 * Synchronizes the stream.  Returns HPS_EINVAL (NULL tflops), HPS_ECUDA. */
int hps_fp64_rate(double *tflops, void *stream);

/* Measure, on this GPU, the kernel choices the builds of these problems would
 * make, and keep the fastest for every later build in this process: for each
 * merge product shape (M, N, K, parents, precision) the tile configuration
 * or the tensor-core product, for each interface-inverse shape (n3, parents,
 * precision) the cluster size or the panel-per-launch regime.  This is the
 * GPU form of the paper's calibration of representative actions (Sec. 3,
 * Table 1, which times a leaf inverse, an interface inverse and a product
 * per level and thread count).  Shapes measured before are skipped.
 *   descs: as for hps_build_batch (the same p, precision, fp64_levels, leaf_form and
 *          fp64_native); their shapes are measured on scratch data.
 *   ntuned: optional, receives the number of shapes measured.
 * With the environment variable HPS_TUNE_CACHE naming a file, the choices
 * found there are taken without measuring and all choices are written back
 * after measuring (text, one shape a line), so that another process makes
 * the same choices.  Synchronizes the stream.  Returns HPS_EINVAL,
 * HPS_ENOTSUP, HPS_ENOMEM, HPS_ECUDA. */
int hps_tune(int nprob, const hps_desc *descs, void *stream, int *ntuned);

/* Sizes and operation counts of the solver hps_build would create for desc,
 * without building it (host only, no device work): the admission check of a
 * request loop.  Same HPS_EINVAL / HPS_ENOTSUP results as hps_build. */
int hps_plan(const hps_desc *desc, hps_info_t *info);

/* Sizes and operation counts of a built handle (host only, no device work). */
int hps_info(const hps_handle *h, hps_info_t *info);

/* Device time of the phases of the handle's build, from CUDA events the
 * build recorded on its stream: ms[0] = the leaf kernel (Sec. 2.1), ms[1+j] =
 * merge level j counted from the leaves up (Sec. 2.2).  Writes at most cap
 * values and returns how many phases there are (1 + levels), or a negative
 * HPS_* code.  Waits for the build to finish. */
int hps_build_times(hps_handle *h, double *ms, int cap);

/* Device time of each tensor-core product kernel of the handle's build (the
 * complex128 products done by the Ozaki scheme, hps_desc.fp64_native == 0),
 * from CUDA events the build recorded on its stream around those kernels
 * alone (not the digit splits): ms[k] and flops[k] = the product's bf16 slice
 * flops (45 slice pairs x 4 real products x 2 M N K), in launch order, for
 * the measurement of that kernel against its roofline.  Writes at most cap
 * of each and returns how many products the build timed (the first 256), or
 * a negative HPS_* code.  Waits for them to finish.  A diagnostic; the paper
 * has no counterpart. */
int hps_build_product_times(hps_handle *h, double *ms, double *flops, int cap);

/* Wait for the handle's work on `stream` and report device-side failures:
 * HPS_ESINGULAR with *level / *box (may be NULL) set to the tree level
 * (leaf level = levels) and box index of the first zero pivot;
 * HPS_ETIMEOUT when a wait inside a tensor-core product gave up (its
 * results are then unspecified; *box = the output tile); or HPS_OK. */
int hps_status(hps_handle *h, void *stream, int *level, int *box);

/* Release the handle and all its device memory.  NULL is allowed. */
int hps_free(hps_handle *h);

/* Static description of an error code. */
const char *hps_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* HPS_H */
