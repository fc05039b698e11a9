// C ABI of the HPS solver (include/hps.h): argument checks, the host-side
// tree planner (index maps per merge level), device memory ownership, and the
// per-level launch sequences of the build (Algorithm 1 / Sec. 2.2) and the
// solve (Algorithm 2).
//
// Tree: m x m leaves in Morton order (x bit lowest); level L = 2 log2 m holds
// the leaves, level 0 the root; the parent of box j on level l+1 is box j/2 on
// level l, alpha = child 2j, beta = child 2j+1.  The merge into level l is
// horizontal (alpha west, beta east, shared vertical edge) when L-1-l is
// even and vertical (alpha south, beta north) otherwise, so the first merge
// above the leaves is horizontal as in Fig. 3 of the paper.
//
// Every box keeps its boundary nodes in the order [I1, I2] that the merge of
// Sec. 2.2 produces (leaves: [S, E, N, W]).  The planner tracks, for every
// position of that order, the side and the offset along the side, and
// derives I1, I2, I3 from it; no reordering pass runs on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "hps.h"
#include "hps_internal.h"

using hps::CopyBatch;
using hps::CopyDesc;
using hps::GemmDesc;
using hps::Mat;

namespace {

struct Canon {
  int side;  // 0 S, 1 E, 2 N, 3 W
  int off;   // offset along the side, in nodes
};

struct Level {
  int lev;         // tree level of the parents
  int P;           // parents on this level
  int horizontal;  // 1: alpha west / beta east
  int nc;          // boundary length of each child
  int n1, n2, n3, nt;
  int f32;         // operators and arithmetic of this level in complex64
  std::vector<int> I1, I2, I3a, I3b;  // positions in the children's orders
  int *d_I1 = nullptr, *d_I2 = nullptr, *d_I3a = nullptr, *d_I3b = nullptr;
  // the leaf and node of both ends of every I3 pair, relative to the parent:
  // [k][4] = (leaf in parent, node in leaf) of alpha's end, then beta's
  std::vector<int> pairs;
  int *d_pairs = nullptr;
  int leaves_per_parent;
  long long jump_off;  // offset of this level's pairs in the flat jump arrays
  // stored operators, per parent contiguous (Sec. 2.4)
  void *Winv = nullptr, *R33a = nullptr, *R33b = nullptr, *R13a = nullptr, *R23b = nullptr;
  void *Phia = nullptr, *Phib = nullptr;
};

constexpr int kLeafRefineSteps = 2;  // refinement steps of the complex64 leaf inverse

struct Plan {
  int m, my, p, e, n, nb, ni, L, leaves, nbdry;  // m: leaves along x, my: along y
  // boundary data points per leaf edge: e (the corner-free Chebyshev nodes),
  // or q Gauss-Legendre nodes (gauss); nbi = 4 qe per leaf
  int qe, nbi;
  bool gauss;
  bool mixed;                   // HPS_MIXED
  int leaf_f32;                 // leaf operators in complex64
  bool leaf_lu;                 // leaf operators as LU factors (else B^{-1})
  bool leaf_refined;            // complex128 B^{-1} by a refined complex64 inverse (else Gauss-Jordan)
  int refine_steps;             // refinement steps of a mixed solve
  bool oz;                      // large complex128 merge products on the tensor cores
  std::vector<Level> lv;        // lv[j]: merge j from the leaves up (parents on level L-1-j)
  std::vector<int> root_src;    // root position -> public boundary index
  std::vector<int> outer;       // public boundary index -> leaf * nb + node
  long long total_pairs = 0;    // I3 pairs over all merges
};

long long cplx_bytes(long long count, int f32 = 0) { return (f32 ? 8LL : 16LL) * count; }

}  // namespace

// Device memory of one build: operators, tables and index maps of one
// problem, or of every problem of a batch (hps_build_batch).  Released with
// the last handle that refers to it.
struct Shared {
  void *arena = nullptr;
  size_t bytes = 0;
  int refs = 0;                 // handles referring to it (guarded by g_shared_mu)
  std::vector<cudaEvent_t> ev;  // [before leaves, after leaves, after merge 0, ...]
  int launches = 0;             // kernels the build launched
  // the build's device work (reads c and every table from the arena), for
  // hps_rebuild, and its captured graph
  std::function<int(cudaStream_t, bool, int &)> compute;
  cudaGraphExec_t graph = nullptr;
  std::vector<hps_handle *> order;  // the handles in build order
  // the build's tensor-core products: events around each product kernel
  static constexpr int kOzTimed = 256;
  std::vector<cudaEvent_t> oz_ev;
  std::vector<double> oz_flops;
  int oz_n = 0;
};
static std::mutex g_shared_mu;

struct hps_handle {
  hps_desc desc;
  Plan plan;
  hps_info_t info;
  Shared *sh = nullptr;
  void *X = nullptr, *GX = nullptr;  // leaf operators (complex64 when plan.leaf_f32)
  // the leaves' interface operators [R | Gamma] on the boundary data points
  // (nbi x (nbi + ni) each; GX itself unless plan.gauss) and, with
  // plan.gauss, the edge interpolation from the Gauss to the Chebyshev nodes
  void *GXi = nullptr;
  long long gxi_ld = 0, gxi_stride = 0;
  const double2 *d_Qcm = nullptr;
  int *lu_perm = nullptr;            // leaf_lu: row k of P D B is row lu_perm[k] of B
  double *lu_dsc = nullptr;          // leaf_lu: d of that row
  double2 *Rroot = nullptr;
  double *c_dev = nullptr;  // c at the interior nodes (for the refinement residual)
  int *d_outer = nullptr;
  void *tables = nullptr;
  int *d_ints = nullptr;
  int *d_root_src = nullptr;
  unsigned int *d_status = nullptr;
  int leaf_cs = 8;
  int device = -1;  // the CUDA device the operators live on (current at build time)
  // solve workspace (grown on demand)
  void *ws = nullptr;
  size_t ws_bytes = 0;
  // staging for host arrays
  void *stage = nullptr;
  size_t stage_bytes = 0;
  // one-launch solve programs for 1 and 2 right-hand sides, without and with
  // the refinement's interface jumps (recorded at the first such solve)
  struct EnProg {
    hps::EnOp *d_ops = nullptr;
    int nops = 0;
    bool lu_tail = false;  // the leaf step (LU form) follows as its own launch
    bool failed = false;   // the solve has a step the engine does not take
  } eng[2][2];
};

namespace {

int check_desc(const hps_desc *d) {
  if (!d) return HPS_EINVAL;
  if (!(d->x1 > d->x0) || !(d->y1 > d->y0)) return HPS_EINVAL;
  if (!std::isfinite(d->x0) || !std::isfinite(d->x1) || !std::isfinite(d->y0) ||
      !std::isfinite(d->y1))
    return HPS_EINVAL;
  if (d->mx < 1 || d->mx > 1024 || (d->mx & (d->mx - 1))) return HPS_EINVAL;
  if (d->my < 1 || d->my > 1024 || (d->my & (d->my - 1))) return HPS_EINVAL;
  if ((long long)d->mx * d->my > (1 << 20)) return HPS_EINVAL;
  if (d->p < 4 || d->p > 32) return HPS_EINVAL;
  if (d->q != 0 && d->q != d->p - 2 && (d->q < 1 || d->q > 64)) return HPS_EINVAL;
  if (!(d->kappa > 0.0) || !std::isfinite(d->kappa)) return HPS_EINVAL;
  if (d->eta_re == 0.0 || !std::isfinite(d->eta_re) || !std::isfinite(d->eta_im)) return HPS_EINVAL;
  if (d->precision != HPS_FP64 && d->precision != HPS_MIXED) return HPS_EINVAL;
  if (d->fp64_levels < 0) return HPS_EINVAL;
  if (d->fp64_native != 0 && d->fp64_native != 1) return HPS_EINVAL;
  if (d->leaf_form != HPS_LEAF_LU && d->leaf_form != HPS_LEAF_INVERSE) return HPS_EINVAL;
  return HPS_OK;
}

// Chebyshev points (increasing) on [a, b] and the differentiation matrix
// (row-major), Sec. 2.1: off-diagonal (c_i/c_j)(-1)^(i+j)/(x_i - x_j) with
// c_0 = c_N = 2, diagonal from the zero row sum of the exact derivative of a
// constant.
void cheb(int p, double a, double b, std::vector<double> &x, std::vector<double> &D) {
  const int N = p - 1;
  std::vector<double> t(p);
  x.assign(p, 0.0);
  D.assign((size_t)p * p, 0.0);
  for (int j = 0; j < p; j++) {
    t[j] = std::sin(M_PI * (2.0 * j - N) / (2.0 * N));
    x[j] = a + 0.5 * (b - a) * (t[j] + 1.0);
  }
  for (int i = 0; i < p; i++) {
    double ci = (i == 0 || i == N) ? 2.0 : 1.0, sum = 0.0;
    for (int j = 0; j < p; j++) {
      if (j == i) continue;
      double cj = (j == 0 || j == N) ? 2.0 : 1.0;
      double v = (ci / cj) * (((i + j) & 1) ? -1.0 : 1.0) / (t[i] - t[j]);
      D[(size_t)i * p + j] = v;
      sum += v;
    }
    D[(size_t)i * p + i] = -sum;
  }
  for (auto &v : D) v *= 2.0 / (b - a);
}

// Grid coordinates (ix, iy) of local node k in the order [S, E, N, W, interior].
void local_grid(int p, int k, int &ix, int &iy) {
  const int e = p - 2;
  if (k < e) { ix = 1 + k; iy = 0; return; }
  k -= e;
  if (k < e) { ix = p - 1; iy = 1 + k; return; }
  k -= e;
  if (k < e) { ix = 1 + k; iy = p - 1; return; }
  k -= e;
  if (k < e) { ix = 0; iy = 1 + k; return; }
  k -= e;
  ix = 1 + k % e;
  iy = 1 + k / e;
}

int log2i(int m) {
  int k = 0;
  while ((1 << k) < m) k++;
  return k;
}

// Directions of the merges of an mx x my grid from the leaves up (0: west /
// east neighbours, halving the boxes along x; 1: south / north): they
// alternate, starting west/east, and once one axis has no halvings left the
// other takes the remaining merges.
std::vector<int> merge_dirs(int mx, int my) {
  int a = log2i(mx), b = log2i(my), want = 0;
  std::vector<int> dir;
  while (a + b > 0) {
    int d = want;
    if (d == 0 && a == 0) d = 1;
    if (d == 1 && b == 0) d = 0;
    dir.push_back(d);
    if (d == 0) a--; else b--;
    want = 1 - d;
  }
  return dir;
}

// Leaf column and row of a public leaf index: bit k of the index belongs to
// merge k, west/east merges giving the column bits and the others the row
// bits (for a square grid: Morton order, x bit lowest).
void leaf_decode(int idx, const std::vector<int> &dir, int &col, int &row) {
  col = row = 0;
  int bc = 0, br = 0;
  for (size_t k = 0; k < dir.size(); k++) {
    const int bit = (idx >> k) & 1;
    if (dir[k] == 0) col |= bit << bc++;
    else row |= bit << br++;
  }
}

void make_plan(const hps_desc &d, Plan &pl) {
  pl.m = d.mx;
  pl.my = d.my;
  pl.p = d.p;
  pl.e = d.p - 2;
  pl.n = d.p * d.p - 4;
  pl.nb = 4 * pl.e;
  pl.ni = pl.e * pl.e;
  pl.gauss = (d.q != 0 && d.q != pl.e);
  pl.qe = pl.gauss ? d.q : pl.e;
  pl.nbi = 4 * pl.qe;
  const std::vector<int> dirs = merge_dirs(d.mx, d.my);
  pl.L = (int)dirs.size();
  pl.leaves = d.mx * d.my;
  pl.nbdry = 2 * (d.mx + d.my) * pl.qe;
  pl.mixed = (d.precision == HPS_MIXED);
  pl.leaf_f32 = pl.mixed ? 1 : 0;
  pl.leaf_lu = (d.leaf_form == HPS_LEAF_LU);
  // the inverse form in complex128: a complex64 inverse refined on the tensor
  // cores (HPS_LEAF_GJ64 set: complex128 Gauss-Jordan on the FP64 pipes)
  pl.leaf_refined = !pl.leaf_lu && !pl.leaf_f32 && !getenv("HPS_LEAF_GJ64");
  pl.refine_steps = d.refine_steps == 0 ? 2 : (d.refine_steps < 0 ? 0 : d.refine_steps);
  pl.oz = (d.fp64_native == 0);
  const int top = std::min(pl.L, d.fp64_levels == 0 ? 4 : d.fp64_levels);
  // the interface bookkeeping runs on the boundary data points of the edges
  const int e = pl.qe;
  std::vector<Canon> cur(pl.nbi);
  // (leaf within the box, node within the leaf) of every boundary position
  std::vector<std::pair<int, int>> at(pl.nbi);
  for (int k = 0; k < pl.nbi; k++) {
    cur[k] = {k / e, k % e};
    at[k] = {0, k};
  }
  int a = 1, b = 1;  // child box size in leaves (width, height)
  int child_leaves = 1;
  pl.lv.clear();
  pl.total_pairs = 0;
  for (int j = 0; j < pl.L; j++) {
    Level L;
    L.lev = pl.L - 1 - j;
    L.P = 1 << L.lev;
    L.horizontal = (dirs[j] == 0);
    L.f32 = (pl.mixed && j < pl.L - top) ? 1 : 0;
    L.nc = (int)cur.size();
    L.leaves_per_parent = 2 * child_leaves;
    const int n3 = L.horizontal ? b * e : a * e;
    L.n3 = n3;
    L.I3a.assign(n3, -1);
    L.I3b.assign(n3, -1);
    std::vector<Canon> parent, from_b;
    std::vector<std::pair<int, int>> pat, pat_b;
    for (int child = 0; child < 2; child++) {
      for (int pos = 0; pos < L.nc; pos++) {
        Canon c = cur[pos];
        bool shared;
        Canon pc = c;
        if (L.horizontal) {
          if (child == 0) {
            shared = (c.side == 1);
          } else {
            shared = (c.side == 3);
            if (c.side == 0 || c.side == 2) pc.off += a * e;
          }
        } else {
          if (child == 0) {
            shared = (c.side == 2);
          } else {
            shared = (c.side == 0);
            if (c.side == 1 || c.side == 3) pc.off += b * e;
          }
        }
        std::pair<int, int> where = {at[pos].first + child * child_leaves, at[pos].second};
        if (shared) {
          (child == 0 ? L.I3a : L.I3b)[c.off] = pos;
        } else if (child == 0) {
          L.I1.push_back(pos);
          parent.push_back(pc);
          pat.push_back(where);
        } else {
          L.I2.push_back(pos);
          from_b.push_back(pc);
          pat_b.push_back(where);
        }
      }
    }
    L.pairs.resize(4 * (size_t)n3);
    for (int k = 0; k < n3; k++) {
      L.pairs[4 * k + 0] = at[L.I3a[k]].first;
      L.pairs[4 * k + 1] = at[L.I3a[k]].second;
      L.pairs[4 * k + 2] = at[L.I3b[k]].first + child_leaves;
      L.pairs[4 * k + 3] = at[L.I3b[k]].second;
    }
    L.jump_off = pl.total_pairs;
    pl.total_pairs += (long long)L.P * n3;
    L.n1 = (int)L.I1.size();
    L.n2 = (int)L.I2.size();
    L.nt = L.n1 + L.n2;
    parent.insert(parent.end(), from_b.begin(), from_b.end());
    pat.insert(pat.end(), pat_b.begin(), pat_b.end());
    cur.swap(parent);
    at.swap(pat);
    if (L.horizontal) a *= 2; else b *= 2;
    child_leaves *= 2;
    pl.lv.push_back(std::move(L));
  }
  // root position -> public boundary index ([S, E, N, W], m e nodes per side),
  // and public boundary index -> the leaf node that carries it
  pl.root_src.resize(cur.size());
  pl.outer.resize(cur.size());
  for (size_t pos = 0; pos < cur.size(); pos++) {
    // public sides S, E, N, W hold mx, my, mx, my leaf edges
    const int side_off[4] = {0, d.mx * e, (d.mx + d.my) * e, (2 * d.mx + d.my) * e};
    const int q = side_off[cur[pos].side] + cur[pos].off;
    pl.root_src[pos] = q;
    pl.outer[q] = at[pos].first * pl.nbi + at[pos].second;
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int cuda_fail(cudaError_t err) {
  if (err == cudaSuccess) return HPS_OK;
  if (err == cudaErrorMemoryAllocation) return HPS_ENOMEM;
  return HPS_ECUDA;
}

#define CK(call)                                 \
  do {                                           \
    cudaError_t err_ = (call);                   \
    if (err_ != cudaSuccess) return cuda_fail(err_); \
  } while (0)
// the same for functions that return minus the error code
#define CK_NEG(call)                                  \
  do {                                                \
    cudaError_t err_ = (call);                        \
    if (err_ != cudaSuccess) return -cuda_fail(err_); \
  } while (0)

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

Mat mat(const void *ptr, long long ld, long long stride, const int *rmap = nullptr,
        const int *cmap = nullptr, int f32 = 0) {
  Mat m;
  m.ptr = ptr;
  m.ld = ld;
  m.stride = stride;
  m.rmap = rmap;
  m.cmap = cmap;
  m.f32 = f32;
  return m;
}

GemmDesc gemm(int M, int N, int K, int batch, Mat A, Mat B, Mat C) {
  GemmDesc g;
  memset(&g, 0, sizeof(g));
  g.M = M;
  g.N = N;
  g.K = K;
  g.batch = batch;
  g.A = A;
  g.B = B;
  g.ksplit = K;
  g.C = C;
  g.alpha = make_double2(1.0, 0.0);
  g.beta = make_double2(0.0, 0.0);
  return g;
}

CopyDesc copy(int M, int N, int batch, Mat src, Mat dst, double alpha = 1.0) {
  CopyDesc c;
  memset(&c, 0, sizeof(c));
  c.M = M;
  c.N = N;
  c.batch = batch;
  c.src = src;
  c.dst = dst;
  c.alpha = make_double2(alpha, 0.0);
  return c;
}

// Stream-ordered scratch (the leaf step's, the merge levels', temporaries)
// comes from a pool the library owns on each device, which keeps up to
// HPS_POOL_KEEP_BYTES (default 16 GiB) of freed memory reserved: the default
// pool returns it at every synchronization, so each build would map its
// gigabytes of scratch afresh (measured: 1.5 ms of host time a 16 x 16 build,
// with the GPU idle).  0 keeps nothing.
cudaMemPool_t lib_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    pool = nullptr;
  } else {
    uint64_t keep = 16ull << 30;
    if (const char *e = getenv("HPS_POOL_KEEP_BYTES")) keep = strtoull(e, nullptr, 10);
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) cudaGetLastError();
  }
  pools[dev] = pool;
  return pool;
}

cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t st) {
  cudaMemPool_t pool = lib_pool();
  return pool ? cudaMallocFromPoolAsync(p, bytes, pool, st) : cudaMallocAsync(p, bytes, st);
}

long long env_cap() {
  const char *s = getenv("HPS_MEM_CAP_BYTES");
  if (!s || !*s) return -1;
  return atoll(s);
}

// Operation counts (real flops; one complex multiply-add = 8) and bytes.
void fill_info(const Plan &pl, hps_info_t &in) {
  in.leaves = pl.leaves;
  in.levels = pl.L;
  in.n_leaf = pl.n;
  in.n_bdry = pl.nbdry;
  in.dof = (long long)pl.leaves * pl.n;
  long long n = pl.n, nb = pl.nb, ni = pl.ni;
  // leaf: Gauss-Jordan n^3 and G X; or LU of [B; G] (n^3/3 + nb n^2/2) and
  // the G-row solve (nb n^2/2), with n pivots and row scales kept
  long long bf = pl.leaf_lu ? (long long)pl.leaves * 8 * (n * n * n / 3 + nb * n * n)
                            : (long long)pl.leaves * 8 * (n * n * n + nb * n * pl.p);
  // refined inverse: the complex64 inverse, then per step the residual
  // product (tensor cores) and the complex64 correction product
  if (pl.leaf_refined) bf += (long long)pl.leaves * 8 * (2LL * kLeafRefineSteps * n * n * n);
  const long long nbi = pl.nbi, qe = pl.qe, e = pl.e;
  long long sf = (long long)pl.leaves * 8 * (nbi * ni + n * n + (pl.gauss ? nb * qe : 0));
  const long long lu_aux = pl.leaf_lu ? (long long)pl.leaves * n * (4 + 8) : 0;
  long long ob = (long long)pl.leaves * cplx_bytes(n * n + nb * n, pl.leaf_f32) + lu_aux;
  long long sb = (long long)pl.leaves * cplx_bytes(n * n + nbi * ni, pl.leaf_f32) + lu_aux;
  if (pl.gauss) {
    // the interface operators [Ph R Qh | Ph Gamma] and the products that form them
    ob += (long long)pl.leaves * cplx_bytes(nbi * (nbi + ni));
    bf += (long long)pl.leaves * 8 * (nbi * e * n + nbi * nb * qe);
  }
  for (const Level &L : pl.lv) {
    long long n1 = L.n1, n2 = L.n2, n3 = L.n3, nt = L.nt, P = L.P;
    bf += P * 8 * (2 * n3 * n3 * n3 + n3 * n3 * n1 + 2 * n3 * n3 * nt + (n1 + n2) * n3 * nt);
    sf += P * 8 * (3 * n3 * n3 + (n1 + n2) * n3 + 2 * n3 * nt);
    long long ops = 3 * n3 * n3 + n1 * n3 + n2 * n3 + 2 * n3 * nt;
    ob += P * cplx_bytes(ops, L.f32);
    sb += P * cplx_bytes(ops, L.f32);
  }
  in.build_flops = bf;
  in.solve_flops = sf;
  in.operator_bytes = ob;
  in.solve_bytes = sb;
  in.build_launches = pl.lv.empty() ? 2 : 1 + 7 * (int)pl.lv.size();
  in.solve_launches = 3 + 6 * (int)pl.lv.size();
  if (pl.gauss) {
    in.build_launches += 5 * (int)((pl.leaves + 2047) / 2048);  // the interface operators, per pass
    in.solve_launches += 1;                                     // t = Qh t_G
  }
  if (pl.mixed) {
    int conv = 0;
    for (size_t j = 0; j < pl.lv.size(); j++)
      if (!pl.lv[j].f32 && (j == 0 ? pl.leaf_f32 : pl.lv[j - 1].f32)) conv++;
    in.build_launches += conv;
    // each refinement step: residual, jumps and outer data, the injections
    // of the correction solve, the correction solve, the update of u
    const int steps = pl.refine_steps;
    in.solve_launches += steps * (2 + (int)pl.lv.size() + in.solve_launches + 1);
    sf *= 1 + steps;
    in.solve_flops = sf;
  }
}

// CTAs a leaf (the leaf kernel's cluster) for a launch over NL leaves, or 0
// when no cluster fits the kernel's shared memory.  Wider clusters split
// each leaf finer, which balances the chip when there are few leaves
// (Gauss-Jordan, measured best: 8 CTAs a leaf for 16 leaves, 4 for 256, 1
// from 1024 leaves on; complex64 leaves are latency-bound: one CTA a leaf
// from 256 leaves on).  The LU kernel also widens until two CTAs fit an SM.
int leaf_cluster(const Plan &pl, long long NL) {
  const bool f32 = pl.leaf_f32 != 0;
  auto smem = [&](int cs) {
    return pl.leaf_lu ? hps::lu_leaf_smem_bytes(pl.n, pl.nb, pl.p, cs, f32)
                      : hps::gj_smem_bytes(pl.n, cs, true, pl.p, false, f32);
  };
  // (LU, measured: 2 CTAs a leaf for 256 and for 4096 leaves; 1 CTA a leaf
  // would hold only one CTA an SM)
  int cs = 1;
  while (cs < 8 && NL * cs < (f32 ? 256 : pl.leaf_lu ? 512 : 1024)) cs *= 2;
  if (pl.leaf_lu)
    while (cs < 8 && smem(cs) > 113 * 1024 && smem(2 * cs) <= 113 * 1024) cs *= 2;
  if (const char *e = getenv("HPS_LEAF_CLUSTER")) {
    int v = atoi(e);
    if (v == 1 || v == 2 || v == 4 || v == 8 || v == 16) cs = v;
  }
  while (cs < 16 && smem(cs) > 227 * 1024) cs *= 2;
  return smem(cs) <= 227 * 1024 ? cs : 0;
}

// Leaves a leaf launch covers: Gauss-Jordan works on a scratch copy of the
// matrices (chunks of ~1 GiB of them), the LU kernel in place (its
// bookkeeping caps a launch at 16384 leaves).
long long leaf_chunk(const Plan &pl, long long NL) {
  const long long esz = pl.leaf_f32 ? 8 : 16, n = pl.n;
  // (refined inverse: ~10 MB of scratch a leaf at p = 16)
  const long long cap = pl.leaf_lu ? 16384 : pl.leaf_refined ? 512 : (1LL << 30) / (esz * n * n);
  return std::max<long long>(1, std::min<long long>(NL, cap));
}

int choose_gj_cs(int n, int batch, bool tglobal, int f32) {
  // smallest cluster whose shared memory fits two CTAs per SM, then wider
  // while the level has too few matrices to fill the chip and every CTA
  // keeps at least two panels
  int cs = 1;
  while (cs < hps::gj_max_cluster() && hps::gj_smem_bytes(n, cs, false, 0, tglobal, f32) > 110 * 1024) cs *= 2;
  while (cs < hps::gj_max_cluster() && (long long)batch * cs < 304 && hps::gj_slab(n, 2 * cs) >= 16)
    cs *= 2;
  return cs;
}

// Measured kernel choices (hps_tune), the GPU form of the paper's
// calibration of representative actions (Sec. 3, Table 1): per product shape
// the tile configuration or the tensor-core product, per interface-inverse
// shape the cluster size or the panel-per-launch regime.  Shapes not in the
// table take the rules below.  Process-wide.
struct TuneKey {
  int kind;  // 0: product (M, N, K, batch, f32), 1: interface inverse (n3, P, f32)
  int M, N, K, batch, f32;
  bool operator<(const TuneKey &o) const {
    if (kind != o.kind) return kind < o.kind;
    if (M != o.M) return M < o.M;
    if (N != o.N) return N < o.N;
    if (K != o.K) return K < o.K;
    if (batch != o.batch) return batch < o.batch;
    return f32 < o.f32;
  }
};
std::map<TuneKey, int> g_tune;  // product: 1..4 tile, 5 tensor cores; inverse: cs > 0, or -G (wide)
std::mutex g_tune_mu;

// The measured choices can be kept in a text file (environment variable
// HPS_TUNE_CACHE): hps_tune reads it before measuring (shapes found there
// are not measured again) and rewrites it after, so that another process
// (a profiler run, whose serialised kernels would time differently) makes
// the same choices.  One line a shape: kind M N K batch f32 choice.
void tune_cache_load() {
  const char *path = getenv("HPS_TUNE_CACHE");
  if (!path || !*path) return;
  FILE *f = fopen(path, "r");
  if (!f) return;
  TuneKey k;
  int v;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  while (fscanf(f, "%d %d %d %d %d %d %d", &k.kind, &k.M, &k.N, &k.K, &k.batch, &k.f32, &v) == 7) g_tune[k] = v;
  fclose(f);
}
void tune_cache_store() {
  const char *path = getenv("HPS_TUNE_CACHE");
  if (!path || !*path) return;
  FILE *f = fopen(path, "w");
  if (!f) return;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (const auto &kv : g_tune)
    fprintf(f, "%d %d %d %d %d %d %d\n", kv.first.kind, kv.first.M, kv.first.N, kv.first.K, kv.first.batch,
            kv.first.f32, kv.second);
  fclose(f);
}

bool tuned(const TuneKey &k, int &v) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  v = it->second;
  return true;
}

// Kernel regime of the interface inverses of one launch: P matrices n3 x n3.
struct GJChoice {
  int cs = 1;            // cluster size of the cluster kernel
  bool tglobal = false;  // cluster kernel: panels read in place from global memory
  int wide = 0;          // > 0: one launch per panel over P * wide CTAs instead
  int kb = 8;            // panel width (8, or 4 for a shorter serial chain)
  // complex128 matrices: a complex64 inverse (the kernel and regime above, in
  // complex64) refined by two complex128 residual steps (w_inverse)
  bool refined = false;
};
// a measured choice as one int of the tuning table: cs, or -wide; panel
// width 4 adds 2^20 to the magnitude, the refined regime 2^21
int gj_encode(const GJChoice &g) {
  const int v = g.wide ? g.wide : g.cs;
  const int m = v + (g.kb == 4 ? (1 << 20) : 0) + (g.refined ? (1 << 21) : 0);
  return g.wide ? -m : m;
}
GJChoice gj_decode(int v) {
  GJChoice g;
  const int m = v < 0 ? -v : v;
  g.kb = ((m >> 20) & 1) ? 4 : 8;
  g.refined = ((m >> 21) & 1) != 0;
  if (v > 0)
    g.cs = m & ((1 << 20) - 1);
  else
    g.wide = m & ((1 << 20) - 1);
  return g;
}

bool choose_gj_rule(int n3, long long P, int f32, GJChoice &g);

// false when no regime fits in the kernels' shared memory
bool choose_gj(int n3, long long P, int f32, GJChoice &g) {
  int v;
  bool ok = false;
  if (P <= (1 << 30) && tuned(TuneKey{1, n3, 0, 0, (int)P, f32}, v) && v != 0) {
    GJChoice t = gj_decode(v);
    const int kf = (f32 || t.refined) ? 1 : 0;  // the precision the elimination runs in
    t.tglobal = hps::gj_smem_bytes(n3, hps::gj_max_cluster(), false, 0, false, kf, t.kb) > 200 * 1024;
    if (t.wide || hps::gj_smem_bytes(n3, t.cs, false, 0, t.tglobal, kf, t.kb) <= 227 * 1024) {
      g = t;
      ok = true;
    }
  }
  if (!ok) {
    ok = choose_gj_rule(n3, P, f32, g);
    // complex128 matrices too few to fill the chip (the panel-per-launch
    // regime): their inverse is a serial chain of panel eliminations on the
    // 1/64-rate FP64 pipe, so refine a complex64 inverse instead
    GJChoice r;
    if (ok && !f32 && g.wide && !getenv("HPS_W_GJ64") && choose_gj_rule(n3, P, 1, r)) {
      g = r;
      g.refined = true;
    }
  }
  // HPS_GJ_KB=4: panels of 4 columns whatever was chosen (it needs less
  // shared memory than 8, so the choice still fits); for tests of that width
  if (ok) {
    const char *e = getenv("HPS_GJ_KB");
    if (e && atoi(e) == 4) g.kb = 4;
  }
  return ok;
}

bool choose_gj_rule(int n3, long long P, int f32, GJChoice &g) {
  // stage the panels in shared memory while they fit beside the rest
  g.tglobal = hps::gj_smem_bytes(n3, hps::gj_max_cluster(), false, 0, false, f32) > 200 * 1024;
  g.cs = choose_gj_cs(n3, (int)std::min<long long>(P, 1 << 30), g.tglobal, f32);
  const bool fits = hps::gj_smem_bytes(n3, g.cs, false, 0, g.tglobal, f32) <= 227 * 1024;
  g.wide = 0;
  // too few matrices to fill the chip with clusters (or a matrix too large
  // for one cluster): one launch per panel over about two CTAs per SM, each
  // with a slab of at least 4 columns
  if (!fits || ((long long)P * g.cs < 152 && n3 >= 64 && !getenv("HPS_NO_WIDE_GJ"))) {
    const long long G = std::min<long long>((2 * 152 + P - 1) / P, n3 / 4 + 1);
    g.wide = (int)std::max<long long>(2, G);
    const int slab = (n3 + g.wide - 2) / (g.wide - 1);
    const bool tg = hps::gj_wide_smem_bytes(n3, slab, f32, false) > 200 * 1024;
    return hps::gj_wide_smem_bytes(n3, slab, f32, tg) <= 227 * 1024;
  }
  return true;
}

int gj_elim_launches(int n3, const GJChoice &g) { return g.wide ? hps::gj_wide_launches(n3, g.kb) : 1; }
bool oz_shape(int M, int N, int K, int batch, int f32, bool oz);
int oz_launches_shape(int M, int N, int K, int batch, int f32 = 0);
// launches of an interface inverse: the elimination, or for the refined
// regime the conversion, the complex64 elimination, the widening copy and
// per step the residual product and the correction product (its FP64
// addition in the epilogue); the second step reuses the first one's split of
// W where the residual runs on the tensor cores
int gj_launches(int n3, long long P, bool oz, const GJChoice &g) {
  if (!g.refined) return gj_elim_launches(n3, g);
  const bool ozr = oz_shape(n3, n3, n3, (int)P, 0, oz);
  const int prod = ozr ? oz_launches_shape(n3, n3, n3, (int)P) : 1;
  return 2 + gj_elim_launches(n3, g) + (prod + 1) + ((ozr ? prod - 2 : 1) + 1);
}

// Does a product of this shape go to the tensor cores (Ozaki scheme: 9
// slices an operand in complex128, 5 for the complex64 products)?  Complex64
// products only where hps_tune measured it faster (at the mixed path's
// shapes it chose the FP32-pipe tiles every time: 64 x 64 leaves, p = 16).
bool oz_shape(int M, int N, int K, int batch, int f32, bool oz) {
  if (!oz) return false;
  int v;
  if (tuned(TuneKey{0, M, N, K, batch, f32}, v)) return v == 5;
  if (f32) return false;
  GemmDesc g;
  memset(&g, 0, sizeof(g));
  g.M = M;
  g.N = N;
  g.K = K;
  g.batch = batch;
  g.cf32 = f32;
  return hps::oz_eligible(g);
}

int oz_launches_shape(int M, int N, int K, int batch, int f32) {
  GemmDesc g;
  memset(&g, 0, sizeof(g));
  g.M = M;
  g.N = N;
  g.K = K;
  g.batch = batch;
  g.cf32 = f32;
  return hps::oz_launches(g);
}

size_t oz_bytes_shape(int M, int N, int K, int batch, int f32 = 0) {
  GemmDesc g;
  memset(&g, 0, sizeof(g));
  g.M = M;
  g.N = N;
  g.K = K;
  g.batch = batch;
  g.cf32 = f32;
  return hps::oz_workspace_bytes(g);
}

// Scratch of the refined interface inverse of P complex128 n3 x n3 matrices:
// W in complex64, its complex64 inverse X0, the residual E, and the
// tensor-core workspace of the residual product where that goes there (it
// keeps W's digits for the second step).
struct WRef {
  size_t w32, x0, e, oz, total;
};
WRef wref_layout(int n3, long long P, bool oz) {
  const size_t n2 = (size_t)n3 * n3 * P;
  WRef L;
  L.w32 = 0;
  L.x0 = align256(8 * n2);
  L.e = L.x0 + align256(8 * n2);  // the residual, in complex64
  L.oz = L.e + align256(8 * n2);
  L.total = L.oz + (oz_shape(n3, n3, n3, (int)P, 0, oz) ? oz_bytes_shape(n3, n3, n3, (int)P) : 0);
  return L;
}

// W^{-1} of P n3 x n3 matrices (Sec. 2.2's interface inverse) into Winv.
// The elimination regimes destroy W; the refined one keeps it (its residuals
// read it): X0 = the complex64 inverse of W, then two steps of E = I - W X
// (complex128-accurate: the Ozaki product on the tensor cores where that shape
// goes there, else the FP64 pipes) and X += X0 E (complex64 arithmetic, added
// in FP64).  W's 1-norm condition numbers stay below ~100 at every workload
// here, so ||I - W X0|| ~ 1e-6 and two steps reach complex128 rounding.
int w_inverse(const GJChoice &g, void *W, void *Winv, int n3, int P, int *meta, unsigned *status, int lev,
              bool f32, char *rscr, bool oz, cudaStream_t st, int &launches) {
  if (!g.refined || f32) {
    if (g.wide)
      CK(hps::launch_gj_wide(W, Winv, n3, P, g.wide, meta, status, lev, f32, st, g.kb));
    else
      CK(hps::launch_gj_inverse(W, Winv, n3, P, meta, status, lev, g.cs, g.tglobal, f32, st, g.kb));
    launches += gj_elim_launches(n3, g);
    return HPS_OK;
  }
  const WRef L = wref_layout(n3, P, oz);
  void *W32 = rscr + L.w32, *X0 = rscr + L.x0;
  float2 *E = (float2 *)(rscr + L.e);
  const long long s2 = (long long)n3 * n3;
  CopyBatch cb;
  cb.count = 1;
  cb.d[0] = copy(n3, n3, P, mat(W, n3, s2), mat(W32, n3, s2, nullptr, nullptr, 1));
  CK(hps::launch_copy(cb, st));
  if (g.wide)
    CK(hps::launch_gj_wide(W32, X0, n3, P, g.wide, meta, status, lev, true, st, g.kb));
  else
    CK(hps::launch_gj_inverse(W32, X0, n3, P, meta, status, lev, g.cs, g.tglobal, true, st, g.kb));
  cb.d[0] = copy(n3, n3, P, mat(X0, n3, s2, nullptr, nullptr, 1), mat(Winv, n3, s2));
  CK(hps::launch_copy(cb, st));
  launches += 2 + gj_elim_launches(n3, g);
  const bool ozr = oz_shape(n3, n3, n3, P, 0, oz);
  for (int it = 0; it < 2; it++) {
    // (E accurate to complex128 rounding, stored in complex64: only the
    // complex64 correction reads it)
    GemmDesc gr = gemm(n3, n3, n3, P, mat(W, n3, s2), mat(Winv, n3, s2), mat(E, n3, s2, nullptr, nullptr, 1));
    gr.alpha = make_double2(-1.0, 0.0);
    gr.addI = 1;
    if (ozr) {
      CK(hps::launch_gemm_oz(gr, rscr + L.oz, L.total - L.oz, st, status, it > 0));
      launches += hps::oz_launches(gr, it > 0);
    } else {
      int v;
      if (tuned(TuneKey{0, n3, n3, n3, P, 0}, v) && v >= 1 && v <= 4) gr.cfg = v;
      CK(hps::launch_gemm(&gr, 1, st));
      launches++;
    }
    // X += X0 E: complex64 product (elementwise complex64 arithmetic: its
    // error is amplified by cond(W) in the next residual), FP64 addition in
    // its epilogue
    GemmDesc gc = gemm(n3, n3, n3, P, mat(X0, n3, s2, nullptr, nullptr, 1), mat(E, n3, s2, nullptr, nullptr, 1),
                       mat(Winv, n3, s2));
    gc.cf32 = 1;
    gc.wide_epilogue = 1;
    gc.D = gc.C;
    gc.beta = make_double2(1.0, 0.0);
    CK(hps::launch_gemm(&gc, 1, st));
    launches += 1;
  }
  return HPS_OK;
}

// The six products of one merge run of P parents (Sec. 2.2): W, Q, Phi_a,
// Phi_b, and the two halves of R^tau, as (M, N, K).
void merge_products(int n1, int n2, int n3, int nt, int (&mnk)[6][3]) {
  const int v[6][3] = {{n3, n3, n3}, {n3, n1, n3}, {n3, nt, n3}, {n3, nt, n3}, {n1, nt, n3}, {n2, nt, n3}};
  memcpy(mnk, v, sizeof(v));
}

// Kernel launches of one merge run: the copy, W^{-1}, and the products (an
// emulated product is four or five launches; the two halves of R^tau share one
// launch when both run on the FP64 pipes).
int merge_launches(int n1, int n2, int n3, int nt, int P, int f32, bool oz, const GJChoice &gj) {
  int mnk[6][3];
  merge_products(n1, n2, n3, nt, mnk);
  int n = 1 + gj_launches(n3, P, oz, gj);
  for (int q = 0; q < 4; q++)
    n += oz_shape(mnk[q][0], mnk[q][1], mnk[q][2], P, f32, oz)
             ? oz_launches_shape(mnk[q][0], mnk[q][1], mnk[q][2], P, f32)
             : 1;
  const bool a = oz_shape(mnk[4][0], mnk[4][1], mnk[4][2], P, f32, oz);
  const bool b = oz_shape(mnk[5][0], mnk[5][1], mnk[5][2], P, f32, oz);
  n += (a ? oz_launches_shape(mnk[4][0], mnk[4][1], mnk[4][2], P, f32) : 0) +
       (b ? oz_launches_shape(mnk[5][0], mnk[5][1], mnk[5][2], P, f32) : 0) + ((!a || !b) ? 1 : 0);
  return n;
}

int grow(void **buf, size_t *have, size_t need) {
  if (*have >= need) return HPS_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *have = 0;
  CK(cudaMalloc(buf, need));
  *have = need;
  // the skinny products' counters at the head of a solve workspace start at zero
  CK(cudaMemset(*buf, 0, std::min(need, hps::gemv_scratch_counters())));
  return HPS_OK;
}

}  // namespace

// element `idx` of an array of complex64 (f32) or complex128 values
static inline void *elem(const void *base, long long idx, int f32) {
  return (char *)base + (f32 ? 8LL : 16LL) * idx;
}

// Solve workspace layout: h per level, t per level, t~3a / t~3b per merge,
// one temporary.  Returns the bytes needed for nrhs right-hand sides.
struct SolveWs {
  static constexpr int kMax = 24;  // merge levels: 2 log2(1024) = 20 at most
  size_t oh[kMax + 1], ot[kMax + 1], ota[kMax], otb[kMax];
  size_t ov = 0, bytes = 0;
  // refinement (HPS_MIXED): residual parts and the correction
  size_t osd = 0, otd = 0, ofu = 0, ogu = 0, oja = 0, ojb = 0, od = 0;
  // products on the tensor cores (wide right-hand-side blocks): digit planes
  size_t ooz = 0, oz_bytes = 0;
  size_t otc = 0;
  // scratch of the skinny products (up to 8 right-hand sides): counters at
  // offset 0 of every workspace (zeroed when it is allocated, left zero by
  // the kernel), partial sums after them
  size_t ogv = 0;
  // one-launch solves (1 or 2 right-hand sides): barrier words and arrival
  // counters (cleared before every launch), then the split products'
  // partial sums
  size_t oen = 0, en_clear = 0, en_part = 0;
};

// The one-launch solve's scratch budget: counters and partial sums of the
// split products of one phase, for grids of up to kEnGridMax CTAs.
constexpr int kEnGridMax = 320;
constexpr long long kEnCounters = 2LL * kEnGridMax;
inline long long en_part_budget(int R) { return 4LL * kEnGridMax * 32 * R; }

// Rows of the first diagonal block when a wide solve in LU form splits each
// leaf's sweeps in two (a multiple of the sweep kernel's 32-row blocks), or
// 0 when the leaf is too small to gain from it.
static int lu_split(int n) {
  const int b1 = (n / 2 + 16) / 32 * 32;
  return (b1 >= 64 && b1 < n) ? b1 : 0;
}

// The complex128 products of a solve with R right-hand sides (M, K, batch),
// Algorithm 2's leaf and level actions.
static void solve_products(const Plan &pl, std::vector<std::array<int, 3>> &out) {
  out.clear();
  if (!pl.leaf_f32) {
    out.push_back({pl.nbi, pl.ni, pl.leaves});
    if (!pl.leaf_lu) {
      out.push_back({pl.n, pl.n, pl.leaves});
    } else if (const int b1 = lu_split(pl.n)) {
      // the off-diagonal blocks of a blocked wide LU solve
      out.push_back({pl.n - b1, b1, pl.leaves});
      out.push_back({b1, pl.n - b1, pl.leaves});
    }
  }
  for (const Level &L : pl.lv) {
    if (L.f32) continue;
    out.push_back({L.n3, L.n3, L.P});
    out.push_back({L.n1, L.n3, L.P});
    out.push_back({L.n2, L.n3, L.P});
    out.push_back({L.n3, L.nt, L.P});
  }
}

static void solve_ws_layout(const Plan &pl, int R, SolveWs &w, bool allow_oz = true) {
  size_t off = align256(hps::gemv_scratch_counters());
  if (R <= 16) {
    w.ogv = off;
    off = align256(off + hps::gemv_part_bytes(R));
  }
  if (R <= 2) {
    w.oen = off;
    w.en_clear = align256(sizeof(unsigned) * (4 + (size_t)kEnCounters));
    w.en_part = w.oen + w.en_clear;
    off = align256(w.en_part + sizeof(double2) * (size_t)en_part_budget(R));
  }
  auto take = [&](long long count) {
    size_t o = off;
    off = align256(off + sizeof(double2) * (size_t)count);
    return o;
  };
  w.oh[0] = take((long long)R * pl.leaves * pl.nbi);
  w.ot[0] = take((long long)R * pl.leaves * pl.nbi);
  // boundary data on Gauss nodes: the leaves' incoming data on their
  // Chebyshev edge nodes (Qh t) before the leaf step
  if (pl.gauss) w.otc = take((long long)R * pl.leaves * pl.nb);
  long long vmax = 1;
  for (size_t j = 0; j < pl.lv.size(); j++) {
    const Level &L = pl.lv[j];
    w.oh[j + 1] = take((long long)R * L.P * L.nt);
    w.ot[j + 1] = take((long long)R * L.P * L.nt);
    w.ota[j] = take((long long)R * L.P * L.n3);
    w.otb[j] = take((long long)R * L.P * L.n3);
    vmax = std::max(vmax, (long long)R * L.P * L.n3);
  }
  w.ov = take(vmax);
  if (pl.mixed && pl.refine_steps > 0) {
    w.osd = take((long long)R * pl.leaves * pl.ni);
    w.otd = take((long long)R * pl.nbdry);
    w.ofu = take((long long)R * pl.leaves * pl.nb);
    w.ogu = take((long long)R * pl.leaves * pl.nb);
    w.oja = take((long long)R * std::max(1LL, pl.total_pairs));
    w.ojb = take((long long)R * std::max(1LL, pl.total_pairs));
    w.od = take((long long)R * pl.leaves * pl.n);
  }
  // room for the tensor-core digit planes of the largest eligible product,
  // in batch chunks of at most 512 MiB (a chunk of one matrix at least)
  w.oz_bytes = 0;
  if (allow_oz && pl.oz && R >= 32) {
    std::vector<std::array<int, 3>> pr;
    solve_products(pl, pr);
    for (const auto &q : pr)
      if (oz_shape(q[0], R, q[1], q[2], 0, true)) {
        const size_t one = oz_bytes_shape(q[0], R, q[1], 1), all = oz_bytes_shape(q[0], R, q[1], q[2]);
        w.oz_bytes = std::max(w.oz_bytes, std::max(one, std::min(all, (size_t)512 << 20)));
      }
    if (w.oz_bytes) {
      w.ooz = off;
      off = align256(off + w.oz_bytes);
    }
  }
  w.bytes = off;
}

// The steps of a solve with one or two right-hand sides as a program for the
// one-launch solve (solve_engine.cu): solve_launch, given a recorder, hands
// it its products and copies instead of launching them.  Operands are
// recorded relative to the call's s, t, u and workspace (so that the program
// serves every later call), or by address (the handle's operators and maps).
struct SolveRec {
  const char *lo[5] = {}, *hi[5] = {};  // ranges of s, t, u, workspace (1..4)
  std::vector<hps::EnOp> ops;
  int phase0 = 0;  // first op of the open phase
  long long part = 0, cnt = 0;
  bool ok = true, lu_tail = false;
  int grid = 0, R = 0;

  hps::EnMat conv(const Mat &m, bool allow_rmap) {
    hps::EnMat e;
    memset(&e, 0, sizeof(e));
    e.base = -1;
    if (!m.ptr) return e;
    if (m.cmap || (m.rmap && !allow_rmap)) ok = false;
    const char *p = (const char *)m.ptr;
    e.base = 0;
    e.off = (long long)(uintptr_t)p;
    for (int b = 1; b <= 4; b++)
      if (p >= lo[b] && p < hi[b]) {
        e.base = b;
        e.off = p - lo[b];
        break;
      }
    e.ld = m.ld;
    e.stride = m.stride;
    e.rmap = m.rmap;
    e.f32 = m.f32;
    return e;
  }
  void open(bool same_phase) {
    if (same_phase && !ops.empty()) {
      ops.back().phase_end = 0;  // reopen the last phase
      return;
    }
    phase0 = (int)ops.size();
    part = cnt = 0;
  }
  void close() {
    if (!ops.empty()) ops.back().phase_end = 1;
    if (part > en_part_budget(R) || cnt > kEnCounters) ok = false;
  }
  int next_unit() const { return (int)ops.size() > phase0 ? ops.back().unit0 + ops.back().units : 0; }
  void gemm(const GemmDesc *gd, int nd) {
    open(false);
    for (int q = 0; q < nd; q++) {
      const GemmDesc &g = gd[q];
      if (g.N != R || g.addI || g.A.rmap || g.A.cmap) ok = false;
      hps::EnOp o;
      memset(&o, 0, sizeof(o));
      o.kind = 0;
      o.M = g.M;
      o.K = g.K;
      o.batch = g.batch;
      o.R = R;
      o.ksplit = g.B2.ptr ? g.ksplit : g.K;
      o.cf32 = g.cf32;
      o.A = conv(g.A, false);
      o.x = conv(g.B, true);
      o.x2 = conv(g.B2, true);
      o.y = conv(g.C, true);
      o.D = conv(g.D, true);
      o.alpha = g.alpha;
      o.beta = g.beta;
      // K cut into chunks when the row blocks alone would leave most of the
      // grid idle
      const int rows = hps::engine_unit_rows();
      o.nrb = (g.M + rows - 1) / rows;
      const long long base = (long long)g.batch * o.nrb;
      int nkc = (g.K + hps::engine_max_kc() - 1) / hps::engine_max_kc();
      if (base < grid / 2 && g.K >= 48)
        nkc = std::max(nkc, (int)std::min<long long>((g.K + 23) / 24, (grid + base - 1) / base));
      o.kc = (g.K + nkc - 1) / nkc;
      o.nkc = (g.K + o.kc - 1) / o.kc;
      o.units = (int)std::min<long long>(base * o.nkc, 1LL << 30);
      o.unit0 = next_unit();
      if (o.nkc > 1) {
        o.part_off = part;
        o.cnt_off = cnt;
        part += base * o.nkc * rows * R;
        cnt += base;
      }
      ops.push_back(o);
    }
    close();
  }
  void copy(const CopyBatch &cb, bool same_phase) {
    open(same_phase);
    for (int q = 0; q < cb.count; q++) {
      const CopyDesc &d = cb.d[q];
      if (d.trans || d.N != R || !d.src.ptr) ok = false;
      hps::EnOp o;
      memset(&o, 0, sizeof(o));
      o.kind = 1;
      o.M = d.M;
      o.batch = d.batch;
      o.R = R;
      o.accumulate = d.accumulate;
      o.x = conv(d.src, true);
      o.y = conv(d.dst, true);
      o.D.base = -1;
      o.alpha = d.alpha;
      const long long el = (long long)d.M * R * d.batch;
      o.units = (int)((el + hps::engine_copy_unit() - 1) / hps::engine_copy_unit());
      o.unit0 = next_unit();
      ops.push_back(o);
    }
    close();
  }
};

// Products of a solve: complex128 ones wide enough for the tensor cores run
// there, the batch cut into chunks whose digit planes fit the workspace's
// region; the rest in one launch.
static int solve_gemm(GemmDesc *gd, int nd, cudaStream_t st, char *wb, const SolveWs &ws, bool oz,
                      unsigned *status) {
  GemmDesc rest[2];
  int nr = 0;
  for (int q = 0; q < nd; q++) {
    GemmDesc &g = gd[q];
    if (g.N <= 16 && ws.ogv) {
      g.part = wb + ws.ogv;
      g.cnt = (unsigned *)wb;
    }
    if (oz && ws.oz_bytes && oz_shape(g.M, g.N, g.K, g.batch, g.cf32, true)) {
      int chunk = g.batch;
      while (chunk > 1 && oz_bytes_shape(g.M, g.N, g.K, chunk, g.cf32) > ws.oz_bytes) chunk = (chunk + 1) / 2;
      if (oz_bytes_shape(g.M, g.N, g.K, chunk, g.cf32) <= ws.oz_bytes) {
        auto shift = [](Mat m, long long b) {
          if (m.ptr) m.ptr = elem(m.ptr, b * m.stride, m.f32);
          return m;
        };
        for (int b0 = 0; b0 < g.batch; b0 += chunk) {
          GemmDesc c = g;
          c.batch = std::min(chunk, g.batch - b0);
          c.A = shift(g.A, b0);
          c.B = shift(g.B, b0);
          c.B2 = shift(g.B2, b0);
          c.C = shift(g.C, b0);
          c.D = shift(g.D, b0);
          CK(hps::launch_gemm_oz(c, wb + ws.ooz, ws.oz_bytes, st, status));
        }
        continue;
      }
    }
    rest[nr++] = g;
  }
  if (nr) CK(hps::launch_gemm(rest, nr, st));
  return HPS_OK;
}

// Algorithm 2 for R right-hand sides on device arrays s, t, u, with the
// workspace at wb (laid out by solve_ws_layout).  Launches kernels only.
// Vectors are complex128; each level computes in its own precision.  JA, JB
// (optional, [R][total_pairs]): residuals of the two interface conditions of
// every I3 pair, injected as h3a -= JB, h3b -= JA before the level's Upsilon
// actions (the right-hand side of t3a = -g3b + JA, t3b = -g3a + JB).
// The leaf step of a solve in LU form: u = B^{-1} [t; s] by the leaves' sweeps.
static cudaError_t lu_leaf_solve(hps_handle *h, const double2 *s, const double2 *tl, double2 *u, int R,
                                 cudaStream_t st) {
  const Plan &pl = h->plan;
  const int n = pl.n, nb = pl.nb, ni = pl.ni, nl = pl.leaves;
  return hps::launch_lu_solve(h->X, h->lu_perm, h->lu_dsc, nl, n, nb, R, tl, (long long)nl * nb, nb, s,
                              (long long)nl * ni, ni, u, (long long)nl * n, n, pl.leaf_f32 != 0, st);
}

static int run_engine(hps_handle *h, const double2 *s, const double2 *t, double2 *u, int R, char *wb,
                      const SolveWs &ws, cudaStream_t st, const double2 *JA, const double2 *JB, bool may_alloc);

static int solve_launch(hps_handle *h, const double2 *s, const double2 *t, double2 *u, int R,
                        char *wb, const SolveWs &ws, cudaStream_t st, const double2 *JA = nullptr,
                        const double2 *JB = nullptr, SolveRec *rec = nullptr, bool may_alloc = true) {
  // one or two right-hand sides: the whole solve as one launch
  if (!rec && R <= 2) {
    const int used = run_engine(h, s, t, u, R, wb, ws, st, JA, JB, may_alloc);
    if (used < 0) return -used;
    if (used > 0) return HPS_OK;
  }
  // with one or two right-hand sides the solve is a chain of small
  // dependent launches: let each be scheduled while the previous one drains
  // (measured at 16 x 16 leaves: 1 RHS 0.85 -> 0.75 ms; with 16 or 64
  // right-hand sides the chained launches were slower)
  std::unique_ptr<hps::LaunchChain> chain;
  if (R <= 2 && !rec) chain.reset(new hps::LaunchChain());
  // the steps, launched or recorded
  auto gemms = [&](GemmDesc *gd, int nd) -> int {
    if (rec) {
      rec->gemm(gd, nd);
      return HPS_OK;
    }
    return solve_gemm(gd, nd, st, wb, ws, h->plan.oz, h->d_status);
  };
  auto copies = [&](const CopyBatch &cb, bool same_phase) -> int {
    if (rec) {
      rec->copy(cb, same_phase);
      return HPS_OK;
    }
    CK(hps::launch_copy(cb, st));
    return HPS_OK;
  };
  const Plan &pl = h->plan;
  const int n = pl.n, nb = pl.nb, ni = pl.ni, nl = pl.leaves, lf = pl.leaf_f32;
  const size_t *oh = ws.oh, *ot = ws.ot, *ota = ws.ota, *otb = ws.otb;
  const size_t ov = ws.ov;
  auto W = [&](size_t o) { return (double2 *)(wb + o); };
  auto F = [&](const void *ptr, long long ld, long long stride, int f32) {
    return mat(ptr, ld, stride, nullptr, nullptr, f32);
  };

  // ---- upward pass ----
  // leaves: h = Gamma s  (Gamma = GX[:, nb:], on the boundary data points: nbi rows)
  const int nbi = pl.nbi;
  const int gf = pl.gauss ? 0 : lf;
  GemmDesc g = gemm(nbi, R, ni, nl, F(elem(h->GXi, h->gxi_ld * nbi, gf), h->gxi_ld, h->gxi_stride, gf),
                    mat(s, (long long)nl * ni, ni), mat(W(oh[0]), (long long)nl * nbi, nbi));
  g.cf32 = lf;
  if (int rc = gemms(&g, 1)) return rc;
  for (size_t j = 0; j < pl.lv.size(); j++) {
    const Level &L = pl.lv[j];
    const int P = L.P, n1 = L.n1, n2 = L.n2, n3 = L.n3, nt = L.nt, nc = L.nc, f = L.f32;
    double2 *hc = W(oh[j]);
    const long long ldh = (long long)2 * P * nc;
    Mat hA = mat(hc, ldh, 2LL * nc), hB = mat(hc + nc, ldh, 2LL * nc);
    Mat h3a = hA, h3b = hB, h1a = hA, h2b = hB;
    h3a.rmap = L.d_I3a;
    h3b.rmap = L.d_I3b;
    h1a.rmap = L.d_I1;
    h2b.rmap = L.d_I2;
    if (JA && JB) {
      CopyBatch cb;
      cb.count = 2;
      cb.d[0] = copy(n3, R, P, mat(JB + L.jump_off, pl.total_pairs, n3), h3a, -1.0);
      cb.d[0].accumulate = 1;
      cb.d[1] = copy(n3, R, P, mat(JA + L.jump_off, pl.total_pairs, n3), h3b, -1.0);
      cb.d[1].accumulate = 1;
      if (int rc = copies(cb, false)) return rc;
    }
    const long long s33 = (long long)n3 * n3, ldv = (long long)P * n3;
    double2 *v = W(ov), *ta = W(ota[j]), *tb = W(otb[j]);
    // v = R33b h3a - h3b ;  t~3a = W^{-1} v  (Upsilon_a [h3a; h3b])
    g = gemm(n3, R, n3, P, F(L.R33b, n3, s33, f), h3a, mat(v, ldv, n3));
    g.D = h3b;
    g.beta = make_double2(-1.0, 0.0);
    g.cf32 = f;
    if (int rc = gemms(&g, 1)) return rc;
    g = gemm(n3, R, n3, P, F(L.Winv, n3, s33, f), mat(v, ldv, n3), mat(ta, ldv, n3));
    g.cf32 = f;
    if (int rc = gemms(&g, 1)) return rc;
    // t~3b = -h3a - R33a t~3a  (Upsilon_b [h3a; h3b])
    g = gemm(n3, R, n3, P, F(L.R33a, n3, s33, f), mat(ta, ldv, n3), mat(tb, ldv, n3));
    g.alpha = make_double2(-1.0, 0.0);
    g.D = h3a;
    g.beta = make_double2(-1.0, 0.0);
    g.cf32 = f;
    if (int rc = gemms(&g, 1)) return rc;
    // h^tau = [h1a + R13a t~3a ; h2b + R23b t~3b]  (Eq. flux_part)
    const long long ldp = (long long)P * nt;
    GemmDesc g2[2];
    g2[0] = gemm(n1, R, n3, P, F(L.R13a, n1, (long long)n1 * n3, f), mat(ta, ldv, n3), mat(W(oh[j + 1]), ldp, nt));
    g2[0].D = h1a;
    g2[0].beta = make_double2(1.0, 0.0);
    g2[0].cf32 = f;
    g2[1] = gemm(n2, R, n3, P, F(L.R23b, n2, (long long)n2 * n3, f), mat(tb, ldv, n3),
                 mat(W(oh[j + 1]) + n1, ldp, nt));
    g2[1].D = h2b;
    g2[1].beta = make_double2(1.0, 0.0);
    g2[1].cf32 = f;
    if (int rc = gemms(g2, 2)) return rc;
  }

  // ---- downward pass ----
  const size_t top = pl.lv.size();
  const int ntop = top ? pl.lv.back().nt : nbi;
  {
    // root incoming data: public [S, E, N, W] order -> the root's [I1, I2] order
    CopyBatch cb;
    cb.count = 1;
    cb.d[0] = copy(ntop, R, 1, mat(t, pl.nbdry, 0, h->d_root_src), mat(W(ot[top]), ntop, 0));
    if (int rc = copies(cb, false)) return rc;
  }
  for (size_t jj = top; jj-- > 0;) {
    const Level &L = pl.lv[jj];
    const int P = L.P, n1 = L.n1, n2 = L.n2, n3 = L.n3, nt = L.nt, nc = L.nc, f = L.f32;
    const double2 *tp = W(ot[jj + 1]);
    double2 *tc = W(ot[jj]);
    const long long ldp = (long long)P * nt, ldc2 = (long long)2 * P * nc, ldv = (long long)P * n3;
    const long long s3t = (long long)n3 * nt;
    // t3a = Phi_a t^tau + t~3a -> alpha rows I3 ; t3b = Phi_b t^tau + t~3b -> beta rows I3
    GemmDesc g2[2];
    g2[0] = gemm(n3, R, nt, P, F(L.Phia, n3, s3t, f), mat(tp, ldp, nt), mat(tc, ldc2, 2LL * nc, L.d_I3a));
    g2[0].D = mat(W(ota[jj]), ldv, n3);
    g2[0].beta = make_double2(1.0, 0.0);
    g2[0].cf32 = f;
    g2[1] = gemm(n3, R, nt, P, F(L.Phib, n3, s3t, f), mat(tp, ldp, nt), mat(tc + nc, ldc2, 2LL * nc, L.d_I3b));
    g2[1].D = mat(W(otb[jj]), ldv, n3);
    g2[1].beta = make_double2(1.0, 0.0);
    g2[1].cf32 = f;
    if (int rc = gemms(g2, 2)) return rc;
    // the rest of the children's incoming data is the parent's: I1 and I2
    CopyBatch cb;
    cb.count = 2;
    cb.d[0] = copy(n1, R, P, mat(tp, ldp, nt), mat(tc, ldc2, 2LL * nc, L.d_I1));
    cb.d[1] = copy(n2, R, P, mat(tp + n1, ldp, nt), mat(tc + nc, ldc2, 2LL * nc, L.d_I2));
    // (rows I1, I2 of the children: independent of the products' rows I3)
    if (int rc = copies(cb, true)) return rc;
  }
  // leaves: u = Psi t + Y s = B^{-1} [t; s], t on the leaves' Chebyshev edge
  // nodes: with boundary data on Gauss nodes, t = Qh t_G first (every
  // (leaf, edge) pair one product with the e x qe table)
  const double2 *tl = W(ot[0]);
  if (pl.gauss) {
    const int qe = pl.qe, e = pl.e;
    GemmDesc gq = gemm(e, R, qe, 4 * nl, mat(h->d_Qcm, e, 0), mat(W(ot[0]), (long long)nl * nbi, qe),
                       mat(W(ws.otc), (long long)nl * nb, e));
    if (int rc = rec ? gemms(&gq, 1) : solve_gemm(&gq, 1, st, wb, ws, false, h->d_status)) return rc;
    tl = W(ws.otc);
  }
  const int b1 = lu_split(n);
  if (pl.leaf_lu && !lf && R >= 32 && b1 && ws.oz_bytes && oz_shape(n - b1, R, b1, nl, 0, pl.oz)) {
    // wide solve: each leaf's sweeps in two diagonal blocks, the products
    // with the off-diagonal blocks L21 and U12 batched over the leaves (on
    // the tensor cores at this width):
    //   y1 = L11^-1 (P D b)_1;  (P D b)_2 -= L21 y1;  y2 = L22^-1 (P D b)_2;
    //   x2 = U22^-1 y2;  y1 -= U12 x2;  x1 = U11^-1 y1
    const long long ldu = (long long)nl * n, s2 = (long long)n * n;
    CK(hps::launch_lu_solve_part(h->X, h->lu_perm, h->lu_dsc, nl, n, nb, R, tl, (long long)nl * nb, nb, s,
                                 (long long)nl * ni, ni, u, ldu, n, false, 0, b1, true, true, false, st));
    GemmDesc gl = gemm(n - b1, R, b1, nl, F(elem(h->X, b1, 0), n, s2, 0), mat(u, ldu, n), mat(u + b1, ldu, n));
    gl.alpha = make_double2(-1.0, 0.0);
    gl.D = mat(u + b1, ldu, n);
    gl.beta = make_double2(1.0, 0.0);
    if (int rc = solve_gemm(&gl, 1, st, wb, ws, pl.oz, h->d_status)) return rc;
    CK(hps::launch_lu_solve_part(h->X, h->lu_perm, h->lu_dsc, nl, n, nb, R, nullptr, 0, 0, nullptr, 0, 0, u, ldu,
                                 n, false, b1, n, false, true, true, st));
    GemmDesc gu = gemm(b1, R, n - b1, nl, F(elem(h->X, (long long)b1 * n, 0), n, s2, 0), mat(u + b1, ldu, n),
                       mat(u, ldu, n));
    gu.alpha = make_double2(-1.0, 0.0);
    gu.D = mat(u, ldu, n);
    gu.beta = make_double2(1.0, 0.0);
    if (int rc = solve_gemm(&gu, 1, st, wb, ws, pl.oz, h->d_status)) return rc;
    CK(hps::launch_lu_solve_part(h->X, h->lu_perm, h->lu_dsc, nl, n, nb, R, nullptr, 0, 0, nullptr, 0, 0, u, ldu,
                                 n, false, 0, b1, false, false, true, st));
  } else if (pl.leaf_lu) {
    if (rec)
      rec->lu_tail = true;  // its own launch after the program
    else
      CK(lu_leaf_solve(h, s, tl, u, R, st));
  } else {
    g = gemm(n, R, n, nl, F(h->X, n, (long long)n * n, lf), mat(tl, (long long)nl * nb, nb),
             mat(u, (long long)nl * n, n));
    g.B2 = mat(s, (long long)nl * ni, ni);
    g.ksplit = nb;
    g.cf32 = lf;
    if (int rc = gemms(&g, 1)) return rc;
  }

  return HPS_OK;
}

// A solve with one or two right-hand sides as one launch: the program of
// the handle for (R, refinement jumps or not), recorded from solve_launch at
// the first such call (may_alloc: its device copy may be allocated now),
// then the engine over this call's s, t, u and workspace, and for leaves in
// LU form their sweeps.  Returns 1 when the solve was launched, 0 when the
// caller launches it step by step, or minus an error code.
static int run_engine(hps_handle *h, const double2 *s, const double2 *t, double2 *u, int R, char *wb,
                      const SolveWs &ws, cudaStream_t st, const double2 *JA, const double2 *JB, bool may_alloc) {
  if (R < 1 || R > 2 || !ws.oen) return 0;
  // opt-in: measured at 16 x 16 leaves, p = 16, 1 right-hand side, the
  // program takes 0.80 ms against 0.59 ms for the step-by-step launches (a
  // grid barrier costs ~2.7 us and a work unit ~4-5 us of dependent-load
  // latency, over 43 dependent phases)
  const char *e = getenv("HPS_SOLVE_ENGINE");
  if (!e || e[0] != '1') return 0;
  const int grid = hps::engine_grid();
  if (grid <= 0 || grid > kEnGridMax) return 0;
  const Plan &pl = h->plan;
  hps_handle::EnProg &pg = h->eng[R - 1][(JA && JB) ? 1 : 0];
  if (pg.failed) return 0;
  if (!pg.d_ops) {
    if (!may_alloc) return 0;
    SolveRec rec;
    rec.grid = grid;
    rec.R = R;
    const char *b[5] = {nullptr, (const char *)s, (const char *)t, (const char *)u, wb};
    const size_t sz[5] = {0, sizeof(double2) * (size_t)R * pl.leaves * pl.ni, sizeof(double2) * (size_t)R * pl.nbdry,
                          sizeof(double2) * (size_t)R * pl.leaves * pl.n, ws.bytes};
    for (int k = 1; k <= 4; k++) {
      rec.lo[k] = b[k];
      rec.hi[k] = b[k] + sz[k];
    }
    for (int k = 1; k <= 3; k++)
      for (int m = k + 1; m <= 3; m++)
        if (rec.lo[k] < rec.hi[m] && rec.lo[m] < rec.hi[k]) rec.ok = false;  // s, t, u overlap
    if (rec.ok) {
      const int rc = solve_launch(h, s, t, u, R, wb, ws, st, JA, JB, &rec);
      if (rc) return -rc;
    }
    if (!rec.ok || rec.ops.empty()) {
      pg.failed = true;
      return 0;
    }
    const size_t bytes = sizeof(hps::EnOp) * rec.ops.size();
    CK_NEG(cudaMalloc((void **)&pg.d_ops, bytes));
    CK_NEG(cudaMemcpy(pg.d_ops, rec.ops.data(), bytes, cudaMemcpyHostToDevice));
    pg.nops = (int)rec.ops.size();
    pg.lu_tail = rec.lu_tail;
  }
  CK_NEG(cudaMemsetAsync(wb + ws.oen, 0, ws.en_clear, st));
  hps::EnArgs a;
  memset(&a, 0, sizeof(a));
  a.ops = pg.d_ops;
  a.nops = pg.nops;
  a.base[0] = nullptr;
  a.base[1] = s;
  a.base[2] = t;
  a.base[3] = u;
  a.base[4] = wb;
  a.bar = (unsigned *)(wb + ws.oen);
  a.cnt = a.bar + 4;
  a.part = (double2 *)(wb + ws.en_part);
  a.status = h->d_status;
  CK_NEG(hps::launch_solve_engine(a, st));
  if (pg.lu_tail) {
    const double2 *tl = (const double2 *)(wb + (pl.gauss ? ws.otc : ws.ot[0]));
    CK_NEG(lu_leaf_solve(h, s, tl, u, R, st));
  }
  return 1;
}

// Iterative refinement of an HPS_MIXED solve: u = S(s, t), then per step the
// complex128 residual of the global collocation system and u += S(residual).
static int solve_refine(hps_handle *h, const double2 *s, const double2 *t, double2 *u, int R, char *wb,
                        const SolveWs &ws, cudaStream_t st) {
  const Plan &pl = h->plan;
  int rc = solve_launch(h, s, t, u, R, wb, ws, st);
  if (rc) return rc;
  auto W = [&](size_t o) { return (double2 *)(wb + o); };
  double2 *sd = W(ws.osd), *td = W(ws.otd), *Fu = W(ws.ofu), *Gu = W(ws.ogu);
  double2 *JA = W(ws.oja), *JB = W(ws.ojb), *d = W(ws.od);
  hps::ResidualSetup rs;
  rs.tab = (const double *)h->tables;
  rs.c = h->c_dev;
  rs.p = pl.p;
  rs.e = pl.e;
  rs.n = pl.n;
  rs.nb = pl.nb;
  rs.ni = pl.ni;
  rs.leaves = pl.leaves;
  rs.nbdry = pl.nbdry;
  rs.eta = make_double2(h->desc.eta_re, h->desc.eta_im);
  rs.kappa2 = h->desc.kappa * h->desc.kappa;
  rs.outer = h->d_outer;
  rs.total_pairs = pl.total_pairs;
  rs.nlev = (int)pl.lv.size();
  for (size_t j = 0; j < pl.lv.size() && j < hps::kMaxLevels; j++) {
    rs.lev[j].pairs = pl.lv[j].d_pairs;
    rs.lev[j].n3 = pl.lv[j].n3;
    rs.lev[j].lpp = pl.lv[j].leaves_per_parent;
    rs.lev[j].off = pl.lv[j].jump_off;
  }
  for (int it = 0; it < pl.refine_steps; it++) {
    CK(hps::launch_residual(rs, u, s, t, sd, td, Fu, Gu, JA, JB, R, st));
    rc = solve_launch(h, sd, td, d, R, wb, ws, st, JA, JB);
    if (rc) return rc;
    CopyBatch cb;
    cb.count = 1;
    cb.d[0] = copy(pl.n * pl.leaves, R, 1, mat(d, (long long)pl.n * pl.leaves, 0),
                   mat(u, (long long)pl.n * pl.leaves, 0));
    cb.d[0].accumulate = 1;
    CK(hps::launch_copy(cb, st));
  }
  return HPS_OK;
}

// ---- fixed workspace of hps_solve_noalloc ----------------------------------
// The array lives in the library's device image: every GPU that loads the
// library holds HPS_NOALLOC_WORKSPACE_BYTES of it until the process exits.
// Host code may not use its name as a device address; the address comes from
// cudaGetSymbolAddress, taken once per device with that device current.
static __device__ __align__(256) unsigned char g_noalloc_ws[HPS_NOALLOC_WORKSPACE_BYTES];

// HPS_OK when the current device is the one the handle's operators live on;
// launches from another device would read them through the wrong context.
static int on_handle_device(const hps_handle *h) {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  return dev == h->device ? HPS_OK : HPS_EINVAL;
}

static int noalloc_ws_ptr(char **out) {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static void *ptrs[kMaxDev] = {nullptr};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) return HPS_ECUDA;
  std::lock_guard<std::mutex> lock(mu);
  if (!ptrs[dev]) {
    void *p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_ws);
    if (err != cudaSuccess || !p) return HPS_ECUDA;
    ptrs[dev] = p;
  }
  *out = (char *)ptrs[dev];
  return HPS_OK;
}

namespace {

// Gauss-Legendre nodes on [-1, 1], increasing: the roots of the Legendre
// polynomial P_q, each by Newton's method from the asymptotic estimate
// -cos(pi (i + 3/4) / (q + 1/2)), with P_q and P_q' from the three-term
// recurrence k P_k = (2k - 1) z P_{k-1} - (k - 1) P_{k-2}.
std::vector<double> gauss_legendre_nodes(int q) {
  const double pi = std::acos(-1.0);
  std::vector<double> x(q);
  for (int i = 0; i < q; i++) {
    double z = -std::cos(pi * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 64; it++) {
      double pm = 1.0, pk = z;  // P_{k-1}, P_k at k = 1
      for (int k = 2; k <= q; k++) {
        const double pn = ((2.0 * k - 1.0) * z * pk - (k - 1.0) * pm) / k;
        pm = pk;
        pk = pn;
      }
      const double dz = pk / (q * (z * pk - pm) / (z * z - 1.0));
      z -= dz;
      if (std::fabs(dz) <= 1e-15) break;
    }
    x[i] = z;
  }
  std::sort(x.begin(), x.end());
  return x;
}

// L[i][j] = l_j(y_i), row-major: the Lagrange basis of the nodes x at the
// points y, i.e. the map from values at x to values at y of the polynomial
// of degree < |x| through them
void lagrange_matrix(const std::vector<double> &x, const std::vector<double> &y, double2 *L) {
  const int n = (int)x.size();
  for (int i = 0; i < (int)y.size(); i++)
    for (int j = 0; j < n; j++) {
      double v = 1.0;
      for (int k = 0; k < n; k++)
        if (k != j) v *= (y[i] - x[k]) / (x[j] - x[k]);
      L[(size_t)i * n + j] = make_double2(v, 0.0);
    }
}

// The root ItI operator in the Gauss-Legendre basis of the boundary data:
// with P the interpolation from the p - 2 corner-free Chebyshev nodes of an
// edge to its q = p - 2 Gauss-Legendre nodes (an invertible change of basis
// between polynomials of degree < q, the same on every edge, which all run
// in increasing coordinate), R_G = diag(P) R diag(P)^-1.  Rt holds R^T
// column-major (the public row-major R) and is overwritten with R_G^T =
// diag(P^-T) R^T diag(P^T): two batched products over the edges, through a
// temporary of the size of R.
int root_R_to_gauss(const Plan &pl, double2 *Rt, cudaStream_t st) {
  const int e = pl.e, nbr = pl.nbdry, edges = nbr / e;
  std::vector<double> xc(e);
  for (int j = 0; j < e; j++) xc[j] = -std::cos(std::acos(-1.0) * (j + 1) / (pl.p - 1));
  const std::vector<double> xg = gauss_legendre_nodes(e);
  std::vector<double2> tab(2 * (size_t)e * e);
  lagrange_matrix(xc, xg, tab.data());                   // P
  lagrange_matrix(xg, xc, tab.data() + (size_t)e * e);   // P^-1
  const size_t tbytes = align256(sizeof(double2) * tab.size());
  char *tmp = nullptr;
  CK(lib_malloc_async((void **)&tmp, tbytes + sizeof(double2) * (size_t)nbr * nbr, st));
  const double2 *dP = (const double2 *)tmp, *dPi = dP + (size_t)e * e;
  double2 *T = (double2 *)(tmp + tbytes);
  // host tables are pageable: the copy has taken them when it returns
  cudaError_t err = cudaMemcpyAsync(tmp, tab.data(), sizeof(double2) * tab.size(), cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) {
    // a row-major P read as a column-major matrix is P^T
    // T = diag(P^-T) R^T: edge r's rows of T from edge r's rows of R^T
    GemmDesc g1 = gemm(e, nbr, e, edges, mat(dPi, e, 0), mat(Rt, nbr, e), mat(T, nbr, e));
    // R_G^T = T diag(P^T): edge c's columns
    GemmDesc g2 = gemm(nbr, e, e, edges, mat(T, nbr, (long long)e * nbr), mat(dP, e, 0),
                       mat(Rt, nbr, (long long)e * nbr));
    err = hps::launch_gemm(&g1, 1, st);
    if (err == cudaSuccess) err = hps::launch_gemm(&g2, 1, st);
  }
  const cudaError_t ferr = cudaFreeAsync(tmp, st);
  if (err != cudaSuccess) return cuda_fail(err);
  return cuda_fail(ferr);
}

}  // namespace

extern "C" {

const char *hps_strerror(int code) {
  switch (code) {
    case HPS_OK: return "success";
    case HPS_EINVAL: return "invalid argument";
    case HPS_ENOMEM: return "out of device memory (or over HPS_MEM_CAP_BYTES)";
    case HPS_ESINGULAR: return "zero pivot in a leaf or interface matrix";
    case HPS_ETIMEOUT: return "bounded device wait timed out";
    case HPS_ECUDA: return "CUDA runtime error";
    case HPS_ENOTSUP: return "not supported for this request (sizes or precision; see the call)";
    case HPS_ETOOBIG: return "request needs more than the fixed no-allocation workspace";
    default: return "unknown error";
  }
}

int hps_nodes(const hps_desc *desc, double *leaf_xy, double *bdry_xy) {
  int st = check_desc(desc);
  if (st) return st;
  const int mx = desc->mx, my = desc->my, p = desc->p, e = p - 2, n = p * p - 4;
  const std::vector<int> dirs = merge_dirs(mx, my);
  const double hx = (desc->x1 - desc->x0) / mx, hy = (desc->y1 - desc->y0) / my;
  std::vector<double> xs, ys, D;
  if (leaf_xy) {
    for (int l = 0; l < mx * my; l++) {
      int col, row;
      leaf_decode(l, dirs, col, row);
      cheb(p, desc->x0 + col * hx, desc->x0 + (col + 1) * hx, xs, D);
      cheb(p, desc->y0 + row * hy, desc->y0 + (row + 1) * hy, ys, D);
      for (int k = 0; k < n; k++) {
        int ix, iy;
        local_grid(p, k, ix, iy);
        leaf_xy[((size_t)l * n + k) * 2] = xs[ix];
        leaf_xy[((size_t)l * n + k) * 2 + 1] = ys[iy];
      }
    }
  }
  if (bdry_xy) {
    // q Gauss-Legendre nodes per leaf edge when q is neither 0 nor p - 2
    const bool gauss = desc->q != 0 && desc->q != e;
    const std::vector<double> zg = gauss ? gauss_legendre_nodes(desc->q) : std::vector<double>();
    size_t q = 0;
    for (int side = 0; side < 4; side++) {
      const bool horiz = (side == 0 || side == 2);
      for (int c = 0; c < (horiz ? mx : my); c++) {
        if (horiz)
          cheb(p, desc->x0 + c * hx, desc->x0 + (c + 1) * hx, xs, D);
        else
          cheb(p, desc->y0 + c * hy, desc->y0 + (c + 1) * hy, ys, D);
        const double lo = horiz ? desc->x0 + c * hx : desc->y0 + c * hy, len = horiz ? hx : hy;
        for (int k = 1; k <= (gauss ? desc->q : e); k++, q++) {
          const double along = gauss ? lo + 0.5 * (zg[k - 1] + 1.0) * len : (horiz ? xs[k] : ys[k]);
          double x = horiz ? along : (side == 1 ? desc->x1 : desc->x0);
          double y = horiz ? (side == 0 ? desc->y0 : desc->y1) : along;
          bdry_xy[2 * q] = x;
          bdry_xy[2 * q + 1] = y;
        }
      }
    }
  }
  return HPS_OK;
}

int hps_free(hps_handle *h) {
  if (!h) return HPS_OK;
  if (Shared *sh = h->sh) {
    bool last;
    {
      std::lock_guard<std::mutex> lock(g_shared_mu);
      last = (--sh->refs == 0);
    }
    if (last) {
      for (cudaEvent_t e : sh->ev) cudaEventDestroy(e);
      for (cudaEvent_t e : sh->oz_ev)
        if (e) cudaEventDestroy(e);
      if (sh->graph) cudaGraphExecDestroy(sh->graph);
      if (sh->arena) cudaFree(sh->arena);
      delete sh;
    }
  }
  if (h->ws) cudaFree(h->ws);
  if (h->stage) cudaFree(h->stage);
  for (auto &row : h->eng)
    for (auto &pg : row)
      if (pg.d_ops) cudaFree(pg.d_ops);
  delete h;
  return HPS_OK;
}

int hps_info(const hps_handle *h, hps_info_t *info) {
  if (!h || !info) return HPS_EINVAL;
  *info = h->info;
  return HPS_OK;
}

// Parents of one merge level that go through the level's kernels together:
// the same precision and the same destination (the level's R buffer, or the
// root block when these parents are roots).
struct BuildRun {
  long long p0;    // first parent of the run in the level's numbering
  int P;           // parents
  int f32;         // complex64 operators and arithmetic
  bool finishing;  // the parents are the roots of their problems
  int k0, nk;      // problems [k0, k0 + nk) in build order
  size_t op[7];    // arena offsets: Winv, R33a, R33b, R13a, R23b, Phia, Phib
  size_t rout;     // byte offset of the run's R^tau in the level's R buffer
  size_t root;     // arena offset of the root block (finishing runs)
  GJChoice gj;
};

// Children of a run: a contiguous range of the level below held by one run
// there (or by the leaves), or several pieces that are gathered first.
struct ChildPiece {
  long long c0, count;  // children [c0, c0 + count) in the lower level's numbering
  int run;              // run of the lower level holding them (-1: the leaves)
};

static std::vector<ChildPiece> child_pieces(const std::vector<std::vector<BuildRun>> &runs, int j,
                                            const BuildRun &r) {
  std::vector<ChildPiece> out;
  const long long c0 = 2 * r.p0, c1 = 2 * (r.p0 + r.P);
  if (j == 0) {
    out.push_back({c0, c1 - c0, -1});
    return out;
  }
  const std::vector<BuildRun> &lo = runs[j - 1];
  for (size_t q = 0; q < lo.size(); q++) {
    const long long a = std::max(c0, lo[q].p0), b = std::min(c1, lo[q].p0 + lo[q].P);
    if (a < b) out.push_back({a, b - a, (int)q});
  }
  return out;
}

// Runs of every merge level of the handles hs (build order) and each
// problem's first parent on each of its levels, with the kernel regime of
// every run's interface inverses.
static int plan_runs(const std::vector<hps_handle *> &hs, std::vector<std::vector<BuildRun>> &runs,
                     std::vector<std::vector<long long>> &first) {
  const int K = (int)hs.size();
  const Plan &P0 = hs[0]->plan;
  const int Lmax = P0.L;
  runs.assign(Lmax, {});
  first.assign(K, {});
  for (int j = 0; j < Lmax; j++) {
    long long pos = 0;
    for (int k = 0; k < K && hs[k]->plan.L > j; k++) {
      const Level &Lk = hs[k]->plan.lv[j];
      const bool fin = (hs[k]->plan.L == j + 1);
      std::vector<BuildRun> &R = runs[j];
      if (!R.empty() && R.back().f32 == Lk.f32 && R.back().finishing == fin) {
        R.back().P += Lk.P;
        R.back().nk++;
      } else {
        BuildRun r{};
        r.p0 = pos;
        r.P = Lk.P;
        r.f32 = Lk.f32;
        r.finishing = fin;
        r.k0 = k;
        r.nk = 1;
        R.push_back(r);
      }
      first[k].push_back(pos);
      pos += Lk.P;
    }
    for (BuildRun &r : runs[j]) {
      if (r.finishing && r.f32) return HPS_ENOTSUP;  // roots are complex128
      if (!choose_gj(P0.lv[j].n3, r.P, r.f32, r.gj)) return HPS_ENOTSUP;
    }
  }
  return HPS_OK;
}

// Algorithm 1 for every handle of hs at once.  hs is in build order: tallest
// tree first, all with the same p, precision and top-level count; each has
// its plan.  Leaves of all problems are numbered problem after problem and
// go through one leaf launch (chunked only to bound the scratch); merge
// level j numbers the parents of every problem that has that level the same
// way, so the parents of a problem's boxes on level j are boxes 2b, 2b+1 of
// level j-1 in that numbering.  The index maps of level j depend on j only
// (the box shape after j merges), so one copy of them serves every problem.
// On success every handle refers to one Shared allocation.
static int build_many(const std::vector<hps_handle *> &hs, const std::vector<const double *> &cin,
                      cudaStream_t st) {
  const int K = (int)hs.size();
  const Plan &P0 = hs[0]->plan;
  const int n = P0.n, nb = P0.nb, ni = P0.ni, p = P0.p, lf = P0.leaf_f32;
  const int Lmax = P0.L;
  const bool mixed = P0.mixed;
  const long long esl = lf ? 8 : 16;
  auto esz = [](int f32) { return f32 ? 8LL : 16LL; };

  std::vector<long long> leaf0(K + 1, 0);
  for (int k = 0; k < K; k++) leaf0[k + 1] = leaf0[k] + hs[k]->plan.leaves;
  const long long NL = leaf0[K];

  // every problem's merge levels must have the tallest tree's shapes (true
  // for square grids of any size; rectangular ones share the first levels
  // with a square grid up to where their axes stop alternating)
  for (int k = 1; k < K; k++)
    for (int j = 0; j < hs[k]->plan.L; j++) {
      const Level &A = P0.lv[j], &B = hs[k]->plan.lv[j];
      if (A.horizontal != B.horizontal || A.nc != B.nc || A.n1 != B.n1 || A.n2 != B.n2 || A.n3 != B.n3)
        return HPS_EINVAL;
    }

  // ---- runs of every merge level, and each problem's first parent there ----
  std::vector<std::vector<BuildRun>> runs;
  std::vector<std::vector<long long>> first;
  {
    int rc = plan_runs(hs, runs, first);
    if (rc != HPS_OK) return rc;
  }

  // ---- one arena: leaf operators, merge operators, roots, tables, maps ----
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const size_t oX = take((size_t)(esl * NL * n * n));
  const size_t oGX = take((size_t)(esl * NL * n * nb));
  const size_t oPerm = P0.leaf_lu ? take(sizeof(int) * (size_t)NL * n) : 0;
  const size_t oDsc = P0.leaf_lu ? take(sizeof(double) * (size_t)NL * n) : 0;
  // boundary data on Gauss-Legendre nodes: the leaves' interface operators
  // [Ph R Qh | Ph Gamma] and the edge interpolation tables P (qe x e) and
  // Q (e x qe), column-major
  const bool gauss = P0.gauss;
  const int nbi = P0.nbi, qe = P0.qe, e0 = P0.e;
  const size_t oGXi = gauss ? take(16ULL * NL * nbi * (nbi + ni)) : 0;
  const size_t oIP = gauss ? take(16ULL * 2 * qe * e0) : 0;
  const size_t gxi_off = gauss ? oGXi : oGX;
  const long long gxi_ld = gauss ? nbi : nb, gxi_stride = gauss ? (long long)nbi * (nbi + ni) : (long long)n * nb;
  const int gxi_f32 = gauss ? 0 : lf;
  const long long gxi_es = gauss ? 16 : esl;
  for (int j = 0; j < Lmax; j++) {
    const Level &S = P0.lv[j];
    const long long n1 = S.n1, n2 = S.n2, n3 = S.n3, nt = S.nt;
    const long long per[7] = {n3 * n3, n3 * n3, n3 * n3, n1 * n3, n2 * n3, n3 * nt, n3 * nt};
    for (BuildRun &r : runs[j]) {
      for (int q = 0; q < 7; q++) r.op[q] = take((size_t)(esz(r.f32) * r.P * per[q]));
      if (r.finishing) r.root = take((size_t)(16LL * r.P * nt * nt));
    }
  }
  // problems with a single leaf: the root is the leaf's R
  int k1 = K;
  while (k1 > 0 && hs[k1 - 1]->plan.L == 0) k1--;
  const size_t oRoot1 = take(16ULL * (K - k1) * nbi * nbi);
  const size_t tab_bytes = sizeof(double) * 4 * p * p + sizeof(int) * (n + p * p);
  std::vector<size_t> oTab(K), oC(K, 0);
  for (int k = 0; k < K; k++) {
    oTab[k] = take(tab_bytes);
    oC[k] = take(sizeof(double) * (size_t)hs[k]->plan.leaves * ni);
  }
  // index maps: per level I1, I2, I3a, I3b, the I3 pairs; per problem the
  // root and outer maps
  std::vector<int> ints;
  std::vector<size_t> imap((size_t)Lmax * 5);
  for (int j = 0; j < Lmax; j++) {
    const Level &L = P0.lv[j];
    const std::vector<int> *v[5] = {&L.I1, &L.I2, &L.I3a, &L.I3b, &L.pairs};
    for (int q = 0; q < 5; q++) {
      imap[5 * j + q] = ints.size();
      ints.insert(ints.end(), v[q]->begin(), v[q]->end());
    }
  }
  std::vector<size_t> root_at(K), outer_at(K);
  for (int k = 0; k < K; k++) {
    const Plan &pk = hs[k]->plan;
    root_at[k] = ints.size();
    ints.insert(ints.end(), pk.root_src.begin(), pk.root_src.end());
    outer_at[k] = ints.size();
    ints.insert(ints.end(), pk.outer.begin(), pk.outer.end());
  }
  const size_t oInts = take(sizeof(int) * (ints.size() + 1));
  const size_t oStatus = take(sizeof(unsigned int));
  const size_t oProbs = take(sizeof(hps::LeafProb) * K);

  long long cap = env_cap();
  if (cap >= 0 && (long long)off > cap) return HPS_ENOMEM;
  Shared *sh = new (std::nothrow) Shared();
  if (!sh) return HPS_ENOMEM;
  sh->bytes = off;
  sh->refs = K;
  {
    cudaError_t err = cudaMalloc(&sh->arena, off);
    if (err != cudaSuccess) {
      delete sh;
      return cuda_fail(err);
    }
  }
  char *base = (char *)sh->arena;
  for (int k = 0; k < K; k++) hs[k]->sh = sh;  // from here on hps_free releases it
  sh->order = hs;

  // ---- every problem's view of the arena ----
  int *d_ints = (int *)(base + oInts);
  unsigned int *d_status = (unsigned int *)(base + oStatus);
  for (int k = 0; k < K; k++) {
    hps_handle *h = hs[k];
    Plan &pl = h->plan;
    h->X = base + oX + esl * leaf0[k] * n * n;
    h->GX = base + oGX + esl * leaf0[k] * n * nb;
    h->GXi = base + gxi_off + gxi_es * leaf0[k] * gxi_stride;
    h->gxi_ld = gxi_ld;
    h->gxi_stride = gxi_stride;
    if (gauss) h->d_Qcm = (const double2 *)(base + oIP) + (size_t)qe * e0;
    if (P0.leaf_lu) {
      h->lu_perm = (int *)(base + oPerm) + leaf0[k] * n;
      h->lu_dsc = (double *)(base + oDsc) + leaf0[k] * n;
    }
    for (int j = 0; j < pl.L; j++) {
      Level &L = pl.lv[j];
      const long long pos = first[k][j];
      const BuildRun *r = nullptr;
      for (const BuildRun &q : runs[j])
        if (pos >= q.p0 && pos < q.p0 + q.P) r = &q;
      const long long d = pos - r->p0, e = esz(r->f32);
      const long long n1 = L.n1, n2 = L.n2, n3 = L.n3, nt = L.nt;
      const long long per[7] = {n3 * n3, n3 * n3, n3 * n3, n1 * n3, n2 * n3, n3 * nt, n3 * nt};
      void **dst[7] = {&L.Winv, &L.R33a, &L.R33b, &L.R13a, &L.R23b, &L.Phia, &L.Phib};
      for (int q = 0; q < 7; q++) *dst[q] = base + r->op[q] + e * d * per[q];
      L.d_I1 = d_ints + imap[5 * j + 0];
      L.d_I2 = d_ints + imap[5 * j + 1];
      L.d_I3a = d_ints + imap[5 * j + 2];
      L.d_I3b = d_ints + imap[5 * j + 3];
      L.d_pairs = d_ints + imap[5 * j + 4];
      if (j == pl.L - 1) h->Rroot = (double2 *)(base + r->root + 16 * d * nt * nt);
    }
    if (pl.L == 0) h->Rroot = (double2 *)(base + oRoot1 + 16ULL * (k - k1) * nbi * nbi);
    h->tables = base + oTab[k];
    h->c_dev = (double *)(base + oC[k]);
    h->d_ints = d_ints;
    h->d_status = d_status;
    h->d_root_src = d_ints + root_at[k];
    h->d_outer = d_ints + outer_at[k];
  }

  // ---- host tables: 1-D differentiation on the leaf, squared, node grid ----
  std::vector<unsigned char> tab(tab_bytes);
  for (int k = 0; k < K; k++) {
    const hps_desc &dk = hs[k]->desc;
    const double hx = (dk.x1 - dk.x0) / hs[k]->plan.m, hy = (dk.y1 - dk.y0) / hs[k]->plan.my;
    std::vector<double> x, D1x, D1y;
    cheb(p, 0.0, hx, x, D1x);
    cheb(p, 0.0, hy, x, D1y);
    double *T = (double *)tab.data();
    for (int i = 0; i < p * p; i++) {
      T[i] = D1x[i];
      T[p * p + i] = D1y[i];
    }
    for (int i = 0; i < p; i++)
      for (int jj = 0; jj < p; jj++) {
        double sx = 0.0, sy = 0.0;
        for (int q = 0; q < p; q++) {
          sx += D1x[i * p + q] * D1x[q * p + jj];
          sy += D1y[i * p + q] * D1y[q * p + jj];
        }
        T[2 * p * p + i * p + jj] = sx;
        T[3 * p * p + i * p + jj] = sy;
      }
    int *G = (int *)(T + 4 * p * p);
    int *Loc = G + n;
    for (int q = 0; q < p * p; q++) Loc[q] = -1;
    for (int q = 0; q < n; q++) {
      int ix, iy;
      local_grid(p, q, ix, iy);
      G[q] = ix | (iy << 8);
      Loc[iy * p + ix] = q;
    }
    CK(cudaMemcpyAsync(hs[k]->tables, tab.data(), tab_bytes, cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemcpyAsync(d_ints, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(d_status, 0, sizeof(unsigned int), st));
  if (gauss) {
    // P: the Chebyshev-edge interpolant at the Gauss nodes; Q: the
    // Gauss-node interpolant at the Chebyshev edge nodes (reference edge)
    std::vector<double> xc(e0);
    for (int j = 0; j < e0; j++) xc[j] = -std::cos(std::acos(-1.0) * (j + 1) / (p - 1));
    const std::vector<double> zg = gauss_legendre_nodes(qe);
    std::vector<double2> Prm((size_t)qe * e0), Qrm((size_t)e0 * qe), tab2(2 * (size_t)qe * e0);
    lagrange_matrix(xc, zg, Prm.data());  // row-major qe x e0
    lagrange_matrix(zg, xc, Qrm.data());  // row-major e0 x qe
    for (int a = 0; a < qe; a++)
      for (int j = 0; j < e0; j++) {
        tab2[(size_t)a + (size_t)j * qe] = Prm[(size_t)a * e0 + j];                 // P column-major
        tab2[(size_t)qe * e0 + j + (size_t)a * e0] = Qrm[(size_t)j * qe + a];       // Q column-major
      }
    // (pageable host memory: the copy has taken the table when it returns)
    CK(cudaMemcpyAsync(base + oIP, tab2.data(), sizeof(double2) * tab2.size(), cudaMemcpyHostToDevice, st));
  }

  // ---- c into the arena (the leaf kernel and the mixed path's residual read
  // it there; hps_rebuild replaces it) ----
  std::vector<hps::LeafProb> probs(K);
  for (int k = 0; k < K; k++) {
    const size_t cb = sizeof(double) * (size_t)hs[k]->plan.leaves * ni;
    CK(cudaMemcpyAsync(hs[k]->c_dev, cin[k], cb, cudaMemcpyDefault, st));
    probs[k].tab = (const double *)hs[k]->tables;
    probs[k].c = hs[k]->c_dev;
    probs[k].leaf0 = leaf0[k];
    probs[k].eta = make_double2(hs[k]->desc.eta_re, hs[k]->desc.eta_im);
    probs[k].kappa2 = hs[k]->desc.kappa * hs[k]->desc.kappa;
  }
  hps::LeafProb *d_probs = (hps::LeafProb *)(base + oProbs);
  CK(cudaMemcpyAsync(d_probs, probs.data(), sizeof(hps::LeafProb) * K, cudaMemcpyHostToDevice, st));

  sh->ev.assign(Lmax + 2, nullptr);
  for (cudaEvent_t &e : sh->ev) CK(cudaEventCreate(&e));
  const std::vector<cudaEvent_t> ev = sh->ev;
  // the device work of the build from here on: run now, and captured into a
  // CUDA graph by hps_rebuild (it reads c and every table from the arena)
  auto compute = [=](cudaStream_t st, bool events, int &launches) mutable -> int {
    // ---- leaves (Sec. 2.1): one cluster launch over every problem's leaves ----
    hps::LeafTables lt;
    lt.p = p;
    lt.e = P0.e;
    lt.n = n;
    lt.nb = nb;
    lt.ni = ni;
    const int lcs = leaf_cluster(P0, NL);
    if (lcs == 0) return HPS_ENOTSUP;
    const int chunk = (int)leaf_chunk(P0, NL);
    void *lscr = nullptr;
    int *lmeta = nullptr;
    const size_t rscr = P0.leaf_refined ? hps::leaf_refined_scratch_bytes(lt, chunk) : 0;
    if (P0.leaf_refined)
      CK(lib_malloc_async(&lscr, rscr, st));
    else if (!P0.leaf_lu)
      CK(lib_malloc_async(&lscr, (size_t)esl * chunk * n * n, st));
    if (!P0.leaf_refined)
      CK(lib_malloc_async((void **)&lmeta,
                         sizeof(int) * (size_t)chunk * (P0.leaf_lu ? hps::lu_meta_ints(n) : hps::gj_meta_ints(n)),
                         st));
    // the complex64 inverse of the refined form: its own cluster rule
    Plan P32 = P0;
    P32.leaf_f32 = 1;
    const int lcs32 = P0.leaf_refined ? leaf_cluster(P32, std::min<long long>(chunk, NL)) : 0;
    if (P0.leaf_refined && lcs32 == 0) return HPS_ENOTSUP;
    if (events) CK(cudaEventRecord(ev[0], st));
    launches = 0;
    for (long long l0 = 0; l0 < NL; l0 += chunk) {
      const int cnt = (int)std::min<long long>(chunk, NL - l0);
      if (P0.leaf_lu) {
        CK(hps::launch_leaf_lu(lt, d_probs, K, l0, cnt, base + oX, base + oGX, (int *)(base + oPerm),
                               (double *)(base + oDsc), lmeta, d_status, Lmax, lcs, lf != 0, st));
        launches++;
      } else if (P0.leaf_refined) {
        CK(hps::launch_leaf_refined(lt, d_probs, K, l0, cnt, base + oX, base + oGX, lscr, rscr, d_status, Lmax,
                                    lcs32, kLeafRefineSteps, st, &launches));
      } else if (lf && hps::gj32_supported(lt)) {
        // complex64 inverse form: 32-column panels, one CTA a leaf
        CK(hps::launch_leaf_gj32(lt, d_probs, K, l0, cnt, base + oX, base + oGX, lscr, d_status, Lmax, st));
        launches++;
      } else {
        CK(hps::launch_leaf(lt, d_probs, K, l0, cnt, base + oX, base + oGX, lscr, lmeta, d_status, Lmax, lcs,
                            lf != 0, st));
        launches++;
      }
    }
    if (gauss) {
      // boundary data on the Gauss nodes: the leaves' interface operators
      // Ph [R | Gamma] then R_G = (Ph R) Qh, with Ph = diag(P, P, P, P),
      // Qh = diag(Q, Q, Q, Q) over the edges [S, E, N, W]: per edge one
      // product with the qe x e (or e x qe) table, batched over the leaves
      const double2 *dP = (const double2 *)(base + oIP), *dQ = dP + (size_t)qe * e0;
      const long long tch = 2048;  // leaves a pass (bounds the temporary)
      double2 *T1 = nullptr;
      CK(lib_malloc_async((void **)&T1, 16ULL * std::min<long long>(tch, NL) * nbi * n, st));
      for (long long l0 = 0; l0 < NL; l0 += tch) {
        const int cnt = (int)std::min<long long>(tch, NL - l0);
        const char *gx = base + oGX + 16 * l0 * n * nb;
        char *gxi = base + oGXi + 16 * l0 * nbi * (nbi + ni);
        GemmDesc gd[4];
        for (int sd = 0; sd < 4; sd++) {  // T1 rows of edge sd = P GX rows of edge sd
          gd[sd] = gemm(qe, n, e0, cnt, mat(dP, qe, 0), mat(gx + 16LL * sd * e0, nb, (long long)n * nb),
                        mat(T1 + (size_t)sd * qe, nbi, (long long)nbi * n));
        }
        CK(hps::launch_gemm(gd, 2, st));
        CK(hps::launch_gemm(gd + 2, 2, st));
        for (int sd = 0; sd < 4; sd++) {  // R_G columns of edge sd = (Ph R) columns of edge sd times Q
          gd[sd] = gemm(nbi, qe, e0, cnt, mat(T1 + (size_t)sd * e0 * nbi, nbi, (long long)nbi * n), mat(dQ, e0, 0),
                        mat(gxi + 16LL * sd * qe * nbi, nbi, (long long)nbi * (nbi + ni)));
        }
        CK(hps::launch_gemm(gd, 2, st));
        CK(hps::launch_gemm(gd + 2, 2, st));
        CopyBatch cg;
        cg.count = 1;  // Gamma_G = Ph Gamma
        cg.d[0] = copy(nbi, ni, cnt, mat(T1 + (size_t)nb * nbi, nbi, (long long)nbi * n),
                       mat(gxi + 16LL * nbi * nbi, nbi, (long long)nbi * (nbi + ni)));
        CK(hps::launch_copy(cg, st));
        launches += 5;
      }
      CK(cudaFreeAsync(T1, st));
    }
    if (events) CK(cudaEventRecord(ev[1], st));
    if (lscr) CK(cudaFreeAsync(lscr, st));
    if (lmeta) CK(cudaFreeAsync(lmeta, st));

    if (k1 < K) {
      // single-leaf problems: the root R is the leaf's R = GX[:, :nb] (on the
      // boundary data points)
      CopyBatch cb;
      cb.count = 1;
      cb.d[0] = copy(nbi, nbi, K - k1, mat(base + gxi_off + gxi_es * leaf0[k1] * gxi_stride, gxi_ld, gxi_stride,
                                           nullptr, nullptr, gxi_f32),
                     mat(base + oRoot1, nbi, (long long)nbi * nbi));
      CK(hps::launch_copy(cb, st));
      launches++;
    }

    // ---- merges (Sec. 2.2), one level at a time (Algorithm 3's level loop) ----
    // scratch: two R buffers (children / parents), then Q, W, converted
    // children (all sized for complex128) and the elimination metadata
    size_t rbytes = 0, qbuf = 0, wbuf = 0, mbuf = 0, cbuf = 0;
    for (int j = 0; j < Lmax; j++) {
      const Level &S = P0.lv[j];
      size_t rb = 0;
      for (BuildRun &r : runs[j]) {
        if (!r.finishing) {
          r.rout = rb;
          rb = align256(rb + (size_t)(esz(r.f32) * r.P * S.nt * S.nt));
        }
        qbuf = std::max(qbuf, (size_t)r.P * S.n3 * S.nt);
        wbuf = std::max(wbuf, (size_t)r.P * S.n3 * S.n3);
        mbuf = std::max(mbuf, (size_t)r.P * hps::gj_meta_ints(S.n3));
        std::vector<ChildPiece> pcs = child_pieces(runs, j, r);
        const int cf = pcs[0].run < 0 ? lf : runs[j - 1][pcs[0].run].f32;
        if (pcs.size() > 1 || cf != r.f32) cbuf = std::max(cbuf, (size_t)2 * r.P * S.nc * S.nc);
      }
      rbytes = std::max(rbytes, rb);
    }
    // workspace of the products done on the tensor cores
    size_t oz_bytes = 0;
    for (int j = 0; j < Lmax; j++) {
      const Level &S = P0.lv[j];
      int mnk[6][3];
      merge_products(S.n1, S.n2, S.n3, S.nt, mnk);
      for (const BuildRun &r : runs[j])
        for (int q = 0; q < 6; q++)
          if (oz_shape(mnk[q][0], mnk[q][1], mnk[q][2], r.P, r.f32, P0.oz))
            oz_bytes = std::max(oz_bytes, oz_bytes_shape(mnk[q][0], mnk[q][1], mnk[q][2], r.P, r.f32));
    }
    // the refined interface inverses' scratch
    size_t wref_bytes = 0;
    for (int j = 0; j < Lmax; j++)
      for (const BuildRun &r : runs[j])
        if (r.gj.refined && !r.f32) wref_bytes = std::max(wref_bytes, wref_layout(P0.lv[j].n3, r.P, P0.oz).total);
    char *scratch = nullptr;
    int *wmeta = nullptr;
    const size_t sbytes = 2 * rbytes + sizeof(double2) * (qbuf + wbuf + cbuf);
    if (Lmax > 0) {
      CK(lib_malloc_async((void **)&scratch, align256(sbytes) + align256(oz_bytes) + wref_bytes, st));
      CK(lib_malloc_async((void **)&wmeta, sizeof(int) * std::max<size_t>(mbuf, 1), st));
    }
    char *Rbuf[2] = {scratch, scratch + rbytes};
    double2 *Q = (double2 *)(scratch + 2 * rbytes);
    double2 *Wscr = Q + qbuf;
    double2 *Rconv = Wscr + wbuf;
    void *ozws = oz_bytes ? scratch + align256(sbytes) : nullptr;
    char *wrscr = wref_bytes ? scratch + align256(sbytes) + align256(oz_bytes) : nullptr;
    // products: emulated ones one at a time, the rest in one launch
    auto run_gemm_on = [&](GemmDesc *gd, int nd, cudaStream_t s) -> int {
      GemmDesc rest[2];
      int nr = 0;
      for (int q = 0; q < nd; q++) {
        int v;
        if (tuned(TuneKey{0, gd[q].M, gd[q].N, gd[q].K, gd[q].batch, gd[q].cf32}, v) && v >= 1 && v <= 7 && v != 5)
          gd[q].cfg = v;
        if (oz_shape(gd[q].M, gd[q].N, gd[q].K, gd[q].batch, gd[q].cf32, P0.oz)) {
          CK(hps::launch_gemm_oz(gd[q], ozws, oz_bytes, s, d_status));
          launches += hps::oz_launches(gd[q]);
        } else {
          rest[nr++] = gd[q];
        }
      }
      if (nr) {
        CK(hps::launch_gemm(rest, nr, s));
        launches++;
      }
      return HPS_OK;
    };
    auto run_gemm = [&](GemmDesc *gd, int nd) -> int { return run_gemm_on(gd, nd, st); };
    // Q = R33b R31a does not depend on W^{-1}: it runs on a side stream while
    // W^{-1} (a chain of small dependent launches) is formed.  (W^{-1} uses
    // no part of the products' workspace, so Q may use it meanwhile.)
    cudaStream_t side = hps::side_stream(st);
    cudaEvent_t fork = nullptr, join = nullptr;
    if (side && (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
                 cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess)) {
      cudaGetLastError();
      side = nullptr;
    }
    struct EvGuard {
      cudaEvent_t &a, &b;
      ~EvGuard() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
      }
    } ev_guard{fork, join};

    auto sub = [&](Mat m, const int *r, const int *c) {
      m.rmap = r;
      m.cmap = c;
      return m;
    };
    for (int j = 0; j < Lmax; j++) {
      const Level &S = P0.lv[j];
      const int n1 = S.n1, n2 = S.n2, n3 = S.n3, nt = S.nt, nc = S.nc;
      const int *dI1 = d_ints + imap[5 * j + 0], *dI2 = d_ints + imap[5 * j + 1];
      const int *dI3a = d_ints + imap[5 * j + 2], *dI3b = d_ints + imap[5 * j + 3];
      for (const BuildRun &r : runs[j]) {
        const int P = r.P, f = r.f32;
        // children's R: in place when one run of this precision holds them all
        const void *Rc;
        int rcf;
        long long ldc, strc;
        std::vector<ChildPiece> pcs = child_pieces(runs, j, r);
        auto piece_src = [&](const ChildPiece &c, int &pf) {
          if (c.run < 0) {
            pf = gxi_f32;
            return mat(base + gxi_off + gxi_es * c.c0 * gxi_stride, gxi_ld, gxi_stride, nullptr, nullptr, gxi_f32);
          }
          const BuildRun &q = runs[j - 1][c.run];
          pf = q.f32;
          return mat(Rbuf[(j - 1) & 1] + q.rout + esz(q.f32) * (c.c0 - q.p0) * nc * nc, nc, (long long)nc * nc,
                     nullptr, nullptr, q.f32);
        };
        int pf0;
        Mat m0 = piece_src(pcs[0], pf0);
        if (pcs.size() == 1 && pf0 == f) {
          Rc = m0.ptr;
          rcf = pf0;
          ldc = m0.ld;
          strc = m0.stride;
        } else {
          // gather (and widen) the children into one complex128 array
          CopyBatch cv;
          cv.count = 0;
          for (const ChildPiece &c : pcs) {
            int pf;
            Mat src = piece_src(c, pf);
            cv.d[cv.count++] = copy(nc, nc, (int)c.count, src,
                                    mat(Rconv + (c.c0 - 2 * r.p0) * nc * nc, nc, (long long)nc * nc));
          }
          CK(hps::launch_copy(cv, st));
          launches++;
          Rc = Rconv;
          rcf = 0;
          ldc = nc;
          strc = (long long)nc * nc;
        }
        void *Rp = r.finishing ? (void *)(base + r.root) : (void *)(Rbuf[j & 1] + r.rout);
        void *Winv = base + r.op[0], *R33a = base + r.op[1], *R33b = base + r.op[2], *R13a = base + r.op[3];
        void *R23b = base + r.op[4], *Phia = base + r.op[5], *Phib = base + r.op[6];
        const long long s2 = 2 * strc;
        Mat Ra = mat(Rc, ldc, s2, nullptr, nullptr, rcf), Rb = mat(elem(Rc, strc, rcf), ldc, s2, nullptr, nullptr, rcf);
        auto M = [&](const void *ptr, long long ld, long long stride) { return mat(ptr, ld, stride, nullptr, nullptr, f); };
        // stored blocks and the parts of Phi_b and R^tau that are copies
        CopyBatch cb;
        cb.count = 0;
        cb.d[cb.count++] = copy(n3, n3, P, sub(Ra, dI3a, dI3a), M(R33a, n3, (long long)n3 * n3));
        cb.d[cb.count++] = copy(n3, n3, P, sub(Rb, dI3b, dI3b), M(R33b, n3, (long long)n3 * n3));
        cb.d[cb.count++] = copy(n1, n3, P, sub(Ra, dI1, dI3a), M(R13a, n1, (long long)n1 * n3));
        cb.d[cb.count++] = copy(n2, n3, P, sub(Rb, dI2, dI3b), M(R23b, n2, (long long)n2 * n3));
        // Q = [R33b R31a | -R32b]: the right block here, the left one by GEMM below
        cb.d[cb.count++] = copy(n3, n2, P, sub(Rb, dI3b, dI2),
                                M(elem(Q, (long long)n1 * n3, f), n3, (long long)n3 * nt), -1.0);
        // Phi_b starts as -[R31a | 0]
        cb.d[cb.count++] = copy(n3, n1, P, sub(Ra, dI3a, dI1), M(Phib, n3, (long long)n3 * nt), -1.0);
        cb.d[cb.count++] = copy(n3, n2, P, mat(nullptr, 0, 0), M(elem(Phib, (long long)n1 * n3, f), n3, (long long)n3 * nt));
        // R^tau starts as diag(R11a, R22b)
        const long long sp = (long long)nt * nt;
        cb.d[cb.count++] = copy(n1, n1, P, sub(Ra, dI1, dI1), M(Rp, nt, sp));
        cb.d[cb.count++] = copy(n2, n2, P, sub(Rb, dI2, dI2), M(elem(Rp, (long long)n1 * nt + n1, f), nt, sp));
        cb.d[cb.count++] = copy(n2, n1, P, mat(nullptr, 0, 0), M(elem(Rp, n1, f), nt, sp));
        cb.d[cb.count++] = copy(n1, n2, P, mat(nullptr, 0, 0), M(elem(Rp, (long long)n1 * nt, f), nt, sp));
        CK(hps::launch_copy(cb, st));

        const long long s33 = (long long)n3 * n3, s3t = (long long)n3 * nt;
        // W = I - R33b R33a (in scratch), then W^{-1} into its stored slot
        GemmDesc g = gemm(n3, n3, n3, P, M(R33b, n3, s33), M(R33a, n3, s33), M(Wscr, n3, s33));
        g.alpha = make_double2(-1.0, 0.0);
        g.addI = 1;
        g.cf32 = f;
        if (int rc = run_gemm(&g, 1)) return rc;
        const int lev = S.lev;  // the tallest tree's level numbering
        // Q(:, :n1) = R33b R31a, beside W^{-1} when there is a side stream
        g = gemm(n3, n1, n3, P, M(R33b, n3, s33), sub(Ra, dI3a, dI1), M(Q, n3, s3t));
        g.cf32 = f;
        if (side) {
          CK(cudaEventRecord(fork, st));
          CK(cudaStreamWaitEvent(side, fork, 0));
          if (int rc = run_gemm_on(&g, 1, side)) return rc;
          CK(cudaEventRecord(join, side));
        } else if (int rc = run_gemm(&g, 1)) {
          return rc;
        }
        if (int rc = w_inverse(r.gj, Wscr, Winv, n3, P, wmeta, d_status, lev, f != 0, wrscr, P0.oz, st, launches))
          return rc;
        if (side) CK(cudaStreamWaitEvent(st, join, 0));
        // Phi_a = W^{-1} Q
        g = gemm(n3, nt, n3, P, M(Winv, n3, s33), M(Q, n3, s3t), M(Phia, n3, s3t));
        g.cf32 = f;
        if (int rc = run_gemm(&g, 1)) return rc;
        // Phi_b = -[R31a | 0] - R33a Phi_a
        g = gemm(n3, nt, n3, P, M(R33a, n3, s33), M(Phia, n3, s3t), M(Phib, n3, s3t));
        g.alpha = make_double2(-1.0, 0.0);
        g.D = g.C;
        g.beta = make_double2(1.0, 0.0);
        g.cf32 = f;
        if (int rc = run_gemm(&g, 1)) return rc;
        // R^tau = diag(R11a, R22b) + diag(R13a, R23b) [Phi_a; Phi_b]
        GemmDesc g2[2];
        g2[0] = gemm(n1, nt, n3, P, M(R13a, n1, (long long)n1 * n3), M(Phia, n3, s3t), M(Rp, nt, sp));
        g2[0].D = g2[0].C;
        g2[0].beta = make_double2(1.0, 0.0);
        g2[0].cf32 = f;
        g2[1] = gemm(n2, nt, n3, P, M(R23b, n2, (long long)n2 * n3), M(Phib, n3, s3t), M(elem(Rp, n1, f), nt, sp));
        g2[1].D = g2[1].C;
        g2[1].beta = make_double2(1.0, 0.0);
        g2[1].cf32 = f;
        if (int rc = run_gemm(g2, 2)) return rc;
        launches += 1;  // the copy (W^{-1} counted by w_inverse)
      }
      if (events) CK(cudaEventRecord(ev[2 + j], st));
    }
    if (scratch) CK(cudaFreeAsync(scratch, st));
    if (wmeta) CK(cudaFreeAsync(wmeta, st));
    return HPS_OK;
  };
  sh->compute = compute;
  int launches = 0;
  // time the product kernels of the tensor-core products of this build
  sh->oz_ev.assign(2 * Shared::kOzTimed, nullptr);  // created as products are launched
  sh->oz_flops.assign(Shared::kOzTimed, 0.0);
  hps::OzTimer timer{sh->oz_ev.data(), sh->oz_flops.data(), Shared::kOzTimed, 0};
  hps::oz_set_timer(&timer);
  int rc = compute(st, true, launches);
  hps::oz_set_timer(nullptr);
  sh->oz_n = timer.n;
  if (rc != HPS_OK) return rc;
  sh->launches = launches;
  return HPS_OK;
}

// Planning shared by hps_build and hps_plan: tree, precisions, kernel
// regimes, sizes.  Returns HPS_OK, HPS_EINVAL or HPS_ENOTSUP.
static int plan_handle(hps_handle *h, const hps_desc *desc) {
  int st0 = check_desc(desc);
  if (st0) return st0;
  h->desc = *desc;
  if (h->desc.q == 0) h->desc.q = desc->p - 2;
  // the mixed path's refinement residual is that of the Chebyshev-edge system
  if (h->desc.q != desc->p - 2 && desc->precision == HPS_MIXED) return HPS_ENOTSUP;
  make_plan(h->desc, h->plan);
  h->leaf_cs = leaf_cluster(h->plan, h->plan.leaves);
  if (h->leaf_cs == 0) return HPS_ENOTSUP;
  fill_info(h->plan, h->info);
  for (const Level &L : h->plan.lv) {
    GJChoice g;
    if (!choose_gj(L.n3, L.P, L.f32, g)) return HPS_ENOTSUP;
    // fill_info counts 7 launches a level
    h->info.build_launches += merge_launches(L.n1, L.n2, L.n3, L.nt, L.P, L.f32, h->plan.oz, g) - 7;
  }
  // transient build memory: the leaf elimination chunk, then the merge scratch
  const Plan &pl = h->plan;
  const long long esz = pl.leaf_f32 ? 8 : 16, n = pl.n;
  const long long chunk = leaf_chunk(pl, pl.leaves);
  const int nchunks = (int)((pl.leaves + chunk - 1) / chunk);
  h->info.build_launches += nchunks - 1;  // leaf chunks
  long long leaf_scr = pl.leaf_lu ? 4LL * chunk * (long long)hps::lu_meta_ints(pl.n)
                                  : esz * chunk * n * n + 4LL * chunk * (long long)hps::gj_meta_ints(pl.n);
  if (pl.leaf_refined) {
    hps::LeafTables lt;
    lt.p = pl.p;
    lt.e = pl.e;
    lt.n = pl.n;
    lt.nb = pl.nb;
    lt.ni = pl.ni;
    leaf_scr = (long long)hps::leaf_refined_scratch_bytes(lt, (int)chunk);
    // per chunk: complex64 inverse, B, X = X0, per step the residual product
    // and the correction (product and FP64 add), G X
    h->info.build_launches += nchunks * (hps::leaf_refined_launches(lt, (int)chunk, kLeafRefineSteps) - 1);
  }
  long long rbuf = 0, qbuf = 0, wbuf = 0, mbuf = 0, cbuf = 0, wref = 0;
  for (size_t j = 0; j < pl.lv.size(); j++) {
    const Level &L = pl.lv[j];
    GJChoice gq;
    if (!L.f32 && choose_gj(L.n3, L.P, 0, gq) && gq.refined)
      wref = std::max(wref, (long long)wref_layout(L.n3, L.P, pl.oz).total);
    rbuf = std::max(rbuf, (long long)L.P * L.nt * L.nt);
    qbuf = std::max(qbuf, (long long)L.P * L.n3 * L.nt);
    wbuf = std::max(wbuf, (long long)L.P * L.n3 * L.n3);
    mbuf = std::max(mbuf, (long long)L.P * (long long)hps::gj_meta_ints(L.n3));
    const int cf = (j == 0) ? pl.leaf_f32 : pl.lv[j - 1].f32;
    if (cf != L.f32) cbuf = std::max(cbuf, 2LL * L.P * L.nc * L.nc);
  }
  const long long merge_scr = 16 * (2 * rbuf + qbuf + wbuf + cbuf) + 4 * mbuf + wref;
  h->info.build_scratch_bytes = std::max(leaf_scr, merge_scr) + (pl.mixed ? 0 : 8LL * pl.leaves * pl.ni);
  SolveWs w1;
  solve_ws_layout(pl, 1, w1);
  h->info.solve_ws_bytes_per_rhs = (long long)w1.bytes;
  return HPS_OK;
}

int hps_zgemm(int M, int N, int K, int batch, const double *A, const double *B, double *C, int emulated,
              void *stream) {
  if (M < 1 || N < 1 || K < 1 || batch < 1 || batch > 65535 || emulated < 0 || emulated > 3) return HPS_EINVAL;
  if (!A || !B || !C || !is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(C)) return HPS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  GemmDesc g = gemm(M, N, K, batch, mat(A, M, (long long)M * K), mat(B, K, (long long)K * N),
                    mat(C, M, (long long)M * N));
  g.cf32 = emulated >= 2 ? 1 : 0;  // the complex64 products: 5 slices, or complex64 arithmetic
  if (emulated == 0 || emulated == 3) {
    CK(hps::launch_gemm(&g, 1, st));
    return HPS_OK;
  }
  const size_t ws = hps::oz_workspace_bytes(g);
  void *w = nullptr;
  CK(lib_malloc_async(&w, ws, st));
  cudaError_t err = hps::launch_gemm_oz(g, w, ws, st);
  cudaError_t err2 = cudaFreeAsync(w, st);
  if (err != cudaSuccess) return cuda_fail(err);
  if (err2 != cudaSuccess) return cuda_fail(err2);
  return HPS_OK;
}

int hps_zinv(int n, int batch, const double *A, double *Ainv, int mode, int *bad, void *stream) {
  if (bad) *bad = -1;
  if (n < 2 || batch < 1 || batch > (1 << 20) || mode < 0 || mode > 1) return HPS_EINVAL;
  if (!A || !Ainv || !is_device_ptr(A) || !is_device_ptr(Ainv)) return HPS_EINVAL;
  // the regime: as the build chooses for P = batch interface matrices of
  // order n (mode 1), or its complex128 elimination (mode 0)
  GJChoice g;
  if (mode == 1 ? !choose_gj(n, batch, 0, g) : !choose_gj_rule(n, batch, 0, g)) return HPS_EINVAL;
  if (mode == 0) g.refined = false;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t elems = (size_t)n * n * batch;
  const size_t o_meta = align256(16 * elems);
  const size_t o_status = o_meta + align256(sizeof(int) * hps::gj_meta_ints(n) * (size_t)batch);
  const size_t o_ref = o_status + 256;
  const size_t total = o_ref + (g.refined ? wref_layout(n, batch, true).total : 0);
  char *w = nullptr;
  CK(lib_malloc_async((void **)&w, total, st));
  unsigned *status = (unsigned *)(w + o_status);
  unsigned word = 0;
  int launches = 0;
  int rc = HPS_OK;
  cudaError_t err = cudaMemsetAsync(status, 0, sizeof(unsigned), st);
  if (err == cudaSuccess) err = cudaMemcpyAsync(w, A, 16 * elems, cudaMemcpyDeviceToDevice, st);
  if (err == cudaSuccess)
    rc = w_inverse(g, w, Ainv, n, batch, (int *)(w + o_meta), status, 0, false, g.refined ? w + o_ref : nullptr,
                   true, st, launches);
  if (err == cudaSuccess && rc == HPS_OK)
    err = cudaMemcpyAsync(&word, status, sizeof(word), cudaMemcpyDeviceToHost, st);
  const cudaError_t err_free = cudaFreeAsync(w, st);
  const cudaError_t err_sync = cudaStreamSynchronize(st);
  if (err != cudaSuccess) return cuda_fail(err);
  if (rc != HPS_OK) return rc;
  if (err_free != cudaSuccess) return cuda_fail(err_free);
  if (err_sync != cudaSuccess) return cuda_fail(err_sync);
  if (!word) return HPS_OK;
  // codes 1, 2: a zero pivot (box = the matrix); 3: a wait of the
  // tensor-core residual product gave up (box = its CTA)
  if ((word >> 28) == 3u) return HPS_ETIMEOUT;
  if (bad) *bad = (int)(word & 0xfffff);
  return HPS_ESINGULAR;
}

int hps_check_wait(int limit_ms, void *stream) {
  if (limit_ms < 1 || limit_ms > 2000) return HPS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned *status = nullptr;
  CK(lib_malloc_async((void **)&status, sizeof(unsigned), st));
  unsigned word = 0;
  cudaError_t err = cudaMemsetAsync(status, 0, sizeof(unsigned), st);
  if (err == cudaSuccess) err = hps::launch_wait_check(status, limit_ms, st);
  if (err == cudaSuccess) err = cudaMemcpyAsync(&word, status, sizeof(word), cudaMemcpyDeviceToHost, st);
  const cudaError_t err_free = cudaFreeAsync(status, st);
  const cudaError_t err_sync = cudaStreamSynchronize(st);
  if (err != cudaSuccess) return cuda_fail(err);
  if (err_free != cudaSuccess) return cuda_fail(err_free);
  if (err_sync != cudaSuccess) return cuda_fail(err_sync);
  if (!word) return HPS_OK;
  return (word >> 28) == 3u ? HPS_ETIMEOUT : HPS_ECUDA;
}

int hps_plan(const hps_desc *desc, hps_info_t *info) {
  if (!info) return HPS_EINVAL;
  hps_handle *h = new (std::nothrow) hps_handle();
  if (!h) return HPS_ENOMEM;
  int st = plan_handle(h, desc);
  if (st == HPS_OK) *info = h->info;
  delete h;
  return st;
}

int hps_build(const hps_desc *desc, const double *c, void *stream, hps_handle **out) {
  return hps_build_batch(1, desc, &c, stream, out);
}

int hps_build_batch(int nprob, const hps_desc *descs, const double *const *c, void *stream,
                    hps_handle **out) {
  if (nprob < 0) return HPS_EINVAL;
  if (nprob == 0) return HPS_OK;
  if (!descs || !c || !out) return HPS_EINVAL;
  for (int k = 0; k < nprob; k++) {
    int st0 = check_desc(&descs[k]);
    if (st0) return st0;
    if (!c[k]) return HPS_EINVAL;
    if (descs[k].p != descs[0].p || descs[k].precision != descs[0].precision ||
        descs[k].fp64_levels != descs[0].fp64_levels || descs[k].fp64_native != descs[0].fp64_native ||
        descs[k].leaf_form != descs[0].leaf_form ||
        (descs[k].q ? descs[k].q : descs[k].p - 2) != (descs[0].q ? descs[0].q : descs[0].p - 2))
      return HPS_EINVAL;
    // host samples of c are checked here (device ones are not scanned)
    if (!is_device_ptr(c[k])) {
      const long long cnt = (long long)descs[k].mx * descs[k].my * (descs[k].p - 2) * (descs[k].p - 2);
      for (long long i = 0; i < cnt; i++)
        if (!std::isfinite(c[k][i])) return HPS_EINVAL;
    }
  }
  std::vector<hps_handle *> hs(nprob, nullptr);
  auto release = [&]() {
    for (hps_handle *x : hs) hps_free(x);
  };
  long long total = 0;
  for (int k = 0; k < nprob; k++) {
    hs[k] = new (std::nothrow) hps_handle();
    if (!hs[k]) {
      release();
      return HPS_ENOMEM;
    }
    int st = plan_handle(hs[k], &descs[k]);
    if (st != HPS_OK) {
      release();
      return st;
    }
    total += hs[k]->info.operator_bytes;
  }
  long long cap = env_cap();
  if (cap >= 0 && total > cap) {
    release();
    return HPS_ENOMEM;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    release();
    return HPS_ECUDA;
  }
  for (hps_handle *x : hs) x->device = dev;
  // build order: tallest tree first (stable), so that on every merge level
  // the problems that still have it come first
  std::vector<int> order(nprob);
  for (int k = 0; k < nprob; k++) order[k] = k;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return hs[a]->plan.L > hs[b]->plan.L; });
  std::vector<hps_handle *> sorted(nprob);
  std::vector<const double *> cs(nprob);
  for (int k = 0; k < nprob; k++) {
    sorted[k] = hs[order[k]];
    cs[k] = c[order[k]];
  }
  int st = build_many(sorted, cs, (cudaStream_t)stream);
  if (st != HPS_OK) {
    release();
    return st;
  }
  for (int k = 0; k < nprob; k++) {
    hs[k]->info.build_launches = hs[k]->sh->launches;
    out[k] = hs[k];
  }
  return HPS_OK;
}

namespace {
// Seeded, well-scaled complex values for the tuning runs (timing does not
// depend on them; the inverse's row swaps do, so they are not diagonal).
__global__ void tune_fill_kernel(void *p, long long count, int n, int f32) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= count) return;
  unsigned long long z = (unsigned long long)id * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
  z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;
  const double re = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  const double im = (double)((z * 0x94D049BB133111EBull) >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  const long long r = n > 0 ? id % ((long long)n * n) : 1;
  const double d = (n > 0 && r % n == r / n) ? 2.0 : 0.0;  // a moderate diagonal
  if (f32)
    ((float2 *)p)[id] = make_float2((float)(re + d), (float)im);
  else
    ((double2 *)p)[id] = make_double2(re + d, im);
}
}  // namespace

int hps_tune(int nprob, const hps_desc *descs, void *stream, int *ntuned) {
  if (nprob < 1 || !descs) return HPS_EINVAL;
  for (int k = 0; k < nprob; k++) {
    int st0 = check_desc(&descs[k]);
    if (st0) return st0;
    if (descs[k].p != descs[0].p || descs[k].precision != descs[0].precision ||
        descs[k].fp64_levels != descs[0].fp64_levels || descs[k].fp64_native != descs[0].fp64_native ||
        descs[k].leaf_form != descs[0].leaf_form)
      return HPS_EINVAL;
  }
  std::vector<hps_handle> hv(nprob);
  std::vector<hps_handle *> hs(nprob);
  for (int k = 0; k < nprob; k++) {
    int st = plan_handle(&hv[k], &descs[k]);
    if (st != HPS_OK) return st;
    hs[k] = &hv[k];
  }
  std::stable_sort(hs.begin(), hs.end(), [](hps_handle *a, hps_handle *b) { return a->plan.L > b->plan.L; });
  const Plan &P0 = hs[0]->plan;
  for (int k = 1; k < nprob; k++)
    for (int j = 0; j < hs[k]->plan.L; j++) {
      const Level &A = P0.lv[j], &B = hs[k]->plan.lv[j];
      if (A.horizontal != B.horizontal || A.nc != B.nc || A.n3 != B.n3) return HPS_EINVAL;
    }
  std::vector<std::vector<BuildRun>> runs;
  std::vector<std::vector<long long>> first;
  int rc = plan_runs(hs, runs, first);
  if (rc != HPS_OK) return rc;
  // the shapes the build would launch
  std::map<TuneKey, int> todo;
  size_t amax = 1, bmax = 1, cmax = 1, smax = 1, mmax = 1;
  for (int j = 0; j < P0.L; j++) {
    const Level &S = P0.lv[j];
    int mnk[6][3];
    merge_products(S.n1, S.n2, S.n3, S.nt, mnk);
    for (const BuildRun &r : runs[j]) {
      for (int q = 0; q < 6; q++) {
        if (mnk[q][1] <= 8) continue;  // the skinny kernel has no choice to make
        todo[TuneKey{0, mnk[q][0], mnk[q][1], mnk[q][2], r.P, r.f32}] = 0;
        amax = std::max(amax, (size_t)mnk[q][0] * mnk[q][2] * r.P);
        bmax = std::max(bmax, (size_t)mnk[q][2] * mnk[q][1] * r.P);
        cmax = std::max(cmax, (size_t)mnk[q][0] * mnk[q][1] * r.P);
      }
      todo[TuneKey{1, S.n3, 0, 0, r.P, r.f32}] = 0;
      smax = std::max(smax, (size_t)S.n3 * S.n3 * r.P);
      mmax = std::max(mmax, (size_t)hps::gj_meta_ints(S.n3) * r.P);
    }
  }
  tune_cache_load();
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (auto it = todo.begin(); it != todo.end();) it = g_tune.count(it->first) ? todo.erase(it) : std::next(it);
  }
  if (ntuned) *ntuned = 0;
  if (todo.empty()) return HPS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  char *buf = nullptr;
  const size_t oA = 0, oB = align256(16 * amax), oC = oB + align256(16 * bmax), oS = oC + align256(16 * cmax);
  const size_t oM = oS + align256(16 * smax), oSt = oM + align256(4 * mmax), total = oSt + 256;
  CK(cudaMalloc((void **)&buf, total));
  void *ozws = nullptr, *wrefws = nullptr;
  size_t ozb = 0, wrefb = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ozws) cudaFree(ozws);
    if (wrefws) cudaFree(wrefws);
    cudaFree(buf);
  };
  auto fail = [&](cudaError_t err) {
    cleanup();
    return cuda_fail(err);
  };
  cudaError_t err;
  if ((err = cudaEventCreate(&e0)) != cudaSuccess || (err = cudaEventCreate(&e1)) != cudaSuccess) return fail(err);
  auto fill = [&](size_t off, size_t count, int n, int f32) {
    tune_fill_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(buf + off, (long long)count, n, f32);
    return cudaGetLastError();
  };
  // device milliseconds of one call of f after one warm-up call (refill runs
  // before each call, outside the timed region)
  auto time_it = [&](auto &&f, auto &&refill, int reps) -> float {
    if (refill() != cudaSuccess || f() != cudaSuccess) {
      cudaGetLastError();
      return -1.0f;
    }
    float best = 1e30f;
    for (int r = 0; r < reps; r++) {
      if (refill() != cudaSuccess) return -1.0f;
      cudaEventRecord(e0, st);
      if (f() != cudaSuccess) {
        cudaGetLastError();
        return -1.0f;
      }
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0f;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms);
    }
    return best;
  };
  int count = 0;
  for (auto &kv : todo) {
    const TuneKey &k = kv.first;
    int best = 0;
    float best_ms = 1e30f;
    if (k.kind == 0) {
      if ((err = fill(oA, (size_t)k.M * k.K * k.batch, 0, k.f32)) != cudaSuccess ||
          (err = fill(oB, (size_t)k.K * k.N * k.batch, 0, k.f32)) != cudaSuccess)
        return fail(err);
      GemmDesc g = gemm(k.M, k.N, k.K, k.batch, mat(buf + oA, k.M, (long long)k.M * k.K, nullptr, nullptr, k.f32),
                        mat(buf + oB, k.K, (long long)k.K * k.N, nullptr, nullptr, k.f32),
                        mat(buf + oC, k.M, (long long)k.M * k.N, nullptr, nullptr, k.f32));
      g.cf32 = k.f32;
      auto none = [&]() { return cudaSuccess; };
      for (int cand = 1; cand <= 7; cand++) {
        if (cand == 5 && (!P0.oz || k.K < 32 || k.batch > 65535)) continue;
        if (cand >= 6 && (!k.f32 || k.M < 96 || k.N < 96)) continue;
        float ms;
        if (cand == 5) {
          const size_t need = hps::oz_workspace_bytes(g);
          if (need > ozb) {
            if (ozws) cudaFree(ozws);
            ozws = nullptr;
            ozb = 0;
            if (cudaMalloc(&ozws, need) != cudaSuccess) {
              cudaGetLastError();
              continue;
            }
            ozb = need;
          }
          ms = time_it([&]() { return hps::launch_gemm_oz(g, ozws, ozb, st); }, none, 3);
        } else {
          GemmDesc gc = g;
          gc.cfg = cand;
          ms = time_it([&]() { return hps::launch_gemm(&gc, 1, st); }, none, 3);
        }
        if (ms >= 0.0f && ms < best_ms) {
          best_ms = ms;
          best = cand;
        }
      }
    } else {
      const int n3 = k.M, P = k.batch;
      GJChoice rule;
      if (!choose_gj_rule(n3, P, k.f32, rule)) continue;
      std::vector<GJChoice> cands;
      // the eliminations in the matrices' own precision, and for complex128
      // matrices the same regimes in complex64 as the start of a refined inverse
      for (int refined = 0; refined <= (k.f32 ? 0 : 1); refined++) {
        const int ef = (k.f32 || refined) ? 1 : 0;
        for (int kb : {8, 4}) {
          const bool tg = hps::gj_smem_bytes(n3, hps::gj_max_cluster(), false, 0, false, ef, kb) > 200 * 1024;
          for (int cs = 1; cs <= hps::gj_max_cluster(); cs *= 2)
            // every CTA of the cluster owns at least one panel
            if (hps::gj_smem_bytes(n3, cs, false, 0, tg, ef, kb) <= 227 * 1024 &&
                (cs - 1) * hps::gj_slab(n3, cs, kb) < n3) {
              GJChoice c;
              c.cs = cs;
              c.tglobal = tg;
              c.kb = kb;
              c.refined = refined != 0;
              cands.push_back(c);
            }
          if (n3 >= 64) {
            const int G0 = rule.wide ? rule.wide : (int)std::max<long long>(2, std::min<long long>((2 * 152 + P - 1) / P, n3 / 4 + 1));
            for (int G : {G0, G0 / 2})
              if (G >= 2) {
                GJChoice c;
                c.wide = G;
                c.kb = kb;
                c.refined = refined != 0;
                cands.push_back(c);
              }
          }
        }
      }
      size_t wrb = 0;
      for (const GJChoice &c : cands)
        if (c.refined) wrb = wref_layout(n3, P, P0.oz).total;
      if (wrb > wrefb) {
        if (wrefws) cudaFree(wrefws);
        wrefws = nullptr;
        wrefb = 0;
        if (cudaMalloc(&wrefws, wrb) == cudaSuccess)
          wrefb = wrb;
        else
          cudaGetLastError();
      }
      auto refill = [&]() { return fill(oS, (size_t)n3 * n3 * P, n3, k.f32); };
      for (const GJChoice &c : cands) {
        float ms;
        if (c.refined) {
          if (!wrefws) continue;
          int nl = 0;
          ms = time_it([&]() {
            return w_inverse(c, buf + oS, buf + oC, n3, P, (int *)(buf + oM), (unsigned *)(buf + oSt), 0, false,
                             (char *)wrefws, P0.oz, st, nl) == HPS_OK ? cudaSuccess : cudaErrorUnknown;
          }, refill, 2);
        } else if (!c.wide)
          ms = time_it([&]() { return hps::launch_gj_inverse(buf + oS, buf + oC, n3, P, (int *)(buf + oM), (unsigned *)(buf + oSt), 0, c.cs, c.tglobal, k.f32 != 0, st, c.kb); }, refill, 2);
        else
          ms = time_it([&]() { return hps::launch_gj_wide(buf + oS, buf + oC, n3, P, c.wide, (int *)(buf + oM), (unsigned *)(buf + oSt), 0, k.f32 != 0, st, c.kb); }, refill, 2);
        if (ms >= 0.0f && ms < best_ms) {
          best_ms = ms;
          best = gj_encode(c);
        }
      }
    }
    if (best != 0) {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tune[k] = best;
      count++;
    }
  }
  cleanup();
  if (ntuned) *ntuned = count;
  tune_cache_store();
  return HPS_OK;
}

int hps_rebuild(int nh, hps_handle *const *hs, const double *const *c, void *stream) {
  if (nh < 1 || !hs || !c || !hs[0] || !hs[0]->sh) return HPS_EINVAL;
  Shared *sh = hs[0]->sh;
  {
    std::lock_guard<std::mutex> lock(g_shared_mu);
    if (sh->refs != (int)sh->order.size()) return HPS_EINVAL;  // a handle of the build was freed
  }
  if (nh != (int)sh->order.size() || !sh->compute) return HPS_EINVAL;
  for (int k = 0; k < nh; k++) {
    if (!hs[k] || hs[k]->sh != sh || !c[k]) return HPS_EINVAL;
    for (int q = 0; q < k; q++)
      if (hs[q] == hs[k]) return HPS_EINVAL;
    if (!is_device_ptr(c[k])) {  // host samples are checked (device ones are not scanned)
      const long long cnt = (long long)hs[k]->plan.leaves * hs[k]->plan.ni;
      for (long long i = 0; i < cnt; i++)
        if (!std::isfinite(c[k][i])) return HPS_EINVAL;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  for (int k = 0; k < nh; k++) {
    const size_t cb = sizeof(double) * (size_t)hs[k]->plan.leaves * hs[k]->plan.ni;
    CK(cudaMemcpyAsync(hs[k]->c_dev, c[k], cb, cudaMemcpyDefault, st));
  }
  CK(cudaMemsetAsync(hs[0]->d_status, 0, sizeof(unsigned int), st));
  if (!sh->graph) {
    // capture the build's device work once, on a stream of our own (the
    // caller's may be the legacy stream, which cannot be captured)
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    int launches = 0, rc = HPS_OK;
    cudaError_t err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (err == cudaSuccess) {
      rc = sh->compute(cs, false, launches);
      err = cudaStreamEndCapture(cs, &g);
    }
    if (err == cudaSuccess && rc == HPS_OK) err = cudaGraphInstantiate(&sh->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (rc != HPS_OK) return rc;
    if (err != cudaSuccess) {
      sh->graph = nullptr;
      return cuda_fail(err);
    }
  }
  CK(cudaGraphLaunch(sh->graph, st));
  return HPS_OK;
}

int hps_build_times(hps_handle *h, double *ms, int cap) {
  if (!h || (!ms && cap > 0) || cap < 0) return -HPS_EINVAL;
  if (!h->sh || h->sh->ev.size() < 2) return -HPS_EINVAL;
  const std::vector<cudaEvent_t> &ev = h->sh->ev;
  const int nph = (int)ev.size() - 1;
  if (cudaEventSynchronize(ev.back()) != cudaSuccess) return -HPS_ECUDA;
  for (int q = 0; q < nph && q < cap; q++) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, ev[q], ev[q + 1]) != cudaSuccess)
      return -HPS_ECUDA;
    ms[q] = t;
  }
  return nph;
}

int hps_build_product_times(hps_handle *h, double *ms, double *flops, int cap) {
  if (!h || cap < 0 || (cap > 0 && (!ms || !flops))) return -HPS_EINVAL;
  if (!h->sh) return -HPS_EINVAL;
  const Shared *sh = h->sh;
  const int n = sh->oz_n;
  for (int k = 0; k < n && k < cap; k++) {
    float t = 0.0f;
    if (cudaEventSynchronize(sh->oz_ev[2 * k + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, sh->oz_ev[2 * k], sh->oz_ev[2 * k + 1]) != cudaSuccess)
      return -HPS_ECUDA;
    ms[k] = t;
    flops[k] = sh->oz_flops[k];
  }
  return n;
}

int hps_status(hps_handle *h, void *stream, int *level, int *box) {
  if (!h) return HPS_EINVAL;
  unsigned int w = 0;
  CK(cudaMemcpyAsync(&w, h->d_status, sizeof(w), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  if (level) *level = w ? (int)((w >> 20) & 0xff) : -1;
  if (box) *box = w ? (int)(w & 0xfffff) : -1;
  if (!w) return HPS_OK;
  // codes 1, 2: a zero pivot of a leaf matrix or an interface matrix; 3: a
  // pipeline wait of the tensor-core product gave up
  return (w >> 28) == 3u ? HPS_ETIMEOUT : HPS_ESINGULAR;
}

int hps_solve(hps_handle *h, const double *s_, const double *t_, double *u_, int nrhs, void *stream) {
  if (!h || nrhs < 0) return HPS_EINVAL;
  if (nrhs == 0) return HPS_OK;
  if (!s_ || !t_ || !u_) return HPS_EINVAL;
  if (int dst = on_handle_device(h)) return dst;
  cudaStream_t st = (cudaStream_t)stream;
  const Plan &pl = h->plan;
  const int n = pl.n, ni = pl.ni, nl = pl.leaves, R = nrhs;

  SolveWs ws;
  solve_ws_layout(pl, R, ws);
  int gst = grow(&h->ws, &h->ws_bytes, ws.bytes);
  if (gst) return gst;

  // stage host arrays
  const bool sdev = is_device_ptr(s_), tdev = is_device_ptr(t_), udev = is_device_ptr(u_);
  size_t sbytes = sizeof(double2) * (size_t)R * nl * ni, tbytes = sizeof(double2) * (size_t)R * pl.nbdry;
  size_t ubytes = sizeof(double2) * (size_t)R * nl * n;
  size_t need = (sdev ? 0 : align256(sbytes)) + (tdev ? 0 : align256(tbytes)) + (udev ? 0 : align256(ubytes));
  if (need) {
    gst = grow(&h->stage, &h->stage_bytes, need);
    if (gst) return gst;
  }
  char *sb = (char *)h->stage;
  const double2 *s = (const double2 *)s_;
  const double2 *t = (const double2 *)t_;
  double2 *u = (double2 *)u_;
  if (!sdev) {
    CK(cudaMemcpyAsync(sb, s_, sbytes, cudaMemcpyHostToDevice, st));
    s = (const double2 *)sb;
    sb += align256(sbytes);
  }
  if (!tdev) {
    CK(cudaMemcpyAsync(sb, t_, tbytes, cudaMemcpyHostToDevice, st));
    t = (const double2 *)sb;
    sb += align256(tbytes);
  }
  if (!udev) u = (double2 *)sb;

  gst = pl.mixed && pl.refine_steps > 0 ? solve_refine(h, s, t, u, R, (char *)h->ws, ws, st)
                                         : solve_launch(h, s, t, u, R, (char *)h->ws, ws, st);
  if (gst) return gst;

  if (!udev) {
    CK(cudaMemcpyAsync(u_, u, ubytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  } else if (!sdev || !tdev) {
    // host inputs were staged: make the call's staging reusable on return
    CK(cudaStreamSynchronize(st));
  }
  return HPS_OK;
}

int hps_reserve(hps_handle *h, int nrhs) {
  if (!h || nrhs < 0) return HPS_EINVAL;
  if (int dst = on_handle_device(h)) return dst;
  const Plan &pl = h->plan;
  SolveWs ws;
  solve_ws_layout(pl, std::max(nrhs, 1), ws);
  int gst = grow(&h->ws, &h->ws_bytes, ws.bytes);
  if (gst) return gst;
  const size_t R = (size_t)std::max(nrhs, 1);
  return grow(&h->stage, &h->stage_bytes,
              align256(sizeof(double2) * R * pl.leaves * pl.ni) + align256(sizeof(double2) * R * pl.nbdry) +
                  align256(sizeof(double2) * R * pl.leaves * pl.n));
}

int hps_solve_batch(hps_handle *h, int nreq, const double *const *s_, const double *const *t_,
                    double *const *u_, const int *nrhs, void *stream) {
  if (!h || nreq < 0) return HPS_EINVAL;
  if (nreq == 0) return HPS_OK;
  if (!s_ || !t_ || !u_ || !nrhs) return HPS_EINVAL;
  if (int dst = on_handle_device(h)) return dst;
  long long Rl = 0;
  bool all_dev = true;
  for (int k = 0; k < nreq; k++) {
    if (nrhs[k] < 0) return HPS_EINVAL;
    if (nrhs[k] == 0) continue;
    if (!s_[k] || !t_[k] || !u_[k]) return HPS_EINVAL;
    Rl += nrhs[k];
    all_dev = all_dev && is_device_ptr(s_[k]) && is_device_ptr(t_[k]) && is_device_ptr(u_[k]);
  }
  if (Rl == 0) return HPS_OK;
  if (Rl > (1LL << 30)) return HPS_EINVAL;
  const int R = (int)Rl;
  cudaStream_t st = (cudaStream_t)stream;
  const Plan &pl = h->plan;
  int gst = hps_reserve(h, R);
  if (gst) return gst;
  SolveWs ws;
  solve_ws_layout(pl, R, ws);
  const size_t sc = (size_t)pl.leaves * pl.ni, tc = (size_t)pl.nbdry, uc = (size_t)pl.leaves * pl.n;
  double2 *S = (double2 *)h->stage;
  double2 *T = (double2 *)((char *)h->stage + align256(sizeof(double2) * R * sc));
  double2 *U = (double2 *)((char *)T + align256(sizeof(double2) * R * tc));
  // gather: request k's columns follow request k-1's
  size_t col = 0;
  for (int k = 0; k < nreq; k++) {
    if (nrhs[k] == 0) continue;
    CK(cudaMemcpyAsync(S + col * sc, s_[k], sizeof(double2) * nrhs[k] * sc, cudaMemcpyDefault, st));
    CK(cudaMemcpyAsync(T + col * tc, t_[k], sizeof(double2) * nrhs[k] * tc, cudaMemcpyDefault, st));
    col += nrhs[k];
  }
  gst = pl.mixed && pl.refine_steps > 0 ? solve_refine(h, S, T, U, R, (char *)h->ws, ws, st)
                                         : solve_launch(h, S, T, U, R, (char *)h->ws, ws, st);
  if (gst) return gst;
  col = 0;
  for (int k = 0; k < nreq; k++) {
    if (nrhs[k] == 0) continue;
    CK(cudaMemcpyAsync(u_[k], U + col * uc, sizeof(double2) * nrhs[k] * uc, cudaMemcpyDefault, st));
    col += nrhs[k];
  }
  if (!all_dev) CK(cudaStreamSynchronize(st));
  return HPS_OK;
}

int hps_solve_noalloc(hps_handle *h, const double *s_, const double *t_, double *u_, int nrhs,
                      void *stream) {
  if (!h || nrhs < 0) return HPS_EINVAL;
  if (nrhs == 0) return HPS_OK;
  if (!s_ || !t_ || !u_) return HPS_EINVAL;
  if (!is_device_ptr(s_) || !is_device_ptr(t_) || !is_device_ptr(u_)) return HPS_EINVAL;
  if (int dst = on_handle_device(h)) return dst;
  if (h->plan.mixed) return HPS_ENOTSUP;  // refinement needs more workspace than the fixed array
  SolveWs ws;
  solve_ws_layout(h->plan, nrhs, ws, false);  // no digit planes: products stay on the FP64 pipes
  if (ws.bytes > (size_t)HPS_NOALLOC_WORKSPACE_BYTES) return HPS_ETOOBIG;
  char *wb = nullptr;
  int st = noalloc_ws_ptr(&wb);
  if (st) return st;
  // The vectors of the workspace are written before they are read, but the
  // split skinny products keep arrival counters at its head that must be
  // zero when a launch starts (each launch leaves them zero when it
  // finishes).  Two calls that overlapped on the GPU can leave them
  // nonzero, so every call clears them first, in stream order; a memset
  // allocates nothing.
  CK(cudaMemsetAsync(wb, 0, hps::gemv_scratch_counters(), (cudaStream_t)stream));
  return solve_launch(h, (const double2 *)s_, (const double2 *)t_, (double2 *)u_, nrhs, wb, ws,
                      (cudaStream_t)stream, nullptr, nullptr, nullptr, false);
}

int hps_root_R(hps_handle *h, double *R, int gauss_basis, void *stream) {
  if (!h || !R || (gauss_basis != 0 && gauss_basis != 1)) return HPS_EINVAL;
  // boundary data on q != p - 2 Gauss nodes: R exists only in that basis
  if (h->plan.gauss && !gauss_basis) return HPS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int nbr = h->plan.nbdry;
  const bool dev = is_device_ptr(R);
  double2 *dst = (double2 *)R;
  size_t bytes = sizeof(double2) * (size_t)nbr * nbr;
  if (!dev) {
    int gst = grow(&h->stage, &h->stage_bytes, bytes);
    if (gst) return gst;
    dst = (double2 *)h->stage;
  }
  const int nr = h->plan.lv.empty() ? h->plan.nbi : h->plan.lv.back().nt;
  // public row-major R[a][b] = root(src^-1 ...): with the root order map
  // root position -> public index, R_pub[pub(i)][pub(j)] = R_root(i, j).
  // As a column-major matrix R_pub^T: element (pub(j), pub(i)) = R_root(i, j),
  // i.e. dst(a=pub(j), b=pub(i)) = src(i, j): a transposed copy with the
  // destination rows and columns mapped by the root map.
  CopyBatch cb;
  cb.count = 1;
  cb.d[0] = copy(nr, nr, 1, mat(h->Rroot, nr, 0), mat(dst, nbr, 0, h->d_root_src, h->d_root_src));
  cb.d[0].trans = 1;
  CK(hps::launch_copy(cb, st));
  if (gauss_basis && !h->plan.gauss)
    if (int rc = root_R_to_gauss(h->plan, dst, st)) return rc;
  if (!dev) {
    CK(cudaMemcpyAsync(R, dst, bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return HPS_OK;
}

int hps_leaf_ops(hps_handle *h, int leaf, double *Psi, double *Y, double *Gam, void *stream) {
  if (!h || leaf < 0 || leaf >= h->plan.leaves) return HPS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = h->plan.n, nb = h->plan.nb, ni = h->plan.ni, lf = h->plan.leaf_f32;
  const void *X = elem(h->X, (long long)leaf * n * n, lf);
  const void *GX = elem(h->GX, (long long)leaf * n * nb, lf);
  int xf = lf;  // precision of the B^{-1} read below
  void *tmp = nullptr;
  if (h->plan.leaf_lu && (Psi || Y)) {
    // B^{-1} from the factors: the leaf's solve with the n unit vectors as
    // right-hand sides ([t; s] = e_c), into a complex128 n x n scratch
    const size_t cnt = (size_t)n * n;
    std::vector<double2> eye(2 * cnt, make_double2(0.0, 0.0));
    double2 *et = eye.data(), *es = et + (size_t)nb * n;
    for (int c = 0; c < n; c++) {
      if (c < nb)
        et[(size_t)c * nb + c] = make_double2(1.0, 0.0);
      else
        es[(size_t)c * ni + (c - nb)] = make_double2(1.0, 0.0);
    }
    CK(lib_malloc_async(&tmp, sizeof(double2) * 3 * cnt, st));
    double2 *dt = (double2 *)tmp, *ds = dt + (size_t)nb * n, *dx = dt + 2 * cnt;
    cudaError_t err = cudaMemcpyAsync(dt, eye.data(), sizeof(double2) * 2 * cnt, cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess)
      err = hps::launch_lu_solve(X, h->lu_perm + (size_t)leaf * n, h->lu_dsc + (size_t)leaf * n, 1, n, nb, n,
                                 dt, nb, 0, ds, ni, 0, dx, n, 0, lf != 0, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) {
      cudaFreeAsync(tmp, st);
      return cuda_fail(err);
    }
    X = dx;
    xf = 0;
  }
  struct Part {
    double *out;
    int rows, cols;
    const void *src;
    long long ld;
    int f32;
  } parts[3] = {{Psi, n, nb, X, n, xf}, {Y, n, ni, elem(X, (long long)nb * n, xf), n, xf},
                {Gam, nb, ni, elem(GX, (long long)nb * nb, lf), nb, lf}};
  int rc = HPS_OK;
  for (const Part &pt : parts) {
    if (rc != HPS_OK) break;
    if (!pt.out) continue;
    size_t bytes = sizeof(double2) * (size_t)pt.rows * pt.cols;
    const bool dev = is_device_ptr(pt.out);
    double2 *dst = (double2 *)pt.out;
    if (!dev) {
      rc = grow(&h->stage, &h->stage_bytes, bytes);
      if (rc) break;
      dst = (double2 *)h->stage;
    }
    // row-major out[i][j] = src(i, j): column-major (j, i) of dst = src(i, j)
    CopyBatch cb;
    cb.count = 1;
    cb.d[0] = copy(pt.cols, pt.rows, 1, mat(pt.src, pt.ld, 0, nullptr, nullptr, pt.f32), mat(dst, pt.cols, 0));
    cb.d[0].trans = 1;
    cudaError_t err = hps::launch_copy(cb, st);
    if (err == cudaSuccess && !dev) err = cudaMemcpyAsync(pt.out, dst, bytes, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess && !dev) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) rc = cuda_fail(err);
  }
  if (tmp) {
    cudaError_t err = cudaFreeAsync(tmp, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess && rc == HPS_OK) rc = cuda_fail(err);
  }
  return rc;
}

}  // extern "C"
