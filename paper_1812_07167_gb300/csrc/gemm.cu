// Batched, index-mapped complex GEMM and copy kernels.
//
// Every dense product of the HPS merge (Sec. 2.2: W = I - R33b R33a,
// Phi_a = W^{-1}[R33b R31a | -R32b], Phi_b, R^tau) and of the solve sweeps
// (Algorithm 2: the leaf matvecs Y s, Gamma s, Psi t and the per-level
// Upsilon / Phi actions) is one launch of these kernels over all boxes of a
// tree level.  Sub-blocks such as R33a = R^alpha(I3, I3) are read through
// index maps, so no gather pass is needed before a product.
//
// The arithmetic is complex128 (DFMA-bound on this part: the tiles only need
// enough reuse to keep shared-memory traffic below the DFMA rate) or
// complex64 for the mixed-precision path; each operand may be stored in
// either precision and is converted when loaded or stored.
#include <algorithm>

#include "hps_internal.h"

namespace hps {

namespace {

struct GemmPack {
  int n;
  GemmDesc d[2];
};

template <class C>
struct CT;
template <>
struct CT<double2> {
  __device__ static double2 make(double x, double y) { return make_double2(x, y); }
};
template <>
struct CT<float2> {
  __device__ static float2 make(double x, double y) { return make_float2((float)x, (float)y); }
};

__device__ __forceinline__ long long mat_off(const Mat &m, int b, int i, int j) {
  long long r = m.rmap ? (long long)__ldg(m.rmap + i) : (long long)i;
  long long c = m.cmap ? (long long)__ldg(m.cmap + j) : (long long)j;
  return (long long)b * m.stride + r + c * m.ld;
}

// element `off` of matrix m (read-only for the kernel), converted to C
template <class C>
__device__ __forceinline__ C ldm(const Mat &m, long long off) {
  if (m.f32) {
    float2 v = __ldg((const float2 *)m.ptr + off);
    return CT<C>::make(v.x, v.y);
  }
  double2 v = __ldg((const double2 *)m.ptr + off);
  return CT<C>::make(v.x, v.y);
}

// plain load, for operands that may alias the output
template <class C>
__device__ __forceinline__ C ldm_rw(const Mat &m, long long off) {
  if (m.f32) {
    float2 v = ((const float2 *)m.ptr)[off];
    return CT<C>::make(v.x, v.y);
  }
  double2 v = ((const double2 *)m.ptr)[off];
  return CT<C>::make(v.x, v.y);
}

template <class C>
__device__ __forceinline__ void stm(const Mat &m, long long off, C v) {
  if (m.f32)
    ((float2 *)m.ptr)[off] = make_float2((float)v.x, (float)v.y);
  else
    ((double2 *)m.ptr)[off] = make_double2((double)v.x, (double)v.y);
}

__device__ __forceinline__ void cmac(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cmac(float2 &acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

template <class C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// alpha * acc + beta * D(i, j) (+ 1 on the diagonal), stored to C(i, j)
template <class C>
__device__ __forceinline__ void epilogue(const GemmDesc &g, int b, int i, int j, C acc) {
  if (g.wide_epilogue) {
    // the product in its arithmetic's precision, the combination in FP64
    // (C = D + AB, the refinement corrections: two additions, since this
    // part's FP64 pipe is slow)
    const double2 a = make_double2((double)acc.x, (double)acc.y);
    if (g.alpha.x == 1.0 && g.alpha.y == 0.0 && g.beta.x == 1.0 && g.beta.y == 0.0 && g.D.ptr && !g.addI) {
      const double2 d = ldm_rw<double2>(g.D, mat_off(g.D, b, i, j));
      stm(g.C, mat_off(g.C, b, i, j), make_double2(d.x + a.x, d.y + a.y));
      return;
    }
    double2 w = cmul(g.alpha, a);
    if (g.D.ptr) {
      const double2 d = ldm_rw<double2>(g.D, mat_off(g.D, b, i, j));
      const double2 t = cmul(g.beta, d);
      w.x += t.x;
      w.y += t.y;
    }
    if (g.addI && i == j) w.x += 1;
    stm(g.C, mat_off(g.C, b, i, j), w);
    return;
  }
  C v = cmul(CT<C>::make(g.alpha.x, g.alpha.y), acc);
  if (g.D.ptr) {
    C t = cmul(CT<C>::make(g.beta.x, g.beta.y), ldm_rw<C>(g.D, mat_off(g.D, b, i, j)));
    v.x += t.x;
    v.y += t.y;
  }
  if (g.addI && i == j) v.x += 1;
  stm(g.C, mat_off(g.C, b, i, j), v);
}

// C tile of BM x BN per CTA; each thread owns TM x TN outputs at rows
// tx + r * (BM/TM) and columns ty + c * (BN/TN).
template <class C, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    gemm_kernel(const __grid_constant__ GemmPack pack) {
  chain_enter();
  constexpr int NTX = BM / TM, NTY = BN / TN, NT = NTX * NTY;
  __shared__ C As[BK][BM];
  __shared__ C Bs[BK][BN];
  const GemmDesc &g = pack.d[blockIdx.z];
  const int tiles_m = (g.M + BM - 1) / BM;
  const int tiles_n = (g.N + BN - 1) / BN;
  if ((int)blockIdx.x >= tiles_m * tiles_n) return;
  const int m0 = (blockIdx.x % tiles_m) * BM;
  const int n0 = (blockIdx.x / tiles_m) * BN;
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;

  for (int b = blockIdx.y; b < g.batch; b += gridDim.y) {
    C acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; r++)
#pragma unroll
      for (int c = 0; c < TN; c++) acc[r][c] = CT<C>::make(0.0, 0.0);

    for (int k0 = 0; k0 < g.K; k0 += BK) {
      // A tile: BM x BK, consecutive threads walk down a column
      for (int e = tid; e < BM * BK; e += NT) {
        int i = e % BM, k = e / BM;
        int gi = m0 + i, gk = k0 + k;
        C v = CT<C>::make(0.0, 0.0);
        if (gi < g.M && gk < g.K) v = ldm<C>(g.A, mat_off(g.A, b, gi, gk));
        As[k][i] = v;
      }
      // B tile: BK x BN
      for (int e = tid; e < BK * BN; e += NT) {
        int k = e % BK, j = e / BK;
        int gk = k0 + k, gj = n0 + j;
        C v = CT<C>::make(0.0, 0.0);
        if (gk < g.K && gj < g.N) {
          if (g.B2.ptr == nullptr || gk < g.ksplit)
            v = ldm<C>(g.B, mat_off(g.B, b, gk, gj));
          else
            v = ldm<C>(g.B2, mat_off(g.B2, b, gk - g.ksplit, gj));
        }
        Bs[k][j] = v;
      }
      __syncthreads();
#pragma unroll 4
      for (int k = 0; k < BK; k++) {
        C a[TM], bv[TN];
#pragma unroll
        for (int r = 0; r < TM; r++) a[r] = As[k][tx + r * NTX];
#pragma unroll
        for (int c = 0; c < TN; c++) bv[c] = Bs[k][ty + c * NTY];
#pragma unroll
        for (int r = 0; r < TM; r++)
#pragma unroll
          for (int c = 0; c < TN; c++) cmac(acc[r][c], a[r], bv[c]);
      }
      __syncthreads();
    }

#pragma unroll
    for (int r = 0; r < TM; r++)
#pragma unroll
      for (int c = 0; c < TN; c++) {
        int i = m0 + tx + r * NTX, j = n0 + ty + c * NTY;
        if (i < g.M && j < g.N) epilogue<C>(g, b, i, j, acc[r][c]);
      }
  }
}

// Complex64 products without index maps (the refinement corrections X0 E,
// the mixed path's dense products): 128 x BN tiles (BN = 128 or 64), 256
// threads with 8 x TN outputs each (TN = BN / 16) at rows tx + 16 r and
// columns ty + 16 c (8 TN complex multiply-adds for 8 + TN shared-memory
// loads a k), K in steps of 16 with the next step's tiles loaded into
// registers while the current one is multiplied.  BN = 64 halves the
// registers, so that two CTAs share an SM.  TA, TB: the storage types of A
// and B (complex64 or complex128, converted on load).
constexpr int kCg = 128, kCgK = 16;
template <class TA, class TB, int BN>
__global__ void __launch_bounds__(256, BN == 128 ? 1 : 2) cgemm64_kernel(const __grid_constant__ GemmPack pack) {
  chain_enter();
  constexpr int TN = BN / 16, QB = BN / 16;  // outputs a thread along N; B elements a thread loads
  __shared__ float2 As[kCgK][kCg];
  __shared__ float2 Bs[kCgK][BN];
  const GemmDesc &g = pack.d[blockIdx.z];
  const int tiles_m = (g.M + kCg - 1) / kCg, tiles_n = (g.N + BN - 1) / BN;
  if ((int)blockIdx.x >= tiles_m * tiles_n) return;
  const int m0 = (blockIdx.x % tiles_m) * kCg, n0 = (blockIdx.x / tiles_m) * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int b = blockIdx.y; b < g.batch; b += gridDim.y) {
    const TA *A = (const TA *)g.A.ptr + (size_t)b * g.A.stride;
    const TB *B = (const TB *)g.B.ptr + (size_t)b * g.B.stride;
    // element q of this thread's share of a tile: A rows (tid % 128), k pairs
    // (tid / 128 + 2 q); B k (tid % 16), columns (tid / 16 + 16 q)
    float2 pa[8], pb[QB];
    auto fetch = [&](int k0) {
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const int i = m0 + (tid & 127), k = k0 + (tid >> 7) + 2 * q;
        float2 v = make_float2(0.f, 0.f);
        if (i < g.M && k < g.K) {
          const TA t = __ldg(A + i + (size_t)k * g.A.ld);
          v = make_float2((float)t.x, (float)t.y);
        }
        pa[q] = v;
      }
#pragma unroll
      for (int q = 0; q < QB; q++) {
        const int kb = k0 + (tid & 15), j = n0 + (tid >> 4) + 16 * q;
        float2 w = make_float2(0.f, 0.f);
        if (kb < g.K && j < g.N) {
          const TB t = __ldg(B + kb + (size_t)j * g.B.ld);
          w = make_float2((float)t.x, (float)t.y);
        }
        pb[q] = w;
      }
    };
    float2 acc[8][TN];
#pragma unroll
    for (int r = 0; r < 8; r++)
#pragma unroll
      for (int c = 0; c < TN; c++) acc[r][c] = make_float2(0.f, 0.f);
    fetch(0);
    for (int k0 = 0; k0 < g.K; k0 += kCgK) {
#pragma unroll
      for (int q = 0; q < 8; q++) As[(tid >> 7) + 2 * q][tid & 127] = pa[q];
#pragma unroll
      for (int q = 0; q < QB; q++) Bs[tid & 15][(tid >> 4) + 16 * q] = pb[q];
      __syncthreads();
      if (k0 + kCgK < g.K) fetch(k0 + kCgK);
#pragma unroll 4
      for (int k = 0; k < kCgK; k++) {
        float2 a[8], bv[TN];
#pragma unroll
        for (int r = 0; r < 8; r++) a[r] = As[k][tx + 16 * r];
#pragma unroll
        for (int c = 0; c < TN; c++) bv[c] = Bs[k][ty + 16 * c];
#pragma unroll
        for (int r = 0; r < 8; r++)
#pragma unroll
          for (int c = 0; c < TN; c++) cmac(acc[r][c], a[r], bv[c]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; r++)
#pragma unroll
      for (int c = 0; c < TN; c++) {
        const int i = m0 + tx + 16 * r, j = n0 + ty + 16 * c;
        if (i < g.M && j < g.N) epilogue<float2>(g, b, i, j, acc[r][c]);
      }
  }
}

// element `off` of a matrix stored as T, converted to C
template <class C, class T>
__device__ __forceinline__ C ldt(const void *ptr, long long off) {
  const T v = __ldg((const T *)ptr + off);
  return CT<C>::make(v.x, v.y);
}

// k-loop of the skinny product with the storage types of A and B fixed
template <class C, class TA, class TB, int NN>
__device__ __forceinline__ void gemv_loop(const GemmDesc &g, int b, int i, int w, int k0, int k1,
                                          C (&acc)[NN]) {
  const long long arow = (long long)b * g.A.stride + (g.A.rmap ? (long long)__ldg(g.A.rmap + i) : i);
#pragma unroll 4
  for (int k = k0 + w; k < k1; k += 8) {
    const long long c = g.A.cmap ? (long long)__ldg(g.A.cmap + k) : k;
    const C a = ldt<C, TA>(g.A.ptr, arow + c * g.A.ld);
    const bool second = (g.B2.ptr != nullptr && k >= g.ksplit);
    const int kk = second ? k - g.ksplit : k;
#pragma unroll
    for (int j = 0; j < NN; j++)
      if (j < g.N) {
        const C bb = second ? ldt<C, TB>(g.B2.ptr, mat_off(g.B2, b, kk, j))
                            : ldt<C, TB>(g.B.ptr, mat_off(g.B, b, kk, j));
        cmac(acc[j], a, bb);
      }
  }
}

// Skinny products (N <= NN: the solve's right-hand sides).  A CTA computes 32
// rows of one batch entry; its 8 warps split its K range (warp w takes
// k = w, w+8, ...), each lane one row, so the 32 loads of A a warp issues are
// one coalesced column segment and B(k, :) is a broadcast.  The 8 partial
// sums meet in shared memory.  When a launch has few row blocks (the top
// levels of a tree), K is also split over gridDim.y CTAs: each writes its
// partial sums to scratch, and the last CTA of a row block to arrive (an
// atomic count) adds them in split order, so results do not depend on
// timing.  B and B2 share one storage type.
template <class C, int NN>
__global__ void __launch_bounds__(256) gemv_kernel(const __grid_constant__ GemmPack pack) {
  chain_enter();
  constexpr int NR = NN < 8 ? NN : 8;  // right-hand sides a reduction round (fits static shared memory)
  __shared__ C red[8][NR][33];
  __shared__ int last;
  const GemmDesc &g = pack.d[blockIdx.z];
  const int rblocks = (g.M + 31) / 32;
  if ((long long)blockIdx.x >= (long long)rblocks * g.batch) return;
  const int b = blockIdx.x / rblocks;
  const int i = (blockIdx.x % rblocks) * 32 + (threadIdx.x & 31);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int ks = gridDim.y, kid = blockIdx.y;
  const int kc = ((g.K + ks - 1) / ks + 7) / 8 * 8;
  const int k0 = min(g.K, kid * kc), k1 = min(g.K, k0 + kc);
  const bool live = i < g.M;
  C acc[NN];
#pragma unroll
  for (int j = 0; j < NN; j++) acc[j] = CT<C>::make(0.0, 0.0);
  if (live) {
    if (g.A.f32) {
      if (g.B.f32)
        gemv_loop<C, float2, float2, NN>(g, b, i, w, k0, k1, acc);
      else
        gemv_loop<C, float2, double2, NN>(g, b, i, w, k0, k1, acc);
    } else {
      if (g.B.f32)
        gemv_loop<C, double2, float2, NN>(g, b, i, w, k0, k1, acc);
      else
        gemv_loop<C, double2, double2, NN>(g, b, i, w, k0, k1, acc);
    }
  }
  C v[NN];
#pragma unroll
  for (int j0 = 0; j0 < NN; j0 += NR) {
    if (j0 > 0) __syncthreads();  // warp 0 has read the previous round
#pragma unroll
    for (int j = 0; j < NR; j++) red[w][j][l] = acc[j0 + j];
    __syncthreads();
    if (w == 0) {
#pragma unroll
      for (int j = 0; j < NR; j++) {
        C t = red[0][j][l];
#pragma unroll
        for (int q = 1; q < 8; q++) {
          t.x += red[q][j][l].x;
          t.y += red[q][j][l].y;
        }
        v[j0 + j] = t;
      }
    }
  }
  if (ks > 1) {
    // partial sums of this split; the last split of the row block finishes
    C *part = (C *)g.part + ((size_t)blockIdx.z * kGemvSlots + (size_t)blockIdx.x * ks) * 32 * NN;
    unsigned *cnt = g.cnt + (size_t)blockIdx.z * kGemvBlocks + blockIdx.x;
    if (w == 0) {
#pragma unroll
      for (int j = 0; j < NN; j++) part[((size_t)kid * NN + j) * 32 + l] = v[j];
      __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(cnt, 1u) == (unsigned)ks - 1) ? 1 : 0;
    __syncthreads();
    if (!last) return;
    if (w == 0) {
      __threadfence();
#pragma unroll
      for (int j = 0; j < NN; j++) {
        C t = CT<C>::make(0.0, 0.0);
        for (int q = 0; q < ks; q++) {
          const C p = __ldcg(part + ((size_t)q * NN + j) * 32 + l);  // other SMs' writes: past L1
          t.x += p.x;
          t.y += p.y;
        }
        v[j] = t;
      }
      if (l == 0) *cnt = 0;  // ready for the next launch
    }
  }
  if (w == 0 && live) {
#pragma unroll
    for (int j = 0; j < NN; j++) {
      if (j >= g.N) continue;
      epilogue<C>(g, b, i, j, v[j]);
    }
  }
}

__global__ void __launch_bounds__(256) copy_kernel(const __grid_constant__ CopyBatch cb) {
  chain_enter();
  const CopyDesc &d = cb.d[blockIdx.z];
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)d.M * d.N;
  if (e >= total) return;
  int i = (int)(e % d.M), j = (int)(e / d.M);
  for (int b = blockIdx.y; b < d.batch; b += gridDim.y) {
    double2 v = make_double2(0.0, 0.0);
    if (d.src.ptr) {
      double2 s = d.trans ? ldm_rw<double2>(d.src, mat_off(d.src, b, j, i))
                          : ldm_rw<double2>(d.src, mat_off(d.src, b, i, j));
      v = cmul(d.alpha, s);
    }
    const long long o = mat_off(d.dst, b, i, j);
    if (d.accumulate) {
      const double2 w = ldm_rw<double2>(d.dst, o);
      v.x += w.x;
      v.y += w.y;
    }
    stm(d.dst, o, v);
  }
}

template <int BM, int BN>
long long cfg_ctas(const GemmPack &pk) {
  long long ctas = 0;
  for (int q = 0; q < pk.n; q++) {
    const GemmDesc &g = pk.d[q];
    ctas += (long long)((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN) * g.batch;
  }
  return ctas;
}

template <class C, int BM, int BN, int BK, int TM, int TN>
cudaError_t launch_cfg(const GemmPack &pk, cudaStream_t st) {
  int maxtiles = 0, maxbatch = 0;
  for (int q = 0; q < pk.n; q++) {
    const GemmDesc &g = pk.d[q];
    int t = ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN);
    if (t > maxtiles) maxtiles = t;
    if (g.batch > maxbatch) maxbatch = g.batch;
  }
  if (maxtiles == 0 || maxbatch == 0) return cudaSuccess;
  dim3 grid(maxtiles, maxbatch < 65535 ? maxbatch : 65535, pk.n);
  return launch_k(gemm_kernel<C, BM, BN, BK, TM, TN>, grid, dim3((BM / TM) * (BN / TN)), 0, st, pk);
}

template <class C, int NN>
cudaError_t launch_gemv(const GemmPack &pk, cudaStream_t st) {
  long long blocks = 0;
  int kmin = 1 << 30;
  bool scratch = true;
  for (int q = 0; q < pk.n; q++) {
    blocks = std::max(blocks, (long long)((pk.d[q].M + 31) / 32) * pk.d[q].batch);
    kmin = std::min(kmin, pk.d[q].K);
    scratch = scratch && pk.d[q].part && pk.d[q].cnt;
  }
  if (blocks == 0) return cudaSuccess;
  // split K over CTAs while the launch has fewer than two CTAs an SM, keeping
  // at least 64 k a split and at most kGemvBlocks row blocks
  int ks = 1;
  if (scratch && blocks <= kGemvBlocks)
    while (ks < 16 && blocks * ks < 2 * 152 && kmin / (2 * ks) >= 64) ks *= 2;
  if (blocks * ks > kGemvSlots) ks = 1;  // (cannot happen: the loop stops below 2 x 304)
  dim3 grid((unsigned)blocks, ks, pk.n);
  return launch_k(gemv_kernel<C, NN>, grid, dim3(256), 0, st, pk);
}

// Complex64 products that the 128 x 128 kernel takes: no index maps, no
// second B, every tile mostly live, and one storage type for A (and for B)
// over the launch's descriptors.
bool cg64_fits(const GemmPack &pk) {
  for (int q = 0; q < pk.n; q++) {
    const GemmDesc &g = pk.d[q];
    if (g.A.rmap || g.A.cmap || g.B.rmap || g.B.cmap || g.B2.ptr || g.C.rmap || g.C.cmap || g.D.rmap ||
        g.D.cmap || g.M < 96 || g.N < 96 || g.A.f32 != pk.d[0].A.f32 || g.B.f32 != pk.d[0].B.f32)
      return false;
  }
  return true;
}

template <int BN>
cudaError_t launch_cg64_bn(const GemmPack &pk, cudaStream_t st) {
  int maxtiles = 0, maxbatch = 0;
  for (int q = 0; q < pk.n; q++) {
    const GemmDesc &g = pk.d[q];
    maxtiles = std::max(maxtiles, ((g.M + kCg - 1) / kCg) * ((g.N + BN - 1) / BN));
    maxbatch = std::max(maxbatch, g.batch);
  }
  if (maxtiles == 0 || maxbatch == 0) return cudaSuccess;
  dim3 grid(maxtiles, maxbatch < 65535 ? maxbatch : 65535, pk.n);
  const bool af = pk.d[0].A.f32, bf = pk.d[0].B.f32;
  if (af && bf) return launch_k(cgemm64_kernel<float2, float2, BN>, grid, dim3(256), 0, st, pk);
  if (af) return launch_k(cgemm64_kernel<float2, double2, BN>, grid, dim3(256), 0, st, pk);
  if (bf) return launch_k(cgemm64_kernel<double2, float2, BN>, grid, dim3(256), 0, st, pk);
  return launch_k(cgemm64_kernel<double2, double2, BN>, grid, dim3(256), 0, st, pk);
}

// 128 x 128 tiles (cfg 6) or 128 x 64 (cfg 7); by rule the narrower tile
// (two CTAs an SM)
cudaError_t launch_cg64(const GemmPack &pk, cudaStream_t st) {
  if (pk.d[0].cfg == 6) return launch_cg64_bn<128>(pk, st);
  return launch_cg64_bn<64>(pk, st);
}

template <class C>
cudaError_t launch_typed(const GemmPack &pk, int maxN, cudaStream_t st) {
  if (maxN <= 1) return launch_gemv<C, 1>(pk, st);
  if (maxN <= 2) return launch_gemv<C, 2>(pk, st);
  if (maxN <= 4) return launch_gemv<C, 4>(pk, st);
  if (maxN <= 8) return launch_gemv<C, 8>(pk, st);
  // 9 .. 16 right-hand sides of a solve (its products carry split-K scratch):
  // the skinny kernel too, which splits K where the level has few row blocks
  bool scratch = true;
  for (int q = 0; q < pk.n; q++) scratch = scratch && pk.d[q].part && pk.d[q].cnt;
  if (maxN <= 16 && scratch) return launch_gemv<C, 16>(pk, st);
  const bool c64 = sizeof(C) == sizeof(float2) && cg64_fits(pk);
  switch (pk.d[0].cfg) {  // a measured choice (hps_tune)
    case 6:
    case 7:
      if (c64) return launch_cg64(pk, st);
      break;
    case 1: return launch_cfg<C, 64, 64, 16, 4, 4>(pk, st);
    case 2: return launch_cfg<C, 32, 32, 16, 2, 2>(pk, st);
    case 3: return launch_cfg<C, 16, 16, 16, 1, 1>(pk, st);
    case 4: return launch_cfg<C, 64, 16, 16, 2, 2>(pk, st);
    default: break;
  }
  if (maxN < 32) return launch_cfg<C, 64, 16, 16, 2, 2>(pk, st);
  // the largest tile that still gives every SM two CTAs (one for the
  // complex64 128 x 128 tiles)
  const long long want = 2 * 152;
  if (c64 && cfg_ctas<128, 128>(pk) >= want / 2) return launch_cg64(pk, st);
  if (cfg_ctas<64, 64>(pk) >= want) return launch_cfg<C, 64, 64, 16, 4, 4>(pk, st);
  if (cfg_ctas<32, 32>(pk) >= want) return launch_cfg<C, 32, 32, 16, 2, 2>(pk, st);
  return launch_cfg<C, 16, 16, 16, 1, 1>(pk, st);
}

}  // namespace

static thread_local bool t_chained = false;
LaunchChain::LaunchChain() : prev(t_chained) { t_chained = true; }
LaunchChain::~LaunchChain() { t_chained = prev; }
bool launch_chained() { return t_chained; }

cudaError_t launch_gemm(const GemmDesc *descs, int ndesc, cudaStream_t st) {
  if (ndesc < 1 || ndesc > 2) return cudaErrorInvalidValue;
  GemmPack pk;
  pk.n = 0;
  int maxN = 0, cf32 = -1;
  for (int q = 0; q < ndesc; q++) {
    const GemmDesc &g = descs[q];
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) continue;
    if (cf32 >= 0 && cf32 != g.cf32) return cudaErrorInvalidValue;  // one precision a launch
    cf32 = g.cf32;
    pk.d[pk.n++] = g;
    if (g.N > maxN) maxN = g.N;
  }
  if (pk.n == 0) return cudaSuccess;
  // K == 0 is legal (C = beta D); the k-loop simply does not run.
  return cf32 ? launch_typed<float2>(pk, maxN, st) : launch_typed<double2>(pk, maxN, st);
}

cudaError_t launch_copy(const CopyBatch &cb, cudaStream_t st) {
  if (cb.count < 1 || cb.count > kMaxCopies) return cudaErrorInvalidValue;
  long long maxel = 0;
  int maxbatch = 0;
  for (int q = 0; q < cb.count; q++) {
    long long el = (long long)cb.d[q].M * cb.d[q].N;
    if (el > maxel) maxel = el;
    if (cb.d[q].batch > maxbatch) maxbatch = cb.d[q].batch;
  }
  if (maxel == 0 || maxbatch == 0) return cudaSuccess;
  dim3 grid((unsigned)((maxel + 255) / 256), maxbatch < 65535 ? maxbatch : 65535, cb.count);
  return launch_k(copy_kernel, grid, dim3(256), 0, st, cb);
}

}  // namespace hps
