// Batched, index-mapped complex128 GEMM and copy kernels.
//
// Every dense product of the HPS merge (Sec. 2.2: W = I - R33b R33a,
// Phi_a = W^{-1}[R33b R31a | -R32b], Phi_b, R^tau) and of the solve sweeps
// (Algorithm 2: the leaf matvecs Y s, Gamma s, Psi t and the per-level
// Upsilon / Phi actions) is one launch of gemm_kernel over all boxes of a
// tree level.  Sub-blocks such as R33a = R^alpha(I3, I3) are read through
// index maps, so no gather pass is needed before a product.
//
// The path is complex FP64 (DFMA-bound on this part: the tile sizes only
// need enough reuse to keep shared-memory traffic well below the DFMA rate).
#include <algorithm>

#include "hps_internal.h"

namespace hps {

namespace {

struct GemmPack {
  int n;
  GemmDesc d[2];
};

__device__ __forceinline__ long long mat_off(const Mat &m, int b, int i, int j) {
  long long r = m.rmap ? (long long)__ldg(m.rmap + i) : (long long)i;
  long long c = m.cmap ? (long long)__ldg(m.cmap + j) : (long long)j;
  return (long long)b * m.stride + r + c * m.ld;
}

__device__ __forceinline__ double2 ld2(const double2 *p) { return __ldg(p); }

__device__ __forceinline__ void cmac(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// C tile of BM x BN per CTA; each thread owns TM x TN outputs at rows
// tx + r * (BM/TM) and columns ty + c * (BN/TN).
template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    gemm_kernel(const __grid_constant__ GemmPack pack) {
  constexpr int NTX = BM / TM, NTY = BN / TN, NT = NTX * NTY;
  __shared__ double2 As[BK][BM];
  __shared__ double2 Bs[BK][BN];
  const GemmDesc &g = pack.d[blockIdx.z];
  const int tiles_m = (g.M + BM - 1) / BM;
  const int tiles_n = (g.N + BN - 1) / BN;
  if ((int)blockIdx.x >= tiles_m * tiles_n) return;
  const int m0 = (blockIdx.x % tiles_m) * BM;
  const int n0 = (blockIdx.x / tiles_m) * BN;
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;

  for (int b = blockIdx.y; b < g.batch; b += gridDim.y) {
  double2 acc[TM][TN];
#pragma unroll
  for (int r = 0; r < TM; r++)
#pragma unroll
    for (int c = 0; c < TN; c++) acc[r][c] = make_double2(0.0, 0.0);

  for (int k0 = 0; k0 < g.K; k0 += BK) {
    // A tile: BM x BK, consecutive threads walk down a column
    for (int e = tid; e < BM * BK; e += NT) {
      int i = e % BM, k = e / BM;
      int gi = m0 + i, gk = k0 + k;
      double2 v = make_double2(0.0, 0.0);
      if (gi < g.M && gk < g.K) v = ld2(g.A.ptr + mat_off(g.A, b, gi, gk));
      As[k][i] = v;
    }
    // B tile: BK x BN
    for (int e = tid; e < BK * BN; e += NT) {
      int k = e % BK, j = e / BK;
      int gk = k0 + k, gj = n0 + j;
      double2 v = make_double2(0.0, 0.0);
      if (gk < g.K && gj < g.N) {
        if (g.B2.ptr == nullptr || gk < g.ksplit)
          v = ld2(g.B.ptr + mat_off(g.B, b, gk, gj));
        else
          v = ld2(g.B2.ptr + mat_off(g.B2, b, gk - g.ksplit, gj));
      }
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < BK; k++) {
      double2 a[TM], bv[TN];
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
      if (i < g.M && j < g.N) {
        double2 v = cmul(g.alpha, acc[r][c]);
        if (g.D.ptr) {
          double2 d = g.D.ptr[mat_off(g.D, b, i, j)];
          double2 t = cmul(g.beta, d);
          v.x += t.x;
          v.y += t.y;
        }
        if (g.addI && i == j) v.x += 1.0;
        const_cast<double2 *>(g.C.ptr)[mat_off(g.C, b, i, j)] = v;
      }
    }
  }
}

__global__ void __launch_bounds__(256) copy_kernel(const __grid_constant__ CopyBatch cb) {
  const CopyDesc &d = cb.d[blockIdx.z];
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)d.M * d.N;
  if (e >= total) return;
  int i = (int)(e % d.M), j = (int)(e / d.M);
  for (int b = blockIdx.y; b < d.batch; b += gridDim.y) {
    double2 v = make_double2(0.0, 0.0);
    if (d.src.ptr) {
      double2 s = d.trans ? d.src.ptr[mat_off(d.src, b, j, i)] : d.src.ptr[mat_off(d.src, b, i, j)];
      v = cmul(d.alpha, s);
    }
    const_cast<double2 *>(d.dst.ptr)[mat_off(d.dst, b, i, j)] = v;
  }
}

// Skinny products (N <= NN: the solve's right-hand sides).  A CTA computes 32
// rows of one batch entry; its 8 warps split K (warp w takes k = w, w+8, ...),
// each lane one row, so the 32 loads of A a warp issues are one coalesced
// column segment and B(k, :) is a broadcast.  The 8 partial sums meet in
// shared memory.  Enough CTAs exist even for one large matrix.
template <int NN>
__global__ void __launch_bounds__(256) gemv_kernel(const __grid_constant__ GemmPack pack) {
  __shared__ double2 red[8][NN][33];
  const GemmDesc &g = pack.d[blockIdx.z];
  const int rblocks = (g.M + 31) / 32;
  if ((long long)blockIdx.x >= (long long)rblocks * g.batch) return;
  const int b = blockIdx.x / rblocks;
  const int i = (blockIdx.x % rblocks) * 32 + (threadIdx.x & 31);
  const int w = threadIdx.x >> 5;
  const bool live = i < g.M;
  double2 acc[NN];
#pragma unroll
  for (int j = 0; j < NN; j++) acc[j] = make_double2(0.0, 0.0);
  if (live) {
    const long long arow = (long long)b * g.A.stride + (g.A.rmap ? (long long)__ldg(g.A.rmap + i) : i);
#pragma unroll 4
    for (int k = w; k < g.K; k += 8) {
      const long long c = g.A.cmap ? (long long)__ldg(g.A.cmap + k) : k;
      const double2 a = ld2(g.A.ptr + arow + c * g.A.ld);
      const bool second = (g.B2.ptr != nullptr && k >= g.ksplit);
      const double2 *bp = second ? g.B2.ptr : g.B.ptr;
      const int *brm = second ? g.B2.rmap : g.B.rmap;
      const int *bcm = second ? g.B2.cmap : g.B.cmap;
      const long long bld = second ? g.B2.ld : g.B.ld;
      const long long bst = second ? g.B2.stride : g.B.stride;
      const int kk = second ? k - g.ksplit : k;
      const long long brow = (long long)b * bst + (brm ? (long long)__ldg(brm + kk) : kk);
#pragma unroll
      for (int j = 0; j < NN; j++)
        if (j < g.N) {
          const long long cj = bcm ? (long long)__ldg(bcm + j) : j;
          cmac(acc[j], a, ld2(bp + brow + cj * bld));
        }
    }
  }
#pragma unroll
  for (int j = 0; j < NN; j++) red[w][j][threadIdx.x & 31] = acc[j];
  __syncthreads();
  if (w == 0 && live) {
    const int l = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < NN; j++) {
      if (j >= g.N) continue;
      double2 v = red[0][j][l];
#pragma unroll
      for (int q = 1; q < 8; q++) {
        v.x += red[q][j][l].x;
        v.y += red[q][j][l].y;
      }
      v = cmul(g.alpha, v);
      if (g.D.ptr) {
        double2 t = cmul(g.beta, g.D.ptr[mat_off(g.D, b, i, j)]);
        v.x += t.x;
        v.y += t.y;
      }
      if (g.addI && i == j) v.x += 1.0;
      const_cast<double2 *>(g.C.ptr)[mat_off(g.C, b, i, j)] = v;
    }
  }
}

template <int BM, int BN, int BK, int TM, int TN>
long long cfg_ctas(const GemmPack &pk) {
  long long ctas = 0;
  for (int q = 0; q < pk.n; q++) {
    const GemmDesc &g = pk.d[q];
    ctas += (long long)((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN) * g.batch;
  }
  return ctas;
}

template <int BM, int BN, int BK, int TM, int TN>
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
  gemm_kernel<BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(pk);
  return cudaGetLastError();
}

template <int NN>
cudaError_t launch_gemv(const GemmPack &pk, cudaStream_t st) {
  long long blocks = 0;
  for (int q = 0; q < pk.n; q++)
    blocks = std::max(blocks, (long long)((pk.d[q].M + 31) / 32) * pk.d[q].batch);
  if (blocks == 0) return cudaSuccess;
  dim3 grid((unsigned)blocks, 1, pk.n);
  gemv_kernel<NN><<<grid, 256, 0, st>>>(pk);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm(const GemmDesc *descs, int ndesc, cudaStream_t st) {
  if (ndesc < 1 || ndesc > 2) return cudaErrorInvalidValue;
  GemmPack pk;
  pk.n = 0;
  int maxN = 0;
  for (int q = 0; q < ndesc; q++) {
    const GemmDesc &g = descs[q];
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) continue;
    pk.d[pk.n++] = g;
    if (g.N > maxN) maxN = g.N;
  }
  if (pk.n == 0) return cudaSuccess;
  // K == 0 is legal (C = beta D); the k-loop simply does not run.
  if (maxN <= 1) return launch_gemv<1>(pk, st);
  if (maxN <= 2) return launch_gemv<2>(pk, st);
  if (maxN <= 4) return launch_gemv<4>(pk, st);
  if (maxN <= 8) return launch_gemv<8>(pk, st);
  if (maxN < 32) return launch_cfg<64, 16, 16, 2, 2>(pk, st);
  // FP64-bound tiles: the largest tile that still gives every SM two CTAs
  const long long want = 2 * 152;
  if (cfg_ctas<64, 64, 16, 4, 4>(pk) >= want) return launch_cfg<64, 64, 16, 4, 4>(pk, st);
  if (cfg_ctas<32, 32, 16, 2, 2>(pk) >= want) return launch_cfg<32, 32, 16, 2, 2>(pk, st);
  return launch_cfg<16, 16, 16, 1, 1>(pk, st);
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
  copy_kernel<<<grid, 256, 0, st>>>(cb);
  return cudaGetLastError();
}

}  // namespace hps
