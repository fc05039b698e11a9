// Complex128 GEMM emulated on the bf16 tensor cores (Ozaki scheme), with the
// products on tcgen05 (accumulators in tensor memory, operand tiles staged in
// shared memory by TMA).
//
// Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59 (2012): split each operand into
// slices whose pairwise products are exact in a fast low-precision unit,
// multiply the slices there and sum the products in high precision.
//
// Splitting.  Row i of A is scaled by 2^-a_i so that its largest real or
// imaginary part lies in [1/4, 1/2); column j of B by 2^-b_j likewise.  Each
// scaled value x (real and imaginary parts separately) is written as
//     x = sum_{s < S} d_s 2^{-6(s+1)} + r,   d_s integers, |d_s| <= 32,
// with |r| <= 2^{-6S-1}: D = round(x 2^{6S}) is formed from the IEEE-754
// fields of x as a 64-bit integer and cut into balanced base-64 digits
// (every step exact; integer work only, since this part's FP64 pipe is 64
// times slower than its integer and FP32 pipes).  The digits are exact in
// bf16.  Both operands' digit planes are stored K-major ([row][k], k
// contiguous), the layout the tensor cores read without transposition.
//
// Products.  The slice pairs (s, t) with s + t < S are taken group by group
// of equal shift e = s + t, whose products all carry the weight 2^{-6(e+2)}.
// A group's complex product over a K chunk of OZ_KC = 896 is accumulated in
// FP32 in tensor memory: a digit product is at most 2^10 in magnitude, a
// complex combination (ar br - ai bi or ar bi + ai br) at most 2^11, and a
// group has at most S = 9 pairs, so every partial sum is an integer below
// 9 * 896 * 2^11 < 2^24 and the FP32 accumulation is exact.  After each
// group (and K chunk) the sum is added, times its weight, into complex128
// partial sums: 9 FP64 updates an output for K <= 896, which keeps this
// part's FP64 pipe (2 operations per clock per SM) well below the
// tensor-core work.  Pairs with s + t >= S are dropped: with the remainders
// they bound the error of every term by ~2^{-6S} max|A_i.| max|B_.j|
// (2^-54 for S = 9), the size of a complex128 rounding.  The result is
// scaled back by 2^{a_i + b_j} and combined as C = alpha AB + beta D (+ I).
//
// Kernels: the exponents of A's rows; the digits of A (64 x 32 blocks
// transposed through shared memory so that both the reads of the
// column-major operand and the K-major digit writes are contiguous); the
// digits of B (a warp per column, lanes over k); and the product kernel, one
// CTA per 128 x BN output tile (BN = 128, or 64 for narrow products) and
// share of the slice pairs:
//   warp 0   one thread issues the TMA copies of the digit tiles (real and
//            imaginary parts of an A slice and a B slice, 64 k each, 128-byte
//            swizzled) into a ring of shared-memory stages;
//   warp 1   allocates the tensor memory; one thread issues tcgen05.mma
//            (M = 128, N = BN, K = 16 per instruction; the real part
//            Re += Ar Br + (-Ai) Bi through the instruction's negate-A bit,
//            the imaginary part Im += Ar Bi + Ai Br) into one of two
//            accumulator buffers, and commits each stage back to its slot and
//            each finished group to the epilogue;
//   warps 2-9  read a finished group's FP32 sums out of tensor memory
//            (tcgen05.ld), hand the buffer back, and add the sums with the
//            group's weight into the tile's complex128 partial sums (global
//            scratch, resident in L2), or, after the last group, write
//            C = alpha 2^(a_i + b_j) sum + beta D (+ I).
// Products with few output tiles split the slice pairs over several CTAs a
// tile and sum the partial results in a last pass.  Every wait on a barrier
// gives up after 2 s (recording a timeout in the status word), so that a
// stalled pipeline ends the kernel with an error instead of hanging the GPU.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "cx.cuh"
#include "hps_internal.h"
#include "tc_desc.h"

namespace hps {

namespace {

// Slices per operand (6 bits each): 9 for complex128 products (every term
// to ~2^-54 of its row and column scale), 5 for the products wanted to
// complex64 accuracy (the cf32 products: ~5 2^-29 a term, at or below the
// rounding of complex64 arithmetic), which take 15 slice pairs instead of 45.
constexpr int OZ_S = 9;
constexpr int OZ_S32 = 5;
inline int oz_slices(const GemmDesc &g) { return g.cf32 ? OZ_S32 : OZ_S; }
constexpr int OZ_KC = 896;                       // K per exact FP32 accumulation of a shift group
constexpr int TC_BM = 128, TC_BK = 64;           // tile rows; k per stage (one 128-byte swizzle row)
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_THREADS = 32 * (2 + TC_EPI_WARPS);
constexpr unsigned kStatusTimeout = 3u;          // status-word code of a pipeline wait that gave up

template <int BN>
struct TcCfg {
  static constexpr int kStages = BN == 128 ? 3 : 4;
  static constexpr int kTileA = TC_BM * TC_BK * 2;  // bytes of one A digit tile (16 KB)
  static constexpr int kTileB = BN * TC_BK * 2;
  static constexpr int kStage = 2 * kTileA + 2 * kTileB;  // Ar, Ai, Br, Bi
  static constexpr size_t kSmem = (size_t)kStages * kStage + 1024;  // + alignment slack
  // two accumulator buffers of [Re | Im] x BN columns; with BN = 64 the other
  // half of tensor memory holds the tile's running complex128 sums (each
  // double as two 32-bit columns: Re of column j at 2 j, Im at 2 (BN + j))
  static constexpr bool kStateInTmem = (BN == 64);
  static constexpr uint32_t kStateCol = 4 * BN;
  static constexpr uint32_t kTmemCols = kStateInTmem ? 8 * BN : 4 * BN;
  static constexpr size_t kAcc = (size_t)TC_BM * 2 * BN;  // doubles of a tile's partial sums
};

int num_sms() {
  static int n = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 148;
    }
  });
  return n;
}

struct OzLayout {
  int Mp, Np, Kp;         // padded sizes (multiples of 128, BN, 64)
  int S, npairs;          // slices per operand; slice pairs (s + t < S)
  int bn;                 // output tile width: 128, or 64 for N <= 64
  int tm, tn;             // output tiles along M and N
  int gp;                 // CTAs per output tile, each summing a share of the slice pairs
  int units, ctas;        // work units (tile, share) and CTAs launched
  bool persistent;        // more tiles than SMs: one CTA an SM loops over them
  size_t a_off, b_off;    // byte offsets of the digit planes
  size_t ea_off, eb_off;  // byte offsets of the row / column exponents
  size_t acc_off;         // complex128 partial sums [gp][batch][tm][tn][2 bn][128]
  size_t total;
};

inline size_t oz_align(size_t x) { return (x + 255) & ~(size_t)255; }

OzLayout oz_layout(const GemmDesc &g, int nsm) {
  OzLayout L;
  // 64-wide tiles (N <= 64) keep their complex128 running sums in tensor
  // memory; 128-wide ones read half the operand bytes per product, which
  // measured faster at every K (1792 x 3584 x 896: 2.06 vs 3.34 ms;
  // 252^3 x 256: 3.22 vs 3.70 ms)
  L.bn = g.N <= 64 ? 64 : 128;
  if (const char *v = getenv("HPS_OZ_BN")) L.bn = atoi(v) == 64 ? 64 : 128;
  L.Mp = (g.M + TC_BM - 1) / TC_BM * TC_BM;
  L.Np = (g.N + L.bn - 1) / L.bn * L.bn;
  L.Kp = (g.K + TC_BK - 1) / TC_BK * TC_BK;
  L.tm = L.Mp / TC_BM;
  L.tn = L.Np / L.bn;
  L.S = oz_slices(g);
  L.npairs = L.S * (L.S + 1) / 2;
  const size_t B = (size_t)g.batch;
  size_t o = 0;
  L.a_off = o;
  o = oz_align(o + B * L.S * 2 * (size_t)L.Mp * L.Kp * sizeof(__nv_bfloat16));
  L.b_off = o;
  o = oz_align(o + B * L.S * 2 * (size_t)L.Np * L.Kp * sizeof(__nv_bfloat16));
  L.ea_off = o;
  o = oz_align(o + B * (size_t)L.Mp * sizeof(int));
  L.eb_off = o;
  o = oz_align(o + B * (size_t)L.Np * sizeof(int));
  // one CTA an SM (the tile's stages fill shared memory): with fewer tiles
  // than SMs the slice pairs are split over up to 9 CTAs a tile (5 pairs or
  // more each), picking the split that leaves the last wave fullest
  const long long tiles = (long long)L.tm * L.tn * g.batch;
  L.gp = 1;
  if (tiles < nsm) {
    double best = 0.0;
    for (int q = 1; q <= std::max(1, L.npairs / 5); q++) {
      const long long ctas = tiles * q;
      const long long waves = (ctas + nsm - 1) / nsm;
      const double eff = (double)ctas / (double)(waves * nsm);
      if (eff > best * 1.02) {
        best = eff;
        L.gp = q;
      }
    }
  }
  while (L.gp > 1 && (long long)g.batch * L.gp > 65535) L.gp--;
  // one CTA an SM: with more tiles than SMs, persistent CTAs loop over the
  // tiles and each keeps one partial-sum slab (L2-resident) for all of them
  L.units = (int)(tiles * L.gp);
  L.persistent = L.gp == 1 && tiles > nsm;
  L.ctas = L.persistent ? nsm : L.units;
  L.acc_off = o;
  o = oz_align(o + (L.persistent ? (size_t)nsm * TC_BM * 2 * L.bn * sizeof(double)
                                 : (size_t)L.gp * B * L.Mp * L.Np * 2 * sizeof(double)));
  L.total = o;
  return L;
}

__device__ __forceinline__ long long oz_off(const Mat &m, int b, int i, int j) {
  long long r = m.rmap ? (long long)__ldg(m.rmap + i) : (long long)i;
  long long c = m.cmap ? (long long)__ldg(m.cmap + j) : (long long)j;
  return (long long)b * m.stride + r + c * m.ld;
}

__device__ __forceinline__ double2 oz_ld(const Mat &m, long long off) {
  if (m.f32) {
    float2 v = __ldg((const float2 *)m.ptr + off);
    return make_double2(v.x, v.y);
  }
  return __ldg((const double2 *)m.ptr + off);
}

// element (k, j) of the B operand (rows from k >= ksplit come from B2)
__device__ __forceinline__ double2 oz_ldb(const GemmDesc &g, int b, int k, int j) {
  if (k < g.ksplit) return oz_ld(g.B, oz_off(g.B, b, k, j));
  return oz_ld(g.B2, oz_off(g.B2, b, k - g.ksplit, j));
}

__device__ __forceinline__ double2 oz_lda(const GemmDesc &g, int b, int i, int k) {
  return oz_ld(g.A, oz_off(g.A, b, i, k));
}

// max(|Re|, |Im|) as the integer image of its IEEE-754 bits (integer order is
// numeric order for non-negative values)
__device__ __forceinline__ unsigned long long oz_mag(double2 v) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(v.x) & 0x7fffffffffffffffull;
  const unsigned long long b = (unsigned long long)__double_as_longlong(v.y) & 0x7fffffffffffffffull;
  return a > b ? a : b;
}

// The scaling exponent sh of a row or column whose largest magnitude has the
// bits m: m 2^-sh lies in [1/4, 1/2) (m = 1.f 2^(E-1023) = 0.1f 2^(E-1022),
// so sh = E - 1021); 0 for an all-zero row.
__device__ __forceinline__ int oz_shift(unsigned long long m) {
  return m ? (int)(m >> 52) - 1021 : 0;
}

// D = round(v 2^(6S - sh)) for |v 2^-sh| < 1/2 (so |D| <= 2^53), from the
// fields of v: v = +-M 2^(E' - 1075) with the 53-bit significand M.
template <int S>
__device__ __forceinline__ long long oz_fixed(double v, int sh) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7ff);
  const unsigned long long M = (b & 0xfffffffffffffull) | (E ? (1ull << 52) : 0ull);
  const int t = (E ? E : 1) - 1075 + 6 * S - sh;  // D = round(M 2^t)
  long long D;
  if (M == 0 || t < -62)
    D = 0;
  else if (t >= 0)
    D = (long long)(M << t);  // only for tiny M: the product stays below 2^53
  else
    D = (long long)((M + (1ull << (-t - 1))) >> -t);
  return (b >> 63) ? -D : D;
}

// the S balanced base-64 digits of D, most significant first:
// D = sum_s d_s 64^(S-1-s), d_s in [-32, 32]
template <int S>
__device__ __forceinline__ void oz_digits(long long D, int (&d)[S]) {
#pragma unroll
  for (int s = S - 1; s > 0; s--) {
    const int v = (int)((D + 32) & 63) - 32;
    d[s] = v;
    D = (D - v) >> 6;
  }
  d[0] = (int)D;
}

// Digits of B, a warp per column, lanes over k (neighbouring k are
// neighbouring in the column-major operands): the column's exponent, then its
// digits ([column][k], k contiguous).  Padding columns and k get zeros.
template <int S>
__global__ void __launch_bounds__(256) oz_split_b_kernel(const __grid_constant__ GemmDesc g, int Np, int Kp,
                                                         __nv_bfloat16 *digits, int *expo) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + warp;
  const int b = blockIdx.y;
  if (j >= Np) return;
  const bool live = j < g.N;
  unsigned long long mx = 0;
  if (live)
    for (int k = lane; k < g.K; k += 32) {
      const unsigned long long m = oz_mag(oz_ldb(g, b, k, j));
      mx = m > mx ? m : mx;
    }
  for (int off = 16; off; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
    mx = o > mx ? o : mx;
  }
  const int sh = oz_shift(mx);
  if (lane == 0) expo[(size_t)b * Np + j] = sh;
  const size_t plane = (size_t)Np * Kp;
  __nv_bfloat16 *base = digits + (size_t)b * S * 2 * plane + (size_t)j * Kp;
  for (int k = lane; k < Kp; k += 32) {
    double2 v = make_double2(0.0, 0.0);
    if (live && k < g.K) v = oz_ldb(g, b, k, j);
    int dr[S], di[S];
    oz_digits<S>(oz_fixed<S>(v.x, sh), dr);
    oz_digits<S>(oz_fixed<S>(v.y, sh), di);
#pragma unroll
    for (int q = 0; q < S; q++) {
      base[(size_t)(2 * q) * plane + k] = __int2bfloat16_rn(dr[q]);
      base[(size_t)(2 * q + 1) * plane + k] = __int2bfloat16_rn(di[q]);
    }
  }
}

// Exponent of each row of A (32 rows a block, 8 threads a row over k,
// combined in shared memory; neighbouring threads on neighbouring rows).
__global__ void __launch_bounds__(256) oz_expo_a_kernel(const __grid_constant__ GemmDesc g, int Mp, int *expo) {
  __shared__ unsigned long long part[8][32];
  const int r = threadIdx.x & 31, kl = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + r, b = blockIdx.y;
  unsigned long long mx = 0;
  if (i < g.M)
    for (int k = kl; k < g.K; k += 8) {
      const unsigned long long m = oz_mag(oz_lda(g, b, i, k));
      mx = m > mx ? m : mx;
    }
  part[kl][r] = mx;
  __syncthreads();
  if (kl == 0 && i < Mp) {
    for (int q = 1; q < 8; q++) mx = part[q][r] > mx ? part[q][r] : mx;
    expo[(size_t)b * Mp + i] = oz_shift(mx);
  }
}

// Digits of A, K-major ([row][k]), for a block of 32 rows x 32 k: each thread
// reads elements with neighbouring threads on neighbouring rows (coalesced
// for the column-major operands), the 18 digit planes are transposed in
// shared memory, and each row's 32 digits leave as four 16-byte stores.
// Padding rows and k get zeros.
constexpr int OZA_R = 32, OZA_K = 32, OZA_LD = OZA_K + 8;  // shared row: 80 bytes (16-byte aligned)
template <int S>
__global__ void __launch_bounds__(256) oz_split_a_kernel(const __grid_constant__ GemmDesc g, int Mp, int Kp,
                                                         __nv_bfloat16 *digits, const int *expo) {
  __shared__ __align__(16) __nv_bfloat16 tile[2 * S][OZA_R][OZA_LD];
  const int r = threadIdx.x & 31, kq = threadIdx.x >> 5;
  const int i0 = blockIdx.x * OZA_R, k0 = blockIdx.y * OZA_K, b = blockIdx.z;
  const int i = i0 + r;
  const int sh = expo[(size_t)b * Mp + i];
  for (int kk = kq; kk < OZA_K; kk += 8) {
    const int k = k0 + kk;
    double2 v = make_double2(0.0, 0.0);
    if (i < g.M && k < g.K) v = oz_lda(g, b, i, k);
    int dr[S], di[S];
    oz_digits<S>(oz_fixed<S>(v.x, sh), dr);
    oz_digits<S>(oz_fixed<S>(v.y, sh), di);
#pragma unroll
    for (int q = 0; q < S; q++) {
      tile[2 * q][r][kk] = __int2bfloat16_rn(dr[q]);
      tile[2 * q + 1][r][kk] = __int2bfloat16_rn(di[q]);
    }
  }
  __syncthreads();
  const size_t plane = (size_t)Mp * Kp;
  __nv_bfloat16 *base = digits + (size_t)b * S * 2 * plane;
  constexpr int VPR = OZA_K / 8;  // 16-byte vectors a row
  for (int v = threadIdx.x; v < 2 * S * OZA_R * VPR; v += 256) {
    const int pl = v / (OZA_R * VPR), rem = v % (OZA_R * VPR), row = rem / VPR, c = rem % VPR;
    const uint4 val = *reinterpret_cast<const uint4 *>(&tile[pl][row][c * 8]);
    *reinterpret_cast<uint4 *>(base + (size_t)pl * plane + (size_t)(i0 + row) * Kp + k0 + c * 8) = val;
  }
}

// ---- PTX wrappers: mbarriers, TMA, tcgen05 ---------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}

constexpr uint64_t kWaitNs = 2000000000ull;  // a wait gives up after 2 s

// L2 cache policy "evict last" and loads / stores that carry it
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ double ld_keep(const double *a, uint64_t pol) {
  double v;
  asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;\n" : "=d"(v) : "l"(a), "l"(pol) : "memory");
  return v;
}
__device__ __forceinline__ void st_keep(double *a, double v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;\n" ::"l"(a), "d"(v), "l"(pol) : "memory");
}

// Wait for the phase of `bar` with the given parity to complete.  Gives up
// (false) when another role of the CTA has given up (*abort set; unless
// drain, for the waits that let work in flight finish before the CTA exits)
// or after limit_ns, then sets *abort and records a timeout in the status word.
__device__ __noinline__ bool bar_wait(uint64_t *bar, uint32_t parity, volatile int *abort, unsigned *status,
                                      bool drain = false, uint64_t limit_ns = kWaitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    for (int q = 0; q < 64; q++)
      if (mbar_try_wait(bar, parity)) return true;
    if (!drain && *abort) return false;
    if (global_ns() - t0 > limit_ns) {
      *abort = 1;
      if (status) record_status(status, kStatusTimeout, 0, (int)(blockIdx.x + gridDim.x * blockIdx.y));
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint64_t *bar, int x, int y,
                                            int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)map) : "memory");
}

__device__ __forceinline__ void tc_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
// D (tensor memory) (+)= A B, A and B from shared-memory descriptors
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive once on `bar` when every tcgen05.mma this thread issued so far has completed
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   smem_u32(bar))
               : "memory");
}
// 32 consecutive 32-bit columns of this thread's tensor-memory lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
// 16 consecutive 32-bit columns of this thread's tensor-memory lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// store 32 consecutive 32-bit columns of this thread's tensor-memory lane
__device__ __forceinline__ void tc_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
      "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
      "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// s 2^k as a double, exactly, for an integer-valued float s with |s| < 2^24
// (a shift group's FP32 sum) and a weight exponent k >= -60: the double is
// assembled from the float's fields with integer instructions (sign; biased
// exponent + 1023 - 127 + k; significand shifted to 52 bits), so a flush
// costs one FP64 add a value on this part's 1/64-rate FP64 pipe instead of
// a conversion and a multiply-add.
__device__ __forceinline__ double oz_term(float s, int k) {
  const unsigned b = __float_as_uint(s);
  if ((b & 0x7fffffffu) == 0u) return 0.0;
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  const unsigned long long ex = (unsigned long long)(((b >> 23) & 0xffu) + 896 + k) << 52;
  const unsigned long long man = (unsigned long long)(b & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(sign | ex | man));
}

// pair index p (ordered by shift e = s + t, then s) -> (e, s)
__device__ __forceinline__ void pair_decode(int p, int &e, int &s) {
  e = 0;
  while (p > e) {
    p -= e + 1;
    e++;
  }
  s = p;
}

struct TcArgs;
__device__ __forceinline__ void oz_out(const TcArgs &a, int b, int i, int j, int sha, double sr, double si);

struct TcArgs {
  GemmDesc g;
  int Mp, Np, Kp;
  int S, npairs;     // slices per operand, slice pairs taken
  int tm, tn;        // output tiles along M and N
  int gp;            // CTAs a tile (shares of the slice pairs)
  int units;         // work units: tn tm batch gp (tile and share), tn fastest
  int persistent;    // 1: CTAs loop over the units with one partial-sum slab each
  double *acc;       // partial sums [gp][batch][tm][tn][2 BN][128] ([Re columns, Im columns][row]),
                     // or [CTA][2 BN][128] when persistent
  const int *ea;     // [batch][Mp]
  const int *eb;     // [batch][Np]
  unsigned *status;  // build status word for timeouts, or null
};

// C(i, j) = alpha 2^(a_i + b_j) (sr + i si) + beta D(i, j) (+ 1 on the diagonal)
__device__ __forceinline__ void oz_out(const TcArgs &a, int b, int i, int j, int sha, double sr, double si) {
  const GemmDesc &g = a.g;
  const int sh = sha + __ldg(a.eb + (size_t)b * a.Np + j);
  const double vre = ldexp(sr, sh), vim = ldexp(si, sh);
  double outr = g.alpha.x * vre - g.alpha.y * vim;
  double outi = g.alpha.x * vim + g.alpha.y * vre;
  if (g.D.ptr) {
    const long long od = oz_off(g.D, b, i, j);
    double2 d;
    if (g.D.f32) {
      const float2 f = ((const float2 *)g.D.ptr)[od];
      d = make_double2(f.x, f.y);
    } else {
      d = ((const double2 *)g.D.ptr)[od];
    }
    outr += g.beta.x * d.x - g.beta.y * d.y;
    outi += g.beta.x * d.y + g.beta.y * d.x;
  }
  if (g.addI && i == j) outr += 1.0;
  const long long oc = oz_off(g.C, b, i, j);
  if (g.C.f32)
    ((float2 *)g.C.ptr)[oc] = make_float2((float)outr, (float)outi);
  else
    ((double2 *)g.C.ptr)[oc] = make_double2(outr, outi);
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    oz_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const __grid_constant__ TcArgs a) {
  using Cfg = TcCfg<BN>;
  constexpr int S_ = Cfg::kStages;
  extern __shared__ unsigned char tc_smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[S_], empty_bar[S_], accf_bar[2], acce_bar[2], drain_bar;
  __shared__ uint32_t tmem_sh;
  __shared__ volatile int abort_sh;
  __shared__ int issued_sh;

  const uint32_t sbase = (smem_u32(tc_smem_raw) + 1023u) & ~1023u;  // 128-byte swizzle atoms: 1 KB aligned
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // work unit u: its output tile (tn, tm), batch entry b and share grp of the
  // slice pairs [p0, p1); a CTA takes units blockIdx.x, + gridDim.x, ...
  struct Unit {
    int tn, tm, b, grp, p0, p1;
  };
  auto unit = [&](int u) {
    Unit w;
    w.tn = u % a.tn;
    w.tm = (u / a.tn) % a.tm;
    const int z = u / (a.tn * a.tm);
    w.b = z / a.gp;
    w.grp = z % a.gp;
    w.p0 = w.grp * a.npairs / a.gp;
    w.p1 = (w.grp + 1) * a.npairs / a.gp;
    return w;
  };
  const int nkb = a.Kp / TC_BK;
  constexpr int CKB = OZ_KC / TC_BK;  // k-blocks of a chunk
  const int nch = (nkb + CKB - 1) / CKB;

  if (threadIdx.x == 0) {
    for (int q = 0; q < S_; q++) {
      mbar_init(&full_bar[q], 1);   // the producer's arrive.expect_tx (+ the copies' bytes)
      mbar_init(&empty_bar[q], 1);  // one tcgen05.commit
    }
    for (int q = 0; q < 2; q++) {
      mbar_init(&accf_bar[q], 1);             // one tcgen05.commit
      mbar_init(&acce_bar[q], TC_EPI_WARPS);  // one arrival per epilogue warp
    }
    mbar_init(&drain_bar, 1);
    abort_sh = 0;
    issued_sh = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tc_alloc(&tmem_sh, Cfg::kTmemCols);
    tc_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    tma_prefetch_map(&tmA);
    tma_prefetch_map(&tmB);
    int it = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < a.units && ok; u += gridDim.x) {
     const Unit w = unit(u);
     const int tm = w.tm, tn = w.tn, b = w.b, p0 = w.p0, p1 = w.p1;
     for (int c = 0; c < nch && ok; c++) {
      const int kb0 = c * CKB, kb1 = min(nkb, kb0 + CKB);
      for (int p = p0; p < p1 && ok; p++) {
        int e, s;
        pair_decode(p, e, s);
        const int zA = (b * a.S + s) * 2, zB = (b * a.S + (e - s)) * 2;
        for (int kb = kb0; kb < kb1; kb++) {
          const int st = it % S_;
          const uint32_t ph = (uint32_t)(it / S_) & 1u;
          if (!bar_wait(&empty_bar[st], ph ^ 1u, &abort_sh, a.status)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full_bar[st], Cfg::kStage);
          const uint32_t sb = sbase + st * Cfg::kStage;
          tma_load_3d(sb, &tmA, &full_bar[st], kb * TC_BK, tm * TC_BM, zA);
          tma_load_3d(sb + Cfg::kTileA, &tmA, &full_bar[st], kb * TC_BK, tm * TC_BM, zA + 1);
          tma_load_3d(sb + 2 * Cfg::kTileA, &tmB, &full_bar[st], kb * TC_BK, tn * BN, zB);
          tma_load_3d(sb + 2 * Cfg::kTileA + Cfg::kTileB, &tmB, &full_bar[st], kb * TC_BK, tn * BN, zB + 1);
          it++;
        }
      }
     }
    }
    issued_sh = it;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    constexpr uint32_t id_pos = tc::idesc_bf16_f32(TC_BM, BN, false);
    constexpr uint32_t id_neg = tc::idesc_bf16_f32(TC_BM, BN, true);
    int it = 0, gi = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < a.units && ok; u += gridDim.x) {
     const Unit w = unit(u);
     const int p0 = w.p0, p1 = w.p1;
     for (int c = 0; c < nch && ok; c++) {
      const int kb0 = c * CKB, kb1 = min(nkb, kb0 + CKB);
      bool open = false, first = true;
      for (int p = p0; p < p1 && ok; p++) {
        int e, s;
        pair_decode(p, e, s);
        const int buf = gi & 1;
        if (!open) {
          // the epilogue has drained this buffer's previous group
          if (!bar_wait(&acce_bar[buf], ((uint32_t)(gi >> 1) & 1u) ^ 1u, &abort_sh, a.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          open = true;
          first = true;
        }
        const uint32_t dre = tmem + (uint32_t)(buf * 2 * BN), dim = dre + BN;
        for (int kb = kb0; kb < kb1; kb++) {
          const int st = it % S_;
          const uint32_t ph = (uint32_t)(it / S_) & 1u;
          if (!bar_wait(&full_bar[st], ph, &abort_sh, a.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sb = sbase + st * Cfg::kStage;
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; kk++) {
            const uint64_t ar = tc::smem_desc_sw128_kmajor(sb + kk * 32);
            const uint64_t ai = tc::smem_desc_sw128_kmajor(sb + Cfg::kTileA + kk * 32);
            const uint64_t br = tc::smem_desc_sw128_kmajor(sb + 2 * Cfg::kTileA + kk * 32);
            const uint64_t bi = tc::smem_desc_sw128_kmajor(sb + 2 * Cfg::kTileA + Cfg::kTileB + kk * 32);
            const uint32_t accum = first ? 0u : 1u;
            tc_mma(dre, ar, br, id_pos, accum);
            tc_mma(dim, ar, bi, id_pos, accum);
            tc_mma(dre, ai, bi, id_neg, 1u);
            tc_mma(dim, ai, br, id_pos, 1u);
            first = false;
          }
          tc_commit(&empty_bar[st]);  // the stage's slot is free once these products are done
          it++;
        }
        if (ok && (s == e || p == p1 - 1)) {
          tc_commit(&accf_bar[buf]);  // the group's sums are complete
          gi++;
          open = false;
        }
      }
     }
    }
    tc_commit(&drain_bar);
  } else if (warp >= 2) {
    // ---- epilogue: FP32 group sums -> complex128 ----
    constexpr int NC = BN / 2;   // columns of each part a warp handles
    constexpr int NL = NC / 32;  // 32-column loads per part
    const int q = warp & 3;      // tensor-memory lanes 32 q .. 32 q + 31 are this warp's
    const int hf = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    const GemmDesc &g = a.g;
    // the running sums stay in L2 while the digit planes stream past them
    const uint64_t keep = l2_evict_last();
    int gi = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < a.units && ok; u += gridDim.x) {
     const Unit w = unit(u);
     const int tm = w.tm, tn = w.tn, b = w.b, p0 = w.p0, p1 = w.p1;
     const int i = tm * TC_BM + row;
     // the running sums: the CTA's own slab when persistent, else the unit's
     double *slab = a.acc + (a.persistent ? (size_t)blockIdx.x
                                          : (((size_t)w.grp * g.batch + b) * a.tm + tm) * a.tn + tn) * Cfg::kAcc;
     const int sha = (i < a.Mp) ? __ldg(a.ea + (size_t)b * a.Mp + i) : 0;
     bool first = true;
     for (int c = 0; c < nch && ok; c++) {
      for (int p = p0; p < p1 && ok; p++) {
        int e, s;
        pair_decode(p, e, s);
        if (!(s == e || p == p1 - 1)) continue;
        const int buf = gi & 1;
        const bool got = bar_wait(&accf_bar[buf], (uint32_t)(gi >> 1) & 1u, &abort_sh, a.status);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 2 * BN + hf * NC);
        const int wk = -6 * (e + 2);  // the group's weight 2^wk
        const bool last = (c == nch - 1) && (p == p1 - 1);
        const bool fin = last && a.gp == 1;
        if constexpr (Cfg::kStateInTmem) {
          // this warp's 32 columns, 16 at a time: the group's FP32 sums and
          // the running complex128 sums, both in tensor memory
          const uint32_t ts = tmem + ((uint32_t)(q * 32) << 16) + Cfg::kStateCol;
#pragma unroll 1
          for (int l = 0; l < NC / 16; l++) {
            const int j0 = hf * NC + l * 16;  // first tile column of this piece
            uint32_t vr[16], vi[16], wr[32], wi[32];
            tc_ld16(tb + l * 16, vr);
            tc_ld16(tb + BN + l * 16, vi);
            if (!first) {
              tc_ld32(ts + 2 * j0, wr);
              tc_ld32(ts + 2 * (BN + j0), wi);
            }
            tc_wait_ld();
            if (l == NC / 16 - 1) {
              // the accumulator buffer is free for the next group but one
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&acce_bar[buf]);
            }
#pragma unroll
            for (int jj = 0; jj < 16; jj++) {
              double sr = oz_term(__uint_as_float(vr[jj]), wk);
              double si = oz_term(__uint_as_float(vi[jj]), wk);
              if (!first) {
                sr += __hiloint2double((int)wr[2 * jj + 1], (int)wr[2 * jj]);
                si += __hiloint2double((int)wi[2 * jj + 1], (int)wi[2 * jj]);
              }
              const int jl = j0 + jj, j = tn * BN + jl;
              if (fin) {
                if (i < g.M && j < g.N) oz_out(a, b, i, j, sha, sr, si);
              } else if (last) {
                // this CTA's share of the slice pairs, for the reduce pass
                slab[(size_t)jl * TC_BM + row] = sr;
                slab[(size_t)(BN + jl) * TC_BM + row] = si;
              } else {
                wr[2 * jj] = (uint32_t)__double2loint(sr);
                wr[2 * jj + 1] = (uint32_t)__double2hiint(sr);
                wi[2 * jj] = (uint32_t)__double2loint(si);
                wi[2 * jj + 1] = (uint32_t)__double2hiint(si);
              }
            }
            if (!last) {
              tc_st32(ts + 2 * j0, wr);
              tc_st32(ts + 2 * (BN + j0), wi);
              tc_wait_st();
            }
          }
        } else {
          // 32 columns of both parts at a time: tensor memory -> registers ->
          // the running complex128 sums in global scratch (or C)
#pragma unroll 1
          for (int l = 0; l < NL; l++) {
            uint32_t vr[32], vi[32];
            tc_ld32(tb + l * 32, vr);
            tc_ld32(tb + BN + l * 32, vi);
            tc_wait_ld();
            if (l == NL - 1) {
              // the buffer is free for the next group but one
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&acce_bar[buf]);
            }
            double *pr = slab + (size_t)(hf * NC + l * 32) * TC_BM + row;
            double *pi = pr + (size_t)BN * TC_BM;
            if (fin) {
#pragma unroll
              for (int jj = 0; jj < 32; jj++) {
                const int j = tn * BN + hf * NC + l * 32 + jj;
                double sr = oz_term(__uint_as_float(vr[jj]), wk);
                double si = oz_term(__uint_as_float(vi[jj]), wk);
                if (!first) {
                  sr += ld_keep(pr + (size_t)jj * TC_BM, keep);
                  si += ld_keep(pi + (size_t)jj * TC_BM, keep);
                }
                if (i < g.M && j < g.N) oz_out(a, b, i, j, sha, sr, si);
              }
            } else if (first) {
#pragma unroll
              for (int jj = 0; jj < 32; jj++) {
                st_keep(pr + (size_t)jj * TC_BM, oz_term(__uint_as_float(vr[jj]), wk), keep);
                st_keep(pi + (size_t)jj * TC_BM, oz_term(__uint_as_float(vi[jj]), wk), keep);
              }
            } else {
#pragma unroll
              for (int jj = 0; jj < 32; jj++) {
                st_keep(pr + (size_t)jj * TC_BM,
                        ld_keep(pr + (size_t)jj * TC_BM, keep) + oz_term(__uint_as_float(vr[jj]), wk), keep);
                st_keep(pi + (size_t)jj * TC_BM,
                        ld_keep(pi + (size_t)jj * TC_BM, keep) + oz_term(__uint_as_float(vi[jj]), wk), keep);
              }
            }
          }
        }
        gi++;
        first = false;
      }
     }
    }
  }

  // ---- teardown: every role has finished or given up ----
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    if (lane == 0) bar_wait(&drain_bar, 0u, &abort_sh, nullptr, true);  // the MMAs this thread issued
    __syncwarp();
  }
  if (warp == 0 && lane == 0 && abort_sh) {
    // copies still in flight after a give-up land before shared memory is released
    const int n = issued_sh;
    for (int k = max(0, n - S_); k < n; k++)
      bar_wait(&full_bar[k % S_], (uint32_t)(k / S_) & 1u, &abort_sh, nullptr, true);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tc_dealloc(tmem, Cfg::kTmemCols);
  }
}

// Sum of the pair groups' partial results of a split product, and the
// epilogue C = alpha 2^(a_i + b_j) sum + beta D (+ I): one thread per entry,
// neighbouring threads on neighbouring rows.
template <int BN>
__global__ void __launch_bounds__(256) oz_reduce_kernel(const __grid_constant__ TcArgs a) {
  const GemmDesc &g = a.g;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)g.M * g.N;
  if (id >= per * g.batch) return;
  const int b = (int)(id / per);
  const long long r = id % per;
  const int j = (int)(r / g.M), i = (int)(r % g.M);
  const int tm = i / TC_BM, il = i % TC_BM, tn = j / BN, jl = j % BN;
  double vr = 0.0, vi = 0.0;
  for (int q = 0; q < a.gp; q++) {
    const double *slab = a.acc + ((((size_t)q * g.batch + b) * a.tm + tm) * a.tn + tn) * TcCfg<BN>::kAcc;
    vr += slab[(size_t)jl * TC_BM + il];
    vi += slab[(size_t)(BN + jl) * TC_BM + il];
  }
  const int sh = __ldg(a.ea + (size_t)b * a.Mp + i) + __ldg(a.eb + (size_t)b * a.Np + j);
  vr = ldexp(vr, sh);
  vi = ldexp(vi, sh);
  double outr = g.alpha.x * vr - g.alpha.y * vi;
  double outi = g.alpha.x * vi + g.alpha.y * vr;
  if (g.D.ptr) {
    const long long od = oz_off(g.D, b, i, j);
    double2 d;
    if (g.D.f32) {
      const float2 f = ((const float2 *)g.D.ptr)[od];
      d = make_double2(f.x, f.y);
    } else {
      d = ((const double2 *)g.D.ptr)[od];
    }
    outr += g.beta.x * d.x - g.beta.y * d.y;
    outi += g.beta.x * d.y + g.beta.y * d.x;
  }
  if (g.addI && i == j) outr += 1.0;
  const long long oc = oz_off(g.C, b, i, j);
  if (g.C.f32)
    ((float2 *)g.C.ptr)[oc] = make_float2((float)outr, (float)outi);
  else
    ((double2 *)g.C.ptr)[oc] = make_double2(outr, outi);
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependence on libcuda)
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  });
  return fn;
}

// Tensor map of `planes` digit planes of rows x Kp bf16 (K-major, k
// contiguous), copied as boxes of 64 k x box_rows rows into 128-byte-swizzled
// shared memory.
bool digit_map(CUtensorMap *m, const void *base, int Kp, int rows, long long planes, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * (cuuint64_t)rows};
  const cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

thread_local OzTimer *g_oz_timer = nullptr;

template <int BN>
cudaError_t launch_product(const OzLayout &L, const TcArgs &a, const void *Ad, const void *Bd, cudaStream_t st) {
  const GemmDesc &g = a.g;
  CUtensorMap mA, mB;
  if (!digit_map(&mA, Ad, L.Kp, L.Mp, (long long)g.batch * L.S * 2, TC_BM) ||
      !digit_map(&mB, Bd, L.Kp, L.Np, (long long)g.batch * L.S * 2, BN))
    return cudaErrorInvalidValue;
  cudaError_t err =
      cudaFuncSetAttribute(oz_tc_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcCfg<BN>::kSmem);
  if (err != cudaSuccess) return err;
  OzTimer *tm = g_oz_timer;
  bool timed = tm && tm->n < tm->cap;
  for (int q = 0; timed && q < 2; q++)
    if (!tm->ev[2 * tm->n + q] && cudaEventCreate(&tm->ev[2 * tm->n + q]) != cudaSuccess) {
      cudaGetLastError();
      timed = false;
    }
  if (timed) cudaEventRecord(tm->ev[2 * tm->n], st);
  oz_tc_kernel<BN><<<L.ctas, TC_THREADS, TcCfg<BN>::kSmem, st>>>(mA, mB, a);
  err = cudaGetLastError();
  if (timed) {
    cudaEventRecord(tm->ev[2 * tm->n + 1], st);
    tm->flops[tm->n] = 8.0 * L.npairs * g.M * g.N * g.K * g.batch;  // slice pairs x 4 real products
    tm->n++;
  }
  if (err != cudaSuccess || L.gp == 1) return err;
  const long long n = (long long)g.M * g.N * g.batch;
  oz_reduce_kernel<BN><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

// One thread waits, with the pipeline's bounded wait, on an mbarrier that
// nothing arrives at: phase 0 of a barrier initialised for one arrival
// completes only with that arrival.  The wait gives up after limit_ns and
// records a timeout in the status word; the kernel then returns.
__global__ void wait_check_kernel(unsigned *status, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int abort_sh;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  abort_sh = 0;
  fence_mbar_init();
  bar_wait(&bar, 0u, &abort_sh, status, false, limit_ns);
}

}  // namespace

void oz_set_timer(OzTimer *t) { g_oz_timer = t; }

int oz_launches(const GemmDesc &g, bool reuse_a) {
  return (oz_layout(g, num_sms()).gp > 1 ? 5 : 4) - (reuse_a ? 2 : 0);
}

bool oz_eligible(const GemmDesc &g) {
  // worth the split passes only for sizeable products whose tiles are mostly
  // live (M padded to 128, N to 64 or 128)
  return g.K >= 64 && g.M >= 96 && g.N >= 48 && g.batch <= 65535 &&
         (double)g.M * g.N * g.K * g.batch >= (double)(1 << 26);
}

size_t oz_workspace_bytes(const GemmDesc &g) { return oz_layout(g, num_sms()).total; }

cudaError_t launch_oz_split_a(const GemmDesc &g, void *ws, size_t ws_bytes, cudaStream_t st) {
  if (g.batch <= 0 || g.M <= 0 || g.N <= 0) return cudaSuccess;
  const OzLayout L = oz_layout(g, num_sms());
  if (!ws || ws_bytes < L.total || g.batch > 65535 || ((uintptr_t)ws & 255)) return cudaErrorInvalidValue;
  char *w = (char *)ws;
  int *ea = (int *)(w + L.ea_off);
  oz_expo_a_kernel<<<dim3(L.Mp / 32, g.batch), 256, 0, st>>>(g, L.Mp, ea);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const dim3 ga(L.Mp / OZA_R, L.Kp / OZA_K, g.batch);
  __nv_bfloat16 *Ad = (__nv_bfloat16 *)(w + L.a_off);
  if (L.S == OZ_S32)
    oz_split_a_kernel<OZ_S32><<<ga, 256, 0, st>>>(g, L.Mp, L.Kp, Ad, ea);
  else
    oz_split_a_kernel<OZ_S><<<ga, 256, 0, st>>>(g, L.Mp, L.Kp, Ad, ea);
  return cudaGetLastError();
}

cudaError_t launch_gemm_oz(const GemmDesc &g, void *ws, size_t ws_bytes, cudaStream_t st, unsigned *status,
                           bool reuse_a) {
  if (g.batch <= 0 || g.M <= 0 || g.N <= 0) return cudaSuccess;
  const OzLayout L = oz_layout(g, num_sms());
  if (!ws || ws_bytes < L.total || g.batch > 65535 || ((uintptr_t)ws & 255)) return cudaErrorInvalidValue;
  char *w = (char *)ws;
  __nv_bfloat16 *Ad = (__nv_bfloat16 *)(w + L.a_off), *Bd = (__nv_bfloat16 *)(w + L.b_off);
  int *ea = (int *)(w + L.ea_off), *eb = (int *)(w + L.eb_off);
  cudaError_t err = cudaSuccess;
  const bool s32 = L.S == OZ_S32;
  if (!reuse_a) {
    oz_expo_a_kernel<<<dim3(L.Mp / 32, g.batch), 256, 0, st>>>(g, L.Mp, ea);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const dim3 ga(L.Mp / OZA_R, L.Kp / OZA_K, g.batch);
    if (s32)
      oz_split_a_kernel<OZ_S32><<<ga, 256, 0, st>>>(g, L.Mp, L.Kp, Ad, ea);
    else
      oz_split_a_kernel<OZ_S><<<ga, 256, 0, st>>>(g, L.Mp, L.Kp, Ad, ea);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  const dim3 gb((L.Np + 7) / 8, g.batch);
  if (s32)
    oz_split_b_kernel<OZ_S32><<<gb, 256, 0, st>>>(g, L.Np, L.Kp, Bd, eb);
  else
    oz_split_b_kernel<OZ_S><<<gb, 256, 0, st>>>(g, L.Np, L.Kp, Bd, eb);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  TcArgs a;
  a.g = g;
  a.Mp = L.Mp;
  a.Np = L.Np;
  a.Kp = L.Kp;
  a.S = L.S;
  a.npairs = L.npairs;
  a.tm = L.tm;
  a.tn = L.tn;
  a.gp = L.gp;
  a.units = L.units;
  a.persistent = L.persistent ? 1 : 0;
  a.acc = (double *)(w + L.acc_off);
  a.ea = ea;
  a.eb = eb;
  a.status = status;
  return L.bn == 64 ? launch_product<64>(L, a, Ad, Bd, st) : launch_product<128>(L, a, Ad, Bd, st);
}

cudaError_t launch_wait_check(unsigned *status, int limit_ms, cudaStream_t st) {
  if (!status || limit_ms < 1) return cudaErrorInvalidValue;
  wait_check_kernel<<<1, 32, 0, st>>>(status, (uint64_t)limit_ms * 1000000ull);
  return cudaGetLastError();
}

}  // namespace hps
