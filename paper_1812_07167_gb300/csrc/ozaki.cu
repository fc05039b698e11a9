// Complex128 GEMM emulated on the bf16 tensor cores (Ozaki scheme).
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
// bf16.
//
// Products.  The slice pairs (s, t) with s + t < S are taken group by group
// of equal shift e = s + t, whose products all carry the weight 2^{-6(e+2)}.
// The tensor core multiplies the digit matrices with FP32 accumulation; a
// digit product is at most 2^10 in magnitude, a complex combination (ar br -
// ai bi or ar bi + ai br) at most 2^11, and a group has at most S = 9 pairs:
// over a K chunk of OZ_KC = 896 every partial sum of a whole group is an
// integer below 9 * 896 * 2^11 < 2^24, so the FP32 accumulation is exact.
// After each group (and K chunk) the sum is added, times its weight, into
// complex128 accumulators: 9 FP64 updates an output for K <= 896, which
// keeps the FP64 pipe (2 operations per clock per SM on this part) well
// below the tensor-core work.  Pairs with s + t >= S are dropped: with the
// remainders they bound the error of every term by ~2^{-6S} max|A_i.|
// max|B_.j| (2^-54 for S = 9), the size of a complex128 rounding.  The
// result is scaled back by 2^{a_i + b_j} and combined as C = alpha AB +
// beta D (+ I).
//
// Kernels: the split of A (row exponents, then the digits k-major), the
// split of B (a warp per column, digits k fastest), and the product kernel:
// 64 x 64 output tiles, 4 warps of 32 x 32, mma.sync m16n8k16 bf16 with FP32
// accumulation on fragments read by ldmatrix (transposing for the k-major A
// tiles), operand tiles staged through shared memory by cp.async with double
// buffering, the complex128 accumulators in shared memory.  Products with few
// output tiles split the slice pairs over several CTAs a tile and sum the
// partial results in a last pass.
#include <cuda_bf16.h>

#include <algorithm>

#include "hps_internal.h"

namespace hps {

namespace {

constexpr int OZ_S = 9;              // slices per operand (6 bits each)
constexpr int OZ_BM = 64, OZ_BN = 64, OZ_BK = 32;
constexpr int OZ_KC = 896;           // K per exact FP32 accumulation of a shift group
constexpr int OZ_LDS = OZ_BK + 8;    // shared row length in bf16: conflict-free fragment loads

constexpr int OZ_PAIRS = OZ_S * (OZ_S + 1) / 2;  // slice pairs with s + t < S

struct OzLayout {
  int Mp, Np, Kp;         // padded sizes (multiples of 64, 64, 32)
  int gp;                 // CTAs per output tile, each summing a share of the slice pairs
  size_t a_off, b_off;    // byte offsets of the digit planes
  size_t ea_off, eb_off;  // byte offsets of the row / column exponents
  size_t part_off;        // gp > 1: per-group complex128 partial sums [gp][batch][Mp][Np]
  size_t total;
};

inline size_t oz_align(size_t x) { return (x + 255) & ~(size_t)255; }

OzLayout oz_layout(const GemmDesc &g) {
  OzLayout L;
  L.Mp = (g.M + OZ_BM - 1) / OZ_BM * OZ_BM;
  L.Np = (g.N + OZ_BN - 1) / OZ_BN * OZ_BN;
  L.Kp = (g.K + OZ_BK - 1) / OZ_BK * OZ_BK;
  const size_t B = (size_t)g.batch;
  size_t o = 0;
  L.a_off = o;
  o = oz_align(o + B * OZ_S * 2 * (size_t)L.Mp * L.Kp * sizeof(__nv_bfloat16));
  L.b_off = o;
  o = oz_align(o + B * OZ_S * 2 * (size_t)L.Np * L.Kp * sizeof(__nv_bfloat16));
  L.ea_off = o;
  o = oz_align(o + B * (size_t)L.Mp * sizeof(int));
  L.eb_off = o;
  o = oz_align(o + B * (size_t)L.Np * sizeof(int));
  // products with few output tiles split the slice pairs over several CTAs
  // a tile, aiming at two waves of one CTA on each SM
  const long long tiles = (long long)(L.Mp / OZ_BM) * (L.Np / OZ_BN) * g.batch;
  L.gp = (int)std::min<long long>(12, std::max<long long>(1, (2 * 152 + tiles - 1) / tiles));
  while (L.gp > 1 && (long long)g.batch * L.gp > 65535) L.gp--;
  L.part_off = o;
  if (L.gp > 1) o = oz_align(o + (size_t)L.gp * B * L.Mp * L.Np * 2 * sizeof(double));
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
__device__ __forceinline__ long long oz_fixed(double v, int sh) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7ff);
  const unsigned long long M = (b & 0xfffffffffffffull) | (E ? (1ull << 52) : 0ull);
  const int t = (E ? E : 1) - 1075 + 6 * OZ_S - sh;  // D = round(M 2^t)
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
__device__ __forceinline__ void oz_digits(long long D, int (&d)[OZ_S]) {
#pragma unroll
  for (int s = OZ_S - 1; s > 0; s--) {
    const int v = (int)((D + 32) & 63) - 32;
    d[s] = v;
    D = (D - v) >> 6;
  }
  d[0] = (int)D;
}

// Digits of B, a warp per column, lanes over k (neighbouring k are
// neighbouring in the column-major operands): the column's exponent, then its
// digits ([column][k], k contiguous).  Padding columns and k get zeros.
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
  __nv_bfloat16 *base = digits + (size_t)b * OZ_S * 2 * plane + (size_t)j * Kp;
  for (int k = lane; k < Kp; k += 32) {
    double2 v = make_double2(0.0, 0.0);
    if (live && k < g.K) v = oz_ldb(g, b, k, j);
    int dr[OZ_S], di[OZ_S];
    oz_digits(oz_fixed(v.x, sh), dr);
    oz_digits(oz_fixed(v.y, sh), di);
#pragma unroll
    for (int q = 0; q < OZ_S; q++) {
      base[(size_t)(2 * q) * plane + k] = __int2bfloat16_rn(dr[q]);
      base[(size_t)(2 * q + 1) * plane + k] = __int2bfloat16_rn(di[q]);
    }
  }
}

// Digits of A in two passes, both reading A with neighbouring threads on
// neighbouring rows (coalesced for the column-major operands).  Pass 1: the
// exponent of each row (32 rows a block, 8 threads a row over k, combined
// in shared memory).  Pass 2: one thread per element, digits written k-major
// ([k][row], rows contiguous).  Padding rows and k get zeros.
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

__global__ void __launch_bounds__(256) oz_split_a_kernel(const __grid_constant__ GemmDesc g, int Mp, int Kp,
                                                         __nv_bfloat16 *digits, const int *expo) {
  const int i = blockIdx.x * 64 + (threadIdx.x & 63);
  const int k = blockIdx.y * 4 + (threadIdx.x >> 6);
  const int b = blockIdx.z;
  if (i >= Mp || k >= Kp) return;
  double2 v = make_double2(0.0, 0.0);
  if (i < g.M && k < g.K) v = oz_lda(g, b, i, k);
  const int sh = expo[(size_t)b * Mp + i];
  const size_t plane = (size_t)Mp * Kp;
  __nv_bfloat16 *base = digits + (size_t)b * OZ_S * 2 * plane + (size_t)k * Mp + i;
  int dr[OZ_S], di[OZ_S];
  oz_digits(oz_fixed(v.x, sh), dr);
  oz_digits(oz_fixed(v.y, sh), di);
#pragma unroll
  for (int q = 0; q < OZ_S; q++) {
    base[(size_t)(2 * q) * plane] = __int2bfloat16_rn(dr[q]);
    base[(size_t)(2 * q + 1) * plane] = __int2bfloat16_rn(di[q]);
  }
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// four 8 x 8 bf16 matrices from shared memory (lane l gives the address of
// row l % 8 of matrix l / 8); register j holds matrix j's row (lane / 4),
// elements 2 (lane % 4) and 2 (lane % 4) + 1
__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const __nv_bfloat16 *p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const __nv_bfloat16 *p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct OzArgs {
  GemmDesc g;
  int Mp, Np, Kp;
  int gp;        // pair groups (CTAs a tile)
  double *part;  // gp > 1: partial sums [gp][batch][Mp][Np][2]
  const __nv_bfloat16 *A;  // [batch][S][2][Kp][Mp] (k-major)
  const __nv_bfloat16 *B;  // [batch][S][2][Np][Kp]
  const int *ea;           // [batch][Mp]
  const int *eb;           // [batch][Np]
};

constexpr int OZ_THREADS = 128;  // 4 warps of 32 x 32 outputs
constexpr int OZ_NACC = 64;      // complex128 outputs x (re, im) per thread
constexpr int OZ_STAGES = 2;     // cp.async pipeline depth
constexpr int OZ_LDA = OZ_BM + 8;  // shared A row (one k) in bf16: conflict-free transposing loads
typedef __nv_bfloat16 TileA[2][OZ_BK][OZ_LDA];  // [re, im][k][row]
typedef __nv_bfloat16 TileB[2][OZ_BN][OZ_LDS];  // [re, im][column][k]
// shared memory: OZ_STAGES stages of A and B digit tiles, then the
// complex128 accumulators ([element][thread]: conflict-free)
constexpr size_t OZ_STAGE = sizeof(TileA) + sizeof(TileB);
constexpr size_t OZ_SMEM = OZ_STAGES * OZ_STAGE + sizeof(double) * OZ_NACC * OZ_THREADS;

__device__ __forceinline__ void cp_async_wait_stages() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(OZ_STAGES - 1) : "memory");
}

__global__ void __launch_bounds__(OZ_THREADS, 2) oz_gemm_kernel(const __grid_constant__ OzArgs a) {
  extern __shared__ __align__(16) unsigned char oz_smem[];
  double *acc = (double *)(oz_smem + OZ_STAGES * OZ_STAGE);
  const GemmDesc &g = a.g;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, grp = lane >> 2, tig = lane & 3;
  const int b = blockIdx.z / a.gp, bm = blockIdx.y * OZ_BM, bn = blockIdx.x * OZ_BN;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  const size_t aplane = (size_t)a.Mp * a.Kp, bplane = (size_t)a.Np * a.Kp;
  const __nv_bfloat16 *Ab = a.A + (size_t)b * OZ_S * 2 * aplane;
  const __nv_bfloat16 *Bb = a.B + (size_t)b * OZ_S * 2 * bplane;
  const int nkb = a.Kp / OZ_BK;
  constexpr int CKB = OZ_KC / OZ_BK;  // k-blocks of a chunk
  auto tileA = [&](int st) -> TileA & { return *(TileA *)(oz_smem + st * OZ_STAGE); };
  auto tileB = [&](int st) -> TileB & { return *(TileB *)(oz_smem + st * OZ_STAGE + sizeof(TileA)); };

  for (int e = 0; e < OZ_NACC; e++) acc[e * OZ_THREADS + tid] = 0.0;

  // this CTA's slice pairs: a contiguous share of the list ordered by shift
  // e = s + t, then s: (0,0), (0,1), (1,0), (0,2), ...
  const int grp_id = blockIdx.z % a.gp;
  const int p0 = grp_id * OZ_PAIRS / a.gp, p1 = (grp_id + 1) * OZ_PAIRS / a.gp;
  struct Pos {
    int c, p, e, s, kb;  // K chunk, pair index, its shift and A slice, k-block
  };
  auto set_pair = [&](Pos &q, int p) {
    q.p = p;
    q.e = 0;
    while (p > q.e) {
      p -= q.e + 1;
      q.e++;
    }
    q.s = p;
  };
  auto chunk_end = [&](int c) { return min(nkb, (c + 1) * CKB); };
  auto advance = [&](Pos &q) {
    if (++q.kb < chunk_end(q.c)) return;
    if (q.p + 1 < p1) {
      q.p++;
      if (++q.s > q.e) {
        q.e++;
        q.s = 0;
      }
      q.kb = q.c * CKB;
    } else {
      q.c++;
      set_pair(q, p0);
      q.kb = q.c * CKB;
    }
  };
  // one pipeline over (chunk, pair, k-block): the next tiles are in flight
  // while the current ones are multiplied
  const int nit = (p1 - p0) * nkb;  // the chunks together cover every k-block once per pair
  auto load = [&](int st, const Pos &q) {
    const __nv_bfloat16 *Ap = Ab + (size_t)(2 * q.s) * aplane;  // real digits; imaginary at + aplane
    const __nv_bfloat16 *Bp = Bb + (size_t)(2 * (q.e - q.s)) * bplane;
    TileA &TA = tileA(st);
    TileB &TB = tileB(st);
    const size_t k0 = (size_t)q.kb * OZ_BK;
#pragma unroll
    for (int c = tid; c < 2 * OZ_BK * (OZ_BM / 8); c += OZ_THREADS) {
      const int ri = c / (OZ_BK * (OZ_BM / 8)), kr = (c / (OZ_BM / 8)) % OZ_BK, ch = c % (OZ_BM / 8);
      cp_async16(&TA[ri][kr][ch * 8], Ap + ri * aplane + (k0 + kr) * (size_t)a.Mp + bm + ch * 8);
    }
#pragma unroll
    for (int c = tid; c < 2 * OZ_BN * 4; c += OZ_THREADS) {
      const int ri = c / (OZ_BN * 4), row = (c >> 2) % OZ_BN, ch = c & 3;
      cp_async16(&TB[ri][row][ch * 8], Bp + ri * bplane + (size_t)(bn + row) * a.Kp + k0 + ch * 8);
    }
  };
  float cr[2][4][4], ci[2][4][4];
#pragma unroll
  for (int mi = 0; mi < 2; mi++)
#pragma unroll
    for (int ni = 0; ni < 4; ni++)
#pragma unroll
      for (int e = 0; e < 4; e++) cr[mi][ni][e] = ci[mi][ni][e] = 0.f;
  Pos cur;
  cur.c = 0;
  set_pair(cur, p0);
  cur.kb = 0;
  Pos ld = cur;
  for (int st = 0; st < OZ_STAGES - 1; st++) {
    if (st < nit) load(st, ld);
    cp_async_commit();
    advance(ld);
  }
  for (int it = 0; it < nit; it++) {
    if (it + OZ_STAGES - 1 < nit) load((it + OZ_STAGES - 1) % OZ_STAGES, ld);
    cp_async_commit();
    advance(ld);
    cp_async_wait_stages();
    __syncthreads();
    TileA &TA = tileA(it % OZ_STAGES);
    TileB &TB = tileB(it % OZ_STAGES);
#pragma unroll
    for (int kk = 0; kk < OZ_BK; kk += 16) {
      unsigned ar[2][4], ai[2][4], br[2][4], bi[2][4];
#pragma unroll
      for (int mi = 0; mi < 2; mi++) {
        // matrix j = lane / 8 of the fragment: rows (k) kk + 8 (j / 2) + lane % 8,
        // columns (m) wm + 16 mi + 8 (j % 2), read transposed
        const int kr = kk + ((lane >> 4) << 3) + (lane & 7);
        const int mc = wm + mi * 16 + (((lane >> 3) & 1) << 3);
        ldsm_x4_t(ar[mi], &TA[0][kr][mc]);
        ldsm_x4_t(ai[mi], &TA[1][kr][mc]);
      }
#pragma unroll
      for (int nj = 0; nj < 2; nj++) {
        // n8 tiles 2 nj and 2 nj + 1: registers b0, b1 of the first, then of the second
        const int n = wn + nj * 16 + (lane & 7) + ((lane >> 4) & 1) * 8;
        const int col = kk + ((lane >> 3) & 1) * 8;
        ldsm_x4(br[nj], &TB[0][n][col]);
        ldsm_x4(bi[nj], &TB[1][n][col]);
      }
      // the four real products in rounds, so that the two products into one
      // accumulator are 16 independent instructions apart
#pragma unroll
      for (int round = 0; round < 4; round++)
#pragma unroll
        for (int mi = 0; mi < 2; mi++)
#pragma unroll
          for (int ni = 0; ni < 4; ni++) {
            const unsigned b0 = br[ni >> 1][2 * (ni & 1)], b1 = br[ni >> 1][2 * (ni & 1) + 1];
            const unsigned c0 = bi[ni >> 1][2 * (ni & 1)], c1 = bi[ni >> 1][2 * (ni & 1) + 1];
            if (round == 0) mma_bf16(cr[mi][ni], ar[mi], b0, b1);
            if (round == 1) mma_bf16(ci[mi][ni], ar[mi], c0, c1);
            if (round == 2) mma_bf16(cr[mi][ni], ai[mi], c0 ^ 0x80008000u, c1 ^ 0x80008000u);  // - Ai Bi
            if (round == 3) mma_bf16(ci[mi][ni], ai[mi], b0, b1);
          }
    }
    __syncthreads();
    // end of a shift group within this chunk: its sums are exact integers,
    // add them into complex128 with the group's weight
    const bool last_kb = cur.kb + 1 == chunk_end(cur.c);
    const bool group_end = cur.p + 1 == p1 || cur.s == cur.e;
    if (last_kb && group_end) {
      const double scale = ldexp(1.0, -6 * (cur.e + 2));
#pragma unroll
      for (int mi = 0; mi < 2; mi++)
#pragma unroll
        for (int ni = 0; ni < 4; ni++)
#pragma unroll
          for (int e = 0; e < 4; e++) {
            const int idx = ((mi * 4 + ni) * 4 + e) * 2;
            double *pr = acc + idx * OZ_THREADS + tid, *pi = pr + OZ_THREADS;
            *pr = fma((double)cr[mi][ni][e], scale, *pr);
            *pi = fma((double)ci[mi][ni][e], scale, *pi);
            cr[mi][ni][e] = ci[mi][ni][e] = 0.f;
          }
    }
    advance(cur);
  }

  if (a.gp > 1) {
    // partial sums of this pair group; oz_reduce_kernel finishes the tile
#pragma unroll
    for (int mi = 0; mi < 2; mi++)
#pragma unroll
      for (int ni = 0; ni < 4; ni++)
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const int i = bm + wm + mi * 16 + grp + ((e >> 1) << 3);
          const int j = bn + wn + ni * 8 + 2 * tig + (e & 1);
          const int idx = ((mi * 4 + ni) * 4 + e) * 2;
          const size_t o = ((((size_t)grp_id * g.batch + b) * a.Mp + i) * a.Np + j) * 2;
          a.part[o] = acc[idx * OZ_THREADS + tid];
          a.part[o + 1] = acc[(idx + 1) * OZ_THREADS + tid];
        }
    return;
  }

  // epilogue: C = alpha 2^(a_i + b_j) acc + beta D (+ I)
#pragma unroll
  for (int mi = 0; mi < 2; mi++)
#pragma unroll
    for (int ni = 0; ni < 4; ni++)
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int i = bm + wm + mi * 16 + grp + ((e >> 1) << 3);
        const int j = bn + wn + ni * 8 + 2 * tig + (e & 1);
        if (i >= g.M || j >= g.N) continue;
        const int idx = ((mi * 4 + ni) * 4 + e) * 2;
        const int sh = __ldg(a.ea + (size_t)b * a.Mp + i) + __ldg(a.eb + (size_t)b * a.Np + j);
        const double vr = ldexp(acc[idx * OZ_THREADS + tid], sh);
        const double vi = ldexp(acc[(idx + 1) * OZ_THREADS + tid], sh);
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
}

// Sum of the pair groups' partial results of a split product, and the
// epilogue C = alpha 2^(a_i + b_j) sum + beta D (+ I): one thread per entry.
__global__ void __launch_bounds__(256) oz_reduce_kernel(const __grid_constant__ OzArgs a) {
  const GemmDesc &g = a.g;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)g.M * g.N;
  if (id >= per * g.batch) return;
  const int b = (int)(id / per);
  const long long r = id % per;
  const int j = (int)(r / g.M), i = (int)(r % g.M);
  double vr = 0.0, vi = 0.0;
  for (int q = 0; q < a.gp; q++) {
    const size_t o = ((((size_t)q * g.batch + b) * a.Mp + i) * a.Np + j) * 2;
    vr += a.part[o];
    vi += a.part[o + 1];
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

}  // namespace

int oz_launches(const GemmDesc &g) { return oz_layout(g).gp > 1 ? 5 : 4; }

bool oz_eligible(const GemmDesc &g) {
  // worth the split passes only for sizeable products; complex128 arithmetic only
  // (measured: from ~2^26 complex multiply-adds a launch the emulation beats
  // the FP64 pipes; 2^23 per product is too small for the fixed costs)
  return !g.cf32 && g.K >= 64 && g.M >= 32 && g.N >= 32 && g.batch <= 65535 &&
         (double)g.M * g.N * g.K * g.batch >= (double)(1 << 26);
}

size_t oz_workspace_bytes(const GemmDesc &g) { return oz_layout(g).total; }

cudaError_t launch_gemm_oz(const GemmDesc &g, void *ws, size_t ws_bytes, cudaStream_t st) {
  if (g.batch <= 0 || g.M <= 0 || g.N <= 0) return cudaSuccess;
  const OzLayout L = oz_layout(g);
  if (!ws || ws_bytes < L.total || g.batch > 65535) return cudaErrorInvalidValue;
  char *w = (char *)ws;
  __nv_bfloat16 *Ad = (__nv_bfloat16 *)(w + L.a_off), *Bd = (__nv_bfloat16 *)(w + L.b_off);
  int *ea = (int *)(w + L.ea_off), *eb = (int *)(w + L.eb_off);
  oz_expo_a_kernel<<<dim3(L.Mp / 32, g.batch), 256, 0, st>>>(g, L.Mp, ea);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  oz_split_a_kernel<<<dim3(L.Mp / 64, L.Kp / 4, g.batch), 256, 0, st>>>(g, L.Mp, L.Kp, Ad, ea);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  oz_split_b_kernel<<<dim3((L.Np + 7) / 8, g.batch), 256, 0, st>>>(g, L.Np, L.Kp, Bd, eb);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  OzArgs a;
  a.g = g;
  a.Mp = L.Mp;
  a.Np = L.Np;
  a.Kp = L.Kp;
  a.A = Ad;
  a.B = Bd;
  a.ea = ea;
  a.eb = eb;
  a.gp = L.gp;
  a.part = L.gp > 1 ? (double *)(w + L.part_off) : nullptr;
  err = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM);
  if (err != cudaSuccess) return err;
  oz_gemm_kernel<<<dim3(L.Np / OZ_BN, L.Mp / OZ_BM, g.batch * L.gp), OZ_THREADS, OZ_SMEM, st>>>(a);
  err = cudaGetLastError();
  if (err != cudaSuccess || L.gp == 1) return err;
  const long long n = (long long)g.M * g.N * g.batch;
  oz_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace hps
