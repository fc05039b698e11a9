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
//     x = sum_{s < S} d_s 2^{-8(s+1)} + r,   d_s integers, |d_s| <= 128,
// taking d_s = rint(256 x_s), x_{s+1} = 256 x_s - d_s (every step exact in
// FP64), so |r| <= 2^{-8S-1}.  The digits are exact in bf16.
//
// Products.  For a slice pair (s, t) the tensor core multiplies the digit
// matrices with FP32 accumulation.  A digit product is at most 2^14 in
// magnitude, a complex combination (ar br - ai bi or ar bi + ai br) at most
// 2^15, and a sum over OZ_KC = 256 of them at most 2^23: every partial sum
// is an integer below 2^24, so the FP32 accumulation is exact.  After each
// chunk of OZ_KC the chunk sum is added, times 2^{-8(s+t+2)}, into complex128
// accumulators.  Pairs with s + t >= S are dropped: with the remainders they
// bound the error of every term by ~2^{-8S} max|A_i.| max|B_.j| (2^-56 for
// S = 7), below the rounding of a complex128 dot product.  The result is
// scaled back by 2^{a_i + b_j} and combined as C = alpha AB + beta D (+ I).
//
// Kernels: one split kernel per operand (a warp per row of A / column of B,
// writing bf16 digit planes laid out as the tensor-core fragments want them:
// k fastest), and the product kernel: 64 x 64 output tiles, 8 warps of
// 32 x 16, mma.sync m16n8k16 bf16 with FP32 accumulation, operand tiles
// staged through shared memory by cp.async with double buffering.
#include <cuda_bf16.h>

#include "hps_internal.h"

namespace hps {

namespace {

constexpr int OZ_S = 7;              // slices per operand
constexpr int OZ_BM = 64, OZ_BN = 64, OZ_BK = 32;
constexpr int OZ_KC = 256;           // K per exact FP32 accumulation
constexpr int OZ_LDS = OZ_BK + 8;    // shared row length in bf16: conflict-free fragment loads

struct OzLayout {
  int Mp, Np, Kp;         // padded sizes (multiples of 64, 64, 32)
  size_t a_off, b_off;    // byte offsets of the digit planes
  size_t ea_off, eb_off;  // byte offsets of the row / column exponents
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

// Digits of one row of A (isb = false) or one column of B (isb = true): a
// warp per line, lanes over k.  Padding rows / columns / k get zeros.
template <bool isb>
__global__ void __launch_bounds__(256) oz_split_kernel(const __grid_constant__ GemmDesc g, int Lp, int Kp,
                                                       __nv_bfloat16 *digits, int *expo) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int line = blockIdx.x * 8 + warp;  // row of A or column of B
  const int b = blockIdx.y;
  if (line >= Lp) return;
  const int nlines = isb ? g.N : g.M;
  const bool live = line < nlines;
  double mx = 0.0;
  if (live)
    for (int k = lane; k < g.K; k += 32) {
      const double2 v = isb ? oz_ldb(g, b, k, line) : oz_lda(g, b, line, k);
      mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
    }
  for (int off = 16; off; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);  // mx = f 2^e, f in [1/2, 1): mx 2^-(e+1) in [1/4, 1/2)
  const int sh = mx > 0.0 ? e + 1 : 0;
  if (lane == 0) expo[(size_t)b * Lp + line] = sh;
  const size_t plane = (size_t)Lp * Kp;
  __nv_bfloat16 *base = digits + (size_t)b * OZ_S * 2 * plane + (size_t)line * Kp;
  for (int k = lane; k < Kp; k += 32) {
    double2 v = make_double2(0.0, 0.0);
    if (live && k < g.K) v = isb ? oz_ldb(g, b, k, line) : oz_lda(g, b, line, k);
    double xr = ldexp(v.x, -sh), xi = ldexp(v.y, -sh);
#pragma unroll
    for (int s = 0; s < OZ_S; s++) {
      xr *= 256.0;
      xi *= 256.0;
      const double dr = rint(xr), di = rint(xi);
      xr -= dr;
      xi -= di;
      base[(size_t)(2 * s) * plane + k] = __float2bfloat16_rn((float)dr);
      base[(size_t)(2 * s + 1) * plane + k] = __float2bfloat16_rn((float)di);
    }
  }
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ unsigned lds32(const __nv_bfloat16 *p) { return *(const unsigned *)p; }

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct OzArgs {
  GemmDesc g;
  int Mp, Np, Kp;
  const __nv_bfloat16 *A;  // [batch][S][2][Mp][Kp]
  const __nv_bfloat16 *B;  // [batch][S][2][Np][Kp]
  const int *ea;           // [batch][Mp]
  const int *eb;           // [batch][Np]
};

__global__ void __launch_bounds__(256) oz_gemm_kernel(const __grid_constant__ OzArgs a) {
  __shared__ __align__(16) __nv_bfloat16 sA[2][2][OZ_BM][OZ_LDS];  // [stage][re, im][row][k]
  __shared__ __align__(16) __nv_bfloat16 sB[2][2][OZ_BN][OZ_LDS];  // [stage][re, im][col][k]
  const GemmDesc &g = a.g;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, grp = lane >> 2, tig = lane & 3;
  const int b = blockIdx.z, bm = blockIdx.y * OZ_BM, bn = blockIdx.x * OZ_BN;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 16;
  const size_t aplane = (size_t)a.Mp * a.Kp, bplane = (size_t)a.Np * a.Kp;
  const __nv_bfloat16 *Ab = a.A + (size_t)b * OZ_S * 2 * aplane;
  const __nv_bfloat16 *Bb = a.B + (size_t)b * OZ_S * 2 * bplane;
  const int nkb = a.Kp / OZ_BK;

  double accr[2][2][4], acci[2][2][4];
#pragma unroll
  for (int mi = 0; mi < 2; mi++)
#pragma unroll
    for (int ni = 0; ni < 2; ni++)
#pragma unroll
      for (int e = 0; e < 4; e++) accr[mi][ni][e] = acci[mi][ni][e] = 0.0;

  for (int s = 0; s < OZ_S; s++) {
    for (int t = 0; s + t < OZ_S; t++) {
      const __nv_bfloat16 *Ap = Ab + (size_t)(2 * s) * aplane;  // real digits; imaginary at + aplane
      const __nv_bfloat16 *Bp = Bb + (size_t)(2 * t) * bplane;
      const double scale = ldexp(1.0, -8 * (s + t + 2));
      float cr[2][2][4], ci[2][2][4];
#pragma unroll
      for (int mi = 0; mi < 2; mi++)
#pragma unroll
        for (int ni = 0; ni < 2; ni++)
#pragma unroll
          for (int e = 0; e < 4; e++) cr[mi][ni][e] = ci[mi][ni][e] = 0.f;

      // stage loader: 2 x 64 rows x 4 chunks of 16 B for A, the same for B
      auto load = [&](int st, int kb) {
        for (int q = tid; q < 1024; q += 256) {
          const int rem = q & 511, ri = rem >> 8, row = (rem >> 2) & 63, ch = rem & 3;
          const size_t koff = (size_t)kb * OZ_BK + ch * 8;
          if (q < 512)
            cp_async16(&sA[st][ri][row][ch * 8], Ap + ri * aplane + (size_t)(bm + row) * a.Kp + koff);
          else
            cp_async16(&sB[st][ri][row][ch * 8], Bp + ri * bplane + (size_t)(bn + row) * a.Kp + koff);
        }
      };
      load(0, 0);
      cp_async_commit();
      for (int kb = 0; kb < nkb; kb++) {
        if (kb + 1 < nkb) load((kb + 1) & 1, kb + 1);
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const int st = kb & 1;
#pragma unroll
        for (int kk = 0; kk < OZ_BK; kk += 16) {
          unsigned ar[2][4], ai[2][4], br[2][2], bi[2][2], nbi[2][2];
#pragma unroll
          for (int mi = 0; mi < 2; mi++) {
            const int r0 = wm + mi * 16 + grp;
            ar[mi][0] = lds32(&sA[st][0][r0][kk + 2 * tig]);
            ar[mi][1] = lds32(&sA[st][0][r0 + 8][kk + 2 * tig]);
            ar[mi][2] = lds32(&sA[st][0][r0][kk + 8 + 2 * tig]);
            ar[mi][3] = lds32(&sA[st][0][r0 + 8][kk + 8 + 2 * tig]);
            ai[mi][0] = lds32(&sA[st][1][r0][kk + 2 * tig]);
            ai[mi][1] = lds32(&sA[st][1][r0 + 8][kk + 2 * tig]);
            ai[mi][2] = lds32(&sA[st][1][r0][kk + 8 + 2 * tig]);
            ai[mi][3] = lds32(&sA[st][1][r0 + 8][kk + 8 + 2 * tig]);
          }
#pragma unroll
          for (int ni = 0; ni < 2; ni++) {
            const int c0 = wn + ni * 8 + grp;
            br[ni][0] = lds32(&sB[st][0][c0][kk + 2 * tig]);
            br[ni][1] = lds32(&sB[st][0][c0][kk + 8 + 2 * tig]);
            bi[ni][0] = lds32(&sB[st][1][c0][kk + 2 * tig]);
            bi[ni][1] = lds32(&sB[st][1][c0][kk + 8 + 2 * tig]);
            nbi[ni][0] = bi[ni][0] ^ 0x80008000u;  // -Bi: flip both bf16 signs
            nbi[ni][1] = bi[ni][1] ^ 0x80008000u;
          }
#pragma unroll
          for (int mi = 0; mi < 2; mi++)
#pragma unroll
            for (int ni = 0; ni < 2; ni++) {
              mma_bf16(cr[mi][ni], ar[mi], br[ni][0], br[ni][1]);
              mma_bf16(cr[mi][ni], ai[mi], nbi[ni][0], nbi[ni][1]);
              mma_bf16(ci[mi][ni], ar[mi], bi[ni][0], bi[ni][1]);
              mma_bf16(ci[mi][ni], ai[mi], br[ni][0], br[ni][1]);
            }
        }
        __syncthreads();
        if (((kb + 1) * OZ_BK) % OZ_KC == 0 || kb + 1 == nkb) {
          // the chunk's sums are exact integers: add them into complex128
#pragma unroll
          for (int mi = 0; mi < 2; mi++)
#pragma unroll
            for (int ni = 0; ni < 2; ni++)
#pragma unroll
              for (int e = 0; e < 4; e++) {
                accr[mi][ni][e] = fma((double)cr[mi][ni][e], scale, accr[mi][ni][e]);
                acci[mi][ni][e] = fma((double)ci[mi][ni][e], scale, acci[mi][ni][e]);
                cr[mi][ni][e] = ci[mi][ni][e] = 0.f;
              }
        }
      }
    }
  }

  // epilogue: C = alpha 2^(a_i + b_j) acc + beta D (+ I)
#pragma unroll
  for (int mi = 0; mi < 2; mi++)
#pragma unroll
    for (int ni = 0; ni < 2; ni++)
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int i = bm + wm + mi * 16 + grp + ((e >> 1) << 3);
        const int j = bn + wn + ni * 8 + 2 * tig + (e & 1);
        if (i >= g.M || j >= g.N) continue;
        const int sh = __ldg(a.ea + (size_t)b * a.Mp + i) + __ldg(a.eb + (size_t)b * a.Np + j);
        const double vr = ldexp(accr[mi][ni][e], sh), vi = ldexp(acci[mi][ni][e], sh);
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

}  // namespace

bool oz_eligible(const GemmDesc &g) {
  // worth the split passes only for sizeable products; complex128 arithmetic only
  return !g.cf32 && g.K >= 64 && g.M >= 32 && g.N >= 32 && g.batch <= 65535 &&
         (double)g.M * g.N * g.K * g.batch >= (double)(1 << 24);
}

size_t oz_workspace_bytes(const GemmDesc &g) { return oz_layout(g).total; }

cudaError_t launch_gemm_oz(const GemmDesc &g, void *ws, size_t ws_bytes, cudaStream_t st) {
  if (g.batch <= 0 || g.M <= 0 || g.N <= 0) return cudaSuccess;
  const OzLayout L = oz_layout(g);
  if (!ws || ws_bytes < L.total || g.batch > 65535) return cudaErrorInvalidValue;
  char *w = (char *)ws;
  __nv_bfloat16 *Ad = (__nv_bfloat16 *)(w + L.a_off), *Bd = (__nv_bfloat16 *)(w + L.b_off);
  int *ea = (int *)(w + L.ea_off), *eb = (int *)(w + L.eb_off);
  oz_split_kernel<false><<<dim3((L.Mp + 7) / 8, g.batch), 256, 0, st>>>(g, L.Mp, L.Kp, Ad, ea);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  oz_split_kernel<true><<<dim3((L.Np + 7) / 8, g.batch), 256, 0, st>>>(g, L.Np, L.Kp, Bd, eb);
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
  oz_gemm_kernel<<<dim3(L.Np / OZ_BN, L.Mp / OZ_BM, g.batch), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace hps
