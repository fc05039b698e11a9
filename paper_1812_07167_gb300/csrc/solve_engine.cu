// One launch for a whole solve with one or two right-hand sides (Algorithm 2).
//
// With one or two right-hand sides every step of the upward and downward
// sweeps is a small batched matrix-vector product or copy, and a solve is a
// chain of ~50 of them, each depending on the one before: as separate
// launches the chain costs a launch latency and a ramp-up and drain per step.
// Here a persistent kernel (cooperative launch: every CTA resident) walks a
// program of such steps recorded on the host for the handle, in phases; the
// steps of a phase are independent, and a grid barrier separates phases.
//
// A product step y = alpha A x (+ beta D) (A: M x K, batch matrices, x with
// one or two columns, rows of x, y and D optionally index-mapped) is cut into
// units of 32 rows x a K chunk (at most 512); a unit stages its chunk of x in
// shared memory, and its 256 threads take 32 rows x 8 interleaved K slices
// (neighbouring threads on neighbouring rows of the column-major A), sum the
// slices in shared memory and, when K was cut into
// chunks, add the chunks' partial sums in chunk order (the last unit of a row
// block to arrive does it, so that the sum is deterministic).  Copy steps are
// element-wise.  Vectors written inside the kernel are read with L2-only
// loads (another SM may have written them since this SM last cached them);
// the operators are read-only and go through the read-only path.
//
// The grid barrier is one arrival counter and a generation word; every wait
// gives up after 2 s (recording a timeout in the build status word and
// setting an abort word that ends every CTA at its next barrier), so a
// stalled kernel returns instead of hanging the GPU.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "cx.cuh"
#include "hps_internal.h"

namespace hps {

namespace {

constexpr int kEnThreads = 256;
constexpr int kEnRows = 32;      // rows of a product unit
constexpr int kEnSlices = 8;     // K slices of a unit
constexpr int kEnMaxKc = 512;    // longest K chunk (its x is staged in shared memory)
constexpr unsigned long long kEnWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long en_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}

__device__ __forceinline__ float en_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double en_fma(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ const char *en_base(const EnArgs &a, const EnMat &m) {
  return (const char *)a.base[m.base] + m.off;
}

// element (i, c) of batch b of a vector operand, written inside the kernel:
// an L2-only load
__device__ __forceinline__ double2 en_ldv(const EnArgs &a, const EnMat &m, int b, int i, int c) {
  const long long r = m.rmap ? (long long)__ldg(m.rmap + i) : (long long)i;
  const long long e = (long long)b * m.stride + (long long)c * m.ld + r;
  if (m.f32) {
    const float2 v = __ldcg((const float2 *)en_base(a, m) + e);
    return make_double2(v.x, v.y);
  }
  return __ldcg((const double2 *)en_base(a, m) + e);
}

__device__ __forceinline__ void en_stv(const EnArgs &a, const EnMat &m, int b, int i, int c, double2 v) {
  const long long r = m.rmap ? (long long)__ldg(m.rmap + i) : (long long)i;
  const long long e = (long long)b * m.stride + (long long)c * m.ld + r;
  if (m.f32)
    ((float2 *)en_base(a, m))[e] = make_float2((float)v.x, (float)v.y);
  else
    ((double2 *)en_base(a, m))[e] = v;
}

// Grid barrier with a bounded wait; false when the kernel is to end.
__device__ bool en_grid_sync(const EnArgs &a, int phase) {
  __shared__ int go;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = a.bar + 1, *abort = a.bar + 2;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(a.bar, 1u);
    bool ok = true;
    if (arrived == gridDim.x - 1) {
      atomicExch(a.bar, 0u);
      __threadfence();
      atomicAdd((unsigned *)(a.bar + 1), 1u);
    } else {
      const unsigned long long t0 = en_ns();
      while (*gen == g) {
        if (*abort) {
          ok = false;
          break;
        }
        if (en_ns() - t0 > kEnWaitNs) {
          *abort = 1u;
          if (a.status) record_status(a.status, 3u, 0, phase);
          ok = false;
          break;
        }
      }
    }
    __threadfence();
    go = ok && !*abort;
  }
  __syncthreads();
  return go != 0;
}

// One unit of a product step: rows [32 rb, 32 rb + 32) of batch entry b,
// K chunk kci.  R = 1 or 2 right-hand sides; T the accumulation type.
template <int R, class T>
__device__ void en_product_unit(const EnArgs &a, const EnOp &o, int u, double2 (*red)[kEnRows][2], int &last_sh,
                                double2 (*xs)[kEnMaxKc]) {
  const int tid = threadIdx.x, r = tid & (kEnRows - 1), ks = tid / kEnRows;
  const int per_b = o.nrb * o.nkc;
  const int b = u / per_b, rem = u - b * per_b, rb = rem / o.nkc, kci = rem - rb * o.nkc;
  const int i = rb * kEnRows + r;
  const int k0 = kci * o.kc, k1 = min(o.K, k0 + o.kc);
  const bool live = i < o.M;
  // issued first, so that their latencies overlap: D of the output rows,
  // the first four of this thread's elements of A, and this chunk of x
  // (rows mapped, both parts) into shared memory
  double2 dpre[R];
  if (tid < kEnRows && live && o.D.base >= 0)
#pragma unroll
    for (int c = 0; c < R; c++) dpre[c] = en_ldv(a, o.D, b, i, c);
  const char *Ab = en_base(a, o.A);
  const long long arow = (long long)b * o.A.stride + i;
  auto lda = [&](int k) -> double2 {
    if (!live || k >= k1) return make_double2(0.0, 0.0);
    if (o.A.f32) {
      const float2 v = __ldg((const float2 *)Ab + arow + (long long)k * o.A.ld);
      return make_double2(v.x, v.y);
    }
    return __ldg((const double2 *)Ab + arow + (long long)k * o.A.ld);
  };
  double2 apre[4];
#pragma unroll
  for (int q = 0; q < 4; q++) apre[q] = lda(k0 + ks + q * kEnSlices);
  for (int e = tid; e < (k1 - k0) * R; e += kEnThreads) {
    const int c = e / (k1 - k0), k = k0 + e - c * (k1 - k0);
    xs[c][k - k0] = (k < o.ksplit) ? en_ldv(a, o.x, b, k, c) : en_ldv(a, o.x2, b, k - o.ksplit, c);
  }
  __syncthreads();
  T acc[R][2];
#pragma unroll
  for (int c = 0; c < R; c++) acc[c][0] = acc[c][1] = T(0);
  auto madd = [&](double2 av, int k) {
#pragma unroll
    for (int c = 0; c < R; c++) {
      const double2 xv = xs[c][k - k0];
      const T tax = (T)av.x, tay = (T)av.y, txx = (T)xv.x, txy = (T)xv.y;
      acc[c][0] = en_fma(tax, txx, acc[c][0]);
      acc[c][0] = en_fma(-tay, txy, acc[c][0]);
      acc[c][1] = en_fma(tax, txy, acc[c][1]);
      acc[c][1] = en_fma(tay, txx, acc[c][1]);
    }
  };
  if (live) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int k = k0 + ks + q * kEnSlices;
      if (k < k1) madd(apre[q], k);
    }
#pragma unroll 4
    for (int k = k0 + ks + 4 * kEnSlices; k < k1; k += kEnSlices) madd(lda(k), k);
  }
#pragma unroll
  for (int c = 0; c < R; c++) red[ks][r][c] = make_double2((double)acc[c][0], (double)acc[c][1]);
  __syncthreads();
  double2 v[R];
  if (tid < kEnRows) {
#pragma unroll
    for (int c = 0; c < R; c++) {
      v[c] = red[0][tid][c];
      for (int q = 1; q < kEnSlices; q++) {
        v[c].x += red[q][tid][c].x;
        v[c].y += red[q][tid][c].y;
      }
    }
  }
  bool fin = true;
  if (o.nkc > 1) {
    // this chunk's partial sums; the last chunk of the row block to arrive
    // adds them up in chunk order
    double2 *part = a.part + o.part_off + ((long long)(b * o.nrb + rb) * o.nkc) * kEnRows * R;
    if (tid < kEnRows)
#pragma unroll
      for (int c = 0; c < R; c++) part[((long long)kci * R + c) * kEnRows + tid] = v[c];
    __syncthreads();
    if (tid == 0) {
      __threadfence();  // (cumulative: the block's stores before the barrier)
      unsigned *cnt = a.cnt + o.cnt_off + b * o.nrb + rb;
      const unsigned old = atomicAdd(cnt, 1u);
      last_sh = old == (unsigned)(o.nkc - 1);
      if (last_sh) {
        atomicExch(cnt, 0u);
        __threadfence();
      }
    }
    __syncthreads();
    fin = last_sh != 0;
    if (fin) {
      if (tid < kEnRows)
#pragma unroll
        for (int c = 0; c < R; c++) {
          double2 s = __ldcg(part + (long long)c * kEnRows + tid);
          for (int q = 1; q < o.nkc; q++) {
            const double2 w = __ldcg(part + ((long long)q * R + c) * kEnRows + tid);
            s.x += w.x;
            s.y += w.y;
          }
          v[c] = s;
        }
    }
  }
  if (fin && tid < kEnRows && i < o.M) {
#pragma unroll
    for (int c = 0; c < R; c++) {
      double2 out = make_double2(o.alpha.x * v[c].x - o.alpha.y * v[c].y, o.alpha.x * v[c].y + o.alpha.y * v[c].x);
      if (o.D.base >= 0) {
        const double2 d = dpre[c];
        out.x += o.beta.x * d.x - o.beta.y * d.y;
        out.y += o.beta.x * d.y + o.beta.y * d.x;
      }
      en_stv(a, o.y, b, i, c, out);
    }
  }
  __syncthreads();  // red and last_sh are reused by the next unit
}

__device__ void en_copy_unit(const EnArgs &a, const EnOp &o, int u) {
  const long long e = (long long)u * kEnThreads + threadIdx.x;
  const long long per_b = (long long)o.M * o.R;
  if (e >= per_b * o.batch) return;
  const int b = (int)(e / per_b);
  const long long rem = e - b * per_b;
  const int c = (int)(rem / o.M), i = (int)(rem - (long long)c * o.M);
  const double2 s = en_ldv(a, o.x, b, i, c);
  double2 v = make_double2(o.alpha.x * s.x - o.alpha.y * s.y, o.alpha.x * s.y + o.alpha.y * s.x);
  if (o.accumulate) {
    const double2 w = en_ldv(a, o.y, b, i, c);
    v.x += w.x;
    v.y += w.y;
  }
  en_stv(a, o.y, b, i, c, v);
}

__global__ void __launch_bounds__(kEnThreads) solve_engine_kernel(const __grid_constant__ EnArgs a) {
  __shared__ double2 red[kEnSlices][kEnRows][2];  // a product unit's K-slice sums
  __shared__ double2 xs[2][kEnMaxKc];              // its chunk of x
  __shared__ int last_sh;
  int op = 0, phase = 0;
  while (op < a.nops) {
    int ope = op;
    while (!a.ops[ope].phase_end) ope++;
    const int total = a.ops[ope].unit0 + a.ops[ope].units;
    for (int u = blockIdx.x; u < total; u += gridDim.x) {
      int q = op;
      while (u >= a.ops[q].unit0 + a.ops[q].units) q++;
      const EnOp &o = a.ops[q];
      const int lu = u - o.unit0;
      if (o.kind == 1)
        en_copy_unit(a, o, lu);
      else if (o.R == 1)
        o.cf32 ? en_product_unit<1, float>(a, o, lu, red, last_sh, xs)
               : en_product_unit<1, double>(a, o, lu, red, last_sh, xs);
      else
        o.cf32 ? en_product_unit<2, float>(a, o, lu, red, last_sh, xs)
               : en_product_unit<2, double>(a, o, lu, red, last_sh, xs);
    }
    op = ope + 1;
    phase++;
    if (op < a.nops && !en_grid_sync(a, phase)) return;
  }
}

}  // namespace

int engine_grid() {
  static int grid = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, solve_engine_kernel, kEnThreads, 0) != cudaSuccess ||
        sms <= 0 || occ <= 0) {
      cudaGetLastError();
      grid = 0;
      return;
    }
    grid = sms * std::min(occ, 2);
  });
  return grid;
}

int engine_unit_rows() { return kEnRows; }
int engine_max_kc() { return kEnMaxKc; }
int engine_copy_unit() { return kEnThreads; }

cudaError_t launch_solve_engine(const EnArgs &a, cudaStream_t st) {
  const int grid = engine_grid();
  if (grid <= 0) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kEnThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, solve_engine_kernel, a);
}

}  // namespace hps
