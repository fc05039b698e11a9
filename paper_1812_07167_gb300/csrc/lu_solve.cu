// The leaf action of the solve in LU form (Algorithm 2's last step):
// u = B^{-1} [t; s] = U^{-1} L^{-1} P D [t; s] for every leaf from the factors
// the LU leaf kernel (lu.cu) stores: L (unit diagonal implied) and U in
// place, the row order pi (row k of P D B is row pi(k) of B) and d_pi(k).
#include "cx.cuh"
#include "hps_internal.h"

namespace hps {

namespace {

constexpr int kThreads = 256;

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

struct LuSolveArgs {
  const void *LU;      // [leaf][n][n]
  const int *perm;     // [leaf][n]
  const double *dsc;   // [leaf][n]
  const double2 *t;    // rows [0, nb): t[c * t_ld + leaf * t_stride + i]
  long long t_ld, t_stride;
  const double2 *s;    // rows [nb, n): s[c * s_ld + leaf * s_stride + i - nb]
  long long s_ld, s_stride;
  double2 *u;          // u[c * u_ld + leaf * u_stride + i]
  long long u_ld, u_stride;
  int n, nb, R;
  // rows [r0, r1) of every leaf: gather (y = P D [t; s] for all n rows, the
  // rows outside [r0, r1) written straight to u) or read y from u; then the
  // forward and/or the backward sweep with the diagonal block of rows
  // [r0, r1) only; then y back to u
  int r0, r1, gather, fwd, bwd;
};

constexpr int kSB = 32;  // rows of a diagonal block of the sweeps

// y[i] -= sum_{kk < jb} A(i, J0 + kk) y[J0 + kk] for CPT of the RB
// right-hand sides (from c0), a = &A(i, J0) (column-major, ld n).  The factor
// entries are loaded KC at a time ahead of their multiply-adds, so a thread
// has KC loads in flight (the sweeps of a 1-RHS solve wait on memory, not on
// arithmetic).
template <class C, int RB, int CPT>
__device__ __forceinline__ void sweep_row(C *y, const C *a, int n, int J0, int jb, int i, int c0) {
  // y points at the row J0 of the shared vector block; row i at y + (i - J0) RB
  constexpr int KC = CPT <= 1 ? 16 : CPT <= 4 ? 8 : 4;
  C acc[CPT];
#pragma unroll
  for (int c = 0; c < CPT; c++) acc[c] = y[(i - J0) * RB + c0 + c];
  for (int k0 = 0; k0 < jb; k0 += KC) {
    C l[KC];
#pragma unroll
    for (int u = 0; u < KC; u++) l[u] = (k0 + u < jb) ? __ldg(a + (size_t)(k0 + u) * n) : CX<C>::make(0.0, 0.0);
#pragma unroll
    for (int u = 0; u < KC; u++) {
      if (k0 + u >= jb) break;
#pragma unroll
      for (int c = 0; c < CPT; c++) acc[c] = cfms(acc[c], l[u], y[(k0 + u) * RB + c0 + c]);
    }
  }
#pragma unroll
  for (int c = 0; c < CPT; c++) y[(i - J0) * RB + c0 + c] = acc[c];
}

// The update of rows [i0, i0 + rows) by the block's jb solved rows: a thread
// per (row, share of the right-hand sides), the right-hand sides split S ways
// while the rows are fewer than the threads, so that short updates keep the
// FP64 pipes of every warp busy.  y: the shared vector block from its row J0
// (rows i and J0 + kk are at (i - J0) and kk; both lie in the block's range).
template <class C, int RB, int S>
__device__ __forceinline__ void sweep_rows_s(C *y, const C *LU, int n, int J0, int jb, int i0, int rows) {
  for (int t = threadIdx.x; t < rows * S; t += blockDim.x) {
    const int i = i0 + t / S, c0 = (t % S) * (RB / S);
    sweep_row<C, RB, RB / S>(y, LU + (size_t)J0 * n + i, n, J0, jb, i, c0);
  }
}

template <class C, int RB>
__device__ __forceinline__ void sweep_rows(C *y, const C *LU, int n, int J0, int jb, int i0, int rows) {
  if (rows <= 0) return;
  const int want = (int)blockDim.x / rows;  // right-hand-side shares that keep every thread busy
  if (RB >= 16 && want >= 16)
    sweep_rows_s<C, RB, (RB >= 16 ? 16 : 1)>(y, LU, n, J0, jb, i0, rows);
  else if (RB >= 8 && want >= 8)
    sweep_rows_s<C, RB, (RB >= 8 ? 8 : 1)>(y, LU, n, J0, jb, i0, rows);
  else if (RB >= 4 && want >= 4)
    sweep_rows_s<C, RB, (RB >= 4 ? 4 : 1)>(y, LU, n, J0, jb, i0, rows);
  else if (RB >= 2 && want >= 2)
    sweep_rows_s<C, RB, (RB >= 2 ? 2 : 1)>(y, LU, n, J0, jb, i0, rows);
  else
    sweep_rows_s<C, RB, 1>(y, LU, n, J0, jb, i0, rows);
}

// One CTA per (leaf, RB right-hand sides): the rows [r0, r1) of y (= P D b,
// gathered here, or the partial result in u) in shared memory, then the
// forward sweep with L and/or the backward sweep with U over those rows in
// blocks of 32: a warp solves the diagonal block for one right-hand side
// with shuffles, then the threads update the rest of the range (a row, or a
// share of a row's right-hand sides, each).  The whole solve is one launch
// over [0, n); a blocked wide solve runs it on two ranges with the products
// between them done elsewhere.
template <class C, int RB>
__global__ void __launch_bounds__(kThreads, 2) lu_solve_kernel(const __grid_constant__ LuSolveArgs a) {
  chain_enter();
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n, nb = a.nb, r0 = a.r0, r1 = a.r1;
  const long long leaf = blockIdx.x;
  const int c0 = blockIdx.y * RB;
  const int nc = min(RB, a.R - c0);
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
  C *y = (C *)smem;                                    // [r1 - r0][RB]: rows r0 ..
  C *Db = (C *)(smem + al16(sizeof(C) * (size_t)n * RB));  // [kSB][kSB + 1]
  C *dinv = Db + kSB * (kSB + 1);                       // [kSB]
  const C *LU = (const C *)a.LU + (size_t)leaf * n * n;
  const int *pm = a.perm + (size_t)leaf * n;
  const double *ds = a.dsc + (size_t)leaf * n;
  double2 *u = a.u + leaf * a.u_stride;

  if (a.gather) {
    for (int idx = tid; idx < n * RB; idx += nthr) {
      const int k = idx / RB, c = idx % RB;
      C v = CX<C>::make(0.0, 0.0);
      if (c < nc) {
        const int i = __ldg(&pm[k]);
        const double d = __ldg(&ds[k]);
        const double2 b = (i < nb) ? a.t[(size_t)(c0 + c) * a.t_ld + leaf * a.t_stride + i]
                                   : a.s[(size_t)(c0 + c) * a.s_ld + leaf * a.s_stride + (i - nb)];
        v = CX<C>::make(d * b.x, d * b.y);
        if (k < r0 || k >= r1) u[(size_t)(c0 + c) * a.u_ld + k] = make_double2(d * b.x, d * b.y);
      }
      if (k >= r0 && k < r1) y[(k - r0) * RB + c] = v;
    }
  } else {
    for (int idx = tid; idx < (r1 - r0) * RB; idx += nthr) {
      const int k = idx / RB, c = idx % RB;
      C v = CX<C>::make(0.0, 0.0);
      if (c < nc) {
        const double2 b = u[(size_t)(c0 + c) * a.u_ld + r0 + k];
        v = CX<C>::make(b.x, b.y);
      }
      y[idx] = v;
    }
  }
  __syncthreads();

  // forward: L y = P D b on the rows [r0, r1)
  if (a.fwd)
    for (int J0 = r0; J0 < r1; J0 += kSB) {
      const int jb = min(kSB, r1 - J0);
      C *yJ = y + (size_t)(J0 - r0) * RB;
#pragma unroll 4
      for (int t = tid; t < jb * kSB; t += nthr) {
        const int kk = t / kSB, i = t % kSB;
        if (i < jb) Db[kk * (kSB + 1) + i] = __ldg(&LU[(size_t)(J0 + kk) * n + J0 + i]);
      }
      __syncthreads();
      for (int c = wid; c < nc; c += nw) {
        C yv = (lane < jb) ? yJ[lane * RB + c] : CX<C>::make(0.0, 0.0);
        for (int kk = 0; kk + 1 < jb; kk++) {
          C yk;
          yk.x = __shfl_sync(0xffffffffu, yv.x, kk);
          yk.y = __shfl_sync(0xffffffffu, yv.y, kk);
          if (lane > kk && lane < jb) yv = cfms(yv, Db[kk * (kSB + 1) + lane], yk);
        }
        if (lane < jb) yJ[lane * RB + c] = yv;
      }
      __syncthreads();
      sweep_rows<C, RB>(yJ, LU, n, J0, jb, J0 + jb, r1 - J0 - jb);
      __syncthreads();
    }
  // backward: U x = y on the rows [r0, r1)
  if (a.bwd) {
    const int nblk = (r1 - r0 + kSB - 1) / kSB;
    for (int bk = nblk - 1; bk >= 0; bk--) {
      const int J0 = r0 + bk * kSB, jb = min(kSB, r1 - J0);
      C *yJ = y + (size_t)(J0 - r0) * RB;
#pragma unroll 4
      for (int t = tid; t < jb * kSB; t += nthr) {
        const int kk = t / kSB, i = t % kSB;
        if (i < jb) Db[kk * (kSB + 1) + i] = __ldg(&LU[(size_t)(J0 + kk) * n + J0 + i]);
      }
      __syncthreads();
      if (tid < jb) dinv[tid] = crecip(Db[tid * (kSB + 1) + tid]);
      __syncthreads();
      for (int c = wid; c < nc; c += nw) {
        C yv = (lane < jb) ? yJ[lane * RB + c] : CX<C>::make(0.0, 0.0);
        for (int kk = jb - 1; kk >= 0; kk--) {
          if (lane == kk) yv = cmul(yv, dinv[kk]);
          C yk;
          yk.x = __shfl_sync(0xffffffffu, yv.x, kk);
          yk.y = __shfl_sync(0xffffffffu, yv.y, kk);
          if (lane < kk) yv = cfms(yv, Db[kk * (kSB + 1) + lane], yk);
        }
        if (lane < jb) yJ[lane * RB + c] = yv;
      }
      __syncthreads();
      sweep_rows<C, RB>(yJ, LU, n, J0, jb, r0, J0 - r0);
      __syncthreads();
    }
  }
  for (int idx = tid; idx < (r1 - r0) * nc; idx += nthr) {
    const int c = idx / (r1 - r0), i = idx % (r1 - r0);
    const C v = y[i * RB + c];
    u[(size_t)(c0 + c) * a.u_ld + r0 + i] = make_double2((double)v.x, (double)v.y);
  }
}

template <class C, int RB>
cudaError_t solve_rb(const LuSolveArgs &a, long long leaves, cudaStream_t st) {
  const size_t smem = al16(sizeof(C) * (size_t)a.n * RB) + sizeof(C) * (kSB * (kSB + 1) + kSB);
  cudaError_t err = cudaFuncSetAttribute(lu_solve_kernel<C, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  dim3 grid((unsigned)leaves, (unsigned)((a.R + RB - 1) / RB), 1);
  return launch_k(lu_solve_kernel<C, RB>, grid, dim3(kThreads), smem, st, a);
}

template <class C>
cudaError_t solve_any(const LuSolveArgs &a, long long leaves, cudaStream_t st) {
  if (a.R <= 1) return solve_rb<C, 1>(a, leaves, st);
  if (a.R <= 2) return solve_rb<C, 2>(a, leaves, st);
  if (a.R <= 4) return solve_rb<C, 4>(a, leaves, st);
  if (a.R <= 8) return solve_rb<C, 8>(a, leaves, st);
  return solve_rb<C, 16>(a, leaves, st);
}

}  // namespace

cudaError_t launch_lu_solve_part(const void *LU, const int *perm, const double *dsc, long long leaves, int n,
                                 int nb, int R, const double2 *t, long long t_ld, long long t_stride,
                                 const double2 *s, long long s_ld, long long s_stride, double2 *u,
                                 long long u_ld, long long u_stride, bool f32, int r0, int r1, bool gather,
                                 bool fwd, bool bwd, cudaStream_t st) {
  if (leaves <= 0 || R <= 0) return cudaSuccess;
  if (r0 < 0 || r1 > n || r0 >= r1) return cudaErrorInvalidValue;
  LuSolveArgs a;
  a.LU = LU;
  a.perm = perm;
  a.dsc = dsc;
  a.t = t;
  a.t_ld = t_ld;
  a.t_stride = t_stride;
  a.s = s;
  a.s_ld = s_ld;
  a.s_stride = s_stride;
  a.u = u;
  a.u_ld = u_ld;
  a.u_stride = u_stride;
  a.n = n;
  a.nb = nb;
  a.R = R;
  a.r0 = r0;
  a.r1 = r1;
  a.gather = gather ? 1 : 0;
  a.fwd = fwd ? 1 : 0;
  a.bwd = bwd ? 1 : 0;
  return f32 ? solve_any<float2>(a, leaves, st) : solve_any<double2>(a, leaves, st);
}

cudaError_t launch_lu_solve(const void *LU, const int *perm, const double *dsc, long long leaves, int n,
                            int nb, int R, const double2 *t, long long t_ld, long long t_stride,
                            const double2 *s, long long s_ld, long long s_stride, double2 *u,
                            long long u_ld, long long u_stride, bool f32, cudaStream_t st) {
  return launch_lu_solve_part(LU, perm, dsc, leaves, n, nb, R, t, t_ld, t_stride, s, s_ld, s_stride, u, u_ld,
                              u_stride, f32, 0, n, true, true, true, st);
}

}  // namespace hps
