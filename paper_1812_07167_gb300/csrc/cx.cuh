// Device helpers shared by the dense kernels (Gauss-Jordan, LU): complex
// arithmetic on double2 / float2, the pivot key, the split cluster barrier
// and the build status word.
#pragma once

#include <cuda_runtime.h>

namespace hps {
namespace {

template <class C>
struct CX;
template <>
struct CX<double2> {
  using R = double;
  __device__ static double2 make(double x, double y) { return make_double2(x, y); }
  __device__ static double fmad(double a, double b, double c) { return fma(a, b, c); }
  // max(|Re|, |Im|) as the integer image of its IEEE-754 bits (for
  // non-negative values integer order is numeric order): the pivot search
  // compares integers instead of spending floating-point instructions
  __device__ static unsigned long long key(double2 z) {
    unsigned long long a = (unsigned long long)__double_as_longlong(z.x) & 0x7fffffffffffffffull;
    unsigned long long b = (unsigned long long)__double_as_longlong(z.y) & 0x7fffffffffffffffull;
    return a > b ? a : b;
  }
};
template <>
struct CX<float2> {
  using R = float;
  __device__ static float2 make(double x, double y) { return make_float2((float)x, (float)y); }
  __device__ static float fmad(float a, float b, float c) { return fmaf(a, b, c); }
  __device__ static unsigned long long key(float2 z) {
    unsigned int a = __float_as_uint(z.x) & 0x7fffffffu;
    unsigned int b = __float_as_uint(z.y) & 0x7fffffffu;
    return a > b ? a : b;
  }
};

template <class C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

template <class C>
__device__ __forceinline__ C cfms(C acc, C a, C b) {  // acc - a b
  acc.x = CX<C>::fmad(-a.x, b.x, acc.x);
  acc.x = CX<C>::fmad(a.y, b.y, acc.x);
  acc.y = CX<C>::fmad(-a.x, b.y, acc.y);
  acc.y = CX<C>::fmad(-a.y, b.x, acc.y);
  return acc;
}

template <class C>
__device__ __forceinline__ C crecip(C z) {
  // 1 / z with Smith's scaling (Smith, CACM 1962)
  using R = typename CX<C>::R;
  C out;
  if (fabs(z.x) >= fabs(z.y)) {
    R r = z.y / z.x, d = z.x + z.y * r;
    out.x = R(1) / d;
    out.y = -r / d;
  } else {
    R r = z.x / z.y, d = z.x * r + z.y;
    out.x = r / d;
    out.y = R(-1) / d;
  }
  return out;
}

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// First error of a build wins: (code << 28) | (level << 20) | box.
__device__ __forceinline__ void record_status(unsigned int *status, unsigned int code, int level,
                                              int box) {
  unsigned int w = (code << 28) | ((unsigned)(level & 0xff) << 20) | ((unsigned)box & 0xfffffu);
  atomicCAS(status, 0u, w);
}

}  // namespace
}  // namespace hps
