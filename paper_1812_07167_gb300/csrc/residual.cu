// Complex128 residual of the global collocation system that the HPS build
// and solve invert: every leaf's interior collocation rows A-hat u = s and
// impedance rows (Sec. 2.1), the outer impedance data F u = t (Eq. (1)), and
// at every pair of coincident nodes on a shared edge the two conditions
// t3a = -g3b and g3a = -t3b of Sec. 2.2.  The mixed-precision solve refines
// its answer against this residual.
#include "hps_internal.h"

namespace hps {

namespace {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double w, double2 a) { return make_double2(w * a.x, w * a.y); }
// i eta z
__device__ __forceinline__ double2 ieta(double2 eta, double2 z) {
  return make_double2(-eta.y * z.x - eta.x * z.y, eta.x * z.x - eta.y * z.y);
}

// one thread per (rhs, leaf, node): interior rows give s - A u, boundary
// nodes give F u and G u
__global__ void __launch_bounds__(256) leaf_residual_kernel(const __grid_constant__ ResidualSetup rs,
                                                            const double2 *u, const double2 *s,
                                                            double2 *sd, double2 *Fu, double2 *Gu, int R) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)R * rs.leaves * rs.n;
  if (gid >= total) return;
  const int p = rs.p, n = rs.n, nb = rs.nb, ni = rs.ni, e = rs.e;
  const int k = (int)(gid % n);
  const long long rl = gid / n;  // rhs * leaves + leaf
  const int leaf = (int)(rl % rs.leaves);
  const double *D1x = rs.tab, *D1y = D1x + p * p, *D2x = D1y + p * p, *D2y = D2x + p * p;
  const int *grid = (const int *)(rs.tab + 4 * p * p);
  const int *loc = grid + n;
  const double2 *ul = u + rl * n;
  const int g = __ldg(grid + k);
  const int ix = g & 0xff, iy = g >> 8;
  if (k >= nb) {
    const int q = k - nb;
    double2 Au = make_double2(0.0, 0.0);
    for (int t = 0; t < p; t++) {
      Au = csub(Au, cscale(__ldg(D2x + ix * p + t), ul[__ldg(loc + iy * p + t)]));
      Au = csub(Au, cscale(__ldg(D2y + iy * p + t), ul[__ldg(loc + t * p + ix)]));
    }
    Au = csub(Au, cscale(rs.kappa2 * __ldg(rs.c + (long long)leaf * ni + q), ul[k]));
    sd[rl * ni + q] = csub(s[rl * ni + q], Au);
  } else {
    const int side = k / e;
    double2 Nu = make_double2(0.0, 0.0);
    for (int t = 0; t < p; t++) {
      double w;
      int node;
      if (side == 0) {
        w = -__ldg(D1y + 0 * p + t);
        node = __ldg(loc + t * p + ix);
      } else if (side == 1) {
        w = __ldg(D1x + (p - 1) * p + t);
        node = __ldg(loc + iy * p + t);
      } else if (side == 2) {
        w = __ldg(D1y + (p - 1) * p + t);
        node = __ldg(loc + t * p + ix);
      } else {
        w = -__ldg(D1x + 0 * p + t);
        node = __ldg(loc + iy * p + t);
      }
      Nu = cadd(Nu, cscale(w, ul[node]));
    }
    const double2 ie = ieta(rs.eta, ul[k]);
    Fu[rl * nb + k] = cadd(Nu, ie);
    Gu[rl * nb + k] = csub(Nu, ie);
  }
}

// one thread per (rhs, I3 pair) and per (rhs, outer boundary node)
__global__ void __launch_bounds__(256) jump_kernel(const __grid_constant__ ResidualSetup rs,
                                                   const double2 *t, const double2 *Fu,
                                                   const double2 *Gu, double2 *td, double2 *JA,
                                                   double2 *JB, int R) {
  const long long per = rs.total_pairs + rs.nbdry;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)R * per) return;
  const int r = (int)(gid / per);
  const long long k = gid % per;
  const long long fb = (long long)r * rs.leaves * rs.nb;
  if (k >= rs.total_pairs) {
    const int q = (int)(k - rs.total_pairs);
    const double2 f = Fu[fb + __ldg(rs.outer + q)];
    td[(long long)r * rs.nbdry + q] = csub(t[(long long)r * rs.nbdry + q], f);
    return;
  }
  int lv = 0;
  while (lv + 1 < rs.nlev && k >= rs.lev[lv + 1].off) lv++;
  const ResidualLevel &L = rs.lev[lv];
  const long long kk = k - L.off;
  const int b = (int)(kk / L.n3), j = (int)(kk % L.n3);
  const int *pr = L.pairs + 4 * j;
  const long long a = fb + ((long long)b * L.lpp + __ldg(pr + 0)) * rs.nb + __ldg(pr + 1);
  const long long c = fb + ((long long)b * L.lpp + __ldg(pr + 2)) * rs.nb + __ldg(pr + 3);
  const double2 fa = Fu[a], ga = Gu[a], fc = Fu[c], gc = Gu[c];
  const double2 ja = cadd(fa, gc), jb = cadd(ga, fc);
  JA[(long long)r * rs.total_pairs + k] = make_double2(-ja.x, -ja.y);
  JB[(long long)r * rs.total_pairs + k] = make_double2(-jb.x, -jb.y);
}

}  // namespace

cudaError_t launch_residual(const ResidualSetup &rs, const double2 *u, const double2 *s,
                            const double2 *t, double2 *sd, double2 *td, double2 *Fu, double2 *Gu,
                            double2 *JA, double2 *JB, int R, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  const long long total = (long long)R * rs.leaves * rs.n;
  leaf_residual_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(rs, u, s, sd, Fu, Gu, R);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const long long jt = (long long)R * (rs.total_pairs + rs.nbdry);
  jump_kernel<<<(unsigned)((jt + 255) / 256), 256, 0, st>>>(rs, t, Fu, Gu, td, JA, JB, R);
  return cudaGetLastError();
}

}  // namespace hps
