// qbx_hk_table.cu -- H0, H1 for complex k along the ray z = k rho.
//
// A call with complex k evaluates H_n(k rho) at every (centre, source) pair;
// the series / Miller / asymptotic evaluation (hankel01_cplx) costs far more
// than the real-axis fits.  But one call has one k, so every argument lies on
// the ray z = (k/|k|) |z|: the modulated amplitudes B_n = H_n(z) e^{-i(z -
// pi/4)} (DLMF 10.17.5: smooth in s = |z|^{-1/2}, no oscillation) are fitted
// once per k on the intervals of the real-axis table, by Chebyshev
// interpolation at QBX_HK_DEG + 1 nodes per interval, and the pair kernels
// evaluate them like the real-axis fits (KW<cplx>).  The values at the nodes
// come from hankel01_cplx for |z| <= 20 and from the asymptotic amplitude
// (hankel_amp_asym_c, finite for any Im z) above.
#include <cuda_runtime.h>
#include "qbx_apply_impl.cuh"
#include "qbx_internal.h"

namespace qbx {
namespace {

constexpr int kN = QBX_HK_DEG + 1;   // nodes and coefficients per interval

__device__ cplx amp_on_ray(cplx z, int n) {
  if (cabs_(z) > 20.0) return hankel_amp_asym_c(z, n);
  cplx h0, h1;
  hankel01_cplx(z, h0, h1);
  return (n == 0 ? h0 : h1) * cexp_(mul_i(cplx{0.78539816339744830962 - z.re, -z.im}));   // e^{-i(z - pi/4)}
}

// one thread per interval i of width w = 2^-LOG2_PER_UNIT in s, [i w, (i+1) w]
__global__ void k_hk_table(double kre, double kim, double* tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= QBX_HK_NI) return;
  const double w = 1.0 / (double)(1 << QBX_HK_LOG2_PER_UNIT);
  const double mid = (i + 0.5) * w, half = 0.5 * w;
  const double ka = hypot(kre, kim);
  const cplx dir{kre / ka, kim / ka};   // k / |k|
  double xs[kN];
  cplx f[2][kN];
  for (int j = 0; j < kN; ++j) {
    xs[j] = cos(3.14159265358979323846 * (j + 0.5) / kN);
    const double s = mid + half * xs[j];
    const cplx z = (1.0 / (s * s)) * dir;
    f[0][j] = amp_on_ray(z, 0);
    f[1][j] = amp_on_ray(z, 1);
  }
  // monomial coefficients of T_0 .. T_{kN-1} in x (T_{m+1} = 2 x T_m - T_{m-1})
  double T[kN][kN];
  for (int m = 0; m < kN; ++m)
    for (int d = 0; d < kN; ++d) T[m][d] = 0.0;
  T[0][0] = 1.0;
  if (kN > 1) T[1][1] = 1.0;
  for (int m = 1; m + 1 < kN; ++m)
    for (int d = 0; d < kN; ++d) T[m + 1][d] = (d > 0 ? 2.0 * T[m][d - 1] : 0.0) - T[m - 1][d];
  double* out = tab + (size_t)i * kN * 4;
  for (int n = 0; n < 2; ++n) {
    // Chebyshev coefficients c_m = (2 - [m = 0]) / kN sum_j f_j T_m(x_j)
    cplx c[kN];
    for (int m = 0; m < kN; ++m) {
      cplx acc{0.0, 0.0};
      for (int j = 0; j < kN; ++j) acc = acc + cos(3.14159265358979323846 * m * (j + 0.5) / kN) * f[n][j];
      c[m] = ((m == 0 ? 1.0 : 2.0) / kN) * acc;
    }
    // p(x) = sum_m c_m T_m(x) in monomials of x, then of u = half x
    double scale = 1.0;
    for (int d = 0; d < kN; ++d) {
      cplx b{0.0, 0.0};
      for (int m = d; m < kN; ++m) b = b + T[m][d] * c[m];
      out[d * 4 + 2 * n] = b.re * scale;
      out[d * 4 + 2 * n + 1] = b.im * scale;
      scale /= half;
    }
  }
}

__global__ void k_debug_hankel_ray(double kre, double kim, const double* tab, const double* rho, int n, cplx* h0,
                                   cplx* h1) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  KW<cplx> kw;
  kw.init(kre, kim, tab);
  double inv, r, y;
  kw.geom(rho[t] * rho[t], inv, r, y);
  cplx a, b, tz;
  kw.hankel(r, inv, y, a, b, tz);
  h0[t] = a;
  h1[t] = b;
}

}  // namespace

int hk_table_doubles() { return QBX_HK_NI * kN * 4; }

cudaError_t launch_hk_table(double kre, double kim, double* tab, cudaStream_t st) {
  k_hk_table<<<(QBX_HK_NI + 63) / 64, 64, 0, st>>>(kre, kim, tab);
  return cudaGetLastError();
}

cudaError_t launch_debug_hankel_ray(double kre, double kim, const double* tab, const double* rho, int n, void* h0,
                                    void* h1, cudaStream_t st) {
  k_debug_hankel_ray<<<(n + 127) / 128, 128, 0, st>>>(kre, kim, tab, rho, n, (cplx*)h0, (cplx*)h1);
  return cudaGetLastError();
}

}  // namespace qbx
