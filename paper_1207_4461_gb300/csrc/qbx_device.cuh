// qbx_device.cuh -- device arithmetic for the QBX kernels: FP64 complex
// numbers, Hankel functions H0^(1), H1^(1) and the Bessel sequence J_0..J_n.
//
// Real argument (Im k == 0): H0, H1 from the library's own piecewise fits
// (special_tables.h, produced by gen_special_tables.py from 34-digit mpmath
// values):
//   z <  2 : ascending series in (z/2)^2 (DLMF 10.2.2, 10.8.1) with log(z/2)
//   z >= 2 : H_n = e^{i(z - pi/4)} B_n(s), s = z^{-1/2}, where
//            B_n = sqrt(2/pi) s e^{-i n pi/2} (P_n + i Q_n) (DLMF 10.17.3) is a
//            degree-4 polynomial on each of 182 intervals of s, and
//            e^{i(z - pi/4)} comes from a 512-entry table + Taylor after
//            Cody-Waite reduction.
// Complex argument (Im z > 0): series for |z| <= 6, Miller's backward
// recurrence with the Neumann series for Y0, Y1 for 6 < |z| <= 20 (DLMF
// 10.23.? / A&S 9.1.88-89), Hankel's asymptotic expansion (DLMF 10.17.5) above.
// J_0..J_n at the expansion targets: Miller's backward recurrence normalised by
// J_0 + 2 sum J_2k = 1 (generating function at t = 1), ascending series for
// |z| < 1/2.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#define QBX_HK_GQUAL static __device__ const
#define QBX_HK_CQUAL static __constant__ const
#include "special_tables.h"

#define QBX_HD __host__ __device__ __forceinline__

namespace qbx {

struct cplx {
  double re, im;
};

__host__ __device__ __forceinline__ cplx mk(double r, double i) { return cplx{r, i}; }
__host__ __device__ __forceinline__ cplx operator+(cplx a, cplx b) { return cplx{a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ cplx operator-(cplx a, cplx b) { return cplx{a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ cplx operator-(cplx a) { return cplx{-a.re, -a.im}; }
__host__ __device__ __forceinline__ cplx operator*(cplx a, cplx b) {
  return cplx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ cplx operator*(double s, cplx a) { return cplx{s * a.re, s * a.im}; }
__host__ __device__ __forceinline__ cplx operator*(cplx a, double s) { return cplx{s * a.re, s * a.im}; }
__host__ __device__ __forceinline__ cplx conj(cplx a) { return cplx{a.re, -a.im}; }
// acc += a b in four FMAs (written out: acc + a * b through the operators
// above costs two extra instructions per part)
__host__ __device__ __forceinline__ void cfma(cplx& acc, cplx a, cplx b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
__host__ __device__ __forceinline__ double abs2(cplx a) { return a.re * a.re + a.im * a.im; }
QBX_HD double cabs_(cplx a) { return hypot(a.re, a.im); }
// 1/b and a/b with the divisor scaled by its larger component, so that
// |b|^2 neither underflows nor overflows (Smith's method).
QBX_HD cplx cinv(cplx b) {
  const double m = fmax(fabs(b.re), fabs(b.im));
  const double br = b.re / m, bi = b.im / m;
  const double s = 1.0 / (m * (br * br + bi * bi));
  return cplx{br * s, -bi * s};
}
QBX_HD cplx cdiv(cplx a, cplx b) { return a * cinv(b); }
QBX_HD cplx clog_(cplx z) { return cplx{log(hypot(z.re, z.im)), atan2(z.im, z.re)}; }
QBX_HD cplx cexp_(cplx z) {
  double s, c;
  sincos(z.im, &s, &c);
  double e = exp(z.re);
  return cplx{e * c, e * s};
}
QBX_HD cplx csqrt_(cplx z) {
  double m = hypot(z.re, z.im);
  double a = sqrt(0.5 * (m + fabs(z.re)));
  if (a == 0.0) return cplx{0.0, 0.0};
  if (z.re >= 0.0) return cplx{a, 0.5 * z.im / a};
  return cplx{0.5 * fabs(z.im) / a, z.im >= 0.0 ? a : -a};
}
// multiply by i
__host__ __device__ __forceinline__ cplx mul_i(cplx a) { return cplx{-a.im, a.re}; }

// Generic "scalar" helpers so kernels can be written once for real k (double
// coefficients) and complex k (cplx coefficients).
QBX_HD cplx to_c(double a) { return cplx{a, 0.0}; }
QBX_HD cplx to_c(cplx a) { return a; }

// 0.5 * 2^53 + 2^52: adding it rounds a double of magnitude < 2^51 to an
// integer held in the low mantissa bits.
#define QBX_ROUND_MAGIC 6755399441055744.0

// e^{i(z - pi/4)} for real z >= 0 (full accuracy for z < 5e4): Cody-Waite
// reduction by 2 pi/1024, a table of e^{i(2 pi j/1024 - pi/4)} and Taylor
// polynomials on |r| <= pi/1024, where cos r = 1 - t/2 + t^2/24 and
// sin r = r (1 - t/6 + t^2/120), t = r^2, are exact to below 1e-17.
__device__ __forceinline__ cplx expi_shift(double z) {
  const double nd = fma(z, QBX_HK_RED_SCALE, QBX_ROUND_MAGIC);
  const double n = nd - QBX_ROUND_MAGIC;
  const int idx = (int)(__double2loint(nd) & (QBX_HK_NT - 1));
  double r = fma(-n, QBX_HK_RED_HI, z);
  r = fma(-n, QBX_HK_RED_LO, r);
  const double t = r * r;
  const double c = fma(fma(1.0 / 24.0, t, -0.5), t, 1.0);
  const double s = fma(r * t, fma(1.0 / 120.0, t, -1.0 / 6.0), r);
  const double2 tcs = __ldg(reinterpret_cast<const double2*>(&qbx_hk_phase[idx][0]));
  const double tc = tcs.x, ts = tcs.y;
  return cplx{fma(tc, c, -ts * s), fma(tc, s, ts * c)};
}

// From rho^2 > 0: y = rho^{-1/2}, inv = 1/rho and rho.  An FP32 seed
// (about 23 bits) is refined by one step of the third-order iteration for
// x^{-1/4}: y <- y (1 + e/4 + 5 e^2/32), e = 1 - x y^4 (the next term,
// 15 e^3/128, is below 1e-19).
__device__ __forceinline__ void rho_powers(double rho2, double& y, double& inv, double& rho) {
  const float r2f = __double2float_rn(rho2);
  const double y0 = (double)sqrtf(rsqrtf(r2f));
  const double y2 = y0 * y0;
  const double e = fma(-rho2, y2 * y2, 1.0);
  y = fma(y0 * e, fma(5.0 / 32.0, e, 0.25), y0);
  inv = y * y;
  rho = rho2 * inv;
}

// The modulated amplitudes B_n(s) = H_n(z) e^{-i(z - pi/4)}, n = 0, 1, at
// s = |z|^{-1/2} <= QBX_HK_S_MAX from a table laid out as qbx_hk_amp
// ([interval][degree][Re B0, Im B0, Re B1, Im B1], intervals of width
// 2^-QBX_HK_LOG2_PER_UNIT in s, polynomials in u = s - mid): the real-axis
// fits, or a table made for one complex k (z = k rho on its ray).
__device__ __forceinline__ void hk_amp_eval(const double* __restrict__ tab, double s, cplx& B0, cplx& B1) {
  const double y = s + 1.0;
  int i = (int)((__double2hiint(y) >> (20 - QBX_HK_LOG2_PER_UNIT)) & ((1 << QBX_HK_LOG2_PER_UNIT) - 1));
  i = i < QBX_HK_NI ? i : QBX_HK_NI - 1;   // floor(s * 2^LOG2_PER_UNIT)
  const double u = y - __ldg(&qbx_hk_mid1[i]);
  // two 16-byte loads per degree
  const double2* A = reinterpret_cast<const double2*>(tab + (size_t)i * (QBX_HK_DEG + 1) * 4);
  double2 c0 = __ldg(&A[2 * QBX_HK_DEG]), c1 = __ldg(&A[2 * QBX_HK_DEG + 1]);
  double b0r = c0.x, b0i = c0.y, b1r = c1.x, b1i = c1.y;
#pragma unroll
  for (int d = QBX_HK_DEG - 1; d >= 0; --d) {
    c0 = __ldg(&A[2 * d]);
    c1 = __ldg(&A[2 * d + 1]);
    b0r = fma(b0r, u, c0.x);
    b0i = fma(b0i, u, c0.y);
    b1r = fma(b1r, u, c1.x);
    b1i = fma(b1i, u, c1.y);
  }
  B0 = cplx{b0r, b0i};
  B1 = cplx{b1r, b1i};
}

// H0(z), H1(z) for real z > 0, given invz = 1/z and s = z^{-1/2}; with
// SCALED, w H0(z) and w H1(z) (w folded into the phase factor).
template <bool SCALED = false>
__device__ __forceinline__ void hankel01_real(double z, double invz, double s, cplx& h0, cplx& h1,
                                              cplx w = cplx{1.0, 0.0}) {
  if (z >= QBX_HK_ZSPLIT) {
    // B_n(s) = H_n(z) e^{-i(z - pi/4)}: piecewise polynomials in s
    cplx B0, B1;
    hk_amp_eval(&qbx_hk_amp[0][0][0], s, B0, B1);
    cplx e = expi_shift(z);
    if constexpr (SCALED) e = w * e;
    h0 = e * B0;
    h1 = e * B1;
  } else {
    double t = 0.25 * z * z;
    double sj0 = qbx_hk_ser[0][QBX_HK_NSER - 1], sj1 = qbx_hk_ser[1][QBX_HK_NSER - 1];
    double sy0 = qbx_hk_ser[2][QBX_HK_NSER - 1], sy1 = qbx_hk_ser[3][QBX_HK_NSER - 1];
#pragma unroll
    for (int m = QBX_HK_NSER - 2; m >= 0; --m) {
      sj0 = fma(sj0, t, qbx_hk_ser[0][m]);
      sj1 = fma(sj1, t, qbx_hk_ser[1][m]);
      sy0 = fma(sy0, t, qbx_hk_ser[2][m]);
      sy1 = fma(sy1, t, qbx_hk_ser[3][m]);
    }
    double j0 = sj0, j1 = 0.5 * z * sj1;
    double L = 0.63661977236758134308 * log(0.5 * z);  // (2/pi) ln(z/2)
    double y0 = fma(L, j0, sy0);
    double y1 = fma(L, j1, fma(z, sy1, -0.63661977236758134308 * invz));
    h0 = cplx{j0, y0};
    h1 = cplx{j1, y1};
    if constexpr (SCALED) {
      h0 = w * h0;
      h1 = w * h1;
    }
  }
}

// ---------------------------------------------------------------------------
// Complex argument, Im z >= 0, z != 0.
// ---------------------------------------------------------------------------
__host__ __device__ inline void jy01_series_c(cplx z, cplx& j0, cplx& j1, cplx& y0, cplx& y1) {
  // sums of t^m c_m, t = (z/2)^2, with the same series coefficients as the
  // real path, evaluated by Horner in complex arithmetic (21 terms for |z|<=6)
  cplx t = 0.25 * (z * z);
  // coefficients beyond the table: generated on the fly from the ratios
  // c_m / c_{m-1}; here simply by direct accumulation of terms.
  cplx tm = cplx{1.0, 0.0};
  cplx sj0{0, 0}, sj1{0, 0}, sy0{0, 0}, sy1{0, 0};
  double f = 1.0, f1 = 1.0;     // m!, (m+1)!
  double psi1 = -0.57721566490153286061;  // psi(m+1)
  double psi2 = psi1 + 1.0;               // psi(m+2)
  for (int m = 0; m < 24; ++m) {
    if (m > 0) {
      f *= m;
      f1 *= (m + 1);
      psi1 += 1.0 / m;
      psi2 += 1.0 / (m + 1);
      tm = tm * (-1.0 * t);
    }
    double a0 = 1.0 / (f * f), a1 = 1.0 / (f * f1);
    sj0 = sj0 + a0 * tm;
    sj1 = sj1 + a1 * tm;
    sy0 = sy0 + (psi1 * a0) * tm;
    sy1 = sy1 + ((psi1 + psi2) * a1) * tm;
  }
  cplx L = 0.63661977236758134308 * clog_(0.5 * z);
  j0 = sj0;
  j1 = 0.5 * (z * sj1);
  y0 = L * j0 - 0.63661977236758134308 * sy0;
  y1 = -0.63661977236758134308 * cinv(z) + L * j1 - (0.15915494309189533577 * z) * sy1;
}

__host__ __device__ inline void jy01_miller_c(cplx z, cplx& j0, cplx& j1, cplx& y0, cplx& y1) {
  double az = cabs_(z);
  int N = 2 * ((int)(az) + 16);          // even start index
  cplx iz2 = 2.0 * cinv(z);              // 2/z
  cplx fp{0.0, 0.0}, f{1e-30, 0.0};      // f_{n+1}, f_n at n = N
  cplx norm = f;                         // J_0 + 2 sum J_2k (f_N counted once here, doubled below)
  norm = 2.0 * f;
  cplx sY0{0, 0}, sY1{0, 0};             // Neumann sums, see below
  cplx f1{0, 0}, f0{0, 0};
  // Neumann sums: Y0 needs sum_{k>=1} (-1)^k J_2k / k, Y1 needs
  // sum_{k>=1} (-1)^k (J_{2k-1} - J_{2k+1}) / (2k).
  // Walk n = N .. 1 computing f_{n-1} = (2n/z) f_n - f_{n+1}.
  cplx fn1 = fp;  // f_{n+1}
  cplx fn = f;    // f_n
  // contributions of f_N itself
  {
    int n = N;  // even
    int kk = n / 2;
    double sg = (kk & 1) ? -1.0 : 1.0;
    sY0 = sY0 + (sg / kk) * fn;
  }
  for (int n = N; n >= 1; --n) {
    cplx fm = (double)n * (iz2 * fn) - fn1;  // f_{n-1}
    int m = n - 1;
    if (m >= 2 && (m & 1) == 0) {
      int kk = m / 2;
      double sg = (kk & 1) ? -1.0 : 1.0;
      norm = norm + 2.0 * fm;
      sY0 = sY0 + (sg / kk) * fm;
    }
    if (m & 1) {
      // f_m with m = 2k-1 enters term k = (m+1)/2 with +, and term k = (m-1)/2 with -
      int ka = (m + 1) / 2;
      double sga = (ka & 1) ? -1.0 : 1.0;
      sY1 = sY1 + (sga / (2.0 * ka)) * fm;
      int kb = (m - 1) / 2;
      if (kb >= 1) {
        double sgb = (kb & 1) ? -1.0 : 1.0;
        sY1 = sY1 - (sgb / (2.0 * kb)) * fm;
      }
    }
    if (m == 1) f1 = fm;
    if (m == 0) f0 = fm;
    fn1 = fn;
    fn = fm;
  }
  norm = norm + f0;
  cplx inv = cinv(norm);
  j0 = f0 * inv;
  j1 = f1 * inv;
  sY0 = sY0 * inv;
  sY1 = sY1 * inv;
  cplx L = clog_(0.5 * z) + cplx{0.57721566490153286061, 0.0};
  y0 = 0.63661977236758134308 * (L * j0) - 1.27323954473516268615 * sY0;
  y1 = -0.63661977236758134308 * (j0 * cinv(z)) + 0.63661977236758134308 * (L * j1) +
       1.27323954473516268615 * sY1;
}

// DLMF 10.17.5 with the series truncated at its smallest term (|z| > 20):
// the modulated amplitude H_nu(z) e^{-i(z - pi/4)} = (2/(pi z))^{1/2}
// e^{-i nu pi/2} sum_k i^k a_k(nu) / z^k (no exponential: finite for any
// Im z >= 0), and H_nu itself.
__host__ __device__ inline cplx hankel_amp_asym_c(cplx z, int nu) {
  double mu = 4.0 * nu * nu;
  cplx iz = cinv(z);
  cplx sum{1.0, 0.0}, term{1.0, 0.0};
  double prev = 1.0;
  for (int k = 1; k < 60; ++k) {
    double a = (mu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) / (8.0 * k);
    cplx nxt = mul_i(a * (term * iz));
    double mag = cabs_(nxt);
    if (mag >= prev) break;
    term = nxt;
    sum = sum + term;
    prev = mag;
    if (mag < 1e-18) break;
  }
  cplx pre = csqrt_(0.63661977236758134308 * iz);
  if (nu & 1) pre = cplx{pre.im, -pre.re};   // e^{-i pi/2}
  return pre * sum;
}

__host__ __device__ inline cplx hankel_asym_c(cplx z, int nu) {
  return hankel_amp_asym_c(z, nu) * cexp_(mul_i(z - cplx{0.78539816339744830962, 0.0}));
}

// H0, H1 for complex z with |z| < 2 (t = z^2/4, |t| < 1): the ascending
// series of the real path (DLMF 10.2.2, 10.8.1) with its coefficient table
// qbx_hk_ser, by Horner in complex arithmetic.
__device__ __forceinline__ void hankel01_cplx_small(cplx z, cplx& h0, cplx& h1) {
  const cplx t = 0.25 * (z * z);
  auto horner = [&](int row) {
    double re = qbx_hk_ser[row][QBX_HK_NSER - 1], im = 0.0;
#pragma unroll
    for (int m = QBX_HK_NSER - 2; m >= 0; --m) {
      const double nre = fma(re, t.re, fma(-im, t.im, qbx_hk_ser[row][m]));
      im = fma(re, t.im, im * t.re);
      re = nre;
    }
    return cplx{re, im};
  };
  const cplx sj0 = horner(0), sj1 = horner(1), sy0 = horner(2), sy1 = horner(3);
  const cplx L = 0.63661977236758134308 * clog_(0.5 * z);   // (2/pi) ln(z/2)
  const cplx j0 = sj0, j1 = 0.5 * (z * sj1);
  const cplx y0 = L * j0 + sy0;
  const cplx y1 = L * j1 + z * sy1 - 0.63661977236758134308 * cinv(z);
  h0 = j0 + mul_i(y0);
  h1 = j1 + mul_i(y1);
}

__host__ __device__ inline void hankel01_cplx(cplx z, cplx& h0, cplx& h1) {
  double az = cabs_(z);
  if (az > 20.0) {
    h0 = hankel_asym_c(z, 0);
    h1 = hankel_asym_c(z, 1);
    return;
  }
  cplx j0, j1, y0, y1;
  if (az <= 6.0) jy01_series_c(z, j0, j1, y0, y1);
  else jy01_miller_c(z, j0, j1, y0, y1);
  h0 = j0 + mul_i(y0);
  h1 = j1 + mul_i(y1);
}

// ---------------------------------------------------------------------------
// J_0..J_nmax at z (a5: Bessel functions at the expansion target).  Writes
// out[l * stride] for l = 0..nmax.  Scalar T = double (real z) or cplx.
// ---------------------------------------------------------------------------
QBX_HD double sc_mul(double a, double b) { return a * b; }
QBX_HD cplx sc_mul(cplx a, cplx b) { return a * b; }
QBX_HD double sc_inv(double a) { return 1.0 / a; }
QBX_HD cplx sc_inv(cplx a) { return cinv(a); }
QBX_HD double sc_abs(double a) { return fabs(a); }
QBX_HD double sc_abs(cplx a) { return cabs_(a); }
QBX_HD double sc_scale(double s, double a) { return s * a; }
QBX_HD cplx sc_scale(double s, cplx a) { return s * a; }
QBX_HD double sc_add(double a, double b) { return a + b; }
QBX_HD cplx sc_add(cplx a, cplx b) { return a + b; }
QBX_HD double sc_sub(double a, double b) { return a - b; }
QBX_HD cplx sc_sub(cplx a, cplx b) { return a - b; }
QBX_HD void sc_zero(double& a) { a = 0.0; }
QBX_HD void sc_zero(cplx& a) { a = cplx{0.0, 0.0}; }
QBX_HD void sc_set(double& a, double v) { a = v; }
QBX_HD void sc_set(cplx& a, double v) { a = cplx{v, 0.0}; }

template <typename T>
__host__ __device__ void besselj_seq(T z, int nmax, T* out, int stride) {
  double az = sc_abs(z);
  if (az < 0.5) {
    // ascending series J_l = sum_m (-1)^m (z/2)^{2m+l} / (m! (m+l)!)
    T hz = sc_scale(0.5, z);
    T mt = sc_mul(hz, hz);
    mt = sc_scale(-1.0, mt);
    T pl;
    sc_set(pl, 1.0);  // (z/2)^l / l!
    for (int l = 0; l <= nmax; ++l) {
      if (l > 0) pl = sc_scale(1.0 / l, sc_mul(pl, hz));
      T term = pl, sum = pl;
      for (int m = 1; m < 12; ++m) {
        term = sc_scale(1.0 / ((double)m * (double)(m + l)), sc_mul(term, mt));
        sum = sc_add(sum, term);
      }
      out[l * stride] = sum;
    }
    return;
  }
  int extra = (int)az + 15;
  if (extra < 20) extra = 20;
  int N = nmax + 1 + extra;
  if (N & 1) ++N;
  T iz2 = sc_scale(2.0, sc_inv(z));
  T fn1, fn, norm;
  sc_zero(fn1);
  sc_set(fn, 1e-30);
  norm = sc_scale(2.0, fn);  // f_N, N even
  for (int n = N; n >= 1; --n) {
    T fm = sc_sub(sc_scale((double)n, sc_mul(iz2, fn)), fn1);
    int m = n - 1;
    if (m <= nmax) out[m * stride] = fm;
    if ((m & 1) == 0) norm = sc_add(norm, m == 0 ? fm : sc_scale(2.0, fm));
    fn1 = fn;
    fn = fm;
    if (sc_abs(fn) > 1e250) {  // rescale (only for tiny |z| relative to N)
      fn = sc_scale(1e-250, fn);
      fn1 = sc_scale(1e-250, fn1);
      norm = sc_scale(1e-250, norm);
      for (int q = m; q <= nmax; ++q) out[q * stride] = sc_scale(1e-250, out[q * stride]);
    }
  }
  T inv = sc_inv(norm);
  for (int l = 0; l <= nmax; ++l) out[l * stride] = sc_mul(out[l * stride], inv);
}

}  // namespace qbx
