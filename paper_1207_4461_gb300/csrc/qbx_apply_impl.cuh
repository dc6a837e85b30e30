// qbx_apply_impl.cuh -- the storage-free QBX apply (the G_p kernel of Sec. 2,
// eq. qbx-kernel; every source adding to the target sum without stored coefficients, Sec. 3.3),
// for any subset of {S, D, grad S} in one pass over the (centre, source)
// pairs.  Included by qbx_apply_real.cu (real k) and qbx_apply_cplx.cu
// (complex k), which instantiate it.
//
// One thread owns one expansion centre c with its on-surface target x
// (x - c = r e^{i theta_t}); a CTA owns 128 consecutive centres and one
// contiguous range of sources (a split), staged through shared memory in
// tiles of 128.  For a pair with x_s - c = rho e^{i theta_s}, psi = theta_t -
// theta_s, z = k rho, the orders come from H0(z), H1(z) by the upward
// recurrence H_{l+1} = (2l/z) H_l - H_{l-1} and from the Chebyshev recurrence
// for cos(l psi), sin(l psi); the kernels are the truncated Graf sums folded
// over +-l (H_{-l} J_{-l} = H_l J_l):
//   S : J0 H0 + 2 sum_{l=1..p} J_l(kr) H_l cos(l psi)        (eq. graf-addition)
//   D : n_s . grad_{x_s} G_p = sum_{m=0..p} e_m H_m - k a J0 H1,
//       e_m = J_{m+1} C_{m+1} + m J_m V_m,  C_m = 2 k a cos(m psi),
//       V_m = (2/rho)(b sin(m psi) - a cos(m psi)),  a = n_s.e_rho, b = n_s.e_theta
//       (eq. graf-coefficient-dlp with H_l' = H_{l-1} - (l/z) H_l)
//   grad S: e_r k [J0' H0 + 2 sum J_l' H_l cos(l psi)] - e_theta (2/r) sum l J_l H_l sin(l psi)
//       (derivative of the local expansion, Sec. 3.2)
// The pair set-up (distance, H0, H1) and the recurrences are shared by all
// requested operators; each operator adds only its own products.  The factor
// i/4, the fixed-order sum over splits and the jump terms are applied by the
// finishing kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "qbx_device.cuh"
#include "qbx_internal.h"

namespace qbx {

// OPB_C: the combined field D - i eta S of one density (Sec. 4.2), one
// component; formed per pair in the group kernel only
enum { OPB_S = 1, OPB_D = 2, OPB_G = 4, OPB_X = 8, OPB_C = kOpsCombined };

// Near-field-first work order: rank r of a launch takes, for the centre
// block whose middle target is tmid, the source split at offset 0, +1, -1,
// +2, ... (mod nsplit) from the block's home split (the one holding the
// sources of the block's own panels; q_tgt, q_src nodes per panel), so the
// items whose pairs take the slower small-argument Hankel branch run first
// and the last wave holds uniform far-field items.
__device__ __forceinline__ int near_first_split(int rank, int tmid, int q_tgt, int q_src, int split_len,
                                                int nsplit) {
  const int home = min(nsplit - 1, (tmid / q_tgt) * q_src / split_len);
  const int off = (rank & 1) ? (rank + 1) / 2 : -(rank / 2);
  return ((home + off) % nsplit + nsplit) % nsplit;
}

// ---- scalar helpers for T = double (real k) or cplx (complex k) ----------
__device__ __forceinline__ void madd(cplx& acc, double e, cplx h) {
  acc.re = fma(e, h.re, acc.re);
  acc.im = fma(e, h.im, acc.im);
}
__device__ __forceinline__ void madd(cplx& acc, cplx e, cplx h) {
  acc.re = fma(e.re, h.re, acc.re);
  acc.re = fma(-e.im, h.im, acc.re);
  acc.im = fma(e.re, h.im, acc.im);
  acc.im = fma(e.im, h.re, acc.im);
}
// acc -= e h
__device__ __forceinline__ void msub(cplx& acc, double e, cplx h) {
  acc.re = fma(-e, h.re, acc.re);
  acc.im = fma(-e, h.im, acc.im);
}
__device__ __forceinline__ void msub(cplx& acc, cplx e, cplx h) {
  acc.re = fma(-e.re, h.re, acc.re);
  acc.re = fma(e.im, h.im, acc.re);
  acc.im = fma(-e.re, h.im, acc.im);
  acc.im = fma(-e.im, h.re, acc.im);
}
__device__ __forceinline__ cplx smul(double e, cplx h) { return cplx{e * h.re, e * h.im}; }
__device__ __forceinline__ cplx smul(cplx e, cplx h) { return e * h; }
__device__ __forceinline__ double rmul(double a, double c) { return a * c; }
__device__ __forceinline__ cplx rmul(cplx a, double c) { return cplx{a.re * c, a.im * c}; }
__device__ __forceinline__ double fmsub_r(double t, double c, double cp) { return fma(t, c, -cp); }
__device__ __forceinline__ cplx fmsub_r(double t, cplx c, cplx cp) {
  return cplx{fma(t, c.re, -cp.re), fma(t, c.im, -cp.im)};
}
// e = a1 * c + a3 * v  (a1, c of type T; a3 of type T; v real)
__device__ __forceinline__ double dcoef(double a2, double c, double a3, double v) { return fma(a2, c, a3 * v); }
__device__ __forceinline__ cplx dcoef(cplx a2, cplx c, cplx a3, double v) {
  return cplx{fma(a3.re, v, a2.re * c.re - a2.im * c.im), fma(a3.im, v, a2.re * c.im + a2.im * c.re)};
}
// H_{l+1} = s_l H_l - H_{l-1},  s_l = 2l/z
__device__ __forceinline__ cplx hrec(double s, cplx h, cplx hm) {
  return cplx{fma(s, h.re, -hm.re), fma(s, h.im, -hm.im)};
}
__device__ __forceinline__ cplx hrec(cplx s, cplx h, cplx hm) {   // four FMAs
  return cplx{fma(s.re, h.re, fma(-s.im, h.im, -hm.re)), fma(s.re, h.im, fma(s.im, h.re, -hm.im))};
}
__device__ __forceinline__ cplx lin2(double a, cplx x, double b, cplx y) {
  return cplx{fma(a, x.re, b * y.re), fma(a, x.im, b * y.im)};
}
__device__ __forceinline__ cplx lin2(cplx a, cplx x, cplx b, cplx y) { return a * x + b * y; }
__device__ __forceinline__ double sadd(double a, double b) { return a + b; }
__device__ __forceinline__ cplx sadd(cplx a, cplx b) { return a + b; }
// complex k: J_l(k r) and the other coefficient columns are complex
template <typename T> struct IsCplx { static constexpr bool value = false; };
template <> struct IsCplx<cplx> { static constexpr bool value = true; };

// Per-pair distance powers and H0, H1 for real k (fitted path, needs
// rho^{-1/2}) or complex k.
template <typename T> struct KW;
template <> struct KW<double> {
  double k, ik, ik2, ksq;  // k, 1/k, 2/k, k^{-1/2}
  __device__ __forceinline__ void init(double kre, double, const double* = nullptr) {
    k = kre;
    ik = 1.0 / kre;
    ik2 = ik + ik;
    ksq = rsqrt(kre);
  }
  __device__ __forceinline__ double kval() const { return k; }
  __device__ __forceinline__ void geom(double rho2, double& inv, double& rho, double& y) const {
    rho_powers(rho2, y, inv, rho);
  }
  __device__ __forceinline__ void hankel(double rho, double inv, double y, cplx& h0, cplx& h1,
                                         double& twoz) const {
    const double z = k * rho, invz = ik * inv;
    twoz = invz + invz;
    hankel01_real(z, invz, y * ksq, h0, h1);
  }
  // w H0, w H1
  __device__ __forceinline__ void hankel_w(double rho, double inv, double y, cplx w, cplx& h0, cplx& h1,
                                           double& twoz) const {
    const double z = k * rho;
    twoz = ik2 * inv;
    hankel01_real<true>(z, 0.5 * twoz, y * ksq, h0, h1, w);   // 1/z used below z = 2 only
  }
};
// Complex k.  With a ray table (tab: the amplitudes B_n along z = k rho, made
// for this k by launch_hk_table), |z| >= 2 takes the fitted amplitudes times
// e^{i(Re k rho - pi/4)} e^{-Im k rho} and |z| < 2 the tabulated series
// (hankel01_cplx_small); without a table, the series / Miller / asymptotic
// evaluation of hankel01_cplx.
template <> struct KW<cplx> {
  cplx k, c2;                 // k, 2 conj(k) / |k|^2 (2/z = c2 / rho)
  double kisq;                // |k|^{-1/2}
  const double* tab;
  __device__ __forceinline__ void init(double kre, double kim, const double* t = nullptr) {
    k = cplx{kre, kim};
    const double a2 = kre * kre + kim * kim;
    c2 = cplx{2.0 * kre / a2, -2.0 * kim / a2};
    kisq = rsqrt(sqrt(a2));
    tab = t;
  }
  __device__ __forceinline__ cplx kval() const { return k; }
  __device__ __forceinline__ void geom(double rho2, double& inv, double& rho, double& y) const {
    if (tab) {
      rho_powers(rho2, y, inv, rho);
    } else {
      inv = rsqrt(rho2);
      rho = rho2 * inv;
      y = 0.0;
    }
  }
  template <bool SCALED>
  __device__ __forceinline__ void hk(double rho, double inv, double y, cplx w, cplx& h0, cplx& h1,
                                     cplx& twoz) const {
    const double s = y * kisq;   // |z|^{-1/2}
    if (tab && s <= QBX_HK_S_MAX) {
      cplx B0, B1;
      hk_amp_eval(tab, s, B0, B1);
      cplx e = exp(-k.im * rho) * expi_shift(k.re * rho);
      if constexpr (SCALED) e = w * e;
      h0 = e * B0;
      h1 = e * B1;
      twoz = c2 * inv;
      return;
    }
    const cplx z = cplx{k.re * rho, k.im * rho};
    twoz = 2.0 * cinv(z);
    if (tab) {
      hankel01_cplx_small(z, h0, h1);   // |z| < 2
    } else {
      hankel01_cplx(z, h0, h1);
    }
    if constexpr (SCALED) {
      h0 = w * h0;
      h1 = w * h1;
    }
  }
  __device__ __forceinline__ void hankel(double rho, double inv, double y, cplx& h0, cplx& h1, cplx& twoz) const {
    hk<false>(rho, inv, y, cplx{1.0, 0.0}, h0, h1, twoz);
  }
  __device__ __forceinline__ void hankel_w(double rho, double inv, double y, cplx w, cplx& h0, cplx& h1,
                                           cplx& twoz) const {
    hk<true>(rho, inv, y, w, h0, h1, twoz);
  }
};

__host__ __device__ constexpr int popc3(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1); }
// several accumulator sets per rhs: at most 4 rhs per launch
__host__ __device__ constexpr bool multi_op(int m) { return popc3(m) > 1 || (m & 8) != 0; }
// partial-sum components: S -> 1, D -> 1, grad S -> 2, grad_{x_s} S -> 2 (in this order),
// D - i eta S -> 1
__host__ __device__ constexpr int ops_ncomp(int m) {
  return (m & 1) + ((m >> 1) & 1) + 2 * ((m >> 2) & 1) + 2 * ((m >> 3) & 1) + ((m >> 4) & 1);
}
// D (or the source-position gradient) taken from grad S's A and B sums (the
// operator sets with grad S and one of them) reads the true J_{p+1} in the
// J column's last row; every other operator set wants 0 there (orders
// |l| <= p, no J_{p+1} term).
__host__ __device__ constexpr bool keeps_jp1(int m) { return (m & OPB_G) && (m & (OPB_D | OPB_X)); }

// Shared memory layout (bytes): source tile x, y [, nx, ny] ; densities
// [nops][tile][NR] (one slot for the one-density instances) ; per-centre
// coefficient columns of type T, kApplyThreads wide: J (J_l, l = 0..p+1;
// J_{p+1} = 0 unless keeps_jp1),
// then with D or grad S  L (l J_l, l = 0..p), then with grad S
// G (J_{l-1} - J_{l+1}, l = 0..p).
template <int OPS, typename T, int NR, bool ONEW = false>
struct ApplySmem {
  static constexpr int kNops = ONEW ? 1 : popc3(OPS);   // density slots (X shares grad S's)
  static constexpr bool kS = OPS & OPB_S, kD = OPS & OPB_D, kG = OPS & OPB_G;
  static constexpr int kGeo = kD ? 4 : 2;
  static __host__ __device__ size_t tile_bytes() {
    return (size_t)kGeo * kSrcTile * 8 + (size_t)kNops * kSrcTile * NR * 16;
  }
  static __host__ __device__ int nslots() { return 1 + ((kD || kG) ? 1 : 0) + (kG ? 1 : 0); }
  static __host__ __device__ size_t bytes(int p) {
    return tile_bytes() + (size_t)((p + 2) + (nslots() - 1) * (p + 1)) * kApplyThreads * sizeof(T);
  }
};

// The kernel values of one (centre, source) pair for the operator set OPS,
// without the factor i/4: GS (S), K (D), GA and GB (grad S: the e_r and
// e_theta sums before scaling), EX and EY (X: the gradient of the S kernel
// with respect to the source position).  (dx, dy) = x_s - c, (nx, ny) = n_s,
// (ux, uy) = unit vector from c to its target, ir = 1/r; cJ, cL, cG: the
// centre's coefficient columns (J_l, l J_l, J_{l-1} - J_{l+1}) with stride
// STRIDE.
template <int OPS, typename T, int STRIDE>
__device__ __forceinline__ void pair_kernels(const KW<T>& kw, const T kk, const T J0, const T kneg_j0,
                                             const T* cJ, const T* cL, const T* cG, int p, double dx,
                                             double dy, double nx, double ny, double ux, double uy, double ir,
                                             cplx& GS, cplx& K, cplx& GA, cplx& GB, cplx& EX, cplx& EY) {
  constexpr bool kS = OPS & OPB_S, kD = OPS & OPB_D, kG = OPS & OPB_G, kX = OPS & OPB_X;
  static_assert(!(kX && kD), "the source-position gradient is not combined with D");
  constexpr bool kDsum = kD && kG;
  constexpr bool kSums = kDsum || kX;   // D1, D3 (and the sin sum GB)
  constexpr bool kB = kG || kX;         // GB = sum l J_l sin(l psi) H_l
  // ---- a2: pair geometry and H0, H1 ----
  const double rho2 = fma(dx, dx, dy * dy);
  double inv, rho, yq;
  kw.geom(rho2, inv, rho, yq);
  double cs, sn = 0.0, av = 0.0, bv = 0.0;
  if constexpr (kD) {
    // four projections: onto the unit vector e_rho first
    const double ex = dx * inv, ey = dy * inv;
    cs = fma(ux, ex, uy * ey);    // cos psi
    sn = fma(uy, ex, -ux * ey);   // sin psi
    av = fma(nx, ex, ny * ey);    // n_s . e_rho
    bv = fma(ny, ex, -nx * ey);   // n_s . e_theta
  } else {
    cs = fma(ux, dx, uy * dy) * inv;
    if (kB) sn = fma(uy, dx, -ux * dy) * inv;
  }
  cplx H0, H1;
  T twoz;
  kw.hankel(rho, inv, yq, H0, H1, twoz);
  const double tw = 2.0 * cs;

  // ---- order sums; l = 0 terms and recurrence seeds ----
  GS = K = GA = GB = cplx{0.0, 0.0};
  if (kG) GA = smul(cG[0], H0);
  cplx Hm = H0, H = H1;
  T s = twoz;
  double cp = 1.0, cl = cs, sp = 0.0, sl = sn;
  if constexpr (kSums && kG) {
    // D and the source-position gradient from grad S's sums: with
    //   T = J0 H0' + 2 sum_{l=1..p} J_l cos(l psi) H_l',  H_l' = (H_{l-1} - H_{l+1})/2,
    // the sum by parts (below) regroups T by H_m with the coefficients
    // t_{m+1} - t_{m-1}, t_m = J_m cos(m psi); writing cos((m +- 1) psi) =
    // cos(m psi) cos psi -+ sin(m psi) sin psi and J_{m+1} -+ J_{m-1} by the
    // Bessel recurrences (-2 J_m', (2m/kr) J_m) gives
    //   T = -cos psi GA - (2 sin psi/(k r)) GB - E,
    //   E = J_{p+1} cos((p+1) psi) H_p + J_p cos(p psi) H_{p+1},
    // GA = sum_{l>=0} G_l cos(l psi) H_l and GB = sum l J_l sin(l psi) H_l
    // the A and B sums of grad S, E what the truncation at order p leaves
    // (the column holds the true J_{p+1}).  So the orders carry only S, GA
    // and GB, and D = k a T + (2/rho) b GB and R = k T take per-pair factors.
    T tc = rmul(cJ[STRIDE], cl);           // t_1
    for (int l = 1; l <= p; ++l) {
      const int o = l * STRIDE;
      if constexpr (IsCplx<T>::value) {
        const cplx Y = cl * H;                   // cos(l psi) H_l once for S and A
        if (kS) madd(GS, cJ[o], Y);
        madd(GA, cG[o], Y);
      } else {
        if (kS) madd(GS, tc, H);
        madd(GA, rmul(cG[o], cl), H);
      }
      madd(GB, rmul(cL[o], sl), H);
      if (l < p) {
        const double cn = fma(tw, cl, -cp);
        cp = cl;
        cl = cn;
        const double sq = fma(tw, sl, -sp);
        sp = sl;
        sl = sq;
        if constexpr (!IsCplx<T>::value) tc = rmul(cJ[o + STRIDE], cl);   // t_{l+1}
        const cplx Hn = hrec(s, H, Hm);
        Hm = H;
        H = Hn;
        s = sadd(s, twoz);
      }
    }
    // E: at p = 0, J_1 cos psi H_0 + J_0 H_1; else (H, Hm) = (H_p, H_{p-1}), tc = t_p
    cplx E;
    if (p == 0) {
      E = smul(tc, Hm);
      madd(E, J0, H);
    } else {
      if constexpr (IsCplx<T>::value) tc = rmul(cJ[p * STRIDE], cl);
      E = smul(rmul(cJ[(p + 1) * STRIDE], fma(tw, cl, -cp)), H);
      madd(E, tc, hrec(s, H, Hm));
    }
    if (kS) GS = smul(J0, H0) + 2.0 * GS;   // J0 H0 + 2 sum_{l>=1}
    const double sr = 2.0 * sn * ir;        // k (2 sin psi/(k r))
    if (kD) {
      // D = -k a cos psi GA + 2 (b/rho - a sin psi/r) GB - k a E
      const T ka = rmul(kk, av);
      K = smul(rmul(ka, -cs), GA) + (2.0 * bv * inv - av * sr) * GB;
      msub(K, ka, E);
    }
    if (kX) {
      // grad_{x_s} of the S kernel: the D kernel is linear in the normal,
      // n . (e_rho R + e_theta Q), R = k T, Q = (2/rho) D2;
      // e_rho = (dx, dy)/rho, e_theta = (-dy, dx)/rho
      cplx R = smul(rmul(kk, -cs), GA) - sr * GB;
      msub(R, kk, E);
      const cplx Q = (2.0 * inv) * GB;
      EX = (dx * R - dy * Q) * inv;
      EY = (dy * R + dx * Q) * inv;
    }
    return;
  }
  if constexpr (kSums && !kG) {
    // the source-position gradient (without grad S) from the sum by parts
    //   T = J0 H0' + 2 sum_{l=1..p} J_l cos(l psi) H_l'
    //     = t_1 H_0 + sum_{m=1..p-1} (t_{m+1} - t_{m-1}) H_m - t_{p-1} H_p - t_p H_{p+1},
    // t_m = J_m cos(m psi) (t_0 = J_0), H_l' = (H_{l-1} - H_{l+1})/2, H_0' = -H_1
    // and D2 = GB
    T tm = J0;                             // t_{l-1}
    T tc = rmul(cJ[STRIDE], cl);           // t_l
    cplx Ts = cplx{0.0, 0.0};
    madd(Ts, tc, H0);
    if (p == 0) msub(Ts, tm, H1);          // (t_1 = 0: the column holds J_{p+1} = 0)
    for (int l = 1; l <= p; ++l) {
      const int o = l * STRIDE;
      if (kS) madd(GS, tc, H);
      madd(GB, rmul(cL[o], sl), H);
      if (l < p) {
        const double cn = fma(tw, cl, -cp);
        cp = cl;
        cl = cn;
        const double sq = fma(tw, sl, -sp);
        sp = sl;
        sl = sq;
        const T tn = rmul(cJ[o + STRIDE], cl);   // t_{l+1}
        madd(Ts, sc_sub(tn, tm), H);
        tm = tc;
        tc = tn;
        const cplx Hn = hrec(s, H, Hm);
        Hm = H;
        H = Hn;
        s = sadd(s, twoz);
      } else {
        msub(Ts, tm, H);                         // - t_{p-1} H_p
        msub(Ts, tc, hrec(s, H, Hm));            // - t_p H_{p+1}
      }
    }
    if (kS) GS = smul(J0, H0) + 2.0 * GS;   // J0 H0 + 2 sum_{l>=1}
    // grad_{x_s} of the S kernel: the D kernel is linear in the normal,
    // n . (e_rho R + e_theta Q), R = k T, Q = (2/rho) D2;
    // e_rho = (dx, dy)/rho, e_theta = (-dy, dx)/rho
    const cplx R = smul(kk, Ts);
    const cplx Q = (2.0 * inv) * GB;
    EX = (dx * R - dy * Q) * inv;
    EY = (dy * R + dx * Q) * inv;
    return;
  }
  if constexpr (kS && kD) {
    // S with D: J_{m+1} C_{m+1} = 2 k a J_{m+1} cos((m+1) psi) is 2 k a times
    // the next order's S product t_{m+1} = J_{m+1} cos((m+1) psi), so
    // e_m = 2 k a t_{m+1} + m J_m V_m needs no C_m recurrence (the column's
    // J_{p+1} = 0 gives t_{p+1} = 0)
    const T tka = rmul(kk, 2.0 * av);                // 2 k a
    const double i2 = 2.0 * inv;
    T tc = rmul(cJ[STRIDE], cl);                     // t_1
    K = smul(rmul(kneg_j0, av), H1);                 // -k a J0 H1
    madd(K, sc_mul(tka, tc), H0);                    // e_0 = 2 k a t_1
    double Vp = -i2 * av;                            // V_0
    double Vc = i2 * fma(bv, sn, -av * cs);          // V_1
    for (int l = 1; l <= p; ++l) {
      const int o = l * STRIDE;
      madd(GS, tc, H);
      T tn;
      double cn = 0.0;
      if (l < p) {
        cn = fma(tw, cl, -cp);
        tn = rmul(cJ[o + STRIDE], cn);               // t_{l+1}
      } else {
        sc_zero(tn);
      }
      madd(K, dcoef(tka, tn, cL[o], Vc), H);         // e_l = 2 k a t_{l+1} + l J_l V_l
      if (l < p) {
        const cplx Hn = hrec(s, H, Hm);
        Hm = H;
        H = Hn;
        s = sadd(s, twoz);
        cp = cl;
        cl = cn;
        tc = tn;
        const double Vn = fma(tw, Vc, -Vp);
        Vp = Vc;
        Vc = Vn;
      }
    }
    GS = smul(J0, H0) + 2.0 * GS;   // J0 H0 + 2 sum_{l>=1}
    return;
  }
  T Cp, Cc;
  double Vp = 0.0, Vc = 0.0;
  if (kD) {
    const T tka = rmul(kk, 2.0 * av);                // C_0 = 2 k a
    const double i2 = 2.0 * inv;
    Cp = tka;
    Cc = rmul(tka, cs);                              // C_1
    K = smul(rmul(kneg_j0, av), H1);                 // -k a J0 H1
    madd(K, sc_mul(cJ[STRIDE], Cc), H0);             // e_0 = J_1 C_1
    const T Cn = fmsub_r(tw, Cc, Cp);                // C_2
    Cp = Cc;
    Cc = Cn;
    Vp = -i2 * av;                                   // V_0
    Vc = i2 * fma(bv, sn, -av * cs);                 // V_1
  }
  for (int l = 1; l <= p; ++l) {
    const int o = l * STRIDE;
    if (kS) madd(GS, rmul(cJ[o], cl), H);            // J_l cos(l psi)
    if (kD) madd(K, dcoef(cJ[o + STRIDE], Cc, cL[o], Vc), H);
    if (kG) madd(GA, rmul(cG[o], cl), H);
    if (kB) madd(GB, rmul(cL[o], sl), H);
    if (l < p) {
      const cplx Hn = hrec(s, H, Hm);
      Hm = H;
      H = Hn;
      s = sadd(s, twoz);
      const double cn = fma(tw, cl, -cp);
      cp = cl;
      cl = cn;
      if (kB) {
        const double sq = fma(tw, sl, -sp);
        sp = sl;
        sl = sq;
      }
      if (kD) {
        const T Cn = fmsub_r(tw, Cc, Cp);
        Cp = Cc;
        Cc = Cn;
        const double Vn = fma(tw, Vc, -Vp);
        Vp = Vc;
        Vc = Vn;
      }
    }
  }
  if (kS) {  // J0 H0 + 2 sum_{l>=1}
    GS = smul(J0, H0) + 2.0 * GS;
  }
}

// One rhs with one weighted density w = (w sigma)_s for every requested
// operator: the seeds H0, H1 are multiplied by w, so every order sum comes
// out weighted (the sums are linear in H_l) and goes straight into the
// centre's accumulators, without the per-pair kernel values and their
// complex products with w.  The cosine and sine recurrences carry
// C_l = 2 cos(l psi), S_l = 2 sin(l psi) (same recurrence, seeds 2, 2 cos psi
// and 0, 2 sin psi), which puts the factor 2 of the folded sums into the
// recurrence: accS receives the S kernel itself, accA and accB twice the A
// and B sums of pair_kernels.  (ux2, uy2) = 2 (ux, uy), so that
// (ux2, uy2) . (dx, dy) / rho = C_1 directly.
// With grad S requested too, D comes from grad S's A and B sums (the
// identity in pair_kernels, here in the doubled C_l, S_l): with A_m = J_m C_m
// (A_0 = 2 J_0), H_l' = (H_{l-1} - H_{l+1})/2 (H_0' = -H_1) and this pair's
//   PA = gA0 H0 + sum_{l=1..p} G_l C_l H_l,  GB = sum_{l=1..p} l J_l S_l H_l,
//   2 [J0 H0' + sum_{l=1..p} A_l H_l'] = -(C_1/2) PA - (S_1/(k r)) GB - E,
//   E = J_{p+1} C_{p+1} H_p + A_p H_{p+1},
//   D = k a [J0 H0' + sum A_l H_l'] + (b/rho) GB
//     = -(k/2) a [(C_1/2) PA + E] + (b/rho - a S_1/(2 r)) GB,
// so the orders carry S, PA and GB only; the J column holds the true J_{p+1}.
// gA0 = 2 (J_{-1} - J_1)/2 = -2 J_1: the l = 0 coefficient of the doubled A
// sum; khalf = k/2, hir = 1/(2 r).
// D with grad S (and S) for NP sources at once (NP = 1 or 2): the identity
// above, with the pairs' recurrences interleaved order by order so that a
// warp holds NP independent dependency chains and the pairs share the
// column loads of each order.
template <int OPS, typename T, int STRIDE, int NP>
__device__ __forceinline__ void pair_dsum_w(const KW<T>& kw, const T J0, const T gA0, const T khalf, double hir,
                                            const T* cJ, const T* cL, const T* cG, int p, const double* dx,
                                            const double* dy, const double* nx, const double* ny, double ux2,
                                            double uy2, const cplx* w, cplx& accS, cplx& accD, cplx& accA,
                                            cplx& accB) {
  constexpr bool kS = OPS & OPB_S;
  double inv[NP], tw[NP], s1[NP], av[NP], bv[NP], cp[NP], cl[NP], sp[NP], sl[NP];
  cplx H[NP], Hm[NP], PA[NP], GB[NP];
  T s[NP], twoz[NP], Ac[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const double rho2 = fma(dx[q], dx[q], dy[q] * dy[q]);
    double rho, yq;
    kw.geom(rho2, inv[q], rho, yq);
    const double ex = dx[q] * inv[q], ey = dy[q] * inv[q];   // e_rho
    tw[q] = fma(ux2, ex, uy2 * ey);                           // C_1 = 2 cos psi
    s1[q] = fma(uy2, ex, -ux2 * ey);                          // S_1 = 2 sin psi
    av[q] = fma(nx[q], ex, ny[q] * ey);                       // n_s . e_rho
    bv[q] = fma(ny[q], ex, -nx[q] * ey);                      // n_s . e_theta
    kw.hankel_w(rho, inv[q], yq, w[q], Hm[q], H[q], twoz[q]);   // w H0, w H1
    s[q] = twoz[q];
    cp[q] = 2.0;
    cl[q] = tw[q];
    sp[q] = 0.0;
    sl[q] = s1[q];
    if (kS) madd(accS, J0, Hm[q]);
    PA[q] = smul(gA0, Hm[q]);
    GB[q] = cplx{0.0, 0.0};
    Ac[q] = rmul(cJ[STRIDE], cl[q]);   // A_1
  }
  for (int l = 1; l <= p; ++l) {
    const int o = l * STRIDE;
    const T Jl = cJ[o], Gl = cG[o], Ll = cL[o];
    T Jn;
    if (!IsCplx<T>::value && l < p) Jn = cJ[o + STRIDE];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      if constexpr (IsCplx<T>::value) {
        // complex columns: C_l H_l once for S and A (2 + 4 + 4 against 2 x (2 + 4))
        const cplx Y = cl[q] * H[q];
        if (kS) madd(accS, Jl, Y);
        madd(PA[q], Gl, Y);
      } else {
        if (kS) madd(accS, Ac[q], H[q]);
        madd(PA[q], rmul(Gl, cl[q]), H[q]);
      }
      madd(GB[q], rmul(Ll, sl[q]), H[q]);
      if (l < p) {
        const double cn = fma(tw[q], cl[q], -cp[q]);
        cp[q] = cl[q];
        cl[q] = cn;
        const double sq = fma(tw[q], sl[q], -sp[q]);
        sp[q] = sl[q];
        sl[q] = sq;
        if constexpr (!IsCplx<T>::value) Ac[q] = rmul(Jn, cn);   // A_{l+1}
        const cplx Hn = hrec(s[q], H[q], Hm[q]);
        Hm[q] = H[q];
        H[q] = Hn;
        s[q] = sadd(s[q], twoz[q]);
      }
    }
  }
  const T Jp = cJ[p * STRIDE], Jp1 = cJ[(p + 1) * STRIDE];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    // E: at p = 0, A_1 H_0 + 2 J_0 H_1; else (H, Hm) = (H_p, H_{p-1}), A_p = J_p C_p
    cplx E;
    if (p == 0) {
      E = smul(Ac[q], Hm[q]);
      madd(E, rmul(J0, 2.0), H[q]);
    } else {
      const T Ap = IsCplx<T>::value ? rmul(Jp, cl[q]) : Ac[q];
      E = smul(rmul(Jp1, fma(tw[q], cl[q], -cp[q])), H[q]);
      madd(E, Ap, hrec(s[q], H[q], Hm[q]));
    }
    madd(E, 0.5 * tw[q], PA[q]);
    msub(accD, rmul(khalf, av[q]), E);
    madd(accD, fma(-av[q] * s1[q], hir, bv[q] * inv[q]), GB[q]);
    accA = accA + PA[q];
    accB = accB + GB[q];
  }
}

template <int OPS, typename T, int STRIDE>
__device__ __forceinline__ void pair_accumulate_w(const KW<T>& kw, const T kk, const T J0, const T kneg_j0,
                                                  const T gA0, const T khalf, double hir, const T* cJ,
                                                  const T* cL, const T* cG, int p, double dx, double dy,
                                                  double nx, double ny, double ux2, double uy2, cplx w,
                                                  cplx& accS, cplx& accD, cplx& accA, cplx& accB) {
  constexpr bool kS = OPS & OPB_S, kD = OPS & OPB_D, kG = OPS & OPB_G;
  static_assert(!(OPS & OPB_X), "the source-position gradient is not formed here");
  if constexpr (kD && kG) {
    pair_dsum_w<OPS, T, STRIDE, 1>(kw, J0, gA0, khalf, hir, cJ, cL, cG, p, &dx, &dy, &nx, &ny, ux2, uy2, &w, accS,
                                   accD, accA, accB);
    return;
  }
  const double rho2 = fma(dx, dx, dy * dy);
  double inv, rho, yq;
  kw.geom(rho2, inv, rho, yq);
  double tw, s1 = 0.0, av = 0.0, bv = 0.0;   // C_1 = 2 cos psi, S_1 = 2 sin psi
  if constexpr (kD) {
    // four projections: onto the unit vector e_rho first
    const double ex = dx * inv, ey = dy * inv;
    tw = fma(ux2, ex, uy2 * ey);
    s1 = fma(uy2, ex, -ux2 * ey);
    av = fma(nx, ex, ny * ey);    // n_s . e_rho
    bv = fma(ny, ex, -nx * ey);   // n_s . e_theta
  } else {
    tw = fma(ux2, dx, uy2 * dy) * inv;
    if (kG) s1 = fma(uy2, dx, -ux2 * dy) * inv;
  }
  cplx H0, H1;
  T twoz;
  kw.hankel_w(rho, inv, yq, w, H0, H1, twoz);   // w H0, w H1
  cplx Hm = H0, H = H1;
  T s = twoz;
  double cp = 2.0, cl = tw, sp = 0.0, sl = s1;  // C_l, S_l at l = 0, 1
  // ---- l = 0 terms and recurrence seeds ----
  if (kS) madd(accS, J0, H0);
  if (kG) madd(accA, gA0, H0);
  T Cp, Cc;
  double Vp = 0.0, Vc = 0.0;
  if (kD) {
    const T ka = rmul(kk, av);
    Cp = rmul(ka, 2.0);                              // C_0 = 2 k a
    Cc = rmul(ka, tw);                               // C_1 = 2 k a cos psi
    madd(accD, rmul(kneg_j0, av), H1);               // -k a J0 H1
    madd(accD, sc_mul(cJ[STRIDE], Cc), H0);          // e_0 = J_1 C_1
    const T Cn = fmsub_r(tw, Cc, Cp);                // C_2
    Cp = Cc;
    Cc = Cn;
    Vp = -2.0 * inv * av;                            // V_0
    Vc = inv * fma(bv, sl, -av * tw);                // V_1 = (2/rho)(b sin psi - a cos psi)
  }
  for (int l = 1; l <= p; ++l) {
    const int o = l * STRIDE;
    if (kS) madd(accS, rmul(cJ[o], cl), H);          // 2 J_l cos(l psi)
    if (kD) madd(accD, dcoef(cJ[o + STRIDE], Cc, cL[o], Vc), H);
    if (kG) {
      madd(accA, rmul(cG[o], cl), H);
      madd(accB, rmul(cL[o], sl), H);
    }
    if (l < p) {
      const cplx Hn = hrec(s, H, Hm);
      Hm = H;
      H = Hn;
      s = sadd(s, twoz);
      const double cn = fma(tw, cl, -cp);
      cp = cl;
      cl = cn;
      if (kG) {
        const double sq = fma(tw, sl, -sp);
        sp = sl;
        sl = sq;
      }
      if (kD) {
        const T Cn = fmsub_r(tw, Cc, Cp);
        Cp = Cc;
        Cc = Cn;
        const double Vn = fma(tw, Vc, -Vp);
        Vp = Vc;
        Vc = Vn;
      }
    }
  }
}

// Near-only QBX (a source far from the centre goes through the smooth rule
// at the target instead of the expansion): the raw kernel values of one
// (target, source) pair in the same form as pair_kernels returns them, with
// (ex, ey) = x_t - x_s, d = |x_t - x_s|:
//   S: H0(kd);  D: k H1(kd) (e . n_s)/d;
//   grad S: -k H1(kd) e/d, returned as GA = (grad . e_r)/k = -H1 (e . e_r)/d and
//   GB = -(grad . e_theta) r/2 = k H1 (e . e_theta) r/(2d), which the
//   epilogue maps back through k GA e_r - (2/r) GB e_theta.
template <int OPS, typename T>
__device__ __forceinline__ void pair_direct(const KW<T>& kw, const T kk, double ex, double ey, double nx, double ny,
                                            double ux, double uy, double r, cplx& GS, cplx& K, cplx& GA,
                                            cplx& GB) {
  constexpr bool kS = OPS & OPB_S, kD = OPS & OPB_D, kG = OPS & OPB_G;
  const double d2 = fma(ex, ex, ey * ey);
  double inv, d, yq;
  kw.geom(d2, inv, d, yq);
  cplx H0, H1;
  T twoz;
  kw.hankel(d, inv, yq, H0, H1, twoz);
  if (kS) GS = H0;
  if (kD) K = smul(rmul(kk, fma(ex, nx, ey * ny) * inv), H1);
  if (kG) {
    GA = H1 * (-fma(ex, ux, ey * uy) * inv);
    GB = smul(rmul(kk, 0.5 * r * fma(ex, -uy, ey * ux) * inv), H1);
  }
}

// pair_direct for the one-density instances: w H0(kd), w H1(kd) and the
// raw kernels added straight into the accumulators (A and B doubled, as in
// pair_accumulate_w).
template <int OPS, typename T>
__device__ __forceinline__ void pair_direct_w(const KW<T>& kw, const T kk, double ex, double ey, double nx,
                                              double ny, double ux, double uy, double r, cplx w, cplx& accS,
                                              cplx& accD, cplx& accA, cplx& accB) {
  constexpr bool kS = OPS & OPB_S, kD = OPS & OPB_D, kG = OPS & OPB_G;
  const double d2 = fma(ex, ex, ey * ey);
  double inv, d, yq;
  kw.geom(d2, inv, d, yq);
  cplx H0, H1;
  T twoz;
  kw.hankel_w(d, inv, yq, w, H0, H1, twoz);
  if (kS) accS = accS + H0;
  if (kD) madd(accD, rmul(kk, fma(ex, nx, ey * ny) * inv), H1);
  if (kG) {
    madd(accA, -2.0 * fma(ex, ux, ey * uy) * inv, H1);
    madd(accB, rmul(kk, r * fma(ex, -uy, ey * ux) * inv), H1);
  }
}

// The storage-free apply (a2-a6 fused): one thread per centre, a CTA of
// kApplyThreads centres against one split of the sources, staged through
// shared memory in tiles of kSrcTile; each pair's order sums go straight
// into the centre's accumulators (split partial sums, finished by
// k_apply_finish).  D with grad S comes from grad S's own sums and two end
// terms (pair_kernels, pair_dsum_w), otherwise from the coefficients e_m
// with the C_m, V_m recurrences (or S's next product, with S).
// LOCAL: the near-only variant (a separate instance, so that the global
// apply carries no per-pair test).  ONEW: one rhs and one density for all
// operators, accumulated through weighted seeds (pair_accumulate_w,
// pair_direct_w).
// Register budget: the two-source D-with-grad-S instances keep three CTAs
// per SM (up to 168 registers), the other one-density instances four.
template <int OPS, bool LOCAL, bool ONEW>
__host__ __device__ constexpr int fused_min_ctas() {
  return !ONEW ? 1 : ((OPS & OPB_D) && (OPS & OPB_G) && !LOCAL) ? 3 : 4;
}

template <int OPS, typename T, int NR, bool LOCAL = false, bool ONEW = false>
__global__ void __launch_bounds__(kApplyThreads, (fused_min_ctas<OPS, LOCAL, ONEW>()))
k_apply_fused(ApplyArgs a) {
  using L = ApplySmem<OPS, T, NR, ONEW>;
  constexpr bool kS = L::kS, kD = L::kD, kG = L::kG, kX = OPS & OPB_X;
  static_assert(!kX || kG, "X is formed with grad S and shares its density");
  static_assert(!ONEW || (NR == 1 && !kX), "one-density instances: one rhs, no X");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s_x = reinterpret_cast<double*>(smem_raw);
  double* s_y = s_x + kSrcTile;
  double* s_nx = s_y + kSrcTile;            // only with D
  double* s_ny = s_nx + kSrcTile;
  cplx* s_wd = reinterpret_cast<cplx*>(smem_raw + (size_t)L::kGeo * kSrcTile * 8);  // [nops][tile][NR]
  T* slot = reinterpret_cast<T*>(smem_raw + L::tile_bytes());
  const int p = a.p;
  T* sJ = slot;                                                   // J_l, p + 2 rows
  T* sL = slot + (p + 2) * kApplyThreads;                         // l J_l, p + 1 rows
  T* sG = sL + ((kD || kG) ? (p + 1) * kApplyThreads : 0);        // J_{l-1} - J_{l+1}, p + 1 rows

  const int tid = threadIdx.x;
  // work item (centre block, source split): rank r = blockIdx.x / nblk;
  // near-field splits first when the grids' node counts are given
  const int nblk = (a.n_ctr + kApplyThreads - 1) / kApplyThreads;
  const int cblk = (int)(blockIdx.x % (unsigned)nblk), rank = (int)(blockIdx.x / (unsigned)nblk);
  const int split = a.near_q_tgt > 0 ? near_first_split(rank, (cblk * kApplyThreads + kApplyThreads / 2) % a.n_tgt,
                                                        a.near_q_tgt, a.near_q_src, a.src_per_split, a.nsplit)
                                     : rank;
  const int c = cblk * kApplyThreads + tid;
  const bool active = c < a.n_ctr;
  const int cc = active ? c : a.n_ctr - 1;

  // ---- per-centre set-up: target direction, J_l(k r) (a5) ----
  const double cx = a.cx[cc], cy = a.cy[cc];
  const int t = cc % a.n_tgt;
  double ux = a.tx[t] - cx, uy = a.ty[t] - cy;
  const double r = hypot(ux, uy);
  const double ir = 1.0 / r;
  ux *= ir;
  uy *= ir;
  // near-only QBX: sources at |x_s - c| >= eta r take the smooth rule
  const double lim2 = (!LOCAL || kX || !(a.eta2 > 0.0)) ? INFINITY : a.eta2 * r * r;
  KW<T> kw;
  kw.init(a.kre, a.kim, a.hk_tab);
  const T kk = kw.kval();
  T* colJ = sJ + tid;
  T* colL = sL + tid;
  T* colG = sG + tid;
  besselj_seq<T>(rmul(kk, r), p + 1, colJ, kApplyThreads);
  const T J0 = colJ[0];
  for (int l = 0; l <= p; ++l) {
    const T jl = colJ[l * kApplyThreads];
    if (kD || kG) colL[l * kApplyThreads] = rmul(jl, (double)l);
    if (kG) {
      const T jn = colJ[(l + 1) * kApplyThreads];
      const T jp = (l == 0) ? jn : colJ[(l - 1) * kApplyThreads];
      colG[l * kApplyThreads] = (l == 0) ? rmul(jn, -1.0) : sc_sub(jp, jn);
    }
  }
  if (!keeps_jp1(OPS)) {
    T z0;
    sc_zero(z0);
    colJ[(p + 1) * kApplyThreads] = z0;  // e_p has no J_{p+1} term (orders |l| <= p)
  }
  const T kneg_j0 = rmul(sc_mul(kk, J0), -1.0);  // -k J0 (D)
  T gA0;
  if (kG) gA0 = rmul(colG[0], 2.0);                // -2 J_1 (one-density grad S)
  const T khalf = rmul(kk, 0.5);
  const double ux2 = ux + ux, uy2 = uy + uy;

  cplx accS[NR], accD[NR], accA[NR], accB[NR], accX[NR], accY[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) accS[q] = accD[q] = accA[q] = accB[q] = accX[q] = accY[q] = cplx{0.0, 0.0};

  const int s_begin = split * a.src_per_split;
  const int s_end = min(a.src.n, s_begin + a.src_per_split);
  const cplx* wdp[3] = {reinterpret_cast<const cplx*>(a.wd[0]), reinterpret_cast<const cplx*>(a.wd[1]),
                        reinterpret_cast<const cplx*>(a.wd[2])};

  for (int base = s_begin; base < s_end; base += kSrcTile) {
    const int nt = min(kSrcTile, s_end - base);
    __syncthreads();
    for (int i = tid; i < nt; i += kApplyThreads) {
      s_x[i] = a.src.x[base + i];
      s_y[i] = a.src.y[base + i];
      if (kD) {
        s_nx[i] = a.src.nx[base + i];
        s_ny[i] = a.src.ny[base + i];
      }
    }
    {
      int slotn = 0;
#pragma unroll
      for (int o = 0; o < 3; ++o) {
        if (!(OPS & (1 << o))) continue;
        if (ONEW && slotn > 0) break;   // one density for all operators
        const cplx* w = wdp[o];
        cplx* dst = s_wd + (size_t)slotn * kSrcTile * NR;
        for (int i = tid; i < nt * NR; i += kApplyThreads) {
          const int s = i / NR, rr = i - s * NR;
          dst[i] = (rr < a.nr) ? w[(size_t)(base + s) * a.nrhs + a.rhs0 + rr] : cplx{0.0, 0.0};
        }
        ++slotn;
      }
    }
    __syncthreads();
    if (!active) continue;

    const T* cJ = colJ;
    const T* cL = colL;
    const T* cG = colG;

    int j0 = 0;
    if constexpr (ONEW && kD && kG && !LOCAL) {
      // two sources per step: two independent recurrence chains per thread
      for (; j0 + 2 <= nt; j0 += 2) {
        double dx2[2], dy2[2], nx2[2], ny2[2];
        cplx w2[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          dx2[q] = s_x[j0 + q] - cx;
          dy2[q] = s_y[j0 + q] - cy;
          nx2[q] = s_nx[j0 + q];
          ny2[q] = s_ny[j0 + q];
          w2[q] = s_wd[j0 + q];
        }
        pair_dsum_w<OPS, T, kApplyThreads, 2>(kw, J0, gA0, khalf, 0.5 * ir, cJ, cL, cG, p, dx2, dy2, nx2, ny2,
                                              ux2, uy2, w2, accS[0], accD[0], accA[0], accB[0]);
      }
    }
    for (int j = j0; j < nt; ++j) {
      const double dx = s_x[j] - cx, dy = s_y[j] - cy;
      double nx = 0.0, ny = 0.0;
      if (kD) {
        nx = s_nx[j];
        ny = s_ny[j];
      }
      if constexpr (ONEW) {
        if (LOCAL && fma(dx, dx, dy * dy) >= lim2) {   // near-only QBX: a distant source
          pair_direct_w<OPS, T>(kw, kk, r * ux - dx, r * uy - dy, nx, ny, ux, uy, r, s_wd[j], accS[0], accD[0],
                                accA[0], accB[0]);
        } else {
          pair_accumulate_w<OPS, T, kApplyThreads>(kw, kk, J0, kneg_j0, gA0, khalf, 0.5 * ir, cJ, cL, cG, p, dx, dy,
                                                    nx, ny, ux2, uy2, s_wd[j], accS[0], accD[0], accA[0],
                                                    accB[0]);
        }
        continue;
      }
      cplx GS, K, GA, GB, EX, EY;
      if (LOCAL && fma(dx, dx, dy * dy) >= lim2) {   // near-only QBX: a distant source
        pair_direct<OPS, T>(kw, kk, r * ux - dx, r * uy - dy, nx, ny, ux, uy, r, GS, K, GA, GB);
      } else {
        pair_kernels<OPS, T, kApplyThreads>(kw, kk, J0, kneg_j0, cJ, cL, cG, p, dx, dy, nx, ny, ux, uy, ir, GS,
                                             K, GA, GB, EX, EY);
      }
      // ---- weighted densities ----
      int slotn = 0;
      if (kS) {
        const cplx* w = s_wd + ((size_t)slotn * kSrcTile + j) * NR;
#pragma unroll
        for (int q = 0; q < NR; ++q) cfma(accS[q], w[q], GS);
        ++slotn;
      }
      if (kD) {
        const cplx* w = s_wd + ((size_t)slotn * kSrcTile + j) * NR;
#pragma unroll
        for (int q = 0; q < NR; ++q) cfma(accD[q], w[q], K);
        ++slotn;
      }
      if (kG) {
        const cplx* w = s_wd + ((size_t)slotn * kSrcTile + j) * NR;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          cfma(accA[q], w[q], GA);
          cfma(accB[q], w[q], GB);
          if (kX) {
            cfma(accX[q], w[q], EX);
            cfma(accY[q], w[q], EY);
          }
        }
      }
    }
  }
  if (!active) return;
  cplx* part = reinterpret_cast<cplx*>(a.part);
  constexpr int ncomp = ops_ncomp(OPS);
  const size_t row = ((size_t)split * a.n_ctr + c) * ncomp;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    if (q >= a.nr) break;
    int comp = 0;
    if (kS) part[(row + comp++) * a.nrhs + a.rhs0 + q] = accS[q];
    if (kD) part[(row + comp++) * a.nrhs + a.rhs0 + q] = accD[q];
    if (kG) {
      // grad = e_r k A - e_theta (1/r) B, B = 2 sum l J_l H_l sin: e_r = (ux, uy), e_theta = (-uy, ux)
      // (the one-density accumulators hold 2 A and 2 B)
      const cplx kA = smul(kk, ONEW ? 0.5 * accA[q] : accA[q]);
      const cplx Bi = accB[q] * ((ONEW ? 1.0 : 2.0) * ir);
      part[(row + comp++) * a.nrhs + a.rhs0 + q] = kA * ux + Bi * uy;
      part[(row + comp++) * a.nrhs + a.rhs0 + q] = kA * uy - Bi * ux;
    }
    if (kX) {
      part[(row + comp++) * a.nrhs + a.rhs0 + q] = accX[q];
      part[(row + comp++) * a.nrhs + a.rhs0 + q] = accY[q];
    }
  }
}

// Percentage of the largest shared-memory carve-out (228 KB) that holds n
// CTAs of smem bytes each (plus the 1 KB CUDA reserves per CTA),
// rounded up; 0 when nothing is to be set.
static inline int carveout_percent(int n, size_t smem) {
  if (n < 1) return 0;
  const size_t need = (size_t)n * (smem + 1024), full = (size_t)228 * 1024;
  if (need >= full) return 0;
  return (int)((need * 100 + full - 1) / full);
}

// Resident CTAs per SM of a one-density instance under the largest
// carve-out (the preference a previous launch left is reset first).
template <typename K>
static cudaError_t onew_occupancy(K kern, size_t smem, int* n) {
  *n = 0;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, kern, kApplyThreads, smem);
  return e;
}

template <int OPS, typename T, int NR, bool LOCAL, bool ONEW = false>
static cudaError_t launch_apply_t(const ApplyArgs& a, cudaStream_t st) {
  const size_t smem = ApplySmem<OPS, T, NR, ONEW>::bytes(a.p);
  auto kern = k_apply_fused<OPS, T, NR, LOCAL, ONEW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if constexpr (ONEW) {
    // the smallest shared-memory carve-out that holds the resident CTAs,
    // which leaves the rest of the SM's 256 KB to L1 (the Hankel tables)
    int n = 0;
    e = onew_occupancy(kern, smem, &n);
    if (e != cudaSuccess) return e;
    const int pct = carveout_percent(n, smem);
    if (pct > 0) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
      if (e != cudaSuccess) return e;
    }
  }
  const unsigned grid = (unsigned)((a.n_ctr + kApplyThreads - 1) / kApplyThreads) * (unsigned)a.nsplit;
  kern<<<grid, kApplyThreads, smem, st>>>(a);
  return cudaGetLastError();
}

// rhs per pass: single operator up to 8, several operators (or the
// near-only variant) up to 4
template <int OPS, typename T, bool LOCAL>
static cudaError_t launch_apply_nr(const ApplyArgs& a, cudaStream_t st) {
  if constexpr (!(OPS & OPB_X)) {
    if (a.nr <= 1 && a.one_w) return launch_apply_t<OPS, T, 1, LOCAL, true>(a, st);
  }
  if (a.nr <= 1) return launch_apply_t<OPS, T, 1, LOCAL>(a, st);
  if constexpr (multi_op(OPS) || LOCAL) {
    return launch_apply_t<OPS, T, 4, LOCAL>(a, st);
  } else {
    if (a.nr <= 4) return launch_apply_t<OPS, T, 4, LOCAL>(a, st);
    return launch_apply_t<OPS, T, 8, LOCAL>(a, st);
  }
}

template <typename T>
static size_t apply_smem_t(int ops, int p, int nr) {
  const int nr_t = nr <= 1 ? 1 : (nr <= 4 || multi_op(ops) ? 4 : 8);
#define QBX_SM(O)                                                                   \
  case O:                                                                           \
    return nr_t == 1 ? ApplySmem<O, T, 1>::bytes(p)                                 \
                     : (nr_t == 4 ? ApplySmem<O, T, 4>::bytes(p) : ApplySmem<O, T, 8>::bytes(p));
  // (ApplySmem is a size calculator only; no kernel is instantiated here)
  switch (ops) {
    QBX_SM(1) QBX_SM(2) QBX_SM(3) QBX_SM(4) QBX_SM(5) QBX_SM(6) QBX_SM(7) QBX_SM(12)
    default: return 0;
  }
#undef QBX_SM
}

// CTAs of the kernel instance that one SM holds at once.
template <int OPS, typename T, bool LOCAL>
static int occupancy_t(int p, int nr, bool one_w) {
  // (the shared-memory opt-in must be set before the query when above 48 KB)
  auto occ = [](auto kern, size_t smem) {
    int n = 0;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kApplyThreads, smem);
    return n;
  };
  if constexpr (!(OPS & OPB_X)) {
    if (nr <= 1 && one_w) {
      int n = 0;
      onew_occupancy(k_apply_fused<OPS, T, 1, LOCAL, true>, ApplySmem<OPS, T, 1, true>::bytes(p), &n);
      return n;
    }
  }
  if (nr <= 1) return occ(k_apply_fused<OPS, T, 1, LOCAL>, ApplySmem<OPS, T, 1>::bytes(p));
  if constexpr (multi_op(OPS) || LOCAL) {
    return occ(k_apply_fused<OPS, T, 4, LOCAL>, ApplySmem<OPS, T, 4>::bytes(p));
  } else {
    if (nr <= 4) return occ(k_apply_fused<OPS, T, 4, LOCAL>, ApplySmem<OPS, T, 4>::bytes(p));
    return occ(k_apply_fused<OPS, T, 8, LOCAL>, ApplySmem<OPS, T, 8>::bytes(p));
  }
}

template <typename T, bool LOCAL = false>
static int apply_occupancy_t(int ops, int p, int nr, bool one_w = false) {
  switch (ops) {
    case OPB_S: return occupancy_t<OPB_S, T, LOCAL>(p, nr, one_w);
    case OPB_D: return occupancy_t<OPB_D, T, LOCAL>(p, nr, one_w);
    case OPB_G: return occupancy_t<OPB_G, T, LOCAL>(p, nr, one_w);
    case OPB_S | OPB_D: return occupancy_t<OPB_S | OPB_D, T, LOCAL>(p, nr, one_w);
    case OPB_S | OPB_G: return occupancy_t<OPB_S | OPB_G, T, LOCAL>(p, nr, one_w);
    case OPB_D | OPB_G: return occupancy_t<OPB_D | OPB_G, T, LOCAL>(p, nr, one_w);
    case OPB_S | OPB_D | OPB_G: return occupancy_t<OPB_S | OPB_D | OPB_G, T, LOCAL>(p, nr, one_w);
    case OPB_G | OPB_X:
      if constexpr (!LOCAL) return occupancy_t<OPB_G | OPB_X, T, false>(p, nr, false);
      return 0;
    default: return 0;
  }
}

template <typename T, bool LOCAL = false>
static cudaError_t launch_apply_ops(const ApplyArgs& a, cudaStream_t st) {
  switch (a.ops) {
    case OPB_S: return launch_apply_nr<OPB_S, T, LOCAL>(a, st);
    case OPB_D: return launch_apply_nr<OPB_D, T, LOCAL>(a, st);
    case OPB_G: return launch_apply_nr<OPB_G, T, LOCAL>(a, st);
    case OPB_S | OPB_D: return launch_apply_nr<OPB_S | OPB_D, T, LOCAL>(a, st);
    case OPB_S | OPB_G: return launch_apply_nr<OPB_S | OPB_G, T, LOCAL>(a, st);
    case OPB_D | OPB_G: return launch_apply_nr<OPB_D | OPB_G, T, LOCAL>(a, st);
    case OPB_S | OPB_D | OPB_G: return launch_apply_nr<OPB_S | OPB_D | OPB_G, T, LOCAL>(a, st);
    case OPB_G | OPB_X:
      if constexpr (!LOCAL) return launch_apply_nr<OPB_G | OPB_X, T, false>(a, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qbx
