// qbx_apply.cu -- the storage-free QBX apply (the G_p kernel of Sec. 2, eq.
// qbx-kernel; "each source adds its contribution directly", Sec. 3.3) and the
// plain-quadrature far-target sum.
//
// One thread owns one expansion centre c with its on-surface target x
// (x - c = r e^{i theta_t}); a CTA owns 128 consecutive centres and one
// contiguous range of sources (a split), staged through shared memory in
// tiles of 128.  For each (centre, source) pair with x_s - c = rho e^{i theta_s},
// psi = theta_t - theta_s, z = k rho, the kernel forms from H0(z), H1(z) the
// orders H_l by the upward recurrence H_{l+1} = (2l/z) H_l - H_{l-1} and the
// Chebyshev recurrence for cos(l psi), sin(l psi), and accumulates
//   S : G   = J0 H0 + 2 sum_{l=1..p} J_l(kr) H_l cos(l psi)
//       (Graf's theorem truncated at |l| <= p, eq. graf-addition; summed over
//        +-l using H_{-l} J_{-l} = H_l J_l)
//   D : n_s . grad_{x_s} G_p
//       = k a [J0 H0' + 2 sum J_l H_l' cos(l psi)] + (2 b / rho) sum l J_l H_l sin(l psi)
//       with a = n_s . e_rho, b = n_s . e_theta at the source (eq. graf-coefficient-dlp)
//   grad S: grad_x G_p = e_r k [J0' H0 + 2 sum J_l' H_l cos] - e_theta (2/r) sum l J_l H_l sin
//       (derivative of the local expansion at the target, Sec. 3.2)
// times the oversampled, weighted density w_s sigma_s of every right-hand
// side.  The factor i/4, the sum over splits (fixed order) and the jump terms
// are applied by the finishing kernel.  Both sides of these identities are
// exact rearrangements of the truncated expansion, so the result equals
// forming alpha_l (eq. graf-coefficient) and evaluating eq. local-exp.
#include <cuda_runtime.h>
#include <stdint.h>
#include "qbx_device.cuh"
#include "qbx_internal.h"

namespace qbx {

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
__device__ __forceinline__ cplx smul(double e, cplx h) { return cplx{e * h.re, e * h.im}; }
__device__ __forceinline__ cplx smul(cplx e, cplx h) { return e * h; }
__device__ __forceinline__ double rmul(double a, double c) { return a * c; }
__device__ __forceinline__ cplx rmul(cplx a, double c) { return cplx{a.re * c, a.im * c}; }
__device__ __forceinline__ double fmsub_r(double t, double c, double cp) { return fma(t, c, -cp); }
__device__ __forceinline__ cplx fmsub_r(double t, cplx c, cplx cp) {
  return cplx{fma(t, c.re, -cp.re), fma(t, c.im, -cp.im)};
}
__device__ __forceinline__ double fmadd2(double a, double x, double b, double y) { return fma(a, x, b * y); }
__device__ __forceinline__ cplx fmadd2(double a, cplx x, double b, double y) {
  return cplx{fma(a, x.re, b * y), a * x.im};
}
__device__ __forceinline__ cplx fmadd2(cplx a, cplx x, cplx b, double y) { return a * x + rmul(b, y); }

template <typename T> struct KW;
template <> struct KW<double> {
  // z = k rho, 2/z, and H0/H1 for real k
  double k, ik;
  __device__ __forceinline__ void init(double kre, double) { k = kre; ik = 1.0 / kre; }
  __device__ __forceinline__ void hankel(double rho, double inv, cplx& h0, cplx& h1, double& twoz) const {
    double z = k * rho, invz = ik * inv;
    twoz = 2.0 * invz;
    hankel01_real(z, invz, h0, h1);
  }
};
template <> struct KW<cplx> {
  cplx k;
  __device__ __forceinline__ void init(double kre, double kim) { k = cplx{kre, kim}; }
  __device__ __forceinline__ void hankel(double rho, double inv, cplx& h0, cplx& h1, cplx& twoz) const {
    cplx z = cplx{k.re * rho, k.im * rho};
    twoz = 2.0 * cinv(z);
    hankel01_cplx(z, h0, h1);
  }
};

// H_{l+1} = s_l H_l - H_{l-1},  s_l = 2l/z
__device__ __forceinline__ cplx hrec(double s, cplx h, cplx hm) {
  return cplx{fma(s, h.re, -hm.re), fma(s, h.im, -hm.im)};
}
__device__ __forceinline__ cplx hrec(cplx s, cplx h, cplx hm) { return s * h - hm; }
__device__ __forceinline__ double sadd(double a, double b) { return a + b; }
__device__ __forceinline__ cplx sadd(cplx a, cplx b) { return a + b; }

template <typename T>
__device__ __forceinline__ T load_k(double kre, double kim);
template <> __device__ __forceinline__ double load_k<double>(double kre, double) { return kre; }
template <> __device__ __forceinline__ cplx load_k<cplx>(double kre, double kim) { return cplx{kre, kim}; }

__host__ __device__ constexpr int op_ncomp(int op) { return op == QBX_OP_GRAD_S ? 2 : 1; }

// Shared memory: source tile (x, y, nx, ny), weighted densities [tile][NR],
// coefficient columns c1, c2 [(p+2)][kApplyThreads] of type T.
template <int OP, typename T, int NR>
__global__ void __launch_bounds__(kApplyThreads)
k_apply_fused(ApplyArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s_x = reinterpret_cast<double*>(smem_raw);
  double* s_y = s_x + kSrcTile;
  double* s_nx = s_y + kSrcTile;
  double* s_ny = s_nx + kSrcTile;
  cplx* s_wd = reinterpret_cast<cplx*>(s_ny + kSrcTile);
  T* s_c1 = reinterpret_cast<T*>(s_wd + kSrcTile * NR);
  T* s_c2 = s_c1 + (a.p + 2) * kApplyThreads;

  const int tid = threadIdx.x;
  const int c = blockIdx.x * kApplyThreads + tid;
  const bool active = c < a.n_ctr;
  const int cc = active ? c : a.n_ctr - 1;
  const int p = a.p;

  // ---- per-centre set-up: target direction, J_l(k r) (a5) ----
  const double cx = a.cx[cc], cy = a.cy[cc];
  const int t = cc % a.n_tgt;
  double ux = a.tx[t] - cx, uy = a.ty[t] - cy;
  const double r = hypot(ux, uy);
  const double ir = 1.0 / r;
  ux *= ir;
  uy *= ir;
  const T kk = load_k<T>(a.kre, a.kim);
  const T kr = rmul(kk, r);
  T* col1 = s_c1 + tid;
  T* col2 = s_c2 + tid;
  besselj_seq<T>(kr, p + 1, col1, kApplyThreads);
  T J0 = col1[0];
  if (OP == QBX_OP_S) {
    for (int l = 1; l <= p; ++l) col1[l * kApplyThreads] = rmul(col1[l * kApplyThreads], 2.0);
  } else if (OP == QBX_OP_D) {
    // c2[m] = m J_m ; c1[m] = J_{m+1} (m < p), 0 at m = p
    for (int m = 0; m <= p; ++m) col2[m * kApplyThreads] = rmul(col1[m * kApplyThreads], (double)m);
    for (int m = 0; m < p; ++m) col1[m * kApplyThreads] = col1[(m + 1) * kApplyThreads];
    T z0;
    sc_zero(z0);
    col1[p * kApplyThreads] = z0;
  } else {
    // c2[l] = 2 l J_l ; c1[l] = J_{l-1} - J_{l+1} (= 2 J_l'), c1[0] = -J_1 (= J_0')
    for (int l = 0; l <= p; ++l) col2[l * kApplyThreads] = rmul(col1[l * kApplyThreads], 2.0 * l);
    T prev = col1[0];
    for (int l = 0; l <= p; ++l) {
      T jl = col1[l * kApplyThreads];
      T jn = col1[(l + 1) * kApplyThreads];
      col1[l * kApplyThreads] = (l == 0) ? rmul(jn, -1.0) : sc_sub(prev, jn);
      prev = jl;
    }
  }
  KW<T> kw;
  kw.init(a.kre, a.kim);
  const T kneg_j0 = rmul(sc_mul(kk, J0), -1.0);  // -k J0 (D only)

  cplx acc[NR], accb[NR];
#pragma unroll
  for (int r2 = 0; r2 < NR; ++r2) {
    acc[r2] = cplx{0.0, 0.0};
    accb[r2] = cplx{0.0, 0.0};
  }

  const int s_begin = blockIdx.y * a.src_per_split;
  const int s_end = min(a.src.n, s_begin + a.src_per_split);
  const cplx* wd = reinterpret_cast<const cplx*>(a.wd);

  for (int base = s_begin; base < s_end; base += kSrcTile) {
    const int nt = min(kSrcTile, s_end - base);
    __syncthreads();
    for (int i = tid; i < nt; i += kApplyThreads) {
      s_x[i] = a.src.x[base + i];
      s_y[i] = a.src.y[base + i];
      if (OP == QBX_OP_D) {
        s_nx[i] = a.src.nx[base + i];
        s_ny[i] = a.src.ny[base + i];
      }
    }
    for (int i = tid; i < nt * NR; i += kApplyThreads) {
      const int s = i / NR, rr = i - s * NR;
      s_wd[i] = (rr < a.nr) ? wd[(size_t)(base + s) * a.nrhs + a.rhs0 + rr] : cplx{0.0, 0.0};
    }
    __syncthreads();
    if (!active) continue;

    for (int j = 0; j < nt; ++j) {
      // ---- a2: pair geometry and H0, H1 ----
      const double dx = s_x[j] - cx, dy = s_y[j] - cy;
      const double rho2 = fma(dx, dx, dy * dy);
      const double inv = rsqrt(rho2);
      const double rho = rho2 * inv;
      const double cs = fma(ux, dx, uy * dy) * inv;   // cos psi
      cplx H0, H1;
      T twoz;
      kw.hankel(rho, inv, H0, H1, twoz);
      const double tw = 2.0 * cs;

      if (OP == QBX_OP_S) {
        // ---- a3 + fused a4..a6 for S ----
        cplx G = smul(col1[0], H0);
        cplx Hm = H0, H = H1;
        T s = twoz;
        double cp = 1.0, cl = cs;
        for (int l = 1; l <= p; ++l) {
          madd(G, rmul(col1[l * kApplyThreads], cl), H);
          const cplx Hn = hrec(s, H, Hm);
          Hm = H;
          H = Hn;
          s = sadd(s, twoz);
          const double cn = fma(tw, cl, -cp);
          cp = cl;
          cl = cn;
        }
#pragma unroll
        for (int r2 = 0; r2 < NR; ++r2) acc[r2] = acc[r2] + s_wd[j * NR + r2] * G;
      } else if (OP == QBX_OP_D) {
        const double nx = s_nx[j], ny = s_ny[j];
        const double av = fma(nx, dx, ny * dy) * inv;     // n_s . e_rho
        const double bv = fma(ny, dx, -nx * dy) * inv;    // n_s . e_theta
        const double sn = fma(uy, dx, -ux * dy) * inv;    // sin psi
        const T tka = rmul(kk, 2.0 * av);                 // 2 k a
        // C_m = 2 k a cos(m psi), V_m = (2/rho)(b sin(m psi) - a cos(m psi))
        T Cp = tka, Cc = rmul(tka, cs);                   // C_0, C_1
        const double i2 = 2.0 * inv;
        double Vp = 0.0, Vc = -i2 * av;                   // V_{-1} unused, V_0
        double Vn1 = i2 * fma(bv, sn, -av * cs);          // V_1
        cplx K = smul(rmul(kneg_j0, av), H1);             // -k a J0 H1
        cplx Hm = H0, H = H0, Hnx = H1;
        T s = twoz;
        // m = 0: e_0 = J_1 C_1
        madd(K, sc_mul(col1[0], Cc), H0);
        // advance: C to (C_1, C_2), V to (V_0, V_1)
        {
          T Cn = fmsub_r(tw, Cc, Cp);
          Cp = Cc;
          Cc = Cn;
          Vp = Vc;
          Vc = Vn1;
        }
        Hm = H0;
        H = H1;
        for (int m = 1; m <= p; ++m) {
          // e_m = J_{m+1} C_{m+1} + m J_m V_m
          const T e = sadd(sc_mul(col1[m * kApplyThreads], Cc), rmul(col2[m * kApplyThreads], Vc));
          madd(K, e, H);
          Hnx = hrec(s, H, Hm);
          Hm = H;
          H = Hnx;
          s = sadd(s, twoz);
          const T Cn = fmsub_r(tw, Cc, Cp);
          Cp = Cc;
          Cc = Cn;
          const double Vn = fma(tw, Vc, -Vp);
          Vp = Vc;
          Vc = Vn;
        }
#pragma unroll
        for (int r2 = 0; r2 < NR; ++r2) acc[r2] = acc[r2] + s_wd[j * NR + r2] * K;
      } else {
        const double sn = fma(uy, dx, -ux * dy) * inv;    // sin psi
        cplx GA = smul(col1[0], H0), GB = cplx{0.0, 0.0};
        cplx Hm = H0, H = H1;
        T s = twoz;
        double cp = 1.0, cl = cs, sp = 0.0, sl = sn;
        for (int l = 1; l <= p; ++l) {
          madd(GA, rmul(col1[l * kApplyThreads], cl), H);
          madd(GB, rmul(col2[l * kApplyThreads], sl), H);
          const cplx Hn = hrec(s, H, Hm);
          Hm = H;
          H = Hn;
          s = sadd(s, twoz);
          const double cn = fma(tw, cl, -cp);
          cp = cl;
          cl = cn;
          const double sq = fma(tw, sl, -sp);
          sp = sl;
          sl = sq;
        }
#pragma unroll
        for (int r2 = 0; r2 < NR; ++r2) {
          acc[r2] = acc[r2] + s_wd[j * NR + r2] * GA;
          accb[r2] = accb[r2] + s_wd[j * NR + r2] * GB;
        }
      }
    }
  }
  if (!active) return;
  cplx* part = reinterpret_cast<cplx*>(a.part);
  const int ncomp = op_ncomp(OP);
  const size_t row = ((size_t)blockIdx.y * a.n_ctr + c) * ncomp;
#pragma unroll
  for (int r2 = 0; r2 < NR; ++r2) {
    if (r2 >= a.nr) break;
    if (OP == QBX_OP_GRAD_S) {
      // grad = e_r k A - e_theta (1/r) B, e_r = (ux, uy), e_theta = (-uy, ux)
      const cplx kA = smul(kk, acc[r2]);
      const cplx Bi = accb[r2] * ir;
      part[(row + 0) * a.nrhs + a.rhs0 + r2] = kA * ux + Bi * uy;
      part[(row + 1) * a.nrhs + a.rhs0 + r2] = kA * uy - Bi * ux;
    } else {
      part[row * a.nrhs + a.rhs0 + r2] = acc[r2];
    }
  }
}

size_t apply_smem_bytes(int op, bool ck, int p, int nr) {
  size_t tile = 4 * kSrcTile * sizeof(double) + (size_t)kSrcTile * nr * 16;
  size_t coef = 2 * (size_t)(p + 2) * kApplyThreads * (ck ? 16 : 8);
  (void)op;
  return tile + coef;
}

template <int OP, typename T, int NR>
static cudaError_t launch_t(const ApplyArgs& a, cudaStream_t st) {
  const size_t smem = apply_smem_bytes(OP, sizeof(T) == 16, a.p, NR);
  auto kern = k_apply_fused<OP, T, NR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.n_ctr + kApplyThreads - 1) / kApplyThreads, a.nsplit);
  kern<<<grid, kApplyThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int OP, typename T>
static cudaError_t launch_nr(const ApplyArgs& a, cudaStream_t st) {
  switch (a.nr) {
    case 1: return launch_t<OP, T, 1>(a, st);
    case 2: return launch_t<OP, T, 2>(a, st);
    case 3:
    case 4: return launch_t<OP, T, 4>(a, st);
    default: return launch_t<OP, T, 8>(a, st);
  }
}

cudaError_t launch_apply_fused(const ApplyArgs& a, cudaStream_t st) {
  const bool ck = a.kim != 0.0;
  switch (a.op) {
    case QBX_OP_S: return ck ? launch_nr<QBX_OP_S, cplx>(a, st) : launch_nr<QBX_OP_S, double>(a, st);
    case QBX_OP_D: return ck ? launch_nr<QBX_OP_D, cplx>(a, st) : launch_nr<QBX_OP_D, double>(a, st);
    default: return ck ? launch_nr<QBX_OP_GRAD_S, cplx>(a, st) : launch_nr<QBX_OP_GRAD_S, double>(a, st);
  }
}

// ---------------------------------------------------------------------------
// Far targets: plain quadrature (a8), partial sums over source splits.
//   S: sum wd H0(kd);  D: sum wd H1(kd) (x - x_s).n_s / d;  grad S: sum wd H1(kd) (x - x_s)/d
// (the factors i/4, ik/4, -ik/4 are applied by the finishing kernel).
// ---------------------------------------------------------------------------
template <int OP, typename T, int NR>
__global__ void __launch_bounds__(kApplyThreads)
k_far(FarArgs a) {
  __shared__ double s_x[kSrcTile], s_y[kSrcTile], s_nx[kSrcTile], s_ny[kSrcTile];
  __shared__ cplx s_wd[kSrcTile * NR];
  const int tid = threadIdx.x;
  const int e = blockIdx.x * kApplyThreads + tid;
  const bool active = e < a.n_far;
  const int ee = active ? e : a.n_far - 1;
  const double x = a.xy[2 * ee], y = a.xy[2 * ee + 1];
  KW<T> kw;
  kw.init(a.kre, a.kim);
  cplx acc[NR], accb[NR];
#pragma unroll
  for (int r2 = 0; r2 < NR; ++r2) {
    acc[r2] = cplx{0.0, 0.0};
    accb[r2] = cplx{0.0, 0.0};
  }
  const int s_begin = blockIdx.y * a.src_per_split;
  const int s_end = min(a.src.n, s_begin + a.src_per_split);
  const cplx* wd = reinterpret_cast<const cplx*>(a.wd);
  for (int base = s_begin; base < s_end; base += kSrcTile) {
    const int nt = min(kSrcTile, s_end - base);
    __syncthreads();
    for (int i = tid; i < nt; i += kApplyThreads) {
      s_x[i] = a.src.x[base + i];
      s_y[i] = a.src.y[base + i];
      s_nx[i] = a.src.nx[base + i];
      s_ny[i] = a.src.ny[base + i];
    }
    for (int i = tid; i < nt * NR; i += kApplyThreads) {
      const int s = i / NR, rr = i - s * NR;
      s_wd[i] = (rr < a.nr) ? wd[(size_t)(base + s) * a.nrhs + a.rhs0 + rr] : cplx{0.0, 0.0};
    }
    __syncthreads();
    if (!active) continue;
    for (int j = 0; j < nt; ++j) {
      const double rx = x - s_x[j], ry = y - s_y[j];
      const double d2 = fma(rx, rx, ry * ry);
      const double inv = rsqrt(d2);
      const double d = d2 * inv;
      cplx H0, H1;
      T twoz;
      kw.hankel(d, inv, H0, H1, twoz);
      if (OP == QBX_OP_S) {
#pragma unroll
        for (int r2 = 0; r2 < NR; ++r2) acc[r2] = acc[r2] + s_wd[j * NR + r2] * H0;
      } else if (OP == QBX_OP_D) {
        const cplx g = H1 * (fma(rx, s_nx[j], ry * s_ny[j]) * inv);
#pragma unroll
        for (int r2 = 0; r2 < NR; ++r2) acc[r2] = acc[r2] + s_wd[j * NR + r2] * g;
      } else {
        const cplx gx = H1 * (rx * inv), gy = H1 * (ry * inv);
#pragma unroll
        for (int r2 = 0; r2 < NR; ++r2) {
          acc[r2] = acc[r2] + s_wd[j * NR + r2] * gx;
          accb[r2] = accb[r2] + s_wd[j * NR + r2] * gy;
        }
      }
    }
  }
  if (!active) return;
  cplx* part = reinterpret_cast<cplx*>(a.part);
  const int ncomp = op_ncomp(OP);
  const size_t row = ((size_t)blockIdx.y * a.n_far + e) * ncomp;
#pragma unroll
  for (int r2 = 0; r2 < NR; ++r2) {
    if (r2 >= a.nr) break;
    part[row * a.nrhs + a.rhs0 + r2] = acc[r2];
    if (OP == QBX_OP_GRAD_S) part[(row + 1) * a.nrhs + a.rhs0 + r2] = accb[r2];
  }
}

template <int OP, typename T>
static cudaError_t launch_far_t(const FarArgs& a, cudaStream_t st) {
  dim3 grid((a.n_far + kApplyThreads - 1) / kApplyThreads, a.nsplit);
  if (a.nr <= 1) k_far<OP, T, 1><<<grid, kApplyThreads, 0, st>>>(a);
  else if (a.nr <= 4) k_far<OP, T, 4><<<grid, kApplyThreads, 0, st>>>(a);
  else k_far<OP, T, 8><<<grid, kApplyThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_far(const FarArgs& a, cudaStream_t st) {
  const bool ck = a.kim != 0.0;
  switch (a.op) {
    case QBX_OP_S: return ck ? launch_far_t<QBX_OP_S, cplx>(a, st) : launch_far_t<QBX_OP_S, double>(a, st);
    case QBX_OP_D: return ck ? launch_far_t<QBX_OP_D, cplx>(a, st) : launch_far_t<QBX_OP_D, double>(a, st);
    default: return ck ? launch_far_t<QBX_OP_GRAD_S, cplx>(a, st) : launch_far_t<QBX_OP_GRAD_S, double>(a, st);
  }
}

}  // namespace qbx
