// qbx_shape.cu -- qbx_apply_shape_adjoint (S) and qbx_apply_shape_adjoint_d
// (D): the reverse-mode gradient of a real functional of the on-surface
// apply with respect to the curve samples (gamma, gamma' at the target and
// source nodes) that qbx_geometry consumed.  The S case is written out
// below; D follows the same chain with the D kernel n_s . grad_{x_s} G in
// place of G (second source derivatives, and the normals n_s, see
// dshape_pair).
//
// With u_t = sum_{c of t} w_c (i/4) sum_s (w sigma)_s G(c, s) (w_c = 1, or 1/2
// for the two-sided average), G the truncated Graf sum of the centre c
// (eq. graf-addition), and L = Re sum_{t,r} conj(g_t) u_t:
//   dL/dx_s = Re sum_r (w sigma)_s conj(Xi_s),  Xi_s  = sum_c g_c conj((i/4) grad_{x_s} G(c, s))
//   dL/dw_s = Re sum_r (P sigma)_s conj(Psi_s), Psi_s = sum_c g_c conj((i/4) G(c, s))
//   dL/dc   = -Re sum_r conj(g_c) (F_c + E_c),  dL/dx_t (direct) = Re sum_r conj(g_c) F_c
// where g_c = w_c g_t, F_c = (i/4) sum_s (w sigma)_s grad_x G (the gradient of
// the local expansion at the target, Sec. 3.2) and E_c = (i/4) sum_s (w sigma)_s
// grad_{x_s} G; G depends on x_t - c and x_s - c only, so grad_c G =
// -grad_{x_t} G - grad_{x_s} G.  The geometry of Sec. 3.3 step 4a then maps
// these to the curve samples: c = x_t -/+ r n_t, r = r_factor h_m,
// h_m = sum of the panel's source weights, w_s = w^GL (t_{m+1}-t_m)/2 |gamma'_s|,
// n = (gamma'_y, -gamma'_x)/|gamma'|.
//
// Device work: one fused forward sweep (lanes = centres) for F and E, one
// transposed sweep (lanes = sources) for Psi and Xi, both recomputing the
// Hankel recurrences, then three short chain-rule kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <algorithm>
#include "../../include/qbx.h"
#include "qbx_apply_impl.cuh"
#include "qbx_internal.h"

using namespace qbx;

namespace {

constexpr int kOpsFwd = (1 << QBX_OP_GRAD_S) | 8;   // grad S and the source-position gradient
constexpr int kOpsAdj = (1 << QBX_OP_S) | 8;        // S and the source-position gradient
constexpr int kNcFwd = 4;                           // F_x, F_y, E_x, E_y
constexpr int kNcAdj = 3;                           // Psi, Xi_x, Xi_y

int sfail(int code, const char* what) {
  char buf[320];
  snprintf(buf, sizeof(buf), "qbx_apply_shape_adjoint: %s", what);
  return host_fail(code, buf);
}

int scuda(cudaError_t e, const char* what) {
  char buf[320];
  snprintf(buf, sizeof(buf), "qbx_apply_shape_adjoint: %s: %s", what, cudaGetErrorString(e));
  return host_fail(QBX_ECUDA, buf);
}

// Re(conj(g) (i/4) z)
__device__ __forceinline__ double re_gi4(cplx g, cplx z) { return 0.25 * (g.im * z.re - g.re * z.im); }
// Re(a conj(b))
__device__ __forceinline__ double re_conj(cplx a, cplx b) { return a.re * b.re + a.im * b.im; }

// gradient carried to each centre: (-i/4) w_c g_t (conj(i/4) = -i/4)
__global__ void k_shape_spread(int n_tgt, int nsides, int nrhs, const cplx* g, cplx* gc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_tgt * nrhs) return;
  const double wgt = nsides == 2 ? 0.5 : 1.0;
  const cplx v = g[idx];
  const cplx s = cplx{0.25 * wgt * v.im, -0.25 * wgt * v.re};
  gc[idx] = s;
  if (nsides == 2) gc[(size_t)n_tgt * nrhs + idx] = s;
}

// Per target: the forward sums of its centre(s) (fixed-order sum over the
// source splits), dL/dc, and the chain through c = x -/+ r n to the target
// samples; qh[t] = the target's share of dL/dh_m.
__global__ void k_shape_targets(int n_tgt, int q_tgt, int nsides, int side0, int nsplit, int nrhs,
                                const cplx* fpart, const cplx* gout, const double* tnx, const double* tny,
                                const double* ctr_r, const double* panel_h, const double* dgam_tgt,
                                double* g_gam, double* g_dgam, double* qh) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tgt) return;
  const int nc = nsides * n_tgt;
  const double wgt = nsides == 2 ? 0.5 : 1.0;
  const double nx = tnx[t], ny = tny[t];
  const double r = ctr_r[t];
  const double rf = r / panel_h[t / q_tgt];
  double gx = 0.0, gy = 0.0, gnx = 0.0, gny = 0.0, q = 0.0;
  for (int sd = 0; sd < nsides; ++sd) {
    const double sg = (side0 + sd) == QBX_SIDE_EXT ? 1.0 : -1.0;   // c = x + sg r n
    const int c = sd * n_tgt + t;
    double fx = 0.0, fy = 0.0, dcx = 0.0, dcy = 0.0;
    for (int rr = 0; rr < nrhs; ++rr) {
      cplx F0{0.0, 0.0}, F1{0.0, 0.0}, E0{0.0, 0.0}, E1{0.0, 0.0};
      for (int k = 0; k < nsplit; ++k) {
        const cplx* row = fpart + (((size_t)k * nc + c) * kNcFwd) * nrhs + rr;
        F0 = F0 + row[0];
        F1 = F1 + row[nrhs];
        E0 = E0 + row[2 * nrhs];
        E1 = E1 + row[3 * nrhs];
      }
      const cplx g = wgt * gout[(size_t)t * nrhs + rr];
      const double ax = re_gi4(g, F0), ay = re_gi4(g, F1);
      fx += ax;
      fy += ay;
      dcx -= ax + re_gi4(g, E0);
      dcy -= ay + re_gi4(g, E1);
    }
    gx += fx + dcx;
    gy += fy + dcy;
    gnx += sg * r * dcx;
    gny += sg * r * dcy;
    q += sg * rf * (dcx * nx + dcy * ny);
  }
  g_gam[2 * t] = gx;
  g_gam[2 * t + 1] = gy;
  // n = R v / |v|: dL/dv = -(g_n . tau) n / |v|, tau = v/|v| = (-n_y, n_x)
  const double vx = dgam_tgt[2 * t], vy = dgam_tgt[2 * t + 1];
  const double sp = hypot(vx, vy);
  const double gt = -gnx * ny + gny * nx;
  g_dgam[2 * t] = -gt * nx / sp;
  g_dgam[2 * t + 1] = -gt * ny / sp;
  qh[t] = q;
}

// dL/dh_m = sum of the panel's targets' shares (fixed order)
__global__ void k_shape_panels(int M, int q_tgt, const double* qh, double* dh) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double s = 0.0;
  for (int i = 0; i < q_tgt; ++i) s += qh[m * q_tgt + i];
  dh[m] = s;
}

// Per source: the transposed sums (fixed-order sum over the centre splits),
// dL/dx_s, dL/dw_s (+ dL/dh_m of its panel), and the chain through
// w_s = w^GL (dt/2) |gamma'_s| to gamma'_s.
__global__ void k_shape_sources(int n_src, int q_src, int nsplit, int nrhs, const cplx* apart, const cplx* wd,
                                const double* w, const double* dh, const double* dgam_src, double* g_gam,
                                double* g_dgam) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_src) return;
  double gx = 0.0, gy = 0.0, gw = 0.0;
  for (int rr = 0; rr < nrhs; ++rr) {
    cplx P{0.0, 0.0}, X0{0.0, 0.0}, X1{0.0, 0.0};
    for (int k = 0; k < nsplit; ++k) {
      const cplx* row = apart + (((size_t)k * n_src + s) * kNcAdj) * nrhs + rr;
      P = P + row[0];
      X0 = X0 + row[nrhs];
      X1 = X1 + row[2 * nrhs];
    }
    const cplx v = wd[(size_t)s * nrhs + rr];
    gx += re_conj(v, X0);
    gy += re_conj(v, X1);
    gw += re_conj(v, P);
  }
  const double ws = w[s];
  gw = gw / ws + dh[s / q_src];
  g_gam[2 * s] = gx;
  g_gam[2 * s + 1] = gy;
  const double vx = dgam_src[2 * s], vy = dgam_src[2 * s + 1];
  const double f = gw * ws / (vx * vx + vy * vy);   // d|v|/dv = v/|v|, w_s / |v| = w^GL dt/2
  g_dgam[2 * s] = f * vx;
  g_dgam[2 * s + 1] = f * vy;
}

// ---------------------------------------------------------------------------
// Shape adjoint of D.  K_D(c, s) = n_s . grad_{x_s} G, G the truncated Graf
// sum of the centre.  With y = x_s - c, x = x_t - c, Y_l = J_l(k|x|) e^{il arg x},
// W_m = H_m(k|y|) e^{im arg y},  G = sum_{|l|<=p} (-1)^l Y_l W_{-l}, and the
// complex derivatives d = d_x - i d_y, db = d_x + i d_y (in x or y) acting as
// db Z_m = -k Z_{m+1}, d Z_m = k Z_{m-1} (Z = Y, W; DLMF 10.6.2), every
// derivative the D shape gradient needs is a sum
//   U_q = sum_{|l|<=p} (-1)^l Y_l W_{q-l} = e^{iq arg y} sum_l (-1)^l J_l H_{q-l} e^{il psi},
// q = -2..2 (psi = arg x - arg y), or one of them with its range shifted by
// one (the mixed x-y derivatives; the truncation leaves two end terms):
//   db_y G = -k U_1,  d_y G = k U_{-1},  db_y^2 G = k^2 U_2,  d_y^2 G = k^2 U_{-2},
//   d_y db_y G = -k^2 G,
//   db_x db_y G = -k^2 (U_2 - t_2(-p) + t_2(p+1)),   db_x d_y G = k^2 (U_0 - t_0(-p) + t_0(p+1)),
//   d_x db_y G = k^2 (U_0 - t_0(p) + t_0(-p-1)),     d_x d_y G = -k^2 (U_{-2} - t_{-2}(p) + t_{-2}(-p-1)),
// t_q(l) the l-th term of U_q; and n . grad = (nu d + conj(nu) db)/2, nu = n_x + i n_y.
// Folding +-l (J_{-l} = (-1)^l J_l, H_{-m} = (-1)^m H_m) turns each U_q into
// cosine and sine sums of J_l against H_{l-q} +- H_{l+q}.
// Outputs (no factor i/4): K = K_D, (Gx, Gy) = grad_y G, (Sx, Sy) = grad_y K_D,
// (Tx, Ty) = grad_x K_D.
template <typename T>
__device__ __forceinline__ void dshape_pair(const KW<T>& kw, const T kk, const T* cJ, int stride, int p, double dx,
                                            double dy, double nx, double ny, double ux, double uy, cplx& K,
                                            cplx& Gx, cplx& Gy, cplx& Sx, cplx& Sy, cplx& Tx, cplx& Ty) {
  const double rho2 = fma(dx, dx, dy * dy);
  double inv, rho, yq;
  kw.geom(rho2, inv, rho, yq);
  cplx H0, H1;
  T twoz;
  kw.hankel(rho, inv, yq, H0, H1, twoz);
  const double cs = fma(ux, dx, uy * dy) * inv, sn = fma(uy, dx, -ux * dy) * inv;   // e^{i psi}
  const double tw = 2.0 * cs;
  // window H_{l-2} .. H_{l+2} at l = 1
  cplx hm2 = -H1, hm1 = H0, h0 = H1;
  T s = twoz;
  cplx hp1 = hrec(s, h0, hm1);   // H_2
  const cplx H2 = hp1;
  s = sadd(s, twoz);
  cplx hp2 = hrec(s, hp1, h0);   // H_3
  s = sadd(s, twoz);
  cplx S0{0.0, 0.0}, X{0.0, 0.0}, Y{0.0, 0.0}, P{0.0, 0.0}, Q{0.0, 0.0};
  double cp = 1.0, cl = cs, sp = 0.0, sl = sn;
  // H_{p-1}, H_p, H_{p+1}, H_{p+2}; cos, sin of p psi
  cplx Hq1 = -H1, Hq = H0, Hr1 = H1, Hr2 = H2;
  double cP = 1.0, sP = 0.0;
  for (int l = 1; l <= p; ++l) {
    const T Jl = cJ[l * stride];
    const T Jc = rmul(Jl, cl), Js = rmul(Jl, sl);
    madd(S0, Jc, h0);
    madd(X, Jc, hp1 - hm1);
    madd(Y, Js, hm1 + hp1);
    madd(P, Jc, hm2 + hp2);
    madd(Q, Js, hm2 - hp2);
    Hq1 = hm1;
    Hq = h0;
    Hr1 = hp1;
    Hr2 = hp2;
    cP = cl;
    sP = sl;
    const double cn = fma(tw, cl, -cp);
    cp = cl;
    cl = cn;
    const double sq = fma(tw, sl, -sp);
    sp = sl;
    sl = sq;
    const cplx hn = hrec(s, hp2, hp1);   // H_{l+3}
    s = sadd(s, twoz);
    hm2 = hm1;
    hm1 = h0;
    h0 = hp1;
    hp1 = hp2;
    hp2 = hn;
  }
  const double cP1 = cl, sP1 = sl;   // cos, sin of (p+1) psi
  const T J0 = cJ[0];
  const cplx j0h0 = smul(J0, H0), j0h1 = smul(J0, H1), j0h2 = smul(J0, H2);
  // folded U_q without e^{iq arg y}
  const cplx U0 = j0h0 + 2.0 * S0;
  const cplx U1 = j0h1 + cplx{X.re + Y.im, X.im - Y.re};        // + X - i Y
  const cplx Um1 = cplx{-X.re + Y.im, -X.im - Y.re} - j0h1;     // - X - i Y - J0 H1
  const cplx U2 = j0h2 + cplx{P.re - Q.im, P.im + Q.re};        // + P + i Q
  const cplx Um2 = j0h2 + cplx{P.re + Q.im, P.im - Q.re};       // + P - i Q
  // end terms of the shifted ranges
  const T Jp = cJ[p * stride], Jp1 = cJ[(p + 1) * stride];
  const cplx ep{cP, sP}, ep1{cP1, sP1};
  const cplx a1 = smul(Jp, Hr2), a2 = smul(Jp1, Hq1), a3 = smul(Jp, Hq), a4 = smul(Jp1, Hr1);
  const cplx M1t = a1 * conj(ep) - a2 * ep1 - U2;        // db_x db_y G = k^2 M1
  const cplx M2 = U0 - a3 * conj(ep) + a4 * ep1;         // db_x d_y G = k^2 M2
  const cplx M3 = U0 - a3 * ep + a4 * conj(ep1);         // d_x db_y G = k^2 M3
  const cplx M4t = a1 * ep - a2 * conj(ep1) - Um2;       // d_x d_y G = k^2 M4
  // phases e^{iq arg y}
  const cplx E1{dx * inv, dy * inv};
  const cplx E2 = E1 * E1;
  const cplx Uf1 = U1 * E1, Ufm1 = Um1 * conj(E1), Uf2 = U2 * E2, Ufm2 = Um2 * conj(E2);
  const cplx M1 = M1t * E2, M4 = M4t * conj(E2);
  const cplx nu{nx, ny}, nub{nx, -ny};
  const cplx k1 = to_c(kk), k2 = k1 * k1;
  const cplx dbG = -(k1 * Uf1), dG = k1 * Ufm1;
  K = 0.5 * (nu * dG + nub * dbG);
  Gx = 0.5 * (dG + dbG);
  Gy = mul_i(0.5 * (dG - dbG));
  const cplx dbK = (0.5 * k2) * (nub * Uf2 - nu * U0), dK = (0.5 * k2) * (nu * Ufm2 - nub * U0);
  Sx = 0.5 * (dK + dbK);
  Sy = mul_i(0.5 * (dK - dbK));
  const cplx dbxK = (0.5 * k2) * (nub * M1 + nu * M2), dxK = (0.5 * k2) * (nu * M4 + nub * M3);
  Tx = 0.5 * (dxK + dbxK);
  Ty = mul_i(0.5 * (dxK - dbxK));
}

constexpr int kDsTile = 64;     // sources per shared-memory tile (forward), centres (transposed)
constexpr int kDsNR = 4;        // rhs per pass
constexpr int kNcFwdD = 4, kNcAdjD = 5;

struct DsArgs {
  int p, nrhs, rhs0, nr;
  double kre, kim;
  const double* hk_tab;
  int n_ctr, n_tgt, n_src;
  const double *cx, *cy, *tx, *ty;
  const double *sx, *sy, *snx, *sny;
  const cplx* wd;     // [n_src][nrhs] (forward)
  const cplx* gc;     // [n_ctr][nrhs] (transposed)
  void* coef;         // [n_ctr][p+2] J_0..J_{p+1} (written by k_dshape_columns)
  double* cgeo;       // [n_ctr][4] ux, uy, r, unused (written by k_dshape_columns)
  int nsplit, per_split;
  cplx* part;
};

template <typename T>
__global__ void k_dshape_columns(DsArgs a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.n_ctr) return;
  KW<T> kw;
  kw.init(a.kre, a.kim, a.hk_tab);
  const double cx = a.cx[c], cy = a.cy[c];
  const int t = c % a.n_tgt;
  const double ux = a.tx[t] - cx, uy = a.ty[t] - cy, r = hypot(ux, uy);
  besselj_seq<T>(rmul(kw.kval(), r), a.p + 1, reinterpret_cast<T*>(a.coef) + (size_t)c * (a.p + 2), 1);
  double* geo = a.cgeo + 4 * (size_t)c;
  geo[0] = ux / r;
  geo[1] = uy / r;
  geo[2] = r;
  geo[3] = 0.0;
}

// lanes = centres: F = sum_s (w mu)_s grad_x K_D, E = sum_s (w mu)_s grad_y K_D
template <typename T>
__global__ void __launch_bounds__(128) k_dshape_fwd(DsArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s_x = reinterpret_cast<double*>(smem_raw);
  double* s_y = s_x + kDsTile;
  double* s_nx = s_y + kDsTile;
  double* s_ny = s_nx + kDsTile;
  cplx* s_w = reinterpret_cast<cplx*>(s_ny + kDsTile);            // [tile][kDsNR]
  T* s_col = reinterpret_cast<T*>(s_w + kDsTile * kDsNR);          // [p+2][128]
  const int nblk = (a.n_ctr + 127) / 128;
  const int cb = blockIdx.x % nblk, split = blockIdx.x / nblk;
  const int c = cb * 128 + threadIdx.x;
  const bool active = c < a.n_ctr;
  const int cc = active ? c : a.n_ctr - 1;
  KW<T> kw;
  kw.init(a.kre, a.kim, a.hk_tab);
  const T kk = kw.kval();
  const T* coef = reinterpret_cast<const T*>(a.coef) + (size_t)cc * (a.p + 2);
  for (int l = 0; l <= a.p + 1; ++l) s_col[l * 128 + threadIdx.x] = coef[l];
  const double cx = a.cx[cc], cy = a.cy[cc];
  const double ux = a.cgeo[4 * (size_t)cc], uy = a.cgeo[4 * (size_t)cc + 1];
  cplx acc[kNcFwdD][kDsNR];
#pragma unroll
  for (int q = 0; q < kNcFwdD; ++q)
#pragma unroll
    for (int r = 0; r < kDsNR; ++r) acc[q][r] = cplx{0.0, 0.0};
  const int s0 = split * a.per_split, s1 = min(a.n_src, s0 + a.per_split);
  for (int base = s0; base < s1; base += kDsTile) {
    const int nt = min(kDsTile, s1 - base);
    __syncthreads();
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
      s_x[i] = a.sx[base + i];
      s_y[i] = a.sy[base + i];
      s_nx[i] = a.snx[base + i];
      s_ny[i] = a.sny[base + i];
    }
    for (int i = threadIdx.x; i < nt * kDsNR; i += blockDim.x) {
      const int j = i / kDsNR, r = i - j * kDsNR;
      s_w[i] = r < a.nr ? a.wd[(size_t)(base + j) * a.nrhs + a.rhs0 + r] : cplx{0.0, 0.0};
    }
    __syncthreads();
    if (!active) continue;
    for (int j = 0; j < nt; ++j) {
      cplx K, Gx, Gy, Sx, Sy, Tx, Ty;
      dshape_pair<T>(kw, kk, s_col + threadIdx.x, 128, a.p, s_x[j] - cx, s_y[j] - cy, s_nx[j], s_ny[j], ux, uy,
                     K, Gx, Gy, Sx, Sy, Tx, Ty);
#pragma unroll
      for (int r = 0; r < kDsNR; ++r) {
        const cplx w = s_w[j * kDsNR + r];
        cfma(acc[0][r], w, Tx);
        cfma(acc[1][r], w, Ty);
        cfma(acc[2][r], w, Sx);
        cfma(acc[3][r], w, Sy);
      }
    }
  }
  if (!active) return;
  const size_t row = ((size_t)split * a.n_ctr + c) * kNcFwdD;
#pragma unroll
  for (int r = 0; r < kDsNR; ++r) {
    if (r >= a.nr) break;
#pragma unroll
    for (int q = 0; q < kNcFwdD; ++q) a.part[(row + q) * a.nrhs + a.rhs0 + r] = acc[q][r];
  }
}

// lanes = sources: Psi = sum_c g_c conj(K_D), Xi = sum_c g_c conj(grad_y K_D),
// N = sum_c g_c conj(grad_y G)
template <typename T>
__global__ void __launch_bounds__(128) k_dshape_adj(DsArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s_cx = reinterpret_cast<double*>(smem_raw);
  double* s_cy = s_cx + kDsTile;
  double* s_ux = s_cy + kDsTile;
  double* s_uy = s_ux + kDsTile;
  cplx* s_g = reinterpret_cast<cplx*>(s_uy + kDsTile);              // [tile][kDsNR]
  T* s_col = reinterpret_cast<T*>(s_g + kDsTile * kDsNR);            // [p+2][tile]
  const int nblk = (a.n_src + 127) / 128;
  const int sb = blockIdx.x % nblk, split = blockIdx.x / nblk;
  const int s = sb * 128 + threadIdx.x;
  const bool active = s < a.n_src;
  const int ss = active ? s : a.n_src - 1;
  KW<T> kw;
  kw.init(a.kre, a.kim, a.hk_tab);
  const T kk = kw.kval();
  const double sx = a.sx[ss], sy = a.sy[ss], snx = a.snx[ss], sny = a.sny[ss];
  const int P2 = a.p + 2;
  cplx acc[kNcAdjD][kDsNR];
#pragma unroll
  for (int q = 0; q < kNcAdjD; ++q)
#pragma unroll
    for (int r = 0; r < kDsNR; ++r) acc[q][r] = cplx{0.0, 0.0};
  const int c0 = split * a.per_split, c1 = min(a.n_ctr, c0 + a.per_split);
  for (int base = c0; base < c1; base += kDsTile) {
    const int nt = min(kDsTile, c1 - base);
    __syncthreads();
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
      s_cx[i] = a.cx[base + i];
      s_cy[i] = a.cy[base + i];
      s_ux[i] = a.cgeo[4 * (size_t)(base + i)];
      s_uy[i] = a.cgeo[4 * (size_t)(base + i) + 1];
    }
    for (int i = threadIdx.x; i < nt * kDsNR; i += blockDim.x) {
      const int j = i / kDsNR, r = i - j * kDsNR;
      s_g[i] = r < a.nr ? a.gc[(size_t)(base + j) * a.nrhs + a.rhs0 + r] : cplx{0.0, 0.0};
    }
    const T* coef = reinterpret_cast<const T*>(a.coef);
    for (int i = threadIdx.x; i < nt * P2; i += blockDim.x) {
      const int j = i / P2, l = i - j * P2;
      s_col[l * kDsTile + j] = coef[(size_t)(base + j) * P2 + l];
    }
    __syncthreads();
    if (!active) continue;
    for (int j = 0; j < nt; ++j) {
      cplx K, Gx, Gy, Sx, Sy, Tx, Ty;
      dshape_pair<T>(kw, kk, s_col + j, kDsTile, a.p, sx - s_cx[j], sy - s_cy[j], snx, sny, s_ux[j], s_uy[j], K,
                     Gx, Gy, Sx, Sy, Tx, Ty);
      const cplx v[kNcAdjD] = {conj(K), conj(Sx), conj(Sy), conj(Gx), conj(Gy)};
#pragma unroll
      for (int r = 0; r < kDsNR; ++r) {
        const cplx g = s_g[j * kDsNR + r];
#pragma unroll
        for (int q = 0; q < kNcAdjD; ++q) cfma(acc[q][r], g, v[q]);
      }
    }
  }
  if (!active) return;
  const size_t row = ((size_t)split * a.n_src + s) * kNcAdjD;
#pragma unroll
  for (int r = 0; r < kDsNR; ++r) {
    if (r >= a.nr) break;
#pragma unroll
    for (int q = 0; q < kNcAdjD; ++q) a.part[(row + q) * a.nrhs + a.rhs0 + r] = acc[q][r];
  }
}

// Per source (D): dL/dx_s from Xi, dL/dw_s from Psi (+ dL/dh_m of its panel),
// dL/dn_s from N, and the chain through w_s = w^GL (dt/2)|gamma'_s| and
// n_s = (gamma'_y, -gamma'_x)/|gamma'_s| to gamma'_s.
__global__ void k_shape_sources_d(int n_src, int q_src, int nsplit, int nrhs, const cplx* apart, const cplx* wd,
                                  const double* w, const double* snx, const double* sny, const double* dh,
                                  const double* dgam_src, double* g_gam, double* g_dgam) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_src) return;
  double gx = 0.0, gy = 0.0, gw = 0.0, gnx = 0.0, gny = 0.0;
  for (int rr = 0; rr < nrhs; ++rr) {
    cplx v5[kNcAdjD];
    for (int q = 0; q < kNcAdjD; ++q) v5[q] = cplx{0.0, 0.0};
    for (int k = 0; k < nsplit; ++k) {
      const cplx* row = apart + (((size_t)k * n_src + s) * kNcAdjD) * nrhs + rr;
      for (int q = 0; q < kNcAdjD; ++q) v5[q] = v5[q] + row[q * nrhs];
    }
    const cplx v = wd[(size_t)s * nrhs + rr];
    gw += re_conj(v, v5[0]);
    gx += re_conj(v, v5[1]);
    gy += re_conj(v, v5[2]);
    gnx += re_conj(v, v5[3]);
    gny += re_conj(v, v5[4]);
  }
  const double ws = w[s];
  gw = gw / ws + dh[s / q_src];
  g_gam[2 * s] = gx;
  g_gam[2 * s + 1] = gy;
  const double vx = dgam_src[2 * s], vy = dgam_src[2 * s + 1];
  const double v2 = vx * vx + vy * vy, sp = sqrt(v2);
  const double f = gw * ws / v2;
  const double nx = snx[s], ny = sny[s];
  const double gt = -gnx * ny + gny * nx;   // g_n . tau, tau = (-n_y, n_x)
  g_dgam[2 * s] = f * vx - gt * nx / sp;
  g_dgam[2 * s + 1] = f * vy - gt * ny / sp;
}

template <typename T>
cudaError_t launch_dshape(const DsArgs& a0, bool fwd, cudaStream_t st) {
  DsArgs a = a0;
  const size_t col = (size_t)(a.p + 2) * (fwd ? 128 : kDsTile) * sizeof(T);
  const size_t smem = 4 * kDsTile * 8 + (size_t)kDsTile * kDsNR * 16 + col;
  auto kern = fwd ? k_dshape_fwd<T> : k_dshape_adj<T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int lanes = fwd ? a.n_ctr : a.n_src;
  const unsigned grid = (unsigned)((lanes + 127) / 128) * (unsigned)a.nsplit;
  for (int r0 = 0; r0 < a.nrhs; r0 += kDsNR) {
    a.rhs0 = r0;
    a.nr = std::min(kDsNR, a.nrhs - r0);
    kern<<<grid, 128, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

struct Layout {
  size_t wd, fpart, gc, coef, cgeo, apart, qh, dh, total;
};

Layout layout(int M, int q_tgt, int q_src, int nc, int p, int nrhs, bool ck, int ns_fwd, int ns_adj,
              int nc_adj = kNcAdj) {
  const size_t n_tgt = (size_t)M * q_tgt, n_src = (size_t)M * q_src;
  Layout L;
  size_t o = 0;
  L.wd = o;
  o += host_align256(n_src * nrhs * 16);
  L.gc = o;
  o += host_align256((size_t)nc * nrhs * 16);
  L.coef = o;
  o += host_align256((size_t)nc * 2 * (p + 2) * (ck ? 16 : 8));
  L.cgeo = o;
  o += host_align256((size_t)nc * 4 * 8);
  L.qh = o;
  o += host_align256(n_tgt * 8);
  L.dh = o;
  o += host_align256((size_t)M * 8);
  L.fpart = o;
  o += host_align256((size_t)ns_fwd * nc * kNcFwd * nrhs * 16);
  L.apart = o;
  o += host_align256((size_t)ns_adj * n_src * nc_adj * nrhs * 16);
  L.total = o + 256;
  return L;
}

}  // namespace

extern "C" size_t qbx_shape_adjoint_workspace_bytes(int M, int q_tgt, int q_src, int p, int nrhs) {
  if (M < 1 || q_tgt < 1 || q_src < 1 || p < 0 || nrhs < 1) return 0;
  return layout(M, q_tgt, q_src, 2 * M * q_tgt, p, nrhs, true, kMaxSplit, kMaxSplit, kNcAdjD).total;
}

static int shape_impl(int op, qbx_plan* plan, const qbx_geom* g, int side, qbx_c64 k, int p,
                      const qbx_c64* dens_tgt, const qbx_c64* gout, int nrhs, const double* dgam_tgt,
                      const double* dgam_src, double* g_gam_tgt, double* g_dgam_tgt, double* g_gam_src,
                      double* g_dgam_src, void* stream) {
  if (!plan) return sfail(QBX_EINVAL, "plan is NULL");
  if (!g) return sfail(QBX_EINVAL, "geometry is NULL");
  int device, q_tgt, q_src, num_sms;
  const double* P;
  host_plan_info(plan, &device, &q_tgt, &q_src, &P);
  void* ws;
  size_t ws_bytes;
  int* status;
  host_plan_workspace(plan, &ws, &ws_bytes, &num_sms, &status);
  if (g->q_tgt != q_tgt || g->q_src != q_src || g->M < 1 || g->n_tgt != g->M * q_tgt || g->n_src != g->M * q_src)
    return sfail(QBX_EINVAL, "geometry inconsistent with the plan");
  if (!g->src_x || !g->src_w || !g->ctr_x || !g->tgt_x || !g->tgt_nx || !g->panel_h || !g->ctr_r)
    return sfail(QBX_EINVAL, "geometry: NULL array");
  if (side != QBX_SIDE_INT && side != QBX_SIDE_EXT && side != QBX_SIDE_TWO) return sfail(QBX_EINVAL, "bad side");
  if (!isfinite(k.re) || !isfinite(k.im) || k.im < 0.0 || (k.im == 0.0 && !(k.re > 0.0)))
    return sfail(QBX_EINVAL, "k must be finite with Im k >= 0 (real k > 0)");
  if (p < 0 || p > QBX_MAX_P) return sfail(QBX_EINVAL, "p outside [0, QBX_MAX_P]");
  if (nrhs < 1 || !dens_tgt || !gout) return sfail(QBX_EINVAL, "bad nrhs or NULL density / gradient");
  if (!dgam_tgt || !dgam_src || !g_gam_tgt || !g_dgam_tgt || !g_gam_src || !g_dgam_src)
    return sfail(QBX_EINVAL, "NULL curve-sample array");
  const bool ck = k.im != 0.0;
  const int n_tgt = g->n_tgt, n_src = g->n_src;
  const int nsides = side == QBX_SIDE_TWO ? 2 : 1;
  const int c0 = side == QBX_SIDE_EXT ? n_tgt : 0;
  const int side0 = side == QBX_SIDE_EXT ? QBX_SIDE_EXT : QBX_SIDE_INT;
  const int nc = nsides * n_tgt;
  const bool opD = op == QBX_OP_D;
  const int nc_adj = opD ? kNcAdjD : kNcAdj;
  const int chunk = apply_chunk(kOpsFwd);
  if (apply_smem_bytes(kOpsFwd, ck, p, chunk) > 220 * 1024) return sfail(QBX_EINVAL, "p too large");
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return scuda(e, "cudaSetDevice");
  // split counts: the forward sweep as the apply chooses them, the transposed
  // sweep about six CTAs per SM; both shrink to fit the workspace
  const Layout L0 = layout(g->M, q_tgt, q_src, nc, p, nrhs, ck, 0, 0, nc_adj);
  if (ws_bytes < L0.total + 512) return sfail(QBX_ENOMEM, "workspace too small");
  const size_t avail = ws_bytes - L0.total - 512;
  const size_t per_fwd = (size_t)nc * kNcFwd * nrhs * 16, per_adj = (size_t)n_src * nc_adj * nrhs * 16;
  const int occ = opD ? 0
                      : (ck ? apply_occupancy_cplx(kOpsFwd, p, std::min(chunk, nrhs))
                            : apply_occupancy_real(kOpsFwd, p, std::min(chunk, nrhs)));
  const int units = (nc + kApplyThreads - 1) / kApplyThreads;
  int ns_fwd = host_choose_split_waves(num_sms, occ, units, n_src, per_fwd, avail / 2);
  const int tiles = opD ? (n_src + 127) / 128 : (n_src + kGrpCentres - 1) / kGrpCentres;
  int ns_adj = std::max(1, (num_sms * 6 + tiles - 1) / tiles);
  ns_adj = std::min(ns_adj, std::max(1, nc / (opD ? kDsTile : kGrpTile)));
  ns_adj = std::min(ns_adj, kMaxSplit);
  ns_adj = (int)std::min<size_t>((size_t)ns_adj, (avail - std::min(avail, (size_t)ns_fwd * per_fwd)) / per_adj);
  if (ns_fwd < 1 || ns_adj < 1) return sfail(QBX_ENOMEM, "workspace too small for the partial sums");
  const Layout L = layout(g->M, q_tgt, q_src, nc, p, nrhs, ck, ns_fwd, ns_adj, nc_adj);
  if (L.total > ws_bytes) return sfail(QBX_ENOMEM, "workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)host_align256((size_t)ws);
  void* wd = base + L.wd;
  // (w sigma)_s
  e = launch_upsample(g->M, q_tgt, q_src, nrhs, P, g->src_w, dens_tgt, wd, st);
  if (e != cudaSuccess) return scuda(e, "upsample");
  const double* hk_tab = host_plan_hk_table(plan, k, st, &e);
  if (e != cudaSuccess) return scuda(e, "complex-k amplitude table");
  if (opD) {
    DsArgs d{};
    d.p = p;
    d.nrhs = nrhs;
    d.kre = k.re;
    d.kim = k.im;
    d.hk_tab = hk_tab;
    d.n_ctr = nc;
    d.n_tgt = n_tgt;
    d.n_src = n_src;
    d.cx = g->ctr_x + c0;
    d.cy = g->ctr_y + c0;
    d.tx = g->tgt_x;
    d.ty = g->tgt_y;
    d.sx = g->src_x;
    d.sy = g->src_y;
    d.snx = g->src_nx;
    d.sny = g->src_ny;
    d.wd = (const cplx*)wd;
    d.gc = (const cplx*)(base + L.gc);
    d.coef = base + L.coef;
    d.cgeo = (double*)(base + L.cgeo);
    // per-centre J_0..J_{p+1} and target direction
    if (ck) k_dshape_columns<cplx><<<(nc + 127) / 128, 128, 0, st>>>(d);
    else k_dshape_columns<double><<<(nc + 127) / 128, 128, 0, st>>>(d);
    e = cudaGetLastError();
    if (e != cudaSuccess) return scuda(e, "coefficient columns");
    // forward sums F = grad_x K_D and E = grad_y K_D against (w mu)_s
    d.nsplit = ns_fwd;
    d.per_split = host_split_len(n_src, ns_fwd);
    d.part = (cplx*)(base + L.fpart);
    e = ck ? launch_dshape<cplx>(d, true, st) : launch_dshape<double>(d, true, st);
    if (e != cudaSuccess) return scuda(e, "forward sweep (D)");
    k_shape_spread<<<(n_tgt * nrhs + 255) / 256, 256, 0, st>>>(n_tgt, nsides, nrhs, (const cplx*)gout,
                                                               (cplx*)(base + L.gc));
    e = cudaGetLastError();
    if (e != cudaSuccess) return scuda(e, "spread kernel");
    // transposed sums Psi, Xi, N
    d.nsplit = ns_adj;
    d.per_split = (nc + ns_adj - 1) / ns_adj;
    d.part = (cplx*)(base + L.apart);
    e = ck ? launch_dshape<cplx>(d, false, st) : launch_dshape<double>(d, false, st);
    if (e != cudaSuccess) return scuda(e, "transposed sweep (D)");
    double* qh = (double*)(base + L.qh);
    double* dh = (double*)(base + L.dh);
    k_shape_targets<<<(n_tgt + 127) / 128, 128, 0, st>>>(n_tgt, q_tgt, nsides, side0, ns_fwd, nrhs,
                                                         (const cplx*)(base + L.fpart), (const cplx*)gout,
                                                         g->tgt_nx, g->tgt_ny, g->ctr_r, g->panel_h, dgam_tgt,
                                                         g_gam_tgt, g_dgam_tgt, qh);
    k_shape_panels<<<(g->M + 127) / 128, 128, 0, st>>>(g->M, q_tgt, qh, dh);
    k_shape_sources_d<<<(n_src + 127) / 128, 128, 0, st>>>(n_src, q_src, ns_adj, nrhs, (const cplx*)(base + L.apart),
                                                           (const cplx*)wd, g->src_w, g->src_nx, g->src_ny, dh,
                                                           dgam_src, g_gam_src, g_dgam_src);
    e = cudaGetLastError();
    if (e != cudaSuccess) return scuda(e, "chain-rule kernels");
    return QBX_OK;
  }
  // forward sums F (grad of the local expansion at the target) and E (source-position gradient)
  ApplyArgs a{};
  a.ops = kOpsFwd;
  a.wd[0] = a.wd[1] = a.wd[2] = wd;
  a.p = p;
  a.kre = k.re;
  a.kim = k.im;
  a.n_ctr = nc;
  a.cx = g->ctr_x + c0;
  a.cy = g->ctr_y + c0;
  a.n_tgt = n_tgt;
  a.tx = g->tgt_x;
  a.ty = g->tgt_y;
  a.src = SrcView{g->src_x, g->src_y, g->src_nx, g->src_ny, n_src};
  a.nrhs = nrhs;
  a.nsplit = ns_fwd;
  a.src_per_split = host_split_len(n_src, ns_fwd);
  a.part = base + L.fpart;
  a.hk_tab = hk_tab;
  for (int r0 = 0; r0 < nrhs; r0 += chunk) {
    a.rhs0 = r0;
    a.nr = std::min(chunk, nrhs - r0);
    e = launch_apply_fused(a, st);
    if (e != cudaSuccess) return scuda(e, "forward sweep");
  }
  // transposed sums Psi, Xi
  k_shape_spread<<<(n_tgt * nrhs + 255) / 256, 256, 0, st>>>(n_tgt, nsides, nrhs, (const cplx*)gout,
                                                             (cplx*)(base + L.gc));
  e = cudaGetLastError();
  if (e != cudaSuccess) return scuda(e, "spread kernel");
  AdjArgs b{};
  b.ops = kOpsAdj;
  b.p = p;
  b.nrhs = nrhs;
  b.kre = k.re;
  b.kim = k.im;
  b.n_ctr = nc;
  b.n_tgt = n_tgt;
  b.n_src = n_src;
  b.cx = g->ctr_x + c0;
  b.cy = g->ctr_y + c0;
  b.tx = g->tgt_x;
  b.ty = g->tgt_y;
  b.sx = g->src_x;
  b.sy = g->src_y;
  b.snx = g->src_nx;
  b.sny = g->src_ny;
  b.gc = base + L.gc;
  b.coef = base + L.coef;
  b.cgeo = (double*)(base + L.cgeo);
  b.nsplit = ns_adj;
  b.ctr_per_split = (nc + ns_adj - 1) / ns_adj;
  b.part = base + L.apart;
  b.hk_tab = a.hk_tab;
  e = ck ? launch_adjoint_cplx(b, st) : launch_adjoint_real(b, st);
  if (e != cudaSuccess) return scuda(e, "transposed sweep");
  // chain rule to the curve samples
  double* qh = (double*)(base + L.qh);
  double* dh = (double*)(base + L.dh);
  k_shape_targets<<<(n_tgt + 127) / 128, 128, 0, st>>>(n_tgt, q_tgt, nsides, side0, ns_fwd, nrhs,
                                                       (const cplx*)(base + L.fpart), (const cplx*)gout,
                                                       g->tgt_nx, g->tgt_ny, g->ctr_r, g->panel_h, dgam_tgt,
                                                       g_gam_tgt, g_dgam_tgt, qh);
  k_shape_panels<<<(g->M + 127) / 128, 128, 0, st>>>(g->M, q_tgt, qh, dh);
  k_shape_sources<<<(n_src + 127) / 128, 128, 0, st>>>(n_src, q_src, ns_adj, nrhs, (const cplx*)(base + L.apart),
                                                       (const cplx*)wd, g->src_w, dh, dgam_src, g_gam_src,
                                                       g_dgam_src);
  e = cudaGetLastError();
  if (e != cudaSuccess) return scuda(e, "chain-rule kernels");
  return QBX_OK;
}

extern "C" int qbx_apply_shape_adjoint(qbx_plan* plan, const qbx_geom* g, int side, qbx_c64 k, int p,
                                       const qbx_c64* dens_tgt, const qbx_c64* gout, int nrhs,
                                       const double* dgam_tgt, const double* dgam_src, double* g_gam_tgt,
                                       double* g_dgam_tgt, double* g_gam_src, double* g_dgam_src,
                                       void* stream) {
  return shape_impl(QBX_OP_S, plan, g, side, k, p, dens_tgt, gout, nrhs, dgam_tgt, dgam_src, g_gam_tgt, g_dgam_tgt,
                    g_gam_src, g_dgam_src, stream);
}

extern "C" int qbx_apply_shape_adjoint_d(qbx_plan* plan, const qbx_geom* g, int side, qbx_c64 k, int p,
                                         const qbx_c64* dens_tgt, const qbx_c64* gout, int nrhs,
                                         const double* dgam_tgt, const double* dgam_src, double* g_gam_tgt,
                                         double* g_dgam_tgt, double* g_gam_src, double* g_dgam_src,
                                         void* stream) {
  return shape_impl(QBX_OP_D, plan, g, side, k, p, dens_tgt, gout, nrhs, dgam_tgt, dgam_src, g_gam_tgt, g_dgam_tgt,
                    g_gam_src, g_dgam_src, stream);
}
