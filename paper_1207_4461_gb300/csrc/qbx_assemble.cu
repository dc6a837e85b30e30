// qbx_assemble.cu -- the Nystrom matrix of the exterior combined-field
// operator (Sec. 4.2; the paper notes the discrete operator can be formed as
// a matrix, Sec. 3.3): A = 1/2 I + D - i eta S with D and S two-sided
// averages, in the sqrt-weight unknowns of Sec. 4.2,
//   At[t][t'] = sqrt(w_t) A[t][t'] / sqrt(w_t'),
// and the GMRES solve whose matvecs are then one complex GEMM (qbx_zgemm.cu, three
// real products per complex multiply-add) for all right-hand sides.
//
// Row t of A collects, for both centres of target t (interior, exterior;
// weight 1/2 each), the truncated Graf sums of D and S against every source
// node x_s, weighted by w_s and carried back to the target grid by the
// per-panel interpolation P (Sec. 3.4.2):
//   A[t][m q_t + i] = (i/4) (1/2) sum_sides sum_j (K_D - i eta K_S)(c, x_{m q_s + j}) w P[j][i]
// plus 1/2 on the diagonal.  A CTA of 4 warps owns 32 targets (one per lane)
// and the panels m = 4 blockIdx.y + g (mod 4 gridDim.y) for warp g; the
// matrix is stored column-major
// (entry (t, t') at t' n + t), so a warp writes 32 consecutive rows of one
// column at a time.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <algorithm>
#include <complex>
#include <vector>
#include "../../include/qbx.h"
#include "qbx_apply_impl.cuh"
#include "qbx_internal.h"

using namespace qbx;

namespace {

constexpr int kAsmLanes = 32, kAsmWarps = 4, kAsmQ = 16;   // targets per CTA, warps, max q_tgt

struct AsmArgs {
  double kre, kim, eta_re, eta_im;
  int p, n_tgt, q_tgt, q_src, M;
  const double *cx, *cy, *tx, *ty, *tw;
  const double *sx, *sy, *snx, *sny, *sw;
  const double* P;     // [q_src][q_tgt]
  cplx* out;           // [n_tgt][n_tgt] column-major
  const double* hk_tab;   // complex k: the amplitude table of this k's ray, or null
};

template <typename T>
__global__ void __launch_bounds__(kAsmLanes * kAsmWarps) k_assemble_cfie(AsmArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sP = reinterpret_cast<double*>(smem_raw);                  // [q_src][q_tgt]
  T* slot = reinterpret_cast<T*>(sP + a.q_src * a.q_tgt + (a.q_src * a.q_tgt & 1));
  const int p = a.p, P2 = (p + 2) * kAsmLanes;
  T* sJ = slot;             // J_l(k r) of the interior centre, [p+2][32]
  T* sL = slot + P2;        // l J_l
  T* sJe = slot + 2 * P2;   // the same for the exterior centre (its radius may differ:
  T* sLe = slot + 3 * P2;   // QBX_RADIUS_ADMISSIBLE lowers each centre's radius separately)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = blockIdx.x * kAsmLanes + lane;
  const bool active = t < a.n_tgt;
  const int tt = active ? t : a.n_tgt - 1;
  for (int i = threadIdx.x; i < a.q_src * a.q_tgt; i += blockDim.x) sP[i] = a.P[i];
  // both centres of the target: u = (x_t - c)/r is n for the interior one and -n for the exterior one
  const double cxi = a.cx[tt], cyi = a.cy[tt], cxe = a.cx[a.n_tgt + tt], cye = a.cy[a.n_tgt + tt];
  double ux = a.tx[tt] - cxi, uy = a.ty[tt] - cyi;
  const double r = hypot(ux, uy);
  ux /= r;
  uy /= r;
  const double re = hypot(a.tx[tt] - cxe, a.ty[tt] - cye);
  KW<T> kw;
  kw.init(a.kre, a.kim, a.hk_tab);
  const T kk = kw.kval();
  if (warp < 2) {
    T* J = warp == 0 ? sJ : sJe;
    T* Lc = warp == 0 ? sL : sLe;
    besselj_seq<T>(rmul(kk, warp == 0 ? r : re), p + 1, J + lane, kAsmLanes);
    for (int l = 0; l <= p; ++l) Lc[l * kAsmLanes + lane] = rmul(J[l * kAsmLanes + lane], (double)l);
    T z0;
    sc_zero(z0);
    J[(p + 1) * kAsmLanes + lane] = z0;
  }
  __syncthreads();
  const T* cJ = sJ + lane;
  const T* cL = sL + lane;
  const T* cJe = sJe + lane;
  const T* cLe = sLe + lane;
  const T J0 = cJ[0], J0e = cJe[0];
  const T kneg_j0 = rmul(sc_mul(kk, J0), -1.0), kneg_j0e = rmul(sc_mul(kk, J0e), -1.0);
  const cplx ieta = cplx{-a.eta_im, a.eta_re};   // i eta
  const double swt = sqrt(a.tw[tt]);
  for (int m = (int)blockIdx.y * kAsmWarps + warp; m < a.M; m += kAsmWarps * (int)gridDim.y) {
    cplx acc[kAsmQ];
#pragma unroll
    for (int i = 0; i < kAsmQ; ++i) acc[i] = cplx{0.0, 0.0};
    for (int j = 0; j < a.q_src; ++j) {
      const int s = m * a.q_src + j;
      const double sx = a.sx[s], sy = a.sy[s], nx = a.snx[s], ny = a.sny[s];
      cplx GS, K, GA, GB, EX, EY, v{0.0, 0.0};
      pair_kernels<OPB_S | OPB_D, T, kAsmLanes>(kw, kk, J0, kneg_j0, cJ, cL, cJ, p, sx - cxi, sy - cyi, nx, ny, ux,
                                               uy, 1.0 / r, GS, K, GA, GB, EX, EY);
      v = K - ieta * GS;
      pair_kernels<OPB_S | OPB_D, T, kAsmLanes>(kw, kk, J0e, kneg_j0e, cJe, cLe, cJe, p, sx - cxe, sy - cye, nx, ny,
                                               -ux, -uy, 1.0 / re, GS, K, GA, GB, EX, EY);
      v = v + K - ieta * GS;
      v = a.sw[s] * v;
      const double* Pj = sP + j * a.q_tgt;
#pragma unroll
      for (int i = 0; i < kAsmQ; ++i) {
        if (i < a.q_tgt) {
          acc[i].re = fma(Pj[i], v.re, acc[i].re);
          acc[i].im = fma(Pj[i], v.im, acc[i].im);
        }
      }
    }
    if (!active) continue;
#pragma unroll
    for (int i = 0; i < kAsmQ; ++i) {
      if (i >= a.q_tgt) break;
      const int col = m * a.q_tgt + i;
      // (i/4)(1/2) acc, the 1/2 of the identity, the sqrt-weight scaling
      cplx e = cplx{-0.125 * acc[i].im, 0.125 * acc[i].re};
      if (col == t) e.re += 0.5;
      const double sc = swt / sqrt(a.tw[col]);
      a.out[(size_t)col * a.n_tgt + t] = cplx{sc * e.re, sc * e.im};
    }
  }
}

template <typename T>
size_t asm_smem(int p, int q_src, int q_tgt) {
  return ((size_t)q_src * q_tgt + 1) * 8 + 4 * (size_t)(p + 2) * kAsmLanes * sizeof(T) + 16;
}

int afail(int code, const char* what) {
  char buf[320];
  snprintf(buf, sizeof(buf), "qbx_assemble: %s", what);
  return host_fail(code, buf);
}

int acuda(cudaError_t e, const char* what) {
  char buf[320];
  snprintf(buf, sizeof(buf), "qbx_assemble: %s: %s", what, cudaGetErrorString(e));
  return host_fail(QBX_ECUDA, buf);
}

}  // namespace

extern "C" int qbx_assemble_cfie(qbx_plan* plan, const qbx_geom* g, qbx_c64 k, qbx_c64 eta, int p, qbx_c64* A,
                                 void* stream) {
  if (!plan || !g || !A) return afail(QBX_EINVAL, "NULL plan, geometry or matrix");
  int device, q_tgt, q_src;
  const double* P;
  host_plan_info(plan, &device, &q_tgt, &q_src, &P);
  if (g->q_tgt != q_tgt || g->q_src != q_src || g->M < 1 || g->n_tgt != g->M * q_tgt || g->n_src != g->M * q_src)
    return afail(QBX_EINVAL, "geometry inconsistent with the plan");
  if (!g->src_x || !g->src_nx || !g->src_w || !g->tgt_x || !g->tgt_w || !g->ctr_x)
    return afail(QBX_EINVAL, "geometry: NULL array");
  if (q_tgt > kAsmQ) return afail(QBX_EINVAL, "q_tgt above 16");
  if (!isfinite(k.re) || !isfinite(k.im) || k.im < 0.0 || (k.im == 0.0 && !(k.re > 0.0)))
    return afail(QBX_EINVAL, "k must be finite with Im k >= 0 (real k > 0)");
  if (!isfinite(eta.re) || !isfinite(eta.im)) return afail(QBX_EINVAL, "eta is not finite");
  if (p < 0 || p > QBX_MAX_P) return afail(QBX_EINVAL, "p outside [0, QBX_MAX_P]");
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return acuda(e, "cudaSetDevice");
  AsmArgs a{};
  a.kre = k.re;
  a.kim = k.im;
  a.eta_re = eta.re;
  a.eta_im = eta.im;
  a.p = p;
  a.n_tgt = g->n_tgt;
  a.q_tgt = q_tgt;
  a.q_src = q_src;
  a.M = g->M;
  a.cx = g->ctr_x;
  a.cy = g->ctr_y;
  a.tx = g->tgt_x;
  a.ty = g->tgt_y;
  a.tw = g->tgt_w;
  a.sx = g->src_x;
  a.sy = g->src_y;
  a.snx = g->src_nx;
  a.sny = g->src_ny;
  a.sw = g->src_w;
  a.P = P;
  a.out = reinterpret_cast<cplx*>(A);
  const bool ck = k.im != 0.0;
  const size_t smem = ck ? asm_smem<cplx>(p, q_src, q_tgt) : asm_smem<double>(p, q_src, q_tgt);
  if (smem > 200 * 1024) return afail(QBX_EINVAL, "p too large");
  // panel groups: about 8192 CTAs in all (some 18 waves of the resident
  // CTAs), so that the last, partly filled wave costs little
  const unsigned gx = (unsigned)((g->n_tgt + kAsmLanes - 1) / kAsmLanes);
  const unsigned gy = (unsigned)std::max(1, std::min((g->M + kAsmWarps - 1) / kAsmWarps, (int)((8192 + gx - 1) / gx)));
  const dim3 grid(gx, gy);
  cudaStream_t st = (cudaStream_t)stream;
  a.hk_tab = host_plan_hk_table(plan, k, st, &e);
  if (e != cudaSuccess) return acuda(e, "complex-k amplitude table");
  if (ck) {
    e = cudaFuncSetAttribute(k_assemble_cfie<cplx>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_assemble_cfie<cplx><<<grid, kAsmLanes * kAsmWarps, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_assemble_cfie<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_assemble_cfie<double><<<grid, kAsmLanes * kAsmWarps, smem, st>>>(a);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? QBX_OK : acuda(e, "assembly kernel");
}
