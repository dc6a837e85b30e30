// qbx_shape.cu -- qbx_apply_shape_adjoint: the reverse-mode gradient of a
// real functional of the on-surface S apply with respect to the curve
// samples (gamma, gamma' at the target and source nodes) that qbx_geometry
// consumed.
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
#include "qbx_device.cuh"
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

struct Layout {
  size_t wd, fpart, gc, coef, cgeo, apart, qh, dh, total;
};

Layout layout(int M, int q_tgt, int q_src, int nc, int p, int nrhs, bool ck, int ns_fwd, int ns_adj) {
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
  o += host_align256((size_t)nc * 3 * 8);
  L.qh = o;
  o += host_align256(n_tgt * 8);
  L.dh = o;
  o += host_align256((size_t)M * 8);
  L.fpart = o;
  o += host_align256((size_t)ns_fwd * nc * kNcFwd * nrhs * 16);
  L.apart = o;
  o += host_align256((size_t)ns_adj * n_src * kNcAdj * nrhs * 16);
  L.total = o + 256;
  return L;
}

}  // namespace

extern "C" size_t qbx_shape_adjoint_workspace_bytes(int M, int q_tgt, int q_src, int p, int nrhs) {
  if (M < 1 || q_tgt < 1 || q_src < 1 || p < 0 || nrhs < 1) return 0;
  return layout(M, q_tgt, q_src, 2 * M * q_tgt, p, nrhs, true, kMaxSplit, kMaxSplit).total;
}

extern "C" int qbx_apply_shape_adjoint(qbx_plan* plan, const qbx_geom* g, int side, qbx_c64 k, int p,
                                       const qbx_c64* dens_tgt, const qbx_c64* gout, int nrhs,
                                       const double* dgam_tgt, const double* dgam_src, double* g_gam_tgt,
                                       double* g_dgam_tgt, double* g_gam_src, double* g_dgam_src,
                                       void* stream) {
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
  const int chunk = apply_chunk(kOpsFwd);
  if (apply_smem_bytes(kOpsFwd, ck, p, chunk) > 220 * 1024) return sfail(QBX_EINVAL, "p too large");
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return scuda(e, "cudaSetDevice");
  // split counts: the forward sweep as the apply chooses them, the transposed
  // sweep about six CTAs per SM; both shrink to fit the workspace
  const Layout L0 = layout(g->M, q_tgt, q_src, nc, p, nrhs, ck, 0, 0);
  if (ws_bytes < L0.total + 512) return sfail(QBX_ENOMEM, "workspace too small");
  const size_t avail = ws_bytes - L0.total - 512;
  const size_t per_fwd = (size_t)nc * kNcFwd * nrhs * 16, per_adj = (size_t)n_src * kNcAdj * nrhs * 16;
  const int occ = ck ? apply_occupancy_cplx(kOpsFwd, p, std::min(chunk, nrhs))
                     : apply_occupancy_real(kOpsFwd, p, std::min(chunk, nrhs));
  const int units = (nc + kApplyThreads - 1) / kApplyThreads;
  int ns_fwd = host_choose_split_waves(num_sms, occ, units, n_src, per_fwd, avail / 2);
  const int tiles = (n_src + kGrpCentres - 1) / kGrpCentres;
  int ns_adj = std::max(1, (num_sms * 6 + tiles - 1) / tiles);
  ns_adj = std::min(ns_adj, std::max(1, nc / kGrpTile));
  ns_adj = std::min(ns_adj, kMaxSplit);
  ns_adj = (int)std::min<size_t>((size_t)ns_adj, (avail - std::min(avail, (size_t)ns_fwd * per_fwd)) / per_adj);
  if (ns_fwd < 1 || ns_adj < 1) return sfail(QBX_ENOMEM, "workspace too small for the partial sums");
  const Layout L = layout(g->M, q_tgt, q_src, nc, p, nrhs, ck, ns_fwd, ns_adj);
  if (L.total > ws_bytes) return sfail(QBX_ENOMEM, "workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)host_align256((size_t)ws);
  void* wd = base + L.wd;
  // (w sigma)_s
  e = launch_upsample(g->M, q_tgt, q_src, nrhs, P, g->src_w, dens_tgt, wd, st);
  if (e != cudaSuccess) return scuda(e, "upsample");
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
  a.hk_tab = host_plan_hk_table(plan, k, st, &e);
  if (e != cudaSuccess) return scuda(e, "complex-k amplitude table");
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
