// qbx_adjoint.cu -- qbx_apply_adjoint: the vector-Jacobian product of the
// on-surface apply of S or D with respect to the density (the transposed
// QBX sweep, targets -> expansions -> sources -> target grid).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <algorithm>
#include "../../include/qbx.h"
#include "qbx_device.cuh"
#include "qbx_internal.h"

using namespace qbx;

namespace {

int afail(int code, const char* what) {
  char buf[320];
  snprintf(buf, sizeof(buf), "qbx_apply_adjoint: %s", what);
  return host_fail(code, buf);
}

int acuda(cudaError_t e, const char* what) {
  char buf[320];
  snprintf(buf, sizeof(buf), "qbx_apply_adjoint: %s: %s", what, cudaGetErrorString(e));
  return host_fail(QBX_ECUDA, buf);
}

// gradient at each centre: (-i/4) * side weight * g_t  (conj(i/4) = -i/4;
// the two-sided average gives each side weight 1/2)
__global__ void k_adj_spread(int n_tgt, int nsides, int nrhs, const cplx* g, cplx* gc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_tgt * nrhs) return;
  const double wgt = nsides == 2 ? 0.5 : 1.0;
  const cplx v = g[idx];
  const cplx s = cplx{0.25 * wgt * v.im, -0.25 * wgt * v.re};   // (-i/4) w v
  gc[idx] = s;
  if (nsides == 2) gc[(size_t)n_tgt * nrhs + idx] = s;
}

// v_s = w_s * sum over centre splits
__global__ void k_adj_reduce(int n_src, int nsplit, int nrhs, const double* w, const cplx* part, cplx* v) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_src * nrhs) return;
  cplx u{0.0, 0.0};
  for (int k = 0; k < nsplit; ++k) u = u + part[(size_t)k * n_src * nrhs + idx];
  v[idx] = w[idx / nrhs] * u;
}

// gdens[m q_tgt + i][r] = sum_j P[j][i] v[m q_src + j][r]  (+ the PV jump term of D)
__global__ void k_adj_interp_t(int n_tgt, int q_tgt, int q_src, int nrhs, const double* P, const cplx* v,
                               double jump, const cplx* g, cplx* out, int* status) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_tgt * nrhs) return;
  const int t = idx / nrhs, r = idx - t * nrhs;
  const int m = t / q_tgt, i = t - m * q_tgt;
  const cplx* vv = v + (size_t)m * q_src * nrhs + r;
  double re = 0.0, im = 0.0;
  for (int j = 0; j < q_src; ++j) {
    const double c = P[(size_t)j * q_tgt + i];
    const cplx x = vv[(size_t)j * nrhs];
    re = fma(c, x.re, re);
    im = fma(c, x.im, im);
  }
  cplx res{re, im};
  if (jump != 0.0) res = res + jump * g[idx];
  out[idx] = res;
  if (!(isfinite(res.re) && isfinite(res.im))) atomicOr(status, 1);
}

}  // namespace

extern "C" int qbx_apply_adjoint(qbx_plan* plan, const qbx_geom* g, int op, int side, int limit, qbx_c64 k,
                                 int p, const qbx_c64* gout, int nrhs, qbx_c64* gdens, void* stream) {
  if (!plan) return afail(QBX_EINVAL, "plan is NULL");
  if (!g) return afail(QBX_EINVAL, "geometry is NULL");
  int device, q_tgt, q_src, num_sms;
  const double* P;
  host_plan_info(plan, &device, &q_tgt, &q_src, &P);
  void* ws;
  size_t ws_bytes;
  int* status;
  host_plan_workspace(plan, &ws, &ws_bytes, &num_sms, &status);
  if (g->q_tgt != q_tgt || g->q_src != q_src || g->M < 1 || g->n_tgt != g->M * q_tgt || g->n_src != g->M * q_src)
    return afail(QBX_EINVAL, "geometry inconsistent with the plan");
  if (!g->src_x || !g->src_w || !g->ctr_x || !g->tgt_x) return afail(QBX_EINVAL, "geometry: NULL array");
  if (op != QBX_OP_S && op != QBX_OP_D) return afail(QBX_EINVAL, "op must be S or D");
  if (side != QBX_SIDE_INT && side != QBX_SIDE_EXT && side != QBX_SIDE_TWO) return afail(QBX_EINVAL, "bad side");
  if (limit != QBX_LIMIT_ONE_SIDED && limit != QBX_LIMIT_PV) return afail(QBX_EINVAL, "bad limit");
  if (!isfinite(k.re) || !isfinite(k.im) || k.im < 0.0 || (k.im == 0.0 && !(k.re > 0.0)))
    return afail(QBX_EINVAL, "k must be finite with Im k >= 0 (real k > 0)");
  if (p < 0 || p > QBX_MAX_P) return afail(QBX_EINVAL, "p outside [0, QBX_MAX_P]");
  if (nrhs < 1 || !gout || !gdens) return afail(QBX_EINVAL, "bad nrhs or NULL array");
  const bool ck = k.im != 0.0;
  const int nsides = side == QBX_SIDE_TWO ? 2 : 1;
  const int c0 = side == QBX_SIDE_EXT ? g->n_tgt : 0;
  const int nc = nsides * g->n_tgt;
  const int nslots = op == QBX_OP_D ? 2 : 1;
  // workspace: gc | coef | cgeo | v | part
  const size_t b_gc = host_align256((size_t)nc * nrhs * 16);
  const size_t b_coef = host_align256((size_t)nc * nslots * (p + 2) * (ck ? 16 : 8));
  const size_t b_geo = host_align256((size_t)nc * 3 * 8);
  const size_t b_v = host_align256((size_t)g->n_src * nrhs * 16);
  const size_t fixed = b_gc + b_coef + b_geo + b_v + 256;
  if (ws_bytes < fixed) return afail(QBX_ENOMEM, "workspace too small");
  const size_t per_split = (size_t)g->n_src * nrhs * 16;
  const int tiles = (g->n_src + kGrpCentres - 1) / kGrpCentres;
  int ns = std::max(1, (num_sms * 6 + tiles - 1) / tiles);
  ns = std::min(ns, std::max(1, nc / kGrpTile));
  ns = std::min(ns, kMaxSplit);
  ns = std::min<long>(ns, (long)((ws_bytes - fixed) / per_split));
  if (ns < 1) return afail(QBX_ENOMEM, "workspace too small for the partial sums");
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return acuda(e, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)host_align256((size_t)ws);
  void* gc = base;
  void* coef = base + b_gc;
  double* cgeo = (double*)(base + b_gc + b_coef);
  void* v = base + b_gc + b_coef + b_geo;
  void* part = base + b_gc + b_coef + b_geo + b_v;
  k_adj_spread<<<(g->n_tgt * nrhs + 255) / 256, 256, 0, st>>>(g->n_tgt, nsides, nrhs, (const cplx*)gout, (cplx*)gc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return acuda(e, "spread kernel");
  AdjArgs a{};
  a.ops = 1 << op;
  a.p = p;
  a.nrhs = nrhs;
  a.kre = k.re;
  a.kim = k.im;
  a.n_ctr = nc;
  a.n_tgt = g->n_tgt;
  a.n_src = g->n_src;
  a.cx = g->ctr_x + c0;
  a.cy = g->ctr_y + c0;
  a.tx = g->tgt_x;
  a.ty = g->tgt_y;
  a.sx = g->src_x;
  a.sy = g->src_y;
  a.snx = g->src_nx;
  a.sny = g->src_ny;
  a.gc = gc;
  a.coef = coef;
  a.cgeo = cgeo;
  a.nsplit = ns;
  a.ctr_per_split = (nc + ns - 1) / ns;
  a.part = part;
  a.hk_tab = host_plan_hk_table(plan, k, st, &e);
  if (e != cudaSuccess) return acuda(e, "complex-k amplitude table");
  e = ck ? launch_adjoint_cplx(a, st) : launch_adjoint_real(a, st);
  if (e != cudaSuccess) return acuda(e, "adjoint kernel");
  k_adj_reduce<<<(g->n_src * nrhs + 255) / 256, 256, 0, st>>>(g->n_src, ns, nrhs, g->src_w, (const cplx*)part,
                                                              (cplx*)v);
  // PV of D: u = lim - sg mu / 2 (sg = +1 exterior, -1 interior): adjoint adds -sg g / 2
  double jump = 0.0;
  if (op == QBX_OP_D && side != QBX_SIDE_TWO && limit == QBX_LIMIT_PV) jump = side == QBX_SIDE_EXT ? -0.5 : 0.5;
  k_adj_interp_t<<<(g->n_tgt * nrhs + 255) / 256, 256, 0, st>>>(g->n_tgt, q_tgt, q_src, nrhs, P, (const cplx*)v,
                                                                jump, (const cplx*)gout, (cplx*)gdens, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return acuda(e, "finish kernels");
  return QBX_OK;
}
