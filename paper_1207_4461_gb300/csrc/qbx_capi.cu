// qbx_capi.cu -- host side of the C ABI declared in include/qbx.h: plans,
// the Gauss-Legendre rule, the per-panel interpolation matrix, argument
// checks and the launch sequence of each call.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>
#include <algorithm>
#include <string>
#include <vector>
#include "../../include/qbx.h"
#include "qbx_internal.h"

using namespace qbx;

struct qbx_plan {
  int device;
  int num_sms;
  int q_tgt, q_src;
  double* d_interp;   // [q_src][q_tgt]
  double* d_wgl_tgt;  // [q_tgt]
  double* d_wgl_src;  // [q_src]
  double* d_diff;     // [q_tgt][q_tgt] d/dxi of the target-grid interpolant at its nodes
  int* d_status;
  void* ws;
  size_t ws_bytes;
  // optional timing of the pair-sum launches of the last apply
  bool timing = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // waves of resident CTAs the split choice aims for (qbx_plan_set_min_waves)
  int min_waves = 1;
  // H0/H1 amplitude table of the ray z = k rho for the last complex k
  // (tab_kim = 0: none made yet)
  double* d_hk_tab;
  double tab_kre, tab_kim;
};

namespace {

thread_local std::string g_err = "";

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(QBX_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call, where)                               \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

// Gauss-Legendre by Newton's method on P_q.  P_q and P_q' come from the
// recurrences (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1} and
// P_n' = n (P_{n-1} - x P_n) / (1 - x^2).  Starting guess: Tricomi's
// asymptotic node formula x_i ~ (1 - (q-1)/(8 q^3)) cos(pi (4i - 1)/(4q + 2)).
void gl_rule(int q, double* x, double* w) {
  for (int i = 1; i <= q; ++i) {
    double th = M_PI * (4.0 * i - 1.0) / (4.0 * q + 2.0);
    double xi = (1.0 - (q - 1.0) / (8.0 * q * q * q)) * cos(th);
    double dp = 1.0;
    for (int it = 0; it < 60; ++it) {
      double pm = 1.0, p = xi;
      for (int n = 1; n < q; ++n) {
        double pn = ((2.0 * n + 1.0) * xi * p - n * pm) / (n + 1.0);
        pm = p;
        p = pn;
      }
      if (q == 1) { p = xi; pm = 1.0; }
      dp = q * (pm - xi * p) / (1.0 - xi * xi);
      double step = p / dp;
      xi -= step;
      if (fabs(step) <= 4e-16 * fabs(xi) + 1e-300) {
        // one more evaluation at the converged point for the weight
        pm = 1.0;
        p = xi;
        for (int n = 1; n < q; ++n) {
          double pn = ((2.0 * n + 1.0) * xi * p - n * pm) / (n + 1.0);
          pm = p;
          p = pn;
        }
        if (q == 1) { p = xi; pm = 1.0; }
        dp = q * (pm - xi * p) / (1.0 - xi * xi);
        break;
      }
    }
    x[q - i] = xi;
    w[q - i] = 2.0 / ((1.0 - xi * xi) * dp * dp);
  }
}

// Legendre polynomials P_0..P_{n-1} at x.
void legendre_all(int n, double x, double* P) {
  P[0] = 1.0;
  if (n > 1) P[1] = x;
  for (int j = 1; j + 1 < n; ++j) P[j + 1] = ((2.0 * j + 1.0) * x * P[j] - j * P[j - 1]) / (j + 1.0);
}

// Interpolation from the q_tgt target nodes to the q_src source nodes of a
// panel through the Legendre expansion of the interpolant:
// f(y) = sum_{n<q_tgt} c_n P_n(y), c_n = (2n+1)/2 sum_i w_i f_i P_n(x_i)
// (exact for degree < q_tgt since the q_tgt-point rule integrates degree
// 2 q_tgt - 1), so M[j][i] = sum_n (2n+1)/2 w_i P_n(x_i) P_n(y_j).
void interp_matrix(int qt, int qs, std::vector<double>& Mx) {
  std::vector<double> xt(qt), wt(qt), xs(qs), ws(qs), Pt(qt * qt), Ps(qt);
  gl_rule(qt, xt.data(), wt.data());
  gl_rule(qs, xs.data(), ws.data());
  for (int i = 0; i < qt; ++i) legendre_all(qt, xt[i], &Pt[i * qt]);
  Mx.assign((size_t)qs * qt, 0.0);
  for (int j = 0; j < qs; ++j) {
    legendre_all(qt, xs[j], Ps.data());
    for (int i = 0; i < qt; ++i) {
      double s = 0.0;
      for (int n = 0; n < qt; ++n) s += (2.0 * n + 1.0) * 0.5 * Pt[i * qt + n] * Ps[n];
      Mx[(size_t)j * qt + i] = s * wt[i];
    }
  }
}

// Differentiation at the target nodes through the same Legendre expansion:
// f'(x_i) = sum_j Dx[i][j] f_j, Dx[i][j] = sum_n (2n+1)/2 w_j P_n(x_j) P_n'(x_i),
// with P'_{n+1} = P'_{n-1} + (2n+1) P_n.
void diff_matrix(int q, std::vector<double>& Dx) {
  std::vector<double> x(q), w(q), P(q * q), dP(q);
  gl_rule(q, x.data(), w.data());
  for (int j = 0; j < q; ++j) legendre_all(q, x[j], &P[j * q]);
  Dx.assign((size_t)q * q, 0.0);
  for (int i = 0; i < q; ++i) {
    dP[0] = 0.0;
    if (q > 1) dP[1] = 1.0;
    for (int n = 1; n + 1 < q; ++n) dP[n + 1] = dP[n - 1] + (2.0 * n + 1.0) * P[i * q + n];
    for (int j = 0; j < q; ++j) {
      double acc = 0.0;
      for (int n = 0; n < q; ++n) acc += (2.0 * n + 1.0) * 0.5 * P[j * q + n] * dP[n];
      Dx[(size_t)i * q + j] = acc * w[j];
    }
  }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int check_plan(const qbx_plan* p) {
  if (!p) return fail(QBX_EINVAL, "plan is NULL");
  return QBX_OK;
}

int check_geom(const qbx_plan* pl, const qbx_geom* g, bool need_ctr) {
  if (!g) return fail(QBX_EINVAL, "geometry is NULL");
  if (g->M < 1) return fail(QBX_EINVAL, "geometry: M = %d < 1", g->M);
  if (g->q_tgt != pl->q_tgt || g->q_src != pl->q_src)
    return fail(QBX_EINVAL, "geometry q (%d, %d) differs from the plan's (%d, %d)", g->q_tgt,
                g->q_src, pl->q_tgt, pl->q_src);
  if (g->n_tgt != g->M * g->q_tgt || g->n_src != g->M * g->q_src)
    return fail(QBX_EINVAL, "geometry: n_tgt/n_src inconsistent with M*q");
  if (!g->src_x || !g->src_y || !g->src_nx || !g->src_ny || !g->src_w || !g->tgt_x || !g->tgt_y ||
      !g->tgt_nx || !g->tgt_ny)
    return fail(QBX_EINVAL, "geometry: NULL node array");
  if (need_ctr && (!g->ctr_x || !g->ctr_y || !g->ctr_r))
    return fail(QBX_EINVAL, "geometry: NULL centre array");
  return QBX_OK;
}

int check_k(qbx_c64 k) {
  if (!isfinite(k.re) || !isfinite(k.im)) return fail(QBX_EINVAL, "k is not finite");
  if (k.im < 0.0) return fail(QBX_EINVAL, "Im k = %g < 0 (need Im k >= 0)", k.im);
  if (k.im == 0.0 && !(k.re > 0.0))
    return fail(QBX_EINVAL, "real k = %g must be > 0 (k = 0 is Laplace; H0 has a cut on the negative axis)", k.re);
  return QBX_OK;
}

int check_p(int p) {
  if (p < 0 || p > QBX_MAX_P) return fail(QBX_EINVAL, "p = %d outside [0, %d]", p, QBX_MAX_P);
  return QBX_OK;
}

int side_range(int side, int n_tgt, int* c0, int* nc) {
  switch (side) {
    case QBX_SIDE_INT: *c0 = 0; *nc = n_tgt; return QBX_OK;
    case QBX_SIDE_EXT: *c0 = n_tgt; *nc = n_tgt; return QBX_OK;
    case QBX_SIDE_TWO: *c0 = 0; *nc = 2 * n_tgt; return QBX_OK;
    default: return fail(QBX_EINVAL, "side = %d is not INT/EXT/TWO", side);
  }
}

int choose_split(const qbx_plan* pl, int n_units, int n_src, size_t bytes_per_split, size_t avail) {
  return qbx::host_choose_split(pl->num_sms, n_units, n_src, bytes_per_split, avail);
}

int split_len(int n_src, int ns) { return qbx::host_split_len(n_src, ns); }

}  // namespace

namespace qbx {

void host_interp_matrix(int qt, int qs, std::vector<double>& Mx) { interp_matrix(qt, qs, Mx); }

int host_fail(int code, const char* msg) { return fail(code, "%s", msg); }

void host_plan_workspace(const qbx_plan* plan, void** ws, size_t* bytes, int* num_sms, int** status) {
  *ws = plan->ws;
  *bytes = plan->ws_bytes;
  *num_sms = plan->num_sms;
  *status = plan->d_status;
}

void host_plan_info(const qbx_plan* plan, int* device, int* q_tgt, int* q_src, const double** interp) {
  *device = plan->device;
  *q_tgt = plan->q_tgt;
  *q_src = plan->q_src;
  *interp = plan->d_interp;
}


// The plan's amplitude table for complex k (made on `st` when k changes;
// later calls on the plan's streams see it in stream order), or null for real k.
const double* host_plan_hk_table(qbx_plan* plan, qbx_c64 k, cudaStream_t st, cudaError_t* err) {
  *err = cudaSuccess;
  if (k.im == 0.0) return nullptr;
  if (plan->tab_kre != k.re || plan->tab_kim != k.im) {
    *err = launch_hk_table(k.re, k.im, plan->d_hk_tab, st);
    if (*err != cudaSuccess) return nullptr;
    plan->tab_kre = k.re;
    plan->tab_kim = k.im;
  }
  return plan->d_hk_tab;
}

size_t host_align256(size_t b) { return align256(b); }

// Number of source splits: fill about two waves of 4 CTAs per SM, bounded by
// kMaxSplit, by one source tile per split, and by the workspace.
int host_choose_split(int num_sms, int n_units, int n_src, size_t bytes_per_split, size_t avail) {
  const int target = num_sms * 8;
  int ns = (target + n_units - 1) / std::max(n_units, 1);
  ns = std::min(ns, kMaxSplit);
  ns = std::min(ns, std::max(1, (n_src + kSrcTile - 1) / kSrcTile));
  ns = std::max(ns, 1);
  if (bytes_per_split > 0) {
    size_t fit = avail / bytes_per_split;
    if ((size_t)ns > fit) ns = (int)fit;
  }
  return ns;
}

// Source splits for the fused and group applies: the fewest splits whose
// items (n_units x ns equal CTAs) make at least `min_waves` waves of the
// kernel's resident CTAs (occ per SM) and fill them to at least 95 %, else
// the best filling; at least 64 sources per split, at most kMaxSplit, and
// within the workspace.  More waves let the block scheduler even out CTAs
// whose pairs take different branches.
int host_choose_split_waves(int num_sms, int occ, int n_units, int n_src, size_t bytes_per_split,
                            size_t avail, int min_waves) {
  if (occ < 1) return host_choose_split(num_sms, n_units, n_src, bytes_per_split, avail);
  const long slots = (long)num_sms * occ;
  long ns_max = std::min<long>(kMaxSplit, std::max(1, n_src / 64));
  if (bytes_per_split > 0) ns_max = std::min<long>(ns_max, (long)(avail / bytes_per_split));
  if (ns_max < 1) return 0;
  const long units = std::max(n_units, 1);
  long best = 1;
  double best_score = -1.0;
  for (long ns = 1; ns <= ns_max; ++ns) {
    const long items = units * ns;
    const long waves = (items + slots - 1) / slots;
    const double fill = (double)items / (double)(waves * slots);
    if (fill >= 0.95 && waves >= min_waves) return (int)ns;
    const double score = fill + (waves >= min_waves ? 1.0 : 0.0) + 1e-3 * std::min<long>(waves, min_waves);
    if (score > best_score + 1e-12) {
      best_score = score;
      best = ns;
    }
  }
  return (int)best;
}

// sources per split (equal shares; the last tile of a split may be partial)
int host_split_len(int n_src, int ns) { return (n_src + ns - 1) / ns; }

}  // namespace qbx

extern "C" {

const char* qbx_last_error(void) { return g_err.c_str(); }

int qbx_version(void) { return 1; }

int qbx_gauss_legendre(int q, double* nodes, double* weights) {
  if (q < 1 || q > QBX_MAX_Q) return fail(QBX_EINVAL, "q = %d outside [1, %d]", q, QBX_MAX_Q);
  if (!nodes || !weights) return fail(QBX_EINVAL, "NULL output");
  gl_rule(q, nodes, weights);
  return QBX_OK;
}

size_t qbx_workspace_bytes(int n_src, int n_ctr, int ncoef, int nrhs) {
  if (n_src < 0 || n_ctr < 0 || ncoef < 0 || nrhs < 0) return 0;
  return 3 * align256((size_t)n_src * nrhs * 16) +
         align256((size_t)kMaxSplit * n_ctr * ncoef * nrhs * 16) + 512;
}

int qbx_plan_create(qbx_plan** plan, int device, int q_tgt, int q_src, size_t workspace_bytes) {
  if (!plan) return fail(QBX_EINVAL, "plan out-pointer is NULL");
  *plan = nullptr;
  if (q_tgt < 1 || q_tgt > QBX_MAX_Q || q_src < 1 || q_src > QBX_MAX_Q)
    return fail(QBX_EINVAL, "q_tgt = %d, q_src = %d outside [1, %d]", q_tgt, q_src, QBX_MAX_Q);
  CK(cudaSetDevice(device), "cudaSetDevice");
  qbx_plan* p = new qbx_plan();
  memset(p, 0, sizeof(*p));
  p->min_waves = 1;
  p->device = device;
  p->q_tgt = q_tgt;
  p->q_src = q_src;
  cudaError_t e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, device);
  std::vector<double> Mx, Dx, xt(q_tgt), wt(q_tgt), xs(q_src), ws(q_src);
  interp_matrix(q_tgt, q_src, Mx);
  diff_matrix(q_tgt, Dx);
  gl_rule(q_tgt, xt.data(), wt.data());
  gl_rule(q_src, xs.data(), ws.data());
  if (e == cudaSuccess) e = cudaMalloc(&p->d_interp, Mx.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_wgl_tgt, q_tgt * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_wgl_src, q_src * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_diff, Dx.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_hk_tab, (size_t)hk_table_doubles() * sizeof(double));
  if (e == cudaSuccess && workspace_bytes > 0) e = cudaMalloc(&p->ws, workspace_bytes);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_diff, Dx.data(), Dx.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_interp, Mx.data(), Mx.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_wgl_tgt, wt.data(), q_tgt * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_wgl_src, ws.data(), q_src * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    qbx_plan_destroy(p);
    return cuda_fail(e, "qbx_plan_create");
  }
  p->ws_bytes = workspace_bytes;
  *plan = p;
  return QBX_OK;
}

int qbx_plan_destroy(qbx_plan* p) {
  if (!p) return QBX_OK;
  cudaSetDevice(p->device);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  cudaFree(p->d_interp);
  cudaFree(p->d_wgl_tgt);
  cudaFree(p->d_wgl_src);
  cudaFree(p->d_status);
  cudaFree(p->d_diff);
  cudaFree(p->d_hk_tab);
  cudaFree(p->ws);
  delete p;
  return QBX_OK;
}

int qbx_plan_set_timing(qbx_plan* p, int on) {
  if (int rc = check_plan(p)) return rc;
  CK(cudaSetDevice(p->device), "cudaSetDevice");
  if (on && !p->ev0) {
    CK(cudaEventCreate(&p->ev0), "cudaEventCreate");
    CK(cudaEventCreate(&p->ev1), "cudaEventCreate");
  }
  p->timing = on != 0;
  return QBX_OK;
}

int qbx_plan_set_min_waves(qbx_plan* p, int waves) {
  if (int rc = check_plan(p)) return rc;
  if (waves < 1 || waves > 64) return fail(QBX_EINVAL, "min_waves = %d outside [1, 64]", waves);
  p->min_waves = waves;
  return QBX_OK;
}

int qbx_plan_kernel_ms(qbx_plan* p, float* ms) {
  if (int rc = check_plan(p)) return rc;
  if (!ms) return fail(QBX_EINVAL, "NULL output");
  if (!p->timing) return fail(QBX_EINVAL, "timing is off (qbx_plan_set_timing)");
  CK(cudaSetDevice(p->device), "cudaSetDevice");
  CK(cudaEventSynchronize(p->ev1), "cudaEventSynchronize");
  CK(cudaEventElapsedTime(ms, p->ev0, p->ev1), "cudaEventElapsedTime");
  return QBX_OK;
}

int qbx_sync_status(qbx_plan* p, void* stream) {
  if (int rc = check_plan(p)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int h = 0;
  CK(cudaMemcpyAsync(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, st), "status copy");
  CK(cudaStreamSynchronize(st), "status sync");
  CK(cudaMemsetAsync(p->d_status, 0, sizeof(int), st), "status clear");
  CK(cudaStreamSynchronize(st), "status sync");
  if (h) return fail(QBX_ENONFINITE, "a kernel produced a non-finite value");
  return QBX_OK;
}

int qbx_geometry_rule(qbx_plan* p, qbx_geom* g, const double* t_edges, const double* gam_tgt,
                      const double* dgam_tgt, const double* gam_src, const double* dgam_src, int rule,
                      double r_factor, void* stream) {
  if (int rc = check_plan(p)) return rc;
  if (!g) return fail(QBX_EINVAL, "geometry is NULL");
  g->n_tgt = g->M * g->q_tgt;
  g->n_src = g->M * g->q_src;
  if (int rc = check_geom(p, g, true)) return rc;
  if (!g->panel_h || !g->ctr_ratio || !g->src_w || !g->tgt_w) return fail(QBX_EINVAL, "geometry: NULL output");
  if (!t_edges || !gam_tgt || !dgam_tgt || !gam_src || !dgam_src) return fail(QBX_EINVAL, "NULL curve samples");
  if (!(r_factor > 0.0) || !isfinite(r_factor)) return fail(QBX_EINVAL, "r_factor must be > 0");
  if (rule != QBX_RADIUS_H && rule != QBX_RADIUS_SQRT_H && rule != QBX_RADIUS_ADMISSIBLE)
    return fail(QBX_EINVAL, "bad radius rule %d", rule);
  CK(cudaSetDevice(p->device), "cudaSetDevice");
  CK(launch_geometry(g->M, g->q_tgt, g->q_src, t_edges, gam_tgt, dgam_tgt, gam_src, dgam_src,
                     p->d_wgl_tgt, p->d_wgl_src, r_factor, rule, *g, (cudaStream_t)stream),
     "geometry kernels");
  return QBX_OK;
}

int qbx_geometry(qbx_plan* p, qbx_geom* g, const double* t_edges, const double* gam_tgt,
                 const double* dgam_tgt, const double* gam_src, const double* dgam_src,
                 double r_factor, void* stream) {
  return qbx_geometry_rule(p, g, t_edges, gam_tgt, dgam_tgt, gam_src, dgam_src, QBX_RADIUS_H, r_factor, stream);
}

int qbx_upsample(qbx_plan* p, const qbx_geom* g, const qbx_c64* dens_tgt, int nrhs,
                 qbx_c64* wdens_src, void* stream) {
  if (int rc = check_plan(p)) return rc;
  if (int rc = check_geom(p, g, false)) return rc;
  if (nrhs < 1) return fail(QBX_EINVAL, "nrhs = %d < 1", nrhs);
  if (!dens_tgt || !wdens_src) return fail(QBX_EINVAL, "NULL density");
  CK(cudaSetDevice(p->device), "cudaSetDevice");
  CK(launch_upsample(g->M, g->q_tgt, g->q_src, nrhs, p->d_interp, g->src_w, dens_tgt, wdens_src,
                     (cudaStream_t)stream),
     "upsample kernel");
  return QBX_OK;
}

int qbx_form_locals(qbx_plan* p, const qbx_geom* g, int kind, int side, qbx_c64 k, int pp,
                    const qbx_c64* wdens_src, int nrhs, qbx_c64* alpha, void* stream) {
  if (int rc = check_plan(p)) return rc;
  if (int rc = check_geom(p, g, true)) return rc;
  if (kind != QBX_OP_S && kind != QBX_OP_D) return fail(QBX_EINVAL, "kind must be S or D");
  if (int rc = check_k(k)) return rc;
  if (int rc = check_p(pp)) return rc;
  if (nrhs < 1) return fail(QBX_EINVAL, "nrhs = %d < 1", nrhs);
  if (!wdens_src || !alpha) return fail(QBX_EINVAL, "NULL array");
  int c0, nc;
  if (int rc = side_range(side, g->n_tgt, &c0, &nc)) return rc;
  CK(cudaSetDevice(p->device), "cudaSetDevice");
  const int ncoef = 2 * pp + 1;
  // rhs per pass limited by the shared-memory accumulators
  int nr = nrhs;
  while (nr > 1 && form_smem_bytes(pp, nr) > 160 * 1024) nr = (nr + 1) / 2;
  if (form_smem_bytes(pp, nr) > 200 * 1024) return fail(QBX_EINVAL, "p = %d too large for form_locals", pp);
  const size_t per_split = (size_t)nc * ncoef * nrhs * 16;
  const int units = (nc + kFormThreads - 1) / kFormThreads;
  const int ns = choose_split(p, units, g->n_src, per_split, p->ws_bytes > 256 ? p->ws_bytes - 256 : 0);
  if (ns < 1) return fail(QBX_ENOMEM, "workspace too small for form_locals (need %zu bytes)", per_split);
  cudaStream_t st = (cudaStream_t)stream;
  void* part = (void*)align256((size_t)p->ws);
  FormArgs a{};
  a.kind = kind;
  a.p = pp;
  a.kre = k.re;
  a.kim = k.im;
  a.n_ctr = nc;
  a.cx = g->ctr_x + c0;
  a.cy = g->ctr_y + c0;
  a.src = SrcView{g->src_x, g->src_y, g->src_nx, g->src_ny, g->n_src};
  a.wd = wdens_src;
  a.nrhs = nrhs;
  a.nsplit = ns;
  a.src_per_split = split_len(g->n_src, ns);
  a.part = part;
  for (int r0 = 0; r0 < nrhs; r0 += nr) {
    a.rhs0 = r0;
    a.nr = std::min(nr, nrhs - r0);
    CK(launch_form(a, st), "form kernel");
  }
  CK(launch_form_finish(nc, ncoef, ns, nrhs, part, alpha, p->d_status, st), "form finish");
  return QBX_OK;
}

int qbx_eval_locals(qbx_plan* p, const qbx_geom* g, int side, qbx_c64 k, int pp, const qbx_c64* alpha,
                    int nrhs, int what, int n_eval, const double* ex, const double* ey,
                    const int* ectr, qbx_c64* out, void* stream) {
  if (int rc = check_plan(p)) return rc;
  if (int rc = check_geom(p, g, true)) return rc;
  if (int rc = check_k(k)) return rc;
  if (int rc = check_p(pp)) return rc;
  if (nrhs < 1) return fail(QBX_EINVAL, "nrhs = %d < 1", nrhs);
  if (what != QBX_VALUE && what != QBX_GRAD) return fail(QBX_EINVAL, "what must be VALUE or GRAD");
  if (!alpha || !out) return fail(QBX_EINVAL, "NULL array");
  int c0, nc;
  if (int rc = side_range(side, g->n_tgt, &c0, &nc)) return rc;
  if (n_eval < 0) return fail(QBX_EINVAL, "n_eval < 0");
  EvalArgs a{};
  if (n_eval == 0) {
    a.n_eval = nc;
    a.ex = a.ey = nullptr;
    a.ectr = nullptr;
  } else {
    if (!ex || !ey || !ectr) return fail(QBX_EINVAL, "n_eval > 0 needs ex, ey, ectr");
    a.n_eval = n_eval;
    a.ex = ex;
    a.ey = ey;
    a.ectr = ectr;
  }
  CK(cudaSetDevice(p->device), "cudaSetDevice");
  a.what = what;
  a.p = pp;
  a.kre = k.re;
  a.kim = k.im;
  a.cx = g->ctr_x + c0;
  a.cy = g->ctr_y + c0;
  a.n_tgt = g->n_tgt;
  a.tx = g->tgt_x;
  a.ty = g->tgt_y;
  a.alpha = alpha;
  a.nrhs = nrhs;
  a.out = out;
  a.n_ctr = nc;
  a.status = p->d_status;
  CK(launch_eval(a, (cudaStream_t)stream), "eval kernel");
  return QBX_OK;
}

static int far_impl(qbx_plan* p, const qbx_geom* g, int op, qbx_c64 k, const qbx_c64* wd, int nrhs,
                    int n_far, const double* x_far, qbx_c64* out, void* part, size_t avail,
                    cudaStream_t st) {
  const int ncomp = op == QBX_OP_GRAD_S ? 2 : 1;
  const size_t per_split = (size_t)n_far * ncomp * nrhs * 16;
  const int units = (n_far + kApplyThreads - 1) / kApplyThreads;
  const int ns = choose_split(p, units, g->n_src, per_split, avail);
  if (ns < 1) return fail(QBX_ENOMEM, "workspace too small for the far targets");
  FarArgs a{};
  a.op = op;
  a.kre = k.re;
  a.kim = k.im;
  a.n_far = n_far;
  a.xy = x_far;
  a.src = SrcView{g->src_x, g->src_y, g->src_nx, g->src_ny, g->n_src};
  a.wd = wd;
  a.nrhs = nrhs;
  a.nsplit = ns;
  a.src_per_split = split_len(g->n_src, ns);
  a.part = part;
  {
    cudaError_t te;
    a.hk_tab = host_plan_hk_table(p, k, st, &te);
    CK(te, "complex-k amplitude table");
  }
  for (int r0 = 0; r0 < nrhs; r0 += 8) {
    a.rhs0 = r0;
    a.nr = std::min(8, nrhs - r0);
    CK(launch_far(a, st), "far kernel");
  }
  CK(launch_far_finish(op, k.re, k.im, n_far, ns, nrhs, part, out, p->d_status, st), "far finish");
  return QBX_OK;
}

int qbx_far(qbx_plan* p, const qbx_geom* g, int op, qbx_c64 k, const qbx_c64* wdens_src, int nrhs,
            int n_far, const double* x_far, qbx_c64* out, void* stream) {
  if (int rc = check_plan(p)) return rc;
  if (int rc = check_geom(p, g, false)) return rc;
  if (op != QBX_OP_S && op != QBX_OP_D && op != QBX_OP_GRAD_S && op != QBX_OP_R)
    return fail(QBX_EINVAL, "bad op %d", op);
  if (int rc = check_k(k)) return rc;
  if (nrhs < 1) return fail(QBX_EINVAL, "nrhs = %d < 1", nrhs);
  if (n_far < 0) return fail(QBX_EINVAL, "n_far < 0");
  if (n_far == 0) return QBX_OK;
  if (!wdens_src || !x_far || !out) return fail(QBX_EINVAL, "NULL array");
  CK(cudaSetDevice(p->device), "cudaSetDevice");
  if (op == QBX_OP_R) {   // D's quadrature with the source tangents (Sec. 3.2, eq. riesz-def)
    const size_t tb = align256((size_t)g->n_src * 16);
    if (p->ws_bytes < tb + 512) return fail(QBX_ENOMEM, "workspace too small for the source tangents");
    char* base = (char*)align256((size_t)p->ws);
    double* tx = (double*)base;
    double* ty = tx + g->n_src;
    cudaStream_t st = (cudaStream_t)stream;
    CK(launch_tangents(g->n_src, g->src_nx, g->src_ny, tx, ty, st), "tangents");
    qbx_geom gt = *g;
    gt.src_nx = tx;
    gt.src_ny = ty;
    return far_impl(p, &gt, QBX_OP_D, k, wdens_src, nrhs, n_far, x_far, out, base + tb, p->ws_bytes - tb - 512, st);
  }
  void* part = (void*)align256((size_t)p->ws);
  return far_impl(p, g, op, k, wdens_src, nrhs, n_far, x_far, out, part,
                  p->ws_bytes > 256 ? p->ws_bytes - 256 : 0, (cudaStream_t)stream);
}

// On-surface apply of the operator subset `ops` (one pass over the pairs for
// all of them), plus far targets when a single operator is requested.
// tangent: the R operator (Sec. 3.2, eq. riesz-def): the D sums with the
// source tangents in place of the normals, and no jump (ops must be D alone).
// cf_eta: the combined field (D - i eta S) mu of one density on both sides
// (Sec. 4.2), formed per pair (group kernel, one component) into out[1].
static int apply_impl(qbx_plan* p, const qbx_geom* g, int ops, int side, int limit, qbx_c64 k, int pp,
                      const qbx_c64* const dens[3], int nrhs, qbx_c64* const out[3], int n_far,
                      const double* x_far, qbx_c64* out_far, void* stream, bool tangent = false,
                      double eta = 0.0, const qbx_c64* cf_eta = nullptr) {
  if (int rc = check_plan(p)) return rc;
  if (int rc = check_geom(p, g, true)) return rc;
  if (ops < 1 || ops > 7) return fail(QBX_EINVAL, "operator set %d is not a non-empty subset of {S, D, grad S}", ops);
  if (limit != QBX_LIMIT_ONE_SIDED && limit != QBX_LIMIT_PV) return fail(QBX_EINVAL, "bad limit %d", limit);
  if (int rc = check_k(k)) return rc;
  if (int rc = check_p(pp)) return rc;
  if (nrhs < 1) return fail(QBX_EINVAL, "nrhs = %d < 1", nrhs);
  const bool cf = cf_eta != nullptr;
  if (cf) {
    if (ops != (QBX_OPS_S | QBX_OPS_D) || side != QBX_SIDE_TWO || dens[0] != dens[1] || n_far != 0 || tangent ||
        eta > 0.0)
      return fail(QBX_EINVAL, "combined field: S and D of one density, both sides, no far targets");
    if (!isfinite(cf_eta->re) || !isfinite(cf_eta->im)) return fail(QBX_EINVAL, "eta is not finite");
    if (!dens[0] || !out[1]) return fail(QBX_EINVAL, "NULL density or output");
  } else {
    for (int o = 0; o < 3; ++o)
      if ((ops >> o & 1) && (!dens[o] || !out[o])) return fail(QBX_EINVAL, "NULL density or output of operator %d", o);
  }
  if (n_far < 0) return fail(QBX_EINVAL, "n_far < 0");
  if (n_far > 0 && (!x_far || !out_far)) return fail(QBX_EINVAL, "n_far > 0 needs x_far and out_far");
  int c0, nc;
  if (int rc = side_range(side, g->n_tgt, &c0, &nc)) return rc;
  // components of a partial-sum row: S 1, D 1, grad S 2 (the combined field 1)
  int comp0[3], ncomp = 0;
  for (int o = 0; o < 3; ++o) {
    comp0[o] = ncomp;
    if (ops >> o & 1) ncomp += (o == QBX_OP_GRAD_S) ? 2 : 1;
  }
  if (cf) {
    comp0[0] = comp0[1] = 0;
    ncomp = 1;
  }
  // one oversampled density per distinct input array
  const qbx_c64* distinct[3];
  int slot_of[3] = {0, 0, 0}, nd = 0;
  for (int o = 0; o < 3; ++o) {
    if (!(ops >> o & 1)) continue;
    int s = 0;
    while (s < nd && distinct[s] != dens[o]) ++s;
    if (s == nd) distinct[nd++] = dens[o];
    slot_of[o] = s;
  }
  const size_t wd_one = align256((size_t)g->n_src * nrhs * 16);
  const size_t tan_bytes = tangent ? align256((size_t)g->n_src * 16) : 0;
  const size_t wd_bytes = wd_one * nd + tan_bytes;
  if (p->ws_bytes < wd_bytes + 512) return fail(QBX_ENOMEM, "workspace too small (%zu < %zu)", p->ws_bytes, wd_bytes + 512);
  const size_t avail = p->ws_bytes - wd_bytes - 512;
  const size_t per_split = (size_t)nc * ncomp * nrhs * 16;
  // many right-hand sides of one density: the group kernel (kernel values
  // formed once per pair for all rhs); otherwise the fused kernel
  const bool ck = k.im != 0.0;
  const bool group = cf || (nrhs >= 16 && nd == 1 && (ops == 1 || ops == 2 || ops == 3 || ops == 7));
  const int gops = cf ? kOpsCombined : ops;   // the group kernel's operator set
  // more than 32 rhs (global apply): eight warps of 8 rhs, so that the kernel
  // values of a pair are formed once per 64 rhs instead of once per 32
  const int rg = (nrhs > 32 && !(eta > 0.0)) ? kGrpRhsWide : 8;
  const int units = group ? (nc + kGrpCentres - 1) / kGrpCentres : (nc + kApplyThreads - 1) / kApplyThreads;
  const bool local = eta > 0.0;
  const int chunk = local ? std::min(4, apply_chunk(ops)) : apply_chunk(ops);
  // one rhs of one density for every operator: the weighted-seed instance
  const bool one_w = !group && nd == 1 && nrhs == 1;
  CK(cudaSetDevice(p->device), "cudaSetDevice");
  int occ;
  if (group && local) occ = group_occupancy_local(ops, ck, pp, rg);
  else if (group) occ = ck ? group_occupancy_cplx(gops, pp, rg) : group_occupancy_real(gops, pp, rg);
  else if (local) occ = apply_occupancy_local(ops, ck, pp, std::min(chunk, nrhs), one_w);
  else occ = ck ? apply_occupancy_cplx(ops, pp, std::min(chunk, nrhs), one_w)
                : apply_occupancy_real(ops, pp, std::min(chunk, nrhs), one_w);
  // the near-only variant's items differ more in cost (distant pairs take the
  // short direct path), and the one-density items (the near-field ones take
  // the slower small-argument Hankel branch) end unevenly: four waves (eight
  // at complex k) let the near-field items spread out (one density,
  // full-size starfish, real k: 63.9 ms with one wave of 3 CTAs per SM, 63.1
  // with four, 64.0 with six or eight; k = 20 + 1i, 2 CTAs per SM: 106.0,
  // 105.1, 103.9 ms with four, six, eight)
  const int waves = local   ? std::max(p->min_waves, 4)
                    : one_w ? std::max(p->min_waves, ck ? 8 : 4)
                            : p->min_waves;
  const int ns = host_choose_split_waves(p->num_sms, occ, units, g->n_src, per_split, avail, waves);
  if (ns < 1) return fail(QBX_ENOMEM, "workspace too small for the apply partial sums");
  if (group ? (ck ? group_smem_cplx(gops, pp, rg) : group_smem_real(gops, pp, rg)) > 220 * 1024
            : apply_smem_bytes(ops, ck, pp, chunk) > 220 * 1024)
    return fail(QBX_EINVAL, "p = %d too large", pp);
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)align256((size_t)p->ws);
  void* part = base + wd_bytes;
  // a1: oversample the densities
  for (int s = 0; s < nd; ++s)
    CK(launch_upsample(g->M, g->q_tgt, g->q_src, nrhs, p->d_interp, g->src_w, distinct[s], base + s * wd_one, st),
       "upsample");
  qbx_geom gtan;
  if (tangent) {   // the same geometry with the source tangents as "normals"
    double* tx = (double*)(base + nd * wd_one);
    double* ty = tx + g->n_src;
    CK(launch_tangents(g->n_src, g->src_nx, g->src_ny, tx, ty, st), "tangents");
    gtan = *g;
    gtan.src_nx = tx;
    gtan.src_ny = ty;
    g = &gtan;
  }
  const void* wd = base;  // far targets (single operator): its oversampled density
  if (p->timing) CK(cudaEventRecord(p->ev0, st), "timing event");
  // a2-a6 fused, per chunk of rhs
  ApplyArgs a{};
  a.ops = ops;
  for (int o = 0; o < 3; ++o) a.wd[o] = base + slot_of[o] * wd_one;
  a.p = pp;
  a.kre = k.re;
  a.kim = k.im;
  a.n_ctr = nc;
  a.cx = g->ctr_x + c0;
  a.cy = g->ctr_y + c0;
  a.n_tgt = g->n_tgt;
  a.tx = g->tgt_x;
  a.ty = g->tgt_y;
  a.src = SrcView{g->src_x, g->src_y, g->src_nx, g->src_ny, g->n_src};
  a.nrhs = nrhs;
  a.nsplit = ns;
  a.src_per_split = split_len(g->n_src, ns);
  a.part = part;
  a.eta2 = eta > 0.0 ? eta * eta : 0.0;
  a.near_q_tgt = g->q_tgt;   // near-field items first
  a.near_q_src = g->q_src;
  a.one_w = one_w ? 1 : 0;
  {
    cudaError_t te;
    a.hk_tab = host_plan_hk_table(p, k, st, &te);
    CK(te, "complex-k amplitude table");
  }
  if (group) {
    GroupArgs ga{};
    ga.ops = gops;
    ga.p = pp;
    ga.nrhs = nrhs;
    if (cf) {
      ga.cf_re = cf_eta->re;
      ga.cf_im = cf_eta->im;
    }
    GroupInst& in = ga.inst0;
    in.kre = k.re;
    in.kim = k.im;
    in.n_src = g->n_src;
    in.n_tgt = g->n_tgt;
    in.n_ctr = nc;
    in.side = side;
    in.nsplit = ns;
    in.M = g->M;
    in.sx = g->src_x;
    in.sy = g->src_y;
    in.snx = g->src_nx;
    in.sny = g->src_ny;
    in.sw = g->src_w;
    in.cx = g->ctr_x + c0;
    in.cy = g->ctr_y + c0;
    in.tx = g->tgt_x;
    in.ty = g->tgt_y;
    in.tnx = g->tgt_nx;
    in.tny = g->tgt_ny;
    in.wd = base;
    in.part = part;
    in.hk_tab = a.hk_tab;
    ga.st_units = units;
    ga.st_nsplit = ns;
    ga.st_split_len = split_len(g->n_src, ns);
    ga.eta2 = a.eta2;
    if (local)
      CK(launch_group_local(ga, ck, rg, units * ns, st), "group kernel (near-only)");
    else
      CK(ck ? launch_group_cplx(ga, rg, units * ns, st) : launch_group_real(ga, rg, units * ns, st), "group kernel");
  } else {
    for (int r0 = 0; r0 < nrhs; r0 += chunk) {
      a.rhs0 = r0;
      a.nr = std::min(chunk, nrhs - r0);
      CK(launch_apply_fused(a, st), "apply kernel");
    }
  }
  if (p->timing) CK(cudaEventRecord(p->ev1, st), "timing event");
  // a7: reduce, i/4, jumps / two-sided average, per operator (the combined
  // field: one finish, the two-sided average as for S and D)
  if (cf) {
    CK(launch_apply_finish(QBX_OP_S, side, limit, g->n_tgt, ns, nc, nrhs, 0, 1, part, dens[0], g->tgt_nx,
                           g->tgt_ny, out[1], p->d_status, st),
       "apply finish");
    return QBX_OK;
  }
  for (int o = 0; o < 3; ++o) {
    if (!(ops >> o & 1)) continue;
    CK(launch_apply_finish(tangent ? QBX_OP_S : o, side, limit, g->n_tgt, ns, nc, nrhs, comp0[o], ncomp, part,
                           dens[o], g->tgt_nx,
                           g->tgt_ny, out[o], p->d_status, st),
       "apply finish");
  }
  // a8: far targets (single operator)
  if (n_far > 0) {
    int op = 0;
    while (!(ops >> op & 1)) ++op;
    return far_impl(p, g, op, k, (const qbx_c64*)wd, nrhs, n_far, x_far, out_far, part, avail, st);
  }
  return QBX_OK;
}

// grad D (Sec. 3.2, eq. dlpderiv): the D coefficients of every centre of the
// side(s) (a4 unfused), the gradient of each expansion at its target (a6),
// and the finish with the tangential jump.  Workspace: oversampled density,
// coefficients, gradients, then the coefficient partial sums.
static int grad_d_impl(qbx_plan* p, const qbx_geom* g, int side, int limit, qbx_c64 k, int pp,
                       const qbx_c64* dens, int nrhs, qbx_c64* out, void* stream) {
  if (int rc = check_plan(p)) return rc;
  if (int rc = check_geom(p, g, true)) return rc;
  if (!g->tgt_w) return fail(QBX_EINVAL, "geometry: NULL target weights");
  if (limit != QBX_LIMIT_ONE_SIDED && limit != QBX_LIMIT_PV) return fail(QBX_EINVAL, "bad limit %d", limit);
  if (int rc = check_k(k)) return rc;
  if (int rc = check_p(pp)) return rc;
  if (nrhs < 1) return fail(QBX_EINVAL, "nrhs = %d < 1", nrhs);
  if (!dens || !out) return fail(QBX_EINVAL, "NULL density or output");
  int c0, nc;
  if (int rc = side_range(side, g->n_tgt, &c0, &nc)) return rc;
  const int nsides = side == QBX_SIDE_TWO ? 2 : 1;
  const int side0 = side == QBX_SIDE_EXT ? QBX_SIDE_EXT : QBX_SIDE_INT;
  const bool ck = k.im != 0.0;
  if (pp >= 1 && nrhs <= 3 && grad_d_fused_smem(ck, pp) <= 200 * 1024) {
    // storage-free sums, one rhs per pass (few rhs: each pass costs a full sweep)
    const size_t b_wd = align256((size_t)g->n_src * nrhs * 16);
    const size_t b_ev = align256((size_t)nc * 2 * nrhs * 16);
    const size_t fixed = b_wd + b_ev + 512;
    if (p->ws_bytes < fixed) return fail(QBX_ENOMEM, "workspace too small for grad D");
    const size_t per_split = (size_t)nc * 2 * nrhs * 16;
    const int units = (nc + kApplyThreads - 1) / kApplyThreads;
    CK(cudaSetDevice(p->device), "cudaSetDevice");
    const int occ = grad_d_fused_occupancy(ck, pp);
    const int ns = host_choose_split_waves(p->num_sms, occ, units, g->n_src, per_split, p->ws_bytes - fixed,
                                           p->min_waves);
    if (ns < 1) return fail(QBX_ENOMEM, "workspace too small for the grad D partial sums");
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)align256((size_t)p->ws);
    void* wd = base;
    void* ev = base + b_wd;
    void* part = base + b_wd + b_ev;
    CK(launch_upsample(g->M, g->q_tgt, g->q_src, nrhs, p->d_interp, g->src_w, dens, wd, st), "upsample");
    if (p->timing) CK(cudaEventRecord(p->ev0, st), "timing event");
    ApplyArgs a{};
    a.p = pp;
    a.kre = k.re;
    a.kim = k.im;
    a.n_ctr = nc;
    a.cx = g->ctr_x + c0;
    a.cy = g->ctr_y + c0;
    a.n_tgt = g->n_tgt;
    a.tx = g->tgt_x;
    a.ty = g->tgt_y;
    a.src = SrcView{g->src_x, g->src_y, g->src_nx, g->src_ny, g->n_src};
    a.wd[0] = a.wd[1] = a.wd[2] = wd;
    a.nrhs = nrhs;
    a.nr = 1;
    a.nsplit = ns;
    a.src_per_split = split_len(g->n_src, ns);
    a.part = part;
    a.near_q_tgt = g->q_tgt;
    a.near_q_src = g->q_src;
    {
      cudaError_t te;
      a.hk_tab = host_plan_hk_table(p, k, st, &te);
      CK(te, "complex-k amplitude table");
    }
    for (int r = 0; r < nrhs; ++r) {
      a.rhs0 = r;
      CK(launch_grad_d_fused(a, st), "grad D kernel");
    }
    CK(launch_form_finish(nc, 2, ns, nrhs, part, ev, p->d_status, st), "grad D reduction");
    if (p->timing) CK(cudaEventRecord(p->ev1, st), "timing event");
    CK(launch_grad_d_finish(g->n_tgt, g->q_tgt, nsides, side0, limit, nrhs, ev, dens, g->tgt_nx, g->tgt_ny,
                            g->tgt_w, p->d_wgl_tgt, p->d_diff, out, p->d_status, st),
       "grad D finish");
    return QBX_OK;
  }
  // otherwise: the D coefficients formed and stored, then the expansion's
  // gradient at each target
  const int ncoef = 2 * pp + 1;
  int nr = nrhs;
  while (nr > 1 && form_smem_bytes(pp, nr) > 160 * 1024) nr = (nr + 1) / 2;
  if (form_smem_bytes(pp, nr) > 200 * 1024) return fail(QBX_EINVAL, "p = %d too large", pp);
  const size_t b_wd = align256((size_t)g->n_src * nrhs * 16);
  const size_t b_al = align256((size_t)nc * ncoef * nrhs * 16);
  const size_t b_ev = align256((size_t)nc * 2 * nrhs * 16);
  const size_t fixed = b_wd + b_al + b_ev + 512;
  if (p->ws_bytes < fixed) return fail(QBX_ENOMEM, "workspace too small for grad D");
  const size_t per_split = (size_t)nc * ncoef * nrhs * 16;
  const int units = (nc + kFormThreads - 1) / kFormThreads;
  const int ns = choose_split(p, units, g->n_src, per_split, p->ws_bytes - fixed);
  if (ns < 1) return fail(QBX_ENOMEM, "workspace too small for the grad D partial sums");
  CK(cudaSetDevice(p->device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)align256((size_t)p->ws);
  void* wd = base;
  void* alpha = base + b_wd;
  void* ev = base + b_wd + b_al;
  void* part = base + b_wd + b_al + b_ev;
  CK(launch_upsample(g->M, g->q_tgt, g->q_src, nrhs, p->d_interp, g->src_w, dens, wd, st), "upsample");
  if (p->timing) CK(cudaEventRecord(p->ev0, st), "timing event");
  FormArgs a{};
  a.kind = QBX_OP_D;
  a.p = pp;
  a.kre = k.re;
  a.kim = k.im;
  a.n_ctr = nc;
  a.cx = g->ctr_x + c0;
  a.cy = g->ctr_y + c0;
  a.src = SrcView{g->src_x, g->src_y, g->src_nx, g->src_ny, g->n_src};
  a.wd = wd;
  a.nrhs = nrhs;
  a.nsplit = ns;
  a.src_per_split = split_len(g->n_src, ns);
  a.part = part;
  for (int r0 = 0; r0 < nrhs; r0 += nr) {
    a.rhs0 = r0;
    a.nr = std::min(nr, nrhs - r0);
    CK(launch_form(a, st), "form kernel");
  }
  CK(launch_form_finish(nc, ncoef, ns, nrhs, part, alpha, p->d_status, st), "form finish");
  EvalArgs e{};
  e.what = QBX_GRAD;
  e.p = pp;
  e.kre = k.re;
  e.kim = k.im;
  e.n_eval = nc;
  e.cx = g->ctr_x + c0;
  e.cy = g->ctr_y + c0;
  e.n_tgt = g->n_tgt;
  e.tx = g->tgt_x;
  e.ty = g->tgt_y;
  e.alpha = alpha;
  e.nrhs = nrhs;
  e.out = ev;
  e.n_ctr = nc;
  e.status = p->d_status;
  CK(launch_eval(e, st), "eval kernel");
  if (p->timing) CK(cudaEventRecord(p->ev1, st), "timing event");
  CK(launch_grad_d_finish(g->n_tgt, g->q_tgt, nsides, side0, limit, nrhs, ev, dens, g->tgt_nx, g->tgt_ny,
                          g->tgt_w, p->d_wgl_tgt, p->d_diff, out, p->d_status, st),
     "grad D finish");
  return QBX_OK;
}

int qbx_apply(qbx_plan* p, const qbx_geom* g, int op, int side, int limit, qbx_c64 k, int pp,
              const qbx_c64* dens_tgt, int nrhs, int n_far, const double* x_far, qbx_c64* out_on,
              qbx_c64* out_far, void* stream) {
  if (op != QBX_OP_S && op != QBX_OP_D && op != QBX_OP_GRAD_S && op != QBX_OP_R && op != QBX_OP_GRAD_D)
    return fail(QBX_EINVAL, "bad op %d", op);
  if (op == QBX_OP_GRAD_D) {
    if (n_far > 0) return fail(QBX_EINVAL, "far targets are not offered with grad D");
    return grad_d_impl(p, g, side, limit, k, pp, dens_tgt, nrhs, out_on, stream);
  }
  const qbx_c64* dens[3] = {dens_tgt, dens_tgt, dens_tgt};
  qbx_c64* out[3] = {out_on, out_on, out_on};
  if (op == QBX_OP_R)
    return apply_impl(p, g, 1 << QBX_OP_D, side, limit, k, pp, dens, nrhs, out, n_far, x_far, out_far, stream, true);
  return apply_impl(p, g, 1 << op, side, limit, k, pp, dens, nrhs, out, n_far, x_far, out_far, stream);
}

int qbx_apply_local(qbx_plan* p, const qbx_geom* g, int ops, int side, int limit, qbx_c64 k, int pp, double eta,
                    const qbx_c64* const dens[3], int nrhs, qbx_c64* const out[3], void* stream) {
  if (!dens || !out) return fail(QBX_EINVAL, "NULL density or output table");
  if (!(eta > 0.0) || !isfinite(eta)) return fail(QBX_EINVAL, "eta must be finite and > 0");
  return apply_impl(p, g, ops, side, limit, k, pp, dens, nrhs, out, 0, nullptr, nullptr, stream, false, eta);
}

int qbx_apply_ops(qbx_plan* p, const qbx_geom* g, int ops, int side, int limit, qbx_c64 k, int pp,
                  const qbx_c64* const dens[3], int nrhs, qbx_c64* const out[3], void* stream) {
  if (!dens || !out) return fail(QBX_EINVAL, "NULL density or output table");
  return apply_impl(p, g, ops, side, limit, k, pp, dens, nrhs, out, 0, nullptr, nullptr, stream);
}

int qbx_apply_cfie(qbx_plan* p, const qbx_geom* g, qbx_c64 k, qbx_c64 eta, int pp, const qbx_c64* dens, int nrhs,
                   qbx_c64* out, void* stream) {
  const qbx_c64* const d3[3] = {dens, dens, nullptr};
  qbx_c64* const o3[3] = {nullptr, out, nullptr};
  return apply_impl(p, g, QBX_OPS_S | QBX_OPS_D, QBX_SIDE_TWO, QBX_LIMIT_ONE_SIDED, k, pp, d3, nrhs, o3, 0,
                    nullptr, nullptr, stream, false, 0.0, &eta);
}

int qbx_assign_centres(qbx_plan* p, const qbx_geom* g, int side, int n, const double* xy, int* out,
                       void* stream) {
  if (int rc = check_plan(p)) return rc;
  if (int rc = check_geom(p, g, true)) return rc;
  int c0, nc;
  if (int rc = side_range(side, g->n_tgt, &c0, &nc)) return rc;
  if (n < 0) return fail(QBX_EINVAL, "n < 0");
  if (n == 0) return QBX_OK;
  if (!xy || !out) return fail(QBX_EINVAL, "NULL array");
  CK(cudaSetDevice(p->device), "cudaSetDevice");
  CK(launch_assign(n, xy, nc, g->ctr_x + c0, g->ctr_y + c0, g->ctr_r + c0, out, (cudaStream_t)stream),
     "assign kernel");
  return QBX_OK;
}

int qbx_debug_hankel01(const qbx_c64* z, int n, qbx_c64* h0, qbx_c64* h1, void* stream) {
  if (n < 0) return fail(QBX_EINVAL, "n < 0");
  if (n == 0) return QBX_OK;
  if (!z || !h0 || !h1) return fail(QBX_EINVAL, "NULL array");
  CK(launch_debug_hankel(z, n, h0, h1, (cudaStream_t)stream), "debug hankel");
  return QBX_OK;
}

int qbx_debug_hankel01_ray(qbx_plan* p, qbx_c64 k, const double* rho, int n, qbx_c64* h0, qbx_c64* h1,
                           void* stream) {
  if (int rc = check_plan(p)) return rc;
  if (int rc = check_k(k)) return rc;
  if (n < 0) return fail(QBX_EINVAL, "n < 0");
  if (n == 0) return QBX_OK;
  if (!rho || !h0 || !h1) return fail(QBX_EINVAL, "NULL array");
  CK(cudaSetDevice(p->device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t te;
  const double* tab = host_plan_hk_table(p, k, st, &te);
  CK(te, "complex-k amplitude table");
  CK(launch_debug_hankel_ray(k.re, k.im, tab, rho, n, h0, h1, st), "debug hankel (ray)");
  return QBX_OK;
}

int qbx_debug_besselj(const qbx_c64* z, int n, int nmax, qbx_c64* j, void* stream) {
  if (n < 0 || nmax < 0 || nmax > QBX_MAX_P + 1) return fail(QBX_EINVAL, "bad n or nmax");
  if (n == 0) return QBX_OK;
  if (!z || !j) return fail(QBX_EINVAL, "NULL array");
  CK(launch_debug_besselj(z, n, nmax, j, (cudaStream_t)stream), "debug besselj");
  return QBX_OK;
}

}  // extern "C"
