// qbx_gmres.cu -- device kernels of the batched GMRES solve for the
// second-kind exterior Dirichlet (sound-soft) problem of Sec. 4.2:
//   (1/2) mu + D mu - i eta S mu = f   (eq. dirichlet-inteq with the exterior
//   sign, D and S as two-sided averages, Sec. 3.5 and Sec. 4.2),
// with unknowns scaled by the square roots of the target weights (Sec. 4.2:
// sqrt-weight unknowns).  Every system (right-hand side) has its own Krylov
// basis; the systems advance in lockstep so that one matvec call serves all.
// Vectors are [n][nrhs] complex; bases [m+1][n][nrhs].  Reductions are
// two-pass in fixed order, so results are deterministic.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include "../../include/qbx.h"
#include "qbx_device.cuh"
#include "qbx_internal.h"

using namespace qbx;

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 152;   // first-pass blocks (one per SM)

// x = y / sqrt(w)  (scaled unknowns -> density) or x = y * sqrt(w)
__global__ void k_scale_sqrtw(int n, int nrhs, const double* w, const cplx* in, cplx* out, int inverse) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * nrhs) return;
  const double s = sqrt(w[idx / nrhs]);
  out[idx] = (inverse ? 1.0 / s : s) * in[idx];
}

// y = sqrt(w) * (x_density / 2 + D - i eta S), x_density = x / sqrt(w);
// s == NULL: d holds (D - i eta S) x_density
__global__ void k_cfie_combine(int n, int nrhs, const double* w, const cplx* xden, const cplx* d, const cplx* s,
                               double eta_re, double eta_im, cplx* y) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * nrhs) return;
  const double sw = sqrt(w[idx / nrhs]);
  const cplx ie = cplx{-eta_im, eta_re};   // i eta
  cplx v = 0.5 * xden[idx] + d[idx];
  if (s) v = v - ie * s[idx];
  y[idx] = sw * v;
}

// partial dots: part[b][j][r] = sum_{i in block b's range} conj(V_j[i][r]) w[i][r],
// grid (kRedBlocks, nv): block (b, j) takes row range b of vector j.  Lanes
// own right-hand sides (rows of [n][nrhs] are read whole and coalesced):
// thread t takes rhs r0 + t % R and every S-th row of the range,
// S = blockDim / R; the S partial sums of each r are then added in a fixed
// order, so the result does not depend on timing.
__global__ void k_dots_pass1(int n, int nrhs, int nv, const cplx* V, const cplx* w, cplx* part) {
  extern __shared__ cplx sred[];
  const int j = blockIdx.y;
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int i0 = blockIdx.x * per, i1 = min(n, i0 + per);
  const int R = min(nrhs, (int)blockDim.x), S = blockDim.x / R;
  const int rr = threadIdx.x % R, sub = threadIdx.x / R;
  const cplx* Vj = V + (size_t)j * n * nrhs;
  for (int r0 = 0; r0 < nrhs; r0 += R) {
    const int r = r0 + rr;
    cplx acc{0.0, 0.0};
    if (sub < S && r < nrhs) {
#pragma unroll 4
      for (int i = i0 + sub; i < i1; i += S) acc = acc + conj(Vj[(size_t)i * nrhs + r]) * w[(size_t)i * nrhs + r];
    }
    sred[threadIdx.x] = acc;
    __syncthreads();
    if (sub == 0 && r < nrhs) {
      cplx tot = sred[rr];
      for (int q = 1; q < S; ++q) tot = tot + sred[q * R + rr];
      part[((size_t)blockIdx.x * nv + j) * nrhs + r] = tot;
    }
    __syncthreads();
  }
}

__global__ void k_dots_pass2(int nblocks, int nrhs, int nv, const cplx* part, cplx* out) {
  const int jr = blockIdx.x * blockDim.x + threadIdx.x;
  if (jr >= nv * nrhs) return;
  cplx acc{0.0, 0.0};
  for (int b = 0; b < nblocks; ++b) acc = acc + part[(size_t)b * nv * nrhs + jr];
  out[jr] = acc;
}

// w -= sum_j V_j h[j][r]
__global__ void k_orth_update(int n, int nrhs, int nv, const cplx* V, const cplx* h, cplx* w) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * nrhs) return;
  const int r = idx % nrhs;
  cplx acc = w[idx];
  for (int j = 0; j < nv; ++j) acc = acc - V[(size_t)j * n * nrhs + idx] * h[(size_t)j * nrhs + r];
  w[idx] = acc;
}

// out[i][r] = a[r] * in[i][r] (a real per rhs; 0 where a is not finite)
__global__ void k_scale_cols(int n, int nrhs, const double* a, const cplx* in, cplx* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * nrhs) return;
  const double s = a[idx % nrhs];
  out[idx] = isfinite(s) ? s * in[idx] : cplx{0.0, 0.0};
}

// x += sum_j V_j y[j][r]
__global__ void k_combine(int n, int nrhs, int nv, const cplx* V, const cplx* y, cplx* x) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * nrhs) return;
  const int r = idx % nrhs;
  cplx acc = x[idx];
  for (int j = 0; j < nv; ++j) acc = acc + V[(size_t)j * n * nrhs + idx] * y[(size_t)j * nrhs + r];
  x[idx] = acc;
}

int gfail(int code, const char* what) {
  char buf[320];
  snprintf(buf, sizeof(buf), "qbx_gmres: %s", what);
  return host_fail(code, buf);
}

int gcuda(cudaError_t e, const char* what) {
  char buf[320];
  snprintf(buf, sizeof(buf), "qbx_gmres: %s: %s", what, cudaGetErrorString(e));
  return host_fail(QBX_ECUDA, buf);
}

inline unsigned blocks(long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

extern "C" {

int qbx_vec_scale_sqrtw(int n, int nrhs, const double* w, const qbx_c64* in, qbx_c64* out, int inverse,
                        void* stream) {
  if (n < 0 || nrhs < 1 || !w || !in || !out) return gfail(QBX_EINVAL, "bad arguments to qbx_vec_scale_sqrtw");
  if (n == 0) return QBX_OK;
  k_scale_sqrtw<<<blocks((long)n * nrhs), 256, 0, (cudaStream_t)stream>>>(n, nrhs, w, (const cplx*)in, (cplx*)out,
                                                                          inverse);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? QBX_OK : gcuda(e, "scale kernel");
}

int qbx_cfie_combine(int n, int nrhs, const double* w, const qbx_c64* xden, const qbx_c64* dmu,
                     const qbx_c64* smu, qbx_c64 eta, qbx_c64* y, void* stream) {
  if (n < 0 || nrhs < 1 || !w || !xden || !dmu || !y) return gfail(QBX_EINVAL, "bad arguments to qbx_cfie_combine");
  if (n == 0) return QBX_OK;
  k_cfie_combine<<<blocks((long)n * nrhs), 256, 0, (cudaStream_t)stream>>>(
      n, nrhs, w, (const cplx*)xden, (const cplx*)dmu, (const cplx*)smu, eta.re, eta.im, (cplx*)y);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? QBX_OK : gcuda(e, "combine kernel");
}

int qbx_vec_dots(int n, int nrhs, int nv, const qbx_c64* V, const qbx_c64* w, qbx_c64* work, qbx_c64* out,
                 void* stream) {
  if (n < 1 || nrhs < 1 || nv < 1 || nv > 65535 || !V || !w || !work || !out)
    return gfail(QBX_EINVAL, "bad arguments to qbx_vec_dots");
  cudaStream_t st = (cudaStream_t)stream;
  k_dots_pass1<<<dim3(kRedBlocks, nv), kRedThreads, kRedThreads * sizeof(cplx), st>>>(n, nrhs, nv, (const cplx*)V,
                                                                            (const cplx*)w, (cplx*)work);
  k_dots_pass2<<<blocks((long)nv * nrhs), 256, 0, st>>>(kRedBlocks, nrhs, nv, (const cplx*)work, (cplx*)out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? QBX_OK : gcuda(e, "dot kernels");
}

size_t qbx_vec_dots_work_bytes(int nrhs, int nv) { return (size_t)kRedBlocks * nv * nrhs * 16; }

int qbx_vec_orth_update(int n, int nrhs, int nv, const qbx_c64* V, const qbx_c64* h, qbx_c64* w, void* stream) {
  if (n < 1 || nrhs < 1 || nv < 0 || !V || !h || !w) return gfail(QBX_EINVAL, "bad arguments to qbx_vec_orth_update");
  if (nv == 0) return QBX_OK;
  k_orth_update<<<blocks((long)n * nrhs), 256, 0, (cudaStream_t)stream>>>(n, nrhs, nv, (const cplx*)V,
                                                                          (const cplx*)h, (cplx*)w);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? QBX_OK : gcuda(e, "orthogonalisation kernel");
}

int qbx_vec_scale_cols(int n, int nrhs, const double* a, const qbx_c64* in, qbx_c64* out, void* stream) {
  if (n < 1 || nrhs < 1 || !a || !in || !out) return gfail(QBX_EINVAL, "bad arguments to qbx_vec_scale_cols");
  k_scale_cols<<<blocks((long)n * nrhs), 256, 0, (cudaStream_t)stream>>>(n, nrhs, a, (const cplx*)in, (cplx*)out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? QBX_OK : gcuda(e, "scale kernel");
}

int qbx_vec_combine(int n, int nrhs, int nv, const qbx_c64* V, const qbx_c64* y, qbx_c64* x, void* stream) {
  if (n < 1 || nrhs < 1 || nv < 0 || !V || !y || !x) return gfail(QBX_EINVAL, "bad arguments to qbx_vec_combine");
  if (nv == 0) return QBX_OK;
  k_combine<<<blocks((long)n * nrhs), 256, 0, (cudaStream_t)stream>>>(n, nrhs, nv, (const cplx*)V, (const cplx*)y,
                                                                      (cplx*)x);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? QBX_OK : gcuda(e, "combine kernel");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The solve: restarted GMRES(m) per right-hand side, all systems in lockstep,
// driven from the device.  Arnoldi by classical Gram-Schmidt with one
// re-orthogonalisation (CGS2); the Hessenberg columns, the Givens rotations,
// the residual estimates |g_{j+1}| / ||f||, the convergence test and the
// back-substitution of each restart cycle run in small kernels on the device
// (one thread per right-hand side), so the host waits for the device once
// per restart cycle.  The kernels of an Arnoldi step read the step index and
// the state (done, matvec count) from a control block in device memory and
// do nothing once the step is inactive (all systems converged, maxiter
// reached or the cycle full); with the assembled matrix one step is
// captured as a CUDA graph and launched `restart` times per cycle.
// ---------------------------------------------------------------------------
#include <vector>

namespace {

// control block
enum { C_J = 0, C_DONE, C_TOTAL, C_MAXITER, C_M, C_ACTIVE, C_NOTCONV, C_JDONE, C_N };

struct Dev {
  void* p = nullptr;
  ~Dev() { cudaFree(p); }
};

struct GraphGuard {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  cudaStream_t cap = nullptr;
  ~GraphGuard() {
    if (x) cudaGraphExecDestroy(x);
    if (g) cudaGraphDestroy(g);
    if (cap) cudaStreamDestroy(cap);
  }
};

// start of a step: is it active?
__global__ void k_gate(int* ctl) {
  ctl[C_ACTIVE] = (!ctl[C_DONE] && ctl[C_TOTAL] < ctl[C_MAXITER] && ctl[C_J] < ctl[C_M]) ? 1 : 0;
}

// out = V_{j + off} (dir 0) or V_{j + off} = in (dir 1)
__global__ void k_basis_copy(long vec, const cplx* V, cplx* Vw, const int* ctl, int off, int dir, const cplx* in,
                             cplx* out) {
  if (!ctl[C_ACTIVE]) return;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= vec) return;
  const long b = (long)(ctl[C_J] + off) * vec;
  if (dir == 0) out[idx] = V[b + idx];
  else Vw[b + idx] = in[idx];
}

// partial dots of the step: which = 0: V_0..V_j against V_{j+1} (nv = j + 1);
// which = 1: V_{j+1} against itself (nv = 1).  Same decomposition and order
// as k_dots_pass1; blocks beyond nv return.
__global__ void k_dots_step1(int n, int nrhs, const cplx* V, const int* ctl, int which, cplx* part) {
  if (!ctl[C_ACTIVE]) return;
  const int j = ctl[C_J];
  const int nv = which == 0 ? j + 1 : 1;
  const int jv = blockIdx.y;
  if (jv >= nv) return;
  extern __shared__ cplx sred[];
  const size_t vec = (size_t)n * nrhs;
  const cplx* Vj = V + (which == 0 ? (size_t)jv : (size_t)(j + 1)) * vec;
  const cplx* w = V + (size_t)(j + 1) * vec;
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int i0 = blockIdx.x * per, i1 = min(n, i0 + per);
  const int R = min(nrhs, (int)blockDim.x), S = blockDim.x / R;
  const int rr = threadIdx.x % R, sub = threadIdx.x / R;
  for (int r0 = 0; r0 < nrhs; r0 += R) {
    const int r = r0 + rr;
    cplx acc{0.0, 0.0};
    if (sub < S && r < nrhs) {
#pragma unroll 4
      for (int i = i0 + sub; i < i1; i += S) acc = acc + conj(Vj[(size_t)i * nrhs + r]) * w[(size_t)i * nrhs + r];
    }
    sred[threadIdx.x] = acc;
    __syncthreads();
    if (sub == 0 && r < nrhs) {
      cplx tot = sred[rr];
      for (int q = 1; q < S; ++q) tot = tot + sred[q * R + rr];
      part[((size_t)blockIdx.x * gridDim.y + jv) * nrhs + r] = tot;
    }
    __syncthreads();
  }
}

__global__ void k_dots_step2(int nblocks, int nrhs, int nvmax, const cplx* part, const int* ctl, int which,
                             cplx* out) {
  if (!ctl[C_ACTIVE]) return;
  const int nv = which == 0 ? ctl[C_J] + 1 : 1;
  const int jr = blockIdx.x * blockDim.x + threadIdx.x;
  if (jr >= nv * nrhs) return;
  cplx acc{0.0, 0.0};
  for (int b = 0; b < nblocks; ++b) acc = acc + part[(size_t)b * nvmax * nrhs + jr];
  out[jr] = acc;
}

// V_{j+1} -= sum_{i <= j} V_i h[i][r]
__global__ void k_orth_step(int n, int nrhs, cplx* V, const cplx* h, const int* ctl) {
  if (!ctl[C_ACTIVE]) return;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * nrhs) return;
  const int r = (int)(idx % nrhs), nv = ctl[C_J] + 1;
  const size_t vec = (size_t)n * nrhs;
  cplx acc = V[(size_t)nv * vec + idx];
  for (int q = 0; q < nv; ++q) acc = acc - V[(size_t)q * vec + idx] * h[(size_t)q * nrhs + r];
  V[(size_t)nv * vec + idx] = acc;
}

// Hessenberg column j of every system: h(i) = h1 + h2 (i <= j), h(j+1) =
// ||V_{j+1}||; the earlier rotations, a new one zeroing h(j+1), the updated
// g and the residual estimate |g_{j+1}| / ||f||; scl = 1 / ||V_{j+1}||.
__global__ void k_givens(int nrhs, int m, const cplx* h1, const cplx* h2, const cplx* hn, cplx* Hm, cplx* cs,
                         cplx* sn, cplx* gv, const double* fnorm, double* rel, double* scl, double tol, int* ctl) {
  if (!ctl[C_ACTIVE]) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const int j = ctl[C_J];
  auto H = [&](int i) -> cplx& { return Hm[((size_t)i * m + j) * nrhs + r]; };
  for (int i = 0; i <= j; ++i) H(i) = h1[(size_t)i * nrhs + r] + h2[(size_t)i * nrhs + r];
  const double hnn = sqrt(fmax(hn[r].re, 0.0));
  H(j + 1) = cplx{hnn, 0.0};
  scl[r] = hnn > 0.0 ? 1.0 / hnn : 0.0;
  for (int i = 0; i < j; ++i) {   // previous rotations
    const cplx c = cs[(size_t)i * nrhs + r], s = sn[(size_t)i * nrhs + r];
    const cplx a = H(i), b = H(i + 1);
    H(i) = conj(c) * a + conj(s) * b;
    H(i + 1) = c * b - s * a;
  }
  const cplx a = H(j), b = H(j + 1);
  const double den = sqrt(abs2(a) + abs2(b));
  const cplx c = den > 0.0 ? (1.0 / den) * a : cplx{1.0, 0.0};
  const cplx s = den > 0.0 ? (1.0 / den) * b : cplx{0.0, 0.0};
  cs[(size_t)j * nrhs + r] = c;
  sn[(size_t)j * nrhs + r] = s;
  H(j) = conj(c) * a + conj(s) * b;
  H(j + 1) = cplx{0.0, 0.0};
  const cplx gj = gv[(size_t)j * nrhs + r];
  gv[(size_t)j * nrhs + r] = conj(c) * gj;
  const cplx gn = -(s * gj);
  gv[(size_t)(j + 1) * nrhs + r] = gn;
  const double e = fnorm[r] > 0.0 ? sqrt(abs2(gn)) / fnorm[r] : 0.0;
  rel[r] = e;
  if (!(e <= tol)) atomicAdd(&ctl[C_NOTCONV], 1);
}

// V_{j+1} *= scl (per rhs; 0 where not finite)
__global__ void k_scale_step(int n, int nrhs, cplx* V, const double* scl, const int* ctl) {
  if (!ctl[C_ACTIVE]) return;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * nrhs) return;
  const double a = scl[idx % nrhs];
  cplx* v = V + (size_t)(ctl[C_J] + 1) * n * nrhs;
  v[idx] = isfinite(a) ? a * v[idx] : cplx{0.0, 0.0};
}

__global__ void k_step_end(int* ctl) {
  if (!ctl[C_ACTIVE]) return;
  ctl[C_J] += 1;
  ctl[C_TOTAL] += 1;
  ctl[C_JDONE] = ctl[C_J];
  ctl[C_DONE] = ctl[C_NOTCONV] == 0;
  ctl[C_NOTCONV] = 0;
}

// start of a restart cycle, from hn = ||f~ - A x~||^2 per rhs: beta, the
// residual estimates, scl = 1/beta for V_0, g = (beta, 0, ...)
__global__ void k_cycle_init(int nrhs, int m, const cplx* hn, const double* fnorm, double* rel, double* scl, cplx* gv,
                             double tol, int* ctl) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const double beta = sqrt(fmax(hn[r].re, 0.0));
  scl[r] = beta > 0.0 ? 1.0 / beta : 0.0;
  const double e = fnorm[r] > 0.0 ? beta / fnorm[r] : 0.0;
  rel[r] = e;
  gv[r] = cplx{beta, 0.0};
  for (int i = 1; i <= m; ++i) gv[(size_t)i * nrhs + r] = cplx{0.0, 0.0};
  if (!(e <= tol)) atomicAdd(&ctl[C_NOTCONV], 1);
}

__global__ void k_cycle_init2(int* ctl) {
  ctl[C_J] = 0;
  ctl[C_JDONE] = 0;
  ctl[C_DONE] = ctl[C_NOTCONV] == 0;
  ctl[C_NOTCONV] = 0;
}

__global__ void k_fnorm(int nrhs, const cplx* hn, double* fnorm) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nrhs) fnorm[r] = sqrt(fmax(hn[r].re, 0.0));
}

// y = H^{-1} g per system (upper triangular, jdone columns)
__global__ void k_backsolve(int nrhs, int m, const cplx* Hm, const cplx* gv, cplx* y, const int* ctl) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const int jd = ctl[C_JDONE];
  for (int i = jd - 1; i >= 0; --i) {
    cplx s = gv[(size_t)i * nrhs + r];
    for (int l = i + 1; l < jd; ++l) s = s - Hm[((size_t)i * m + l) * nrhs + r] * y[(size_t)l * nrhs + r];
    const cplx d = Hm[((size_t)i * m + i) * nrhs + r];
    y[(size_t)i * nrhs + r] = abs2(d) > 0.0 ? cdiv(s, d) : cplx{0.0, 0.0};
  }
}

// x += sum_{i < jdone} V_i y[i][r]
__global__ void k_combine_cycle(int n, int nrhs, const cplx* V, const cplx* y, cplx* x, const int* ctl) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * nrhs) return;
  const int r = (int)(idx % nrhs), nv = ctl[C_JDONE];
  cplx acc = x[idx];
  for (int q = 0; q < nv; ++q) acc = acc + V[(size_t)q * n * nrhs + idx] * y[(size_t)q * nrhs + r];
  x[idx] = acc;
}

// V_0 = f~ - w
__global__ void k_sub(long nel, const cplx* f, const cplx* w, cplx* out) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < nel) out[idx] = f[idx] - w[idx];
}

}  // namespace

// Adense: the sqrt-weighted matrix from qbx_assemble_cfie (column-major), or
// NULL for matrix-free matvecs through qbx_apply_cfie.
static int solve_impl(qbx_plan* plan, const qbx_geom* g, qbx_c64 k, qbx_c64 eta, int p, const qbx_c64* Adense,
                      const qbx_c64* f, int nrhs, double tol, int restart, int maxiter, qbx_c64* mu, int* iters,
                      double* resid, void* stream) {
  if (!plan || !g || !f || !mu || nrhs < 1 || restart < 1 || maxiter < 1 || !(tol > 0.0))
    return gfail(QBX_EINVAL, "bad arguments to qbx_solve_exterior_dirichlet");
  const int n = g->n_tgt;
  const size_t vec = (size_t)n * nrhs;
  cudaStream_t st = (cudaStream_t)stream;
  const int m = restart;
  const size_t zw = Adense ? qbx_matmul_cm_work_bytes(n, nrhs) : 0;
  if (Adense && zw == 0) return gfail(QBX_ECUDA, "matrix product set-up failed");
  Dev V, W, X, F, DEN, DM, WORK, ST, ZW, CTL;
  // small state: h1, h2 [(m+1)][nrhs], hn [nrhs], Hm [(m+1)][m][nrhs], cs, sn [m][nrhs],
  // gv [(m+1)][nrhs], y [m][nrhs] (complex); fnorm, rel, scl [nrhs] (real)
  const size_t nst = (size_t)nrhs * (2 * (m + 1) + 1 + (size_t)(m + 1) * m + 2 * m + (m + 1) + m);
  cudaError_t e = cudaMalloc(&V.p, (size_t)(m + 1) * vec * 16);
  if (e == cudaSuccess) e = cudaMalloc(&W.p, vec * 16);
  if (e == cudaSuccess) e = cudaMalloc(&X.p, vec * 16);
  if (e == cudaSuccess) e = cudaMalloc(&F.p, vec * 16);
  if (e == cudaSuccess) e = cudaMalloc(&DEN.p, vec * 16);
  if (e == cudaSuccess && !Adense) e = cudaMalloc(&DM.p, vec * 16);   // (D - i eta S) of the density
  if (e == cudaSuccess) e = cudaMalloc(&WORK.p, qbx_vec_dots_work_bytes(nrhs, m + 1));
  if (e == cudaSuccess) e = cudaMalloc(&ST.p, nst * 16 + 3 * (size_t)nrhs * 8);
  if (e == cudaSuccess && Adense) e = cudaMalloc(&ZW.p, zw);
  if (e == cudaSuccess) e = cudaMalloc(&CTL.p, C_N * sizeof(int));
  if (e != cudaSuccess) return gcuda(e, "allocation");
  cplx* Vb = (cplx*)V.p;
  cplx* h1 = (cplx*)ST.p;
  cplx* h2 = h1 + (size_t)(m + 1) * nrhs;
  cplx* hn = h2 + (size_t)(m + 1) * nrhs;
  cplx* Hm = hn + nrhs;
  cplx* cs = Hm + (size_t)(m + 1) * m * nrhs;
  cplx* sn = cs + (size_t)m * nrhs;
  cplx* gv = sn + (size_t)m * nrhs;
  cplx* yv = gv + (size_t)(m + 1) * nrhs;
  double* fnorm = (double*)(yv + (size_t)m * nrhs);
  double* rel = fnorm + nrhs;
  double* scl = rel + nrhs;
  int* ctl = (int*)CTL.p;
  {
    const int init[C_N] = {0, 0, 0, maxiter, m, 0, 0, 0};
    e = cudaMemcpyAsync(ctl, init, sizeof(init), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // (init lives on the host stack)
    if (e != cudaSuccess) return gcuda(e, "control block");
  }
  const unsigned ebl = blocks((long)vec), rbl = (unsigned)((nrhs + 127) / 128);
  int rc;
  // scaled right-hand side and initial guess: f~ = sqrt(w) f, x~ = sqrt(w) mu
  if ((rc = qbx_vec_scale_sqrtw(n, nrhs, g->tgt_w, f, (qbx_c64*)F.p, 0, stream))) return rc;
  if ((rc = qbx_vec_scale_sqrtw(n, nrhs, g->tgt_w, mu, (qbx_c64*)X.p, 0, stream))) return rc;
  // y = A~ x~ : density x~/sqrt(w), (D - i eta S) two-sided with the two
  // kernel values of each pair combined (qbx_apply_cfie), plus x/2; or one
  // complex matrix product with the assembled A~ (qbx_matmul_cm)
  auto matvec = [&](const qbx_c64* xs, qbx_c64* y, cudaStream_t s) -> int {
    int r;
    if (Adense) return qbx_matmul_cm(n, nrhs, Adense, xs, y, ZW.p, zw, s);
    if ((r = qbx_vec_scale_sqrtw(n, nrhs, g->tgt_w, xs, (qbx_c64*)DEN.p, 1, s))) return r;
    if ((r = qbx_apply_cfie(plan, g, k, eta, p, (qbx_c64*)DEN.p, nrhs, (qbx_c64*)DM.p, s))) return r;
    return qbx_cfie_combine(n, nrhs, g->tgt_w, (qbx_c64*)DEN.p, (qbx_c64*)DM.p, nullptr, eta, y, s);
  };
  // one Arnoldi step on stream s, every kernel gated by the control block:
  // V_j -> W, W = A~ W, W -> V_{j+1}, CGS2 against V_0..V_j, the norm, the
  // Givens update and the convergence count, V_{j+1} normalised
  auto step = [&](cudaStream_t s) -> int {
    k_gate<<<1, 1, 0, s>>>(ctl);
    k_basis_copy<<<ebl, 256, 0, s>>>((long)vec, Vb, Vb, ctl, 0, 0, nullptr, (cplx*)W.p);
    if (Adense) {
      if (int r = matmul_cm_gated(n, nrhs, Adense, (qbx_c64*)W.p, (qbx_c64*)DEN.p, ZW.p, zw, ctl + C_ACTIVE, s))
        return r;
      k_basis_copy<<<ebl, 256, 0, s>>>((long)vec, Vb, Vb, ctl, 1, 1, (const cplx*)DEN.p, nullptr);
    } else {
      if (int r = matvec((qbx_c64*)W.p, (qbx_c64*)W.p, s)) return r;   // (host-checked: runs only when active)
      k_basis_copy<<<ebl, 256, 0, s>>>((long)vec, Vb, Vb, ctl, 1, 1, (const cplx*)W.p, nullptr);
    }
    for (int pass = 0; pass < 2; ++pass) {   // CGS2
      cplx* hh = pass == 0 ? h1 : h2;
      k_dots_step1<<<dim3(kRedBlocks, m + 1), kRedThreads, kRedThreads * sizeof(cplx), s>>>(n, nrhs, Vb, ctl, 0,
                                                                                         (cplx*)WORK.p);
      k_dots_step2<<<blocks((long)(m + 1) * nrhs), 256, 0, s>>>(kRedBlocks, nrhs, m + 1, (const cplx*)WORK.p, ctl, 0,
                                                               hh);
      k_orth_step<<<ebl, 256, 0, s>>>(n, nrhs, Vb, hh, ctl);
    }
    k_dots_step1<<<dim3(kRedBlocks, m + 1), kRedThreads, kRedThreads * sizeof(cplx), s>>>(n, nrhs, Vb, ctl, 1,
                                                                                       (cplx*)WORK.p);
    k_dots_step2<<<blocks(nrhs), 256, 0, s>>>(kRedBlocks, nrhs, m + 1, (const cplx*)WORK.p, ctl, 1, hn);
    k_givens<<<rbl, 128, 0, s>>>(nrhs, m, h1, h2, hn, Hm, cs, sn, gv, fnorm, rel, scl, tol, ctl);
    k_scale_step<<<ebl, 256, 0, s>>>(n, nrhs, Vb, scl, ctl);
    k_step_end<<<1, 1, 0, s>>>(ctl);
    cudaError_t ee = cudaGetLastError();
    return ee == cudaSuccess ? QBX_OK : gcuda(ee, "Arnoldi step kernels");
  };
  // ||f~|| per rhs
  if ((rc = qbx_vec_dots(n, nrhs, 1, (qbx_c64*)F.p, (qbx_c64*)F.p, (qbx_c64*)WORK.p, (qbx_c64*)hn, stream)))
    return rc;
  k_fnorm<<<rbl, 128, 0, st>>>(nrhs, hn, fnorm);
  // the assembled operator: one Arnoldi step as a CUDA graph
  GraphGuard gg;
  if (Adense) {
    e = cudaStreamCreateWithFlags(&gg.cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(gg.cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return gcuda(e, "graph capture");
    rc = step(gg.cap);
    e = cudaStreamEndCapture(gg.cap, &gg.g);
    if (rc) return rc;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gg.x, gg.g, 0);
    if (e != cudaSuccess) return gcuda(e, "Arnoldi step graph");
  }
  int hctl[C_N] = {0};
  bool done = false;
  int total = 0;
  while (!done && total < maxiter) {
    // r = f~ - A~ x~, beta, V_0 = r / beta, g = beta e_1
    if ((rc = matvec((qbx_c64*)X.p, (qbx_c64*)W.p, st))) return rc;
    k_sub<<<ebl, 256, 0, st>>>((long)vec, (const cplx*)F.p, (const cplx*)W.p, Vb);
    if ((rc = qbx_vec_dots(n, nrhs, 1, (qbx_c64*)Vb, (qbx_c64*)Vb, (qbx_c64*)WORK.p, (qbx_c64*)hn, stream)))
      return rc;
    k_cycle_init<<<rbl, 128, 0, st>>>(nrhs, m, hn, fnorm, rel, scl, gv, tol, ctl);
    k_cycle_init2<<<1, 1, 0, st>>>(ctl);
    if ((rc = qbx_vec_scale_cols(n, nrhs, scl, (qbx_c64*)Vb, (qbx_c64*)Vb, stream))) return rc;
    if (Adense) {
      for (int j = 0; j < m; ++j) {   // gated steps: those after convergence do nothing
        e = cudaGraphLaunch(gg.x, st);
        if (e != cudaSuccess) return gcuda(e, "Arnoldi step graph launch");
      }
    } else {
      for (int j = 0; j < m; ++j) {   // one host check per step (each step is a full QBX apply)
        e = cudaMemcpyAsync(hctl, ctl, sizeof(hctl), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return gcuda(e, "control block copy");
        if (hctl[C_DONE] || hctl[C_TOTAL] >= maxiter || hctl[C_J] >= m) break;
        if ((rc = step(st))) return rc;
      }
    }
    // y = H^{-1} g per system; x~ += V y
    k_backsolve<<<rbl, 128, 0, st>>>(nrhs, m, Hm, gv, yv, ctl);
    k_combine_cycle<<<ebl, 256, 0, st>>>(n, nrhs, Vb, yv, (cplx*)X.p, ctl);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hctl, ctl, sizeof(hctl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the one wait of the cycle
    if (e != cudaSuccess) return gcuda(e, "end of restart cycle");
    done = hctl[C_DONE] != 0;
    total = hctl[C_TOTAL];
  }
  // mu = x~ / sqrt(w); residual estimates of the last cycle
  if ((rc = qbx_vec_scale_sqrtw(n, nrhs, g->tgt_w, (qbx_c64*)X.p, mu, 1, stream))) return rc;
  if (resid) e = cudaMemcpyAsync(resid, rel, (size_t)nrhs * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return gcuda(e, "final sync");
  if (iters) *iters = total;
  if (!done) return gfail(QBX_ENOCONV, "GMRES did not reach the tolerance within maxiter iterations");
  return QBX_OK;
}

extern "C" int qbx_solve_exterior_dirichlet(qbx_plan* plan, const qbx_geom* g, qbx_c64 k, qbx_c64 eta, int p,
                                            const qbx_c64* f, int nrhs, double tol, int restart, int maxiter,
                                            qbx_c64* mu, int* iters, double* resid, void* stream) {
  return solve_impl(plan, g, k, eta, p, nullptr, f, nrhs, tol, restart, maxiter, mu, iters, resid, stream);
}

extern "C" int qbx_solve_exterior_dirichlet_assembled(qbx_plan* plan, const qbx_geom* g, const qbx_c64* A,
                                                      const qbx_c64* f, int nrhs, double tol, int restart,
                                                      int maxiter, qbx_c64* mu, int* iters, double* resid,
                                                      void* stream) {
  if (!A) return gfail(QBX_EINVAL, "NULL matrix");
  return solve_impl(plan, g, qbx_c64{1.0, 0.0}, qbx_c64{0.0, 0.0}, 0, A, f, nrhs, tol, restart, maxiter, mu, iters,
                    resid, stream);
}
