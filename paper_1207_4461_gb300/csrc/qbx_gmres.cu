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

// y = sqrt(w) * (x_density / 2 + D - i eta S), x_density = x / sqrt(w)
__global__ void k_cfie_combine(int n, int nrhs, const double* w, const cplx* xden, const cplx* d, const cplx* s,
                               double eta_re, double eta_im, cplx* y) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * nrhs) return;
  const double sw = sqrt(w[idx / nrhs]);
  const cplx ie = cplx{-eta_im, eta_re};   // i eta
  const cplx v = 0.5 * xden[idx] + d[idx] - ie * s[idx];
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
  if (n < 0 || nrhs < 1 || !w || !xden || !dmu || !smu || !y) return gfail(QBX_EINVAL, "bad arguments to qbx_cfie_combine");
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
// The solve: restarted GMRES(m) per right-hand side, all systems in lockstep.
// Arnoldi by classical Gram-Schmidt with one re-orthogonalisation (CGS2) on
// the device; the (m+1) x m Hessenberg columns come to the host, where
// Givens rotations update the residual estimates |g_{j+1}|.
// ---------------------------------------------------------------------------
#include <cublas_v2.h>
#include <complex>
#include <vector>

namespace {

typedef std::complex<double> zc;

struct Dev {
  void* p = nullptr;
  ~Dev() { cudaFree(p); }
};

}  // namespace

// Adense: the sqrt-weighted matrix from qbx_assemble_cfie (column-major), or
// NULL for matrix-free matvecs through qbx_apply_ops.
static int solve_impl(qbx_plan* plan, const qbx_geom* g, qbx_c64 k, qbx_c64 eta, int p, const qbx_c64* Adense,
                      const qbx_c64* f, int nrhs, double tol, int restart, int maxiter, qbx_c64* mu, int* iters,
                      double* resid, void* stream) {
  if (!plan || !g || !f || !mu || nrhs < 1 || restart < 1 || maxiter < 1 || !(tol > 0.0))
    return gfail(QBX_EINVAL, "bad arguments to qbx_solve_exterior_dirichlet");
  const int n = g->n_tgt;
  const size_t vec = (size_t)n * nrhs;
  cudaStream_t st = (cudaStream_t)stream;
  const int m = restart;
  Dev V, W, X, F, DEN, SM, DM, H, WORK, SCL;
  cudaError_t e = cudaMalloc(&V.p, (size_t)(m + 1) * vec * 16);
  if (e == cudaSuccess) e = cudaMalloc(&W.p, vec * 16);
  if (e == cudaSuccess) e = cudaMalloc(&X.p, vec * 16);
  if (e == cudaSuccess) e = cudaMalloc(&F.p, vec * 16);
  if (e == cudaSuccess) e = cudaMalloc(&DEN.p, vec * 16);
  if (e == cudaSuccess) e = cudaMalloc(&SM.p, vec * 16);
  if (e == cudaSuccess) e = cudaMalloc(&DM.p, vec * 16);
  if (e == cudaSuccess) e = cudaMalloc(&H.p, (size_t)(m + 1) * nrhs * 16);
  if (e == cudaSuccess) e = cudaMalloc(&WORK.p, qbx_vec_dots_work_bytes(nrhs, m + 1));
  if (e == cudaSuccess) e = cudaMalloc(&SCL.p, (size_t)nrhs * 8);
  if (e != cudaSuccess) return gcuda(e, "allocation");
  cplx* Vb = (cplx*)V.p;
  auto Vj = [&](int j) { return (qbx_c64*)(Vb + (size_t)j * vec); };
  int rc;
  // scaled right-hand side and initial guess: f~ = sqrt(w) f, x~ = sqrt(w) mu
  if ((rc = qbx_vec_scale_sqrtw(n, nrhs, g->tgt_w, f, (qbx_c64*)F.p, 0, stream))) return rc;
  if ((rc = qbx_vec_scale_sqrtw(n, nrhs, g->tgt_w, mu, (qbx_c64*)X.p, 0, stream))) return rc;
  const int ops = QBX_OPS_S | QBX_OPS_D;
  cublasHandle_t blas = nullptr;   // the plan's handle (kept for later solves)
  if (Adense) {
    blas = (cublasHandle_t)host_plan_blas(plan);
    if (!blas) return gfail(QBX_ECUDA, "cublasCreate failed");
    if (cublasSetStream(blas, st) != CUBLAS_STATUS_SUCCESS) return gfail(QBX_ECUDA, "cublasSetStream failed");
  }
  // y = A~ x~ : density x~/sqrt(w), S and D two-sided in one pass, combine;
  // or one complex GEMM with the assembled A~ (row-major [n][nrhs] vectors are
  // the column-major nrhs x n matrices X^T, Y^T = X^T A~^T), in the
  // three-real-product form (cublasZgemm3m: 104 ms against 130 ms for
  // n = 16384, 64 rhs, at errors of the same size for this use)
  auto matvec = [&](const qbx_c64* xs, qbx_c64* y) -> int {
    int r;
    if (Adense) {
      const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
      cublasStatus_t cs = cublasZgemm3m(blas, CUBLAS_OP_N, CUBLAS_OP_T, nrhs, n, n, &one,
                                        reinterpret_cast<const cuDoubleComplex*>(xs), nrhs,
                                        reinterpret_cast<const cuDoubleComplex*>(Adense), n, &zero,
                                        reinterpret_cast<cuDoubleComplex*>(y), nrhs);
      return cs == CUBLAS_STATUS_SUCCESS ? QBX_OK : gfail(QBX_ECUDA, "cublasZgemm3m failed");
    }
    if ((r = qbx_vec_scale_sqrtw(n, nrhs, g->tgt_w, xs, (qbx_c64*)DEN.p, 1, stream))) return r;
    const qbx_c64* dens[3] = {(qbx_c64*)DEN.p, (qbx_c64*)DEN.p, nullptr};
    qbx_c64* outs[3] = {(qbx_c64*)SM.p, (qbx_c64*)DM.p, nullptr};
    if ((r = qbx_apply_ops(plan, g, ops, QBX_SIDE_TWO, QBX_LIMIT_ONE_SIDED, k, p, dens, nrhs, outs, stream))) return r;
    return qbx_cfie_combine(n, nrhs, g->tgt_w, (qbx_c64*)DEN.p, (qbx_c64*)DM.p, (qbx_c64*)SM.p, eta, y, stream);
  };
  auto dots = [&](int nv, const qbx_c64* base, const qbx_c64* w, std::vector<zc>& out) -> int {
    int r = qbx_vec_dots(n, nrhs, nv, base, w, (qbx_c64*)WORK.p, (qbx_c64*)H.p, stream);
    if (r) return r;
    out.resize((size_t)nv * nrhs);
    cudaError_t ee = cudaMemcpyAsync(out.data(), H.p, (size_t)nv * nrhs * 16, cudaMemcpyDeviceToHost, st);
    if (ee == cudaSuccess) ee = cudaStreamSynchronize(st);
    return ee == cudaSuccess ? QBX_OK : gcuda(ee, "dot copy");
  };
  std::vector<zc> tmp;
  if ((rc = dots(1, (qbx_c64*)F.p, (qbx_c64*)F.p, tmp))) return rc;
  std::vector<double> fnorm(nrhs);
  for (int r = 0; r < nrhs; ++r) fnorm[r] = std::sqrt(std::max(tmp[r].real(), 0.0));
  std::vector<double> rel(nrhs, 1.0);
  int total = 0;
  bool done = false;
  while (!done && total < maxiter) {
    // r = f~ - A~ x~
    if ((rc = matvec((qbx_c64*)X.p, (qbx_c64*)W.p))) return rc;
    {
      // V_0 = f~ - W (via combine with y = -1 on W, then add f~)
      std::vector<double> one(nrhs, 1.0);
      e = cudaMemcpyAsync(Vj(0), F.p, vec * 16, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return gcuda(e, "copy");
      std::vector<zc> minus1(nrhs, zc(-1.0, 0.0));
      e = cudaMemcpyAsync(H.p, minus1.data(), nrhs * 16, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return gcuda(e, "copy");
      if ((rc = qbx_vec_combine(n, nrhs, 1, (qbx_c64*)W.p, (qbx_c64*)H.p, Vj(0), stream))) return rc;
    }
    if ((rc = dots(1, Vj(0), Vj(0), tmp))) return rc;
    std::vector<double> beta(nrhs), inv(nrhs);
    for (int r = 0; r < nrhs; ++r) {
      beta[r] = std::sqrt(std::max(tmp[r].real(), 0.0));
      inv[r] = beta[r] > 0.0 ? 1.0 / beta[r] : 0.0;
      rel[r] = fnorm[r] > 0.0 ? beta[r] / fnorm[r] : 0.0;
    }
    done = true;
    for (int r = 0; r < nrhs; ++r) done = done && rel[r] <= tol;
    if (done) break;
    e = cudaMemcpyAsync(SCL.p, inv.data(), nrhs * 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return gcuda(e, "copy");
    if ((rc = qbx_vec_scale_cols(n, nrhs, (double*)SCL.p, Vj(0), Vj(0), stream))) return rc;
    // Hessenberg columns and Givens rotations per system
    std::vector<zc> Hm((size_t)(m + 1) * m * nrhs, zc(0, 0)), cs((size_t)m * nrhs), sn((size_t)m * nrhs);
    std::vector<zc> gv((size_t)(m + 1) * nrhs, zc(0, 0));
    for (int r = 0; r < nrhs; ++r) gv[r] = beta[r];
    int jdone = 0;
    for (int j = 0; j < m && total < maxiter; ++j) {
      if ((rc = matvec(Vj(j), Vj(j + 1)))) return rc;
      ++total;
      // CGS2
      std::vector<zc> h1, h2;
      if ((rc = dots(j + 1, Vj(0), Vj(j + 1), h1))) return rc;
      e = cudaMemcpyAsync(H.p, h1.data(), (size_t)(j + 1) * nrhs * 16, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return gcuda(e, "copy");
      if ((rc = qbx_vec_orth_update(n, nrhs, j + 1, Vj(0), (qbx_c64*)H.p, Vj(j + 1), stream))) return rc;
      if ((rc = dots(j + 1, Vj(0), Vj(j + 1), h2))) return rc;
      e = cudaMemcpyAsync(H.p, h2.data(), (size_t)(j + 1) * nrhs * 16, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return gcuda(e, "copy");
      if ((rc = qbx_vec_orth_update(n, nrhs, j + 1, Vj(0), (qbx_c64*)H.p, Vj(j + 1), stream))) return rc;
      if ((rc = dots(1, Vj(j + 1), Vj(j + 1), tmp))) return rc;
      std::vector<double> hn(nrhs), ihn(nrhs);
      for (int r = 0; r < nrhs; ++r) {
        hn[r] = std::sqrt(std::max(tmp[r].real(), 0.0));
        ihn[r] = hn[r] > 0.0 ? 1.0 / hn[r] : 0.0;
      }
      e = cudaMemcpyAsync(SCL.p, ihn.data(), nrhs * 8, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return gcuda(e, "copy");
      if ((rc = qbx_vec_scale_cols(n, nrhs, (double*)SCL.p, Vj(j + 1), Vj(j + 1), stream))) return rc;
      bool all = true;
      for (int r = 0; r < nrhs; ++r) {
        auto h = [&](int i) -> zc& { return Hm[((size_t)i * m + j) * nrhs + r]; };
        for (int i = 0; i <= j; ++i) h(i) = h1[(size_t)i * nrhs + r] + h2[(size_t)i * nrhs + r];
        h(j + 1) = hn[r];
        for (int i = 0; i < j; ++i) {   // previous rotations
          const zc c = cs[(size_t)i * nrhs + r], s = sn[(size_t)i * nrhs + r];
          const zc a = h(i), b = h(i + 1);
          h(i) = std::conj(c) * a + std::conj(s) * b;
          h(i + 1) = -s * a + c * b;
        }
        const zc a = h(j), b = h(j + 1);
        const double den = std::sqrt(std::norm(a) + std::norm(b));
        zc c = den > 0 ? a / den : zc(1, 0), s = den > 0 ? b / den : zc(0, 0);
        cs[(size_t)j * nrhs + r] = c;
        sn[(size_t)j * nrhs + r] = s;
        h(j) = std::conj(c) * a + std::conj(s) * b;
        h(j + 1) = 0.0;
        const zc gj = gv[(size_t)j * nrhs + r];
        gv[(size_t)j * nrhs + r] = std::conj(c) * gj;
        gv[(size_t)(j + 1) * nrhs + r] = -s * gj;
        rel[r] = fnorm[r] > 0.0 ? std::abs(gv[(size_t)(j + 1) * nrhs + r]) / fnorm[r] : 0.0;
        all = all && rel[r] <= tol;
      }
      jdone = j + 1;
      if (all) break;
    }
    // y = H^{-1} g per system; x~ += V y
    std::vector<zc> y((size_t)jdone * nrhs, zc(0, 0));
    for (int r = 0; r < nrhs; ++r) {
      for (int i = jdone - 1; i >= 0; --i) {
        zc s = gv[(size_t)i * nrhs + r];
        for (int l = i + 1; l < jdone; ++l) s -= Hm[((size_t)i * m + l) * nrhs + r] * y[(size_t)l * nrhs + r];
        const zc d = Hm[((size_t)i * m + i) * nrhs + r];
        y[(size_t)i * nrhs + r] = std::abs(d) > 0 ? s / d : zc(0, 0);
      }
    }
    if (jdone > 0) {
      e = cudaMemcpyAsync(H.p, y.data(), (size_t)jdone * nrhs * 16, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return gcuda(e, "copy");
      if ((rc = qbx_vec_combine(n, nrhs, jdone, Vj(0), (qbx_c64*)H.p, (qbx_c64*)X.p, stream))) return rc;
    }
    done = true;
    for (int r = 0; r < nrhs; ++r) done = done && rel[r] <= tol;
  }
  // mu = x~ / sqrt(w); true residual of the last restart start is in rel
  if ((rc = qbx_vec_scale_sqrtw(n, nrhs, g->tgt_w, (qbx_c64*)X.p, mu, 1, stream))) return rc;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return gcuda(e, "final sync");
  if (iters) *iters = total;
  if (resid)
    for (int r = 0; r < nrhs; ++r) resid[r] = rel[r];
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
