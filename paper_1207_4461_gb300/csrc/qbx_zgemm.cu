// qbx_zgemm.cu -- the matrix product of the assembled solve: y = A x for the
// column-major n x n complex Nystrom matrix A (entry (i, j) at A[j n + i])
// and nrhs vectors x, y stored [n][nrhs], in FP64 with three real products
// per complex multiply-add:
//   T1 = sum Re A Re x,  T2 = sum Im A Im x,  T3 = sum (Re A + Im A)(Re x + Im x),
//   Re y = T1 - T2,  Im y = T3 - T1 - T2,
// the sums Re + Im formed once per staged element.  Sec. 3.3 remarks that the
// discrete operator may be stored as a matrix; with many right-hand sides its
// application is this dense contraction, bound by the FP64 pipe (FP64
// multiply-adds are not the tensor cores' work on this part).
//
// A CTA of 256 threads computes a 64-row x 64-rhs tile of one K range (a
// split of the columns of A): per step it stages a 64 x 16 tile of A and a
// 16 x 64 tile of x in shared memory as three real planes (re, im, re + im),
// and each thread accumulates a 4 x 4 block of the three real products.
// Split partial sums go to a work array and are added in split order by a
// second kernel (deterministic); the split count fills whole waves of the
// resident CTAs.
#include <cuda_runtime.h>
#include <stdio.h>
#include <algorithm>
#include "../../include/qbx.h"
#include "qbx_device.cuh"
#include "qbx_internal.h"

using namespace qbx;

namespace {

constexpr int kBM = 64, kBK = 16, kThreads = 256, kTM = 4;

template <int TN>
__global__ void __launch_bounds__(kThreads, 2)
k_zgemm3m(int n, int nrhs, const cplx* __restrict__ A, const cplx* __restrict__ x, cplx* __restrict__ part,
          int kchunk, const int* gate) {
  if (gate && !*gate) return;
  constexpr int BN = 16 * TN;
  __shared__ double sA[3][kBK][kBM];
  __shared__ double sX[3][kBK][BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * kBM, r0 = blockIdx.y * BN;
  const int j0 = blockIdx.z * kchunk, j1 = min(n, j0 + kchunk);
  double t1[kTM][TN], t2[kTM][TN], t3[kTM][TN];
#pragma unroll
  for (int a = 0; a < kTM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) t1[a][b] = t2[a][b] = t3[a][b] = 0.0;

  for (int jb = j0; jb < j1; jb += kBK) {
    // stage A (64 rows x 16 columns: 4 per thread, consecutive rows per warp) and x
#pragma unroll
    for (int q = 0; q < kBM * kBK / kThreads; ++q) {
      const int ii = tid & (kBM - 1), jj = (tid >> 6) + q * (kThreads / kBM);
      const int i = i0 + ii, j = jb + jj;
      const cplx v = (i < n && j < j1) ? A[(size_t)j * n + i] : cplx{0.0, 0.0};
      sA[0][jj][ii] = v.re;
      sA[1][jj][ii] = v.im;
      sA[2][jj][ii] = v.re + v.im;
    }
#pragma unroll
    for (int q = 0; q < kBK * BN / kThreads; ++q) {
      const int idx = tid + q * kThreads, jj = idx / BN, rr = idx - jj * BN;
      const int j = jb + jj, r = r0 + rr;
      const cplx v = (j < j1 && r < nrhs) ? x[(size_t)j * nrhs + r] : cplx{0.0, 0.0};
      sX[0][jj][rr] = v.re;
      sX[1][jj][rr] = v.im;
      sX[2][jj][rr] = v.re + v.im;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < kBK; ++jj) {
      double a[kTM], b[TN];
#pragma unroll
      for (int m = 0; m < kTM; ++m) a[m] = sA[0][jj][ty + 16 * m];
#pragma unroll
      for (int q = 0; q < TN; ++q) b[q] = sX[0][jj][tx + 16 * q];
#pragma unroll
      for (int m = 0; m < kTM; ++m)
#pragma unroll
        for (int q = 0; q < TN; ++q) t1[m][q] = fma(a[m], b[q], t1[m][q]);
#pragma unroll
      for (int m = 0; m < kTM; ++m) a[m] = sA[1][jj][ty + 16 * m];
#pragma unroll
      for (int q = 0; q < TN; ++q) b[q] = sX[1][jj][tx + 16 * q];
#pragma unroll
      for (int m = 0; m < kTM; ++m)
#pragma unroll
        for (int q = 0; q < TN; ++q) t2[m][q] = fma(a[m], b[q], t2[m][q]);
#pragma unroll
      for (int m = 0; m < kTM; ++m) a[m] = sA[2][jj][ty + 16 * m];
#pragma unroll
      for (int q = 0; q < TN; ++q) b[q] = sX[2][jj][tx + 16 * q];
#pragma unroll
      for (int m = 0; m < kTM; ++m)
#pragma unroll
        for (int q = 0; q < TN; ++q) t3[m][q] = fma(a[m], b[q], t3[m][q]);
    }
    __syncthreads();
  }
  cplx* out = part + (size_t)blockIdx.z * n * nrhs;
#pragma unroll
  for (int m = 0; m < kTM; ++m) {
    const int i = i0 + ty + 16 * m;
    if (i >= n) continue;
#pragma unroll
    for (int q = 0; q < TN; ++q) {
      const int r = r0 + tx + 16 * q;
      if (r >= nrhs) continue;
      const double re = t1[m][q] - t2[m][q];
      out[(size_t)i * nrhs + r] = cplx{re, t3[m][q] - t1[m][q] - t2[m][q]};
    }
  }
}

// y = sum over splits in order
__global__ void k_zgemm_reduce(long nel, int nsplit, const cplx* part, cplx* y, const int* gate) {
  if (gate && !*gate) return;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nel) return;
  cplx acc = part[idx];
  for (int s = 1; s < nsplit; ++s) acc = acc + part[(size_t)s * nel + idx];
  y[idx] = acc;
}

int zfail(int code, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "qbx_matmul_cm: %s", what);
  return host_fail(code, buf);
}

int zcuda(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "qbx_matmul_cm: %s: %s", what, cudaGetErrorString(e));
  return host_fail(QBX_ECUDA, buf);
}

// rhs per CTA: 64 (TN = 4) or, for at most 16 rhs, 16 (TN = 1)
int tn_of(int nrhs) { return nrhs <= 16 ? 1 : 4; }

// Split count: the fewest K splits whose CTAs fill whole waves of the
// resident CTAs to >= 95 % (at most 32 splits, each at least 4 tiles of
// kBK columns).
int choose_splits(int n, int nrhs, int* kchunk) {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const cudaError_t e = tn_of(nrhs) == 1
                            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_zgemm3m<1>, kThreads, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_zgemm3m<4>, kThreads, 0);
  if (e != cudaSuccess || occ < 1) return 0;
  const int BN = 16 * tn_of(nrhs);
  const long tiles = (long)((n + kBM - 1) / kBM) * ((nrhs + BN - 1) / BN);
  const long slots = (long)sms * occ;
  const int smax = std::max(1, std::min(32, (n + 4 * kBK - 1) / (4 * kBK)));
  int best = 1;
  double best_fill = -1.0;
  for (int s = 1; s <= smax; ++s) {
    const long items = tiles * s, waves = (items + slots - 1) / slots;
    const double fill = (double)items / (double)(waves * slots);
    if (fill >= 0.95) {
      best = s;
      break;
    }
    if (fill > best_fill + 1e-12) {
      best_fill = fill;
      best = s;
    }
  }
  int chunk = (n + best - 1) / best;
  chunk = (chunk + kBK - 1) / kBK * kBK;
  *kchunk = chunk;
  return (n + chunk - 1) / chunk;
}

}  // namespace

extern "C" size_t qbx_matmul_cm_work_bytes(int n, int nrhs) {
  if (n < 1 || nrhs < 1) return 0;
  int kchunk = 0;
  const int ns = choose_splits(n, nrhs, &kchunk);
  return ns < 1 ? 0 : (size_t)ns * n * nrhs * 16;
}

namespace qbx {

int matmul_cm_gated(int n, int nrhs, const qbx_c64* A, const qbx_c64* x, qbx_c64* y, void* work,
                    size_t work_bytes, const int* gate, void* stream) {
  if (n < 1 || nrhs < 1 || !A || !x || !y || !work) return zfail(QBX_EINVAL, "bad arguments");
  int kchunk = 0;
  const int ns = choose_splits(n, nrhs, &kchunk);
  if (ns < 1) return zfail(QBX_ECUDA, "device query failed");
  if (work_bytes < (size_t)ns * n * nrhs * 16) return zfail(QBX_ENOMEM, "work array smaller than qbx_matmul_cm_work_bytes");
  cudaStream_t st = (cudaStream_t)stream;
  const int BN = 16 * tn_of(nrhs);
  const dim3 grid((unsigned)((n + kBM - 1) / kBM), (unsigned)((nrhs + BN - 1) / BN), (unsigned)ns);
  if (tn_of(nrhs) == 1)
    k_zgemm3m<1><<<grid, kThreads, 0, st>>>(n, nrhs, (const cplx*)A, (const cplx*)x, (cplx*)work, kchunk, gate);
  else
    k_zgemm3m<4><<<grid, kThreads, 0, st>>>(n, nrhs, (const cplx*)A, (const cplx*)x, (cplx*)work, kchunk, gate);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return zcuda(e, "product kernel");
  const long nel = (long)n * nrhs;
  k_zgemm_reduce<<<(unsigned)((nel + 255) / 256), 256, 0, st>>>(nel, ns, (const cplx*)work, (cplx*)y, gate);
  e = cudaGetLastError();
  return e == cudaSuccess ? QBX_OK : zcuda(e, "reduction kernel");
}

}  // namespace qbx

extern "C" int qbx_matmul_cm(int n, int nrhs, const qbx_c64* A, const qbx_c64* x, qbx_c64* y, void* work,
                             size_t work_bytes, void* stream) {
  return qbx::matmul_cm_gated(n, nrhs, A, x, y, work, work_bytes, nullptr, stream);
}
