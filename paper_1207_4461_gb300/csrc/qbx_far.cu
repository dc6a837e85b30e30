// qbx_far.cu -- far targets by the plain smooth quadrature rule (a8; Sec. 1,
// Sec. 2: targets where the smooth rule is accurate), partial sums over source splits:
//   S: sum wd H0(kd);  D: sum wd H1(kd) (x - x_s).n_s / d;  grad S: sum wd H1(kd) (x - x_s)/d
// (the factors i/4, ik/4, -ik/4 are applied by the finishing kernel).
#include "qbx_apply_impl.cuh"

namespace qbx {

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
  kw.init(a.kre, a.kim, a.hk_tab);
  cplx acc[NR], accb[NR];
#pragma unroll
  for (int r2 = 0; r2 < NR; ++r2) acc[r2] = accb[r2] = cplx{0.0, 0.0};
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
      double inv, d, yq;
      kw.geom(d2, inv, d, yq);
      cplx H0, H1;
      T twoz;
      kw.hankel(d, inv, yq, H0, H1, twoz);
      if (OP == QBX_OP_S) {
#pragma unroll
        for (int r2 = 0; r2 < NR; ++r2) cfma(acc[r2], s_wd[j * NR + r2], H0);
      } else if (OP == QBX_OP_D) {
        const cplx g = H1 * (fma(rx, s_nx[j], ry * s_ny[j]) * inv);
#pragma unroll
        for (int r2 = 0; r2 < NR; ++r2) cfma(acc[r2], s_wd[j * NR + r2], g);
      } else {
        const cplx gx = H1 * (rx * inv), gy = H1 * (ry * inv);
#pragma unroll
        for (int r2 = 0; r2 < NR; ++r2) {
          cfma(acc[r2], s_wd[j * NR + r2], gx);
          cfma(accb[r2], s_wd[j * NR + r2], gy);
        }
      }
    }
  }
  if (!active) return;
  cplx* part = reinterpret_cast<cplx*>(a.part);
  const int ncomp = OP == QBX_OP_GRAD_S ? 2 : 1;
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
