// qbx_grad_d.cu -- storage-free grad D (Sec. 3.2, eq. dlpderiv): the
// gradient at the target of the D expansion about each centre, summed pair
// by pair without forming the coefficients (Sec. 3.3's remark that every
// source may add to the target sum directly).
//
// With x - c = r e^{i theta_t}, x_s - c = rho e^{i theta_s}, psi = theta_t -
// theta_s, the truncated Graf kernel is G_p = sum_{|l|<=p} H_l(k rho)
// e^{-i l theta_s} J_l(k r) e^{i l theta_t}.  Writing d = d_x - i d_y and
// dbar = d_x + i d_y, the Bessel identities dbar[Z_m e^{i m theta}] =
// -k Z_{m+1} e^{i(m+1) theta}, d[Z_m e^{i m theta}] = k Z_{m-1} e^{i(m-1) theta}
// (Z = J or H) give, for n_s . grad_{x_s} G_p differentiated at the target,
//   d D    =  (k^2/2) e^{-i theta_t} [-nu~ R(psi)  + conj(nu~) Q(-psi)],
//   dbar D = -(k^2/2) e^{ i theta_t} [-nu~ Q(psi)  + conj(nu~) R(-psi)],
// nu~ = (a + i b) e^{-i psi}, a = n_s . e_rho, b = n_s . e_theta, and
//   Q(psi) = sum_{m=-p+1}^{p+1} H_m J_m     e^{i m psi},
//   R(psi) = sum_{m=-p+1}^{p+1} H_m J_{m-2} e^{i m psi}.
// Folding +-m over |m| <= p-1 (H_{-m} = (-1)^m H_m, J likewise):
//   Q(+-psi) = H_0 J_0 + 2 sum_{m=1}^{p-1} J_m cos(m psi) H_m + edges,
//   R(+-psi) = H_0 J_2 + sum_{m=1}^{p-1} [(J_{m-2}+J_{m+2}) cos(m psi)
//              +- i (J_{m-2}-J_{m+2}) sin(m psi)] H_m + edges,
// the edges being the orders m = p, p+1 with e^{+-i m psi}.  Then
// grad = ((d D + dbar D)/2, i (d D - dbar D)/2).  Per order: three sums and
// the H and Chebyshev recurrences; one rhs per pass with the weighted
// density multiplied into the seeds H0, H1 (every sum is linear in H_m).
#include <cuda_runtime.h>
#include "qbx_apply_impl.cuh"
#include "qbx_internal.h"

namespace qbx {
namespace {

constexpr int kGdThreads = kApplyThreads;   // one centre per thread, 128-centre CTAs

// shared memory: source tile x, y, nx, ny, w; columns J (J_0..J_{p+1}),
// C (J_{m-2}+J_{m+2})/2 and S (J_{m-2}-J_{m+2})/2 for m = 1..p-1 (row m).
template <typename T>
__host__ __device__ size_t gd_smem(int p) {
  return (size_t)kSrcTile * (4 * 8 + 16) + (size_t)((p + 2) + 2 * p) * kGdThreads * sizeof(T);
}

template <typename T>
__device__ __forceinline__ T jl_signed(const T* cJ, int l) {   // J_l for l >= -1 from the column
  return l >= 0 ? cJ[l * kGdThreads] : rmul(cJ[kGdThreads], -1.0);
}

template <typename T>
__global__ void __launch_bounds__(kGdThreads) k_grad_d_fused(ApplyArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s_x = reinterpret_cast<double*>(smem_raw);
  double* s_y = s_x + kSrcTile;
  double* s_nx = s_y + kSrcTile;
  double* s_ny = s_nx + kSrcTile;
  cplx* s_w = reinterpret_cast<cplx*>(s_ny + kSrcTile);
  T* sJ = reinterpret_cast<T*>(s_w + kSrcTile);
  const int p = a.p;
  T* sC = sJ + (p + 2) * kGdThreads;
  T* sS = sC + p * kGdThreads;

  const int tid = threadIdx.x;
  // work item (centre block, source split), near-field splits first
  const int nblk = (a.n_ctr + kGdThreads - 1) / kGdThreads;
  const int cblk = (int)(blockIdx.x % (unsigned)nblk), rank = (int)(blockIdx.x / (unsigned)nblk);
  const int split = a.near_q_tgt > 0 ? near_first_split(rank, (cblk * kGdThreads + kGdThreads / 2) % a.n_tgt,
                                                        a.near_q_tgt, a.near_q_src, a.src_per_split, a.nsplit)
                                     : rank;
  const int c = cblk * kGdThreads + tid;
  const bool active = c < a.n_ctr;
  const int cc = active ? c : a.n_ctr - 1;

  // ---- per-centre set-up ----
  const double cx = a.cx[cc], cy = a.cy[cc];
  const int t = cc % a.n_tgt;
  double ux = a.tx[t] - cx, uy = a.ty[t] - cy;
  const double r = hypot(ux, uy);
  ux /= r;
  uy /= r;
  KW<T> kw;
  kw.init(a.kre, a.kim, a.hk_tab);
  const T kk = kw.kval();
  T* colJ = sJ + tid;
  T* colC = sC + tid;
  T* colS = sS + tid;
  besselj_seq<T>(rmul(kk, r), p + 1, colJ, kGdThreads);
  for (int m = 1; m <= p - 1; ++m) {
    const T jm2 = jl_signed(colJ, m - 2), jp2 = colJ[(m + 2) * kGdThreads];
    colC[m * kGdThreads] = rmul(sadd(jm2, jp2), 0.5);
    colS[m * kGdThreads] = rmul(sc_sub(jm2, jp2), 0.5);
  }
  const T J0 = colJ[0], J2 = colJ[2 * kGdThreads];
  // edge coefficients (halved: the Chebyshev values below are doubled)
  const T eQ0 = rmul(colJ[p * kGdThreads], 0.5), eQ1 = rmul(colJ[(p + 1) * kGdThreads], 0.5);
  const T eR0 = rmul(jl_signed(colJ, p - 2), 0.5), eR1 = rmul(colJ[(p - 1) * kGdThreads], 0.5);

  cplx accP{0.0, 0.0}, accM{0.0, 0.0};   // sums of the d and dbar brackets
  const int s_begin = split * a.src_per_split;
  const int s_end = min(a.src.n, s_begin + a.src_per_split);
  const cplx* wd = reinterpret_cast<const cplx*>(a.wd[0]);
  for (int base = s_begin; base < s_end; base += kSrcTile) {
    const int nt = min(kSrcTile, s_end - base);
    __syncthreads();
    for (int i = tid; i < nt; i += kGdThreads) {
      s_x[i] = a.src.x[base + i];
      s_y[i] = a.src.y[base + i];
      s_nx[i] = a.src.nx[base + i];
      s_ny[i] = a.src.ny[base + i];
      s_w[i] = wd[(size_t)(base + i) * a.nrhs + a.rhs0];
    }
    __syncthreads();
    if (!active) continue;
    for (int j = 0; j < nt; ++j) {
      const double dx = s_x[j] - cx, dy = s_y[j] - cy;
      const double nx = s_nx[j], ny = s_ny[j];
      const double rho2 = fma(dx, dx, dy * dy);
      double inv, rho, yq;
      kw.geom(rho2, inv, rho, yq);
      const double cs = fma(ux, dx, uy * dy) * inv;   // cos psi
      const double sn = fma(uy, dx, -ux * dy) * inv;  // sin psi
      const double av = fma(nx, dx, ny * dy) * inv;   // n_s . e_rho
      const double bv = fma(ny, dx, -nx * dy) * inv;  // n_s . e_theta
      cplx H0, H1;
      T twoz;
      kw.hankel_w(rho, inv, yq, s_w[j], H0, H1, twoz);   // w H0, w H1
      // core sums over m = 1..p-1 with 2 cos(m psi), 2 sin(m psi)
      cplx SQ{0.0, 0.0}, CR{0.0, 0.0}, SR{0.0, 0.0};
      const double tw = 2.0 * cs;
      cplx Hm = H0, H = H1;
      T s = twoz;
      double cp = 2.0, cl = tw, sp = 0.0, sl = sn + sn;
      for (int m = 1; m < p; ++m) {
        const int o = m * kGdThreads;
        madd(SQ, rmul(colJ[o], cl), H);
        madd(CR, rmul(colC[o], cl), H);
        madd(SR, rmul(colS[o], sl), H);
        const cplx Hn = hrec(s, H, Hm);
        Hm = H;
        H = Hn;
        s = sadd(s, twoz);
        const double cn = fma(tw, cl, -cp), sq = fma(tw, sl, -sp);
        cp = cl;
        cl = cn;
        sp = sl;
        sl = sq;
      }
      // edges: orders p (H, cl, sl) and p + 1
      const cplx Hp1 = hrec(s, H, Hm);
      const double cl1 = fma(tw, cl, -cp), sl1 = fma(tw, sl, -sp);
      cplx A1Q{0.0, 0.0}, A2Q{0.0, 0.0}, A1R{0.0, 0.0}, A2R{0.0, 0.0};
      madd(A1Q, rmul(eQ0, cl), H);
      madd(A1Q, rmul(eQ1, cl1), Hp1);
      madd(A2Q, rmul(eQ0, sl), H);
      madd(A2Q, rmul(eQ1, sl1), Hp1);
      madd(A1R, rmul(eR0, cl), H);
      madd(A1R, rmul(eR1, cl1), Hp1);
      madd(A2R, rmul(eR0, sl), H);
      madd(A2R, rmul(eR1, sl1), Hp1);
      // Q(+-psi) = Qa +- i Qb, R(+-psi) = Ra +- i Rb
      cplx Qa = SQ + A1Q, Ra = CR + A1R;
      madd(Qa, J0, H0);
      madd(Ra, J2, H0);
      const cplx Qb = A2Q, Rb = SR + A2R;
      const cplx iQb{-Qb.im, Qb.re}, iRb{-Rb.im, Rb.re};
      // nu~ = (a + i b) e^{-i psi}
      const cplx nu{fma(av, cs, bv * sn), fma(bv, cs, -av * sn)};
      const cplx nuc = conj(nu);
      // d bracket: -nu~ R(psi) + conj(nu~) Q(-psi); dbar bracket: -nu~ Q(psi) + conj(nu~) R(-psi)
      cfma(accP, nuc, Qa - iQb);
      cfma(accP, -nu, Ra + iRb);
      cfma(accM, nuc, Ra - iRb);
      cfma(accM, -nu, Qa + iQb);
    }
  }
  if (!active) return;
  // d D = (k^2/2) e^{-i theta_t} P, dbar D = -(k^2/2) e^{i theta_t} M (without the factor i/4)
  const cplx h = 0.5 * sc_mul(to_c(kk), to_c(kk));
  const cplx et{ux, uy};
  const cplx dD = h * (conj(et) * accP);
  const cplx dbD = -(h * (et * accM));
  const cplx gx = 0.5 * (dD + dbD);
  const cplx dm = dD - dbD;
  const cplx gy = cplx{-0.5 * dm.im, 0.5 * dm.re};
  cplx* part = reinterpret_cast<cplx*>(a.part);
  const size_t row = ((size_t)split * a.n_ctr + c) * 2;
  part[row * a.nrhs + a.rhs0] = gx;
  part[(row + 1) * a.nrhs + a.rhs0] = gy;
}

template <typename T>
cudaError_t launch_gd(const ApplyArgs& a, cudaStream_t st) {
  const size_t smem = gd_smem<T>(a.p);
  cudaError_t e = cudaFuncSetAttribute(k_grad_d_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((a.n_ctr + kGdThreads - 1) / kGdThreads) * (unsigned)a.nsplit;
  k_grad_d_fused<T><<<grid, kGdThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
int occ_gd(int p) {
  const size_t smem = gd_smem<T>(p);
  int n = 0;
  if (cudaFuncSetAttribute(k_grad_d_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_grad_d_fused<T>, kGdThreads, smem) != cudaSuccess) return 0;
  return n;
}

}  // namespace

cudaError_t launch_grad_d_fused(const ApplyArgs& a, cudaStream_t st) {
  return a.kim == 0.0 ? launch_gd<double>(a, st) : launch_gd<cplx>(a, st);
}
size_t grad_d_fused_smem(bool ck, int p) { return ck ? gd_smem<cplx>(p) : gd_smem<double>(p); }
int grad_d_fused_occupancy(bool ck, int p) { return ck ? occ_gd<cplx>(p) : occ_gd<double>(p); }

}  // namespace qbx
