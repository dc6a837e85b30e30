// qbx_adjoint_impl.cuh -- the transposed QBX sweep: the adjoint of the
// on-surface apply of S or D with respect to the density, and (operator set
// S|X) the sums over centres that the shape adjoint of S needs: conj(K) g_c
// and conj(grad_{x_s} K) g_c per source.  For
// u = (i/4) K W P sigma (kernel values K(c, x_s), source weights W, per-panel
// interpolation P), the vector-Jacobian product of a gradient g on the
// targets is  P^T W K^H (-i/4) g  (plus the self-adjoint jump term for PV).
// Here a CTA of 4 warps owns 32 sources (one per lane) and runs through the
// centres in tiles of 32: phase 1 forms K(c, x_s) (recomputing H0, H1 and the
// recurrences, nothing stored between calls) for the tile, phase 2 adds
// conj(K) g_c into each warp's group of right-hand sides.  The per-centre
// Bessel coefficient columns are formed once per call into the workspace.
#pragma once
#include "qbx_apply_impl.cuh"

namespace qbx {

// Per-centre coefficient columns [n_ctr][nslots][p+2] (J_l, l J_l, J_{l-1}-J_{l+1})
// and the centre's target direction (ux, uy, 1/r).
template <int OPS, typename T>
__global__ void k_coef_columns(AdjArgs a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.n_ctr) return;
  constexpr bool kD = OPS & OPB_D, kG = OPS & OPB_G, kX = OPS & OPB_X;
  constexpr int ns = 1 + ((kD || kG || kX) ? 1 : 0) + (kG ? 1 : 0);
  const int P2 = a.p + 2;
  T* col = reinterpret_cast<T*>(a.coef) + (size_t)c * ns * P2;
  KW<T> kw;
  kw.init(a.kre, a.kim, a.hk_tab);
  const T kk = kw.kval();
  const double cx = a.cx[c], cy = a.cy[c];
  const int t = c % a.n_tgt;
  double ux = a.tx[t] - cx, uy = a.ty[t] - cy;
  const double r = hypot(ux, uy);
  besselj_seq<T>(rmul(kk, r), a.p + 1, col, 1);
  for (int l = 0; l <= a.p; ++l) {
    const T jl = col[l];
    if (kD || kG || kX) col[P2 + l] = rmul(jl, (double)l);
    if (kG) {
      const T jn = col[l + 1];
      const T jp = (l == 0) ? jn : col[l - 1];
      col[2 * P2 + l] = (l == 0) ? rmul(jn, -1.0) : sc_sub(jp, jn);
    }
  }
  if (!keeps_jp1(OPS)) {
    T z0;
    sc_zero(z0);
    col[a.p + 1] = z0;
  }
  double* geo = a.cgeo + 3 * (size_t)c;
  geo[0] = ux / r;
  geo[1] = uy / r;
  geo[2] = 1.0 / r;
}

template <int OPS, typename T, int RG>
struct AdjSmem {
  static constexpr int kNc = ops_ncomp(OPS);
  static constexpr bool kD = OPS & OPB_D, kG = OPS & OPB_G, kX = OPS & OPB_X;
  static __host__ __device__ constexpr int nslots() { return 1 + ((kD || kG || kX) ? 1 : 0) + (kG ? 1 : 0); }
  static __host__ __device__ size_t bytes(int p) {
    return 5 * kGrpTile * 8 +                                   // centre x, y, ux, uy, 1/r
           (size_t)kGrpTile * kGrpWarps * RG * 16 +              // gradients [centre][4 RG]
           (size_t)kNc * kGrpTile * kGrpCentres * 16 +           // kernel values [comp][centre][source]
           (size_t)nslots() * (p + 2) * kGrpTile * sizeof(T);    // coefficient columns [slot][l][centre]
  }
};

// items: blockIdx.x = source tile * nsplit + centre split
template <int OPS, typename T, int RG>
__global__ void __launch_bounds__(kGrpCentres * kGrpWarps)
k_adjoint(AdjArgs a) {
  using L = AdjSmem<OPS, T, RG>;
  constexpr bool kS = OPS & OPB_S, kD = OPS & OPB_D, kX = OPS & OPB_X;
  constexpr int kNc = L::kNc;
  constexpr int kRP = kGrpWarps * RG;
  constexpr int ns = L::nslots();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s_cx = reinterpret_cast<double*>(smem_raw);
  double* s_cy = s_cx + kGrpTile;
  double* s_ux = s_cy + kGrpTile;
  double* s_uy = s_ux + kGrpTile;
  double* s_ir = s_uy + kGrpTile;
  cplx* s_g = reinterpret_cast<cplx*>(s_ir + kGrpTile);     // [centre][kRP]
  cplx* s_kv = s_g + kGrpTile * kRP;                         // [comp][centre][source]
  T* s_col = reinterpret_cast<T*>(s_kv + kNc * kGrpTile * kGrpCentres);  // [slot][l][centre]
  const int p = a.p, P2 = p + 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  const int item = blockIdx.x;
  const int stile = item / a.nsplit, split = item % a.nsplit;
  const int c_begin = split * a.ctr_per_split;
  const int c_end = min(a.n_ctr, c_begin + a.ctr_per_split);
  const int s = stile * kGrpCentres + lane;
  const bool active = s < a.n_src;
  const int ss = active ? s : a.n_src - 1;
  const double sx = a.sx[ss], sy = a.sy[ss];
  double snx = 0.0, sny = 0.0;
  if (kD) {
    snx = a.snx[ss];
    sny = a.sny[ss];
  }
  KW<T> kw;
  kw.init(a.kre, a.kim, a.hk_tab);
  const T kk = kw.kval();
  const cplx* gin = reinterpret_cast<const cplx*>(a.gc);
  const T* coef = reinterpret_cast<const T*>(a.coef);

  for (int r0 = 0; r0 < a.nrhs; r0 += kRP) {
    cplx acc[kNc][RG];
#pragma unroll
    for (int q = 0; q < kNc; ++q)
#pragma unroll
      for (int g = 0; g < RG; ++g) acc[q][g] = cplx{0.0, 0.0};
    for (int base = c_begin; base < c_end; base += kGrpTile) {
      const int nt = min(kGrpTile, c_end - base);
      __syncthreads();
      for (int i = threadIdx.x; i < nt; i += blockDim.x) {
        s_cx[i] = a.cx[base + i];
        s_cy[i] = a.cy[base + i];
        s_ux[i] = a.cgeo[3 * (size_t)(base + i)];
        s_uy[i] = a.cgeo[3 * (size_t)(base + i) + 1];
        s_ir[i] = a.cgeo[3 * (size_t)(base + i) + 2];
      }
      for (int i = threadIdx.x; i < kGrpTile * kRP; i += blockDim.x) {
        const int c = i / kRP, rr = i - c * kRP;
        s_g[i] = (c < nt && r0 + rr < a.nrhs) ? gin[(size_t)(base + c) * a.nrhs + r0 + rr] : cplx{0.0, 0.0};
      }
      for (int i = threadIdx.x; i < nt * ns * P2; i += blockDim.x) {
        const int c = i / (ns * P2), rem = i - c * ns * P2;   // rem = slot * P2 + l
        s_col[rem * kGrpTile + c] = coef[(size_t)(base + c) * ns * P2 + rem];
      }
      __syncthreads();
      // ---- phase 1: K(c_j, x_s) for this warp's centres ----
      for (int j = warp; j < nt; j += kGrpWarps) {
        const double dx = sx - s_cx[j], dy = sy - s_cy[j];
        const T* cJ = s_col + j;
        const T* cL = s_col + P2 * kGrpTile + j;
        const T* cG = s_col + 2 * P2 * kGrpTile + j;
        const T J0 = cJ[0];
        const T kneg_j0 = rmul(sc_mul(kk, J0), -1.0);
        cplx GS, K, GA, GB, EX, EY;
        pair_kernels<OPS, T, kGrpTile>(kw, kk, J0, kneg_j0, cJ, cL, cG, p, dx, dy, snx, sny, s_ux[j], s_uy[j],
                                       s_ir[j], GS, K, GA, GB, EX, EY);
        int q = 0;
        if (kS) s_kv[(q++ * kGrpTile + j) * kGrpCentres + lane] = GS;
        if (kD) s_kv[(q++ * kGrpTile + j) * kGrpCentres + lane] = K;
        if (kX) {
          s_kv[(q++ * kGrpTile + j) * kGrpCentres + lane] = EX;
          s_kv[(q++ * kGrpTile + j) * kGrpCentres + lane] = EY;
        }
      }
      __syncthreads();
      // ---- phase 2: sum_c conj(K) g_c for this warp's rhs ----
      for (int j = 0; j < nt; ++j) {
        const cplx* g = s_g + j * kRP + warp * RG;
#pragma unroll
        for (int q = 0; q < kNc; ++q) {
          const cplx kv = conj(s_kv[(q * kGrpTile + j) * kGrpCentres + lane]);
#pragma unroll
          for (int gg = 0; gg < RG; ++gg) cfma(acc[q][gg], g[gg], kv);
        }
      }
    }
    if (active) {
      cplx* part = reinterpret_cast<cplx*>(a.part);
      const size_t row = ((size_t)split * a.n_src + s) * kNc;
#pragma unroll
      for (int gg = 0; gg < RG; ++gg) {
        const int rr = r0 + warp * RG + gg;
        if (rr >= a.nrhs) break;
#pragma unroll
        for (int q = 0; q < kNc; ++q) part[(row + q) * a.nrhs + rr] = acc[q][gg];
      }
    }
  }
}

template <int OPS, typename T, int RG>
static cudaError_t launch_adjoint_t(const AdjArgs& a, cudaStream_t st) {
  k_coef_columns<OPS, T><<<(a.n_ctr + 127) / 128, 128, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = AdjSmem<OPS, T, RG>::bytes(a.p);
  auto kern = k_adjoint<OPS, T, RG>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int tiles = (a.n_src + kGrpCentres - 1) / kGrpCentres;
  kern<<<tiles * a.nsplit, kGrpCentres * kGrpWarps, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_adjoint_any(const AdjArgs& a, cudaStream_t st) {
  const bool many = a.nrhs > 8;
  switch (a.ops) {
    case OPB_S: return many ? launch_adjoint_t<OPB_S, T, 8>(a, st) : launch_adjoint_t<OPB_S, T, 2>(a, st);
    case OPB_D: return many ? launch_adjoint_t<OPB_D, T, 8>(a, st) : launch_adjoint_t<OPB_D, T, 2>(a, st);
    case OPB_S | OPB_X:
      return many ? launch_adjoint_t<OPB_S | OPB_X, T, 8>(a, st) : launch_adjoint_t<OPB_S | OPB_X, T, 2>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qbx
