// qbx_group_impl.cuh -- the QBX apply for many right-hand sides and for
// batches of curves (the "group" kernel).  Same per-pair mathematics as
// k_apply_fused (pair_kernels), different work decomposition:
//
// A CTA of 4 warps owns 32 centres of one curve (one per lane) and works
// through a range of its sources in tiles of 32.  Phase 1: warp w forms the
// kernel values of its 8 sources of the tile for the 32 centres (H0, H1 and
// the order recurrences once per pair) and stores them in shared memory.
// Phase 2: warp g multiplies them into its own group of RG right-hand sides.
// Kernel generation is therefore paid once per pair however many densities
// there are, and each thread keeps only RG accumulators per component.
//
// Items (32 centres x a source range) come either from blockIdx (one curve,
// static split of the sources) or from a longest-first item list through an
// atomic counter (a batch: persistent CTAs, no waits between CTAs).
#pragma once
#include "qbx_apply_impl.cuh"

namespace qbx {

// Phase 2 is a small complex matrix product (centres x sources) x (sources x
// rhs).  With at most two components it runs on three real products per
// complex multiply-add (re = T1 - T2, im = T3 - T1 - T2 with T1 = sum a c,
// T2 = sum b d, T3 = sum (a + b)(c + d)), the sums a + b and c + d formed
// once per stored value; kernel values and densities then sit in shared
// memory as three real planes.  Otherwise four FMAs per complex product.
template <int OPS, typename T, int RG, int W = kGrpWarps>
struct GroupSmem {
  static constexpr int kNc = ops_ncomp(OPS);   // raw components: S 1, D 1, grad S 2; D - i eta S 1
  static constexpr bool kD = (OPS & OPB_D) || (OPS & OPB_C), kG = OPS & OPB_G;
  static constexpr bool k3M = kNc <= 2;
  static constexpr int kVal = k3M ? 24 : 16;   // bytes per stored complex value
  static __host__ __device__ int nslots() { return 1 + ((kD || kG) ? 1 : 0) + (kG ? 1 : 0); }
  static __host__ __device__ size_t bytes(int p) {
    return 4 * kGrpTile * 8 +                                  // x, y, nx, ny
           (size_t)kGrpTile * W * RG * kVal +                   // densities [tile][W RG]
           (size_t)kNc * kGrpTile * kGrpCentres * kVal +        // kernel values [comp][tile][centre]
           (size_t)nslots() * (p + 2) * kGrpCentres * sizeof(T) +  // coefficient columns
           16;                                                  // item index
  }
};

// LOCAL: near-only QBX (sources at |x_s - c| >= eta r by the smooth rule at
// the target, pair_direct), a separate instance.  W warps per CTA: W RG rhs
// per pass (kernel values are formed once per pass; W = 8 serves 64 rhs in
// one pass, the GMRES matvec's count).  OPS = OPB_C: the S and D kernel
// values of a pair are combined into D - i eta S before phase 2, so the
// rhs products are one complex multiply-add per rhs instead of two.
template <int OPS, typename T, int RG, bool LOCAL = false, int W = kGrpWarps>
__global__ void __launch_bounds__(kGrpCentres * W)
k_apply_group(GroupArgs a) {
  using L = GroupSmem<OPS, T, RG, W>;
  constexpr bool kC = OPS & OPB_C;
  constexpr int PK = kC ? (OPB_S | OPB_D) : OPS;   // the pair kernels formed
  constexpr bool kS = PK & OPB_S, kD = PK & OPB_D, kG = PK & OPB_G;
  constexpr int kNc = L::kNc;
  constexpr int kRP = W * RG;   // rhs per pass
  constexpr bool k3M = L::k3M;
  constexpr int kNW = kGrpTile * kRP, kNK = kNc * kGrpTile * kGrpCentres;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s_x = reinterpret_cast<double*>(smem_raw);
  double* s_y = s_x + kGrpTile;
  double* s_nx = s_y + kGrpTile;
  double* s_ny = s_nx + kGrpTile;
  unsigned char* w_raw = reinterpret_cast<unsigned char*>(s_ny + kGrpTile);
  unsigned char* k_raw = w_raw + (size_t)kNW * L::kVal;
  cplx* s_wd = reinterpret_cast<cplx*>(w_raw);                 // [tile][kRP]  (4 FMAs)
  double* s_wa = reinterpret_cast<double*>(w_raw);             // re, im, re + im planes (3M)
  double* s_wb = s_wa + kNW;
  double* s_ws = s_wb + kNW;
  cplx* s_kv = reinterpret_cast<cplx*>(k_raw);                 // [comp][tile][centre]
  double* s_ka = reinterpret_cast<double*>(k_raw);
  double* s_kb = s_ka + kNK;
  double* s_ks = s_kb + kNK;
  T* slot = reinterpret_cast<T*>(k_raw + (size_t)kNK * L::kVal);
  const int p = a.p;
  const int P2 = (p + 2) * kGrpCentres;
  T* sJ = slot;
  T* sL = slot + P2;
  T* sG = sL + ((kD || kG) ? P2 : 0);
  int* s_item = reinterpret_cast<int*>(slot + L::nslots() * P2);

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool dynamic = a.items != nullptr;
  const int n_items = dynamic ? a.n_items : a.st_units * a.st_nsplit;

  for (int it = dynamic ? -1 : (int)blockIdx.x;;) {
    // ---- next item ----
    if (dynamic) {
      __syncthreads();
      if (threadIdx.x == 0) s_item[0] = atomicAdd(a.counter, 1);
      __syncthreads();
      it = s_item[0];
    }
    if (it >= n_items) break;
    GroupItem item;
    if (dynamic) {
      item = a.items[it];
    } else {
      // rank r of the launch takes the 32-centre units' splits near-field
      // first, as the fused apply
      item.inst = 0;
      const int unit = it % a.st_units, rank = it / a.st_units;
      const int q_t = a.inst0.n_tgt / a.inst0.M, q_s = a.inst0.n_src / a.inst0.M;
      item.ctr0 = unit * kGrpCentres;
      item.split = near_first_split(rank, (unit * kGrpCentres + kGrpCentres / 2) % a.inst0.n_tgt, q_t, q_s,
                                    a.st_split_len, a.st_nsplit);
      item.src0 = item.split * a.st_split_len;
      item.src1 = min(a.inst0.n_src, item.src0 + a.st_split_len);
    }
    const GroupInst& in = dynamic ? a.inst[item.inst] : a.inst0;

    // ---- per-centre set-up (every warp keeps its lane's centre geometry) ----
    const int c = item.ctr0 + lane;
    const bool active = c < in.n_ctr;
    const int cc = active ? c : in.n_ctr - 1;
    const double cx = in.cx[cc], cy = in.cy[cc];
    const int t = cc % in.n_tgt;
    double ux = in.tx[t] - cx, uy = in.ty[t] - cy;
    const double r = hypot(ux, uy);
    const double ir = 1.0 / r;
    ux *= ir;
    uy *= ir;
    const double lim2 = LOCAL ? a.eta2 * r * r : INFINITY;
    KW<T> kw;
    kw.init(in.kre, in.kim, in.hk_tab);
    const T kk = kw.kval();
    T* colJ = sJ + lane;
    T* colL = sL + lane;
    T* colG = sG + lane;
    __syncthreads();   // previous item's coefficient columns are no longer read
    if (warp == 0) {
      besselj_seq<T>(rmul(kk, r), p + 1, colJ, kGrpCentres);
      for (int l = 0; l <= p; ++l) {
        const T jl = colJ[l * kGrpCentres];
        if (kD || kG) colL[l * kGrpCentres] = rmul(jl, (double)l);
        if (kG) {
          const T jn = colJ[(l + 1) * kGrpCentres];
          const T jp = (l == 0) ? jn : colJ[(l - 1) * kGrpCentres];
          colG[l * kGrpCentres] = (l == 0) ? rmul(jn, -1.0) : sc_sub(jp, jn);
        }
      }
      if (!keeps_jp1(PK)) {
        T z0;
        sc_zero(z0);
        colJ[(p + 1) * kGrpCentres] = z0;
      }
    }
    __syncthreads();
    const T J0 = colJ[0];
    const T kneg_j0 = rmul(sc_mul(kk, J0), -1.0);
    const cplx* wd = reinterpret_cast<const cplx*>(in.wd);

    for (int r0 = 0; r0 < a.nrhs; r0 += kRP) {
      cplx acc[kNc][RG];
      double t1[k3M ? kNc : 1][RG], t2[k3M ? kNc : 1][RG], t3[k3M ? kNc : 1][RG];
#pragma unroll
      for (int q = 0; q < kNc; ++q)
#pragma unroll
        for (int g = 0; g < RG; ++g) acc[q][g] = cplx{0.0, 0.0};
#pragma unroll
      for (int q = 0; q < (k3M ? kNc : 1); ++q)
#pragma unroll
        for (int g = 0; g < RG; ++g) t1[q][g] = t2[q][g] = t3[q][g] = 0.0;

      for (int base = item.src0; base < item.src1; base += kGrpTile) {
        const int nt = min(kGrpTile, item.src1 - base);
        __syncthreads();   // previous tile's values consumed
        for (int i = threadIdx.x; i < nt; i += blockDim.x) {
          s_x[i] = in.sx[base + i];
          s_y[i] = in.sy[base + i];
          if (kD) {
            s_nx[i] = in.snx[base + i];
            s_ny[i] = in.sny[base + i];
          }
        }
        for (int i = threadIdx.x; i < kGrpTile * kRP; i += blockDim.x) {
          const int s = i / kRP, rr = i - s * kRP;
          const cplx v = (s < nt && r0 + rr < a.nrhs) ? wd[(size_t)(base + s) * a.nrhs + r0 + rr] : cplx{0.0, 0.0};
          if constexpr (k3M) {
            s_wa[i] = v.re;
            s_wb[i] = v.im;
            s_ws[i] = v.re + v.im;
          } else {
            s_wd[i] = v;
          }
        }
        __syncthreads();
        // ---- phase 1: kernel values of this warp's sources ----
        for (int j = warp; j < nt; j += W) {
          const double dx = s_x[j] - cx, dy = s_y[j] - cy;
          double nx = 0.0, ny = 0.0;
          if (kD) {
            nx = s_nx[j];
            ny = s_ny[j];
          }
          cplx GS, K, GA, GB, EX, EY;
          if (LOCAL && fma(dx, dx, dy * dy) >= lim2) {   // near-only QBX: a distant source
            pair_direct<PK, T>(kw, kk, r * ux - dx, r * uy - dy, nx, ny, ux, uy, r, GS, K, GA, GB);
          } else {
            pair_kernels<PK, T, kGrpCentres>(kw, kk, J0, kneg_j0, colJ, colL, colG, p, dx, dy, nx, ny, ux,
                                             uy, ir, GS, K, GA, GB, EX, EY);
          }
          auto put = [&](int q, cplx v) {
            const int idx = (q * kGrpTile + j) * kGrpCentres + lane;
            if constexpr (k3M) {
              s_ka[idx] = v.re;
              s_kb[idx] = v.im;
              s_ks[idx] = v.re + v.im;
            } else {
              s_kv[idx] = v;
            }
          };
          if constexpr (kC) {
            // K - (i eta) GS, i eta = (-eta_im, eta_re)
            put(0, cplx{fma(a.cf_im, GS.re, fma(a.cf_re, GS.im, K.re)),
                        fma(a.cf_im, GS.im, fma(-a.cf_re, GS.re, K.im))});
          } else {
            int q = 0;
            if (kS) put(q++, GS);
            if (kD) put(q++, K);
            if (kG) {
              put(q++, GA);
              put(q++, GB);
            }
          }
        }
        __syncthreads();
        // ---- phase 2: this warp's rhs group ----
        if constexpr (k3M) {
          for (int j = 0; j < nt; ++j) {
            const int w0 = j * kRP + warp * RG;
#pragma unroll
            for (int q = 0; q < kNc; ++q) {
              const int idx = (q * kGrpTile + j) * kGrpCentres + lane;
              const double ka = s_ka[idx], kb = s_kb[idx], ks = s_ks[idx];
#pragma unroll
              for (int g = 0; g < RG; ++g) {
                t1[q][g] = fma(ka, s_wa[w0 + g], t1[q][g]);
                t2[q][g] = fma(kb, s_wb[w0 + g], t2[q][g]);
                t3[q][g] = fma(ks, s_ws[w0 + g], t3[q][g]);
              }
            }
          }
        } else {
          for (int j = 0; j < nt; ++j) {
            const cplx* w = s_wd + j * kRP + warp * RG;
#pragma unroll
            for (int q = 0; q < kNc; ++q) {
              const cplx kv = s_kv[(q * kGrpTile + j) * kGrpCentres + lane];
#pragma unroll
              for (int g = 0; g < RG; ++g) cfma(acc[q][g], w[g], kv);
            }
          }
        }
      }
      if constexpr (k3M) {
#pragma unroll
        for (int q = 0; q < kNc; ++q)
#pragma unroll
          for (int g = 0; g < RG; ++g)
            acc[q][g] = cplx{t1[q][g] - t2[q][g], t3[q][g] - t1[q][g] - t2[q][g]};
      }
      // ---- raw sums of this item (grad S already turned into x, y) ----
      if (active) {
        cplx* part = reinterpret_cast<cplx*>(in.part);
        const size_t row = ((size_t)item.split * in.n_ctr + c) * kNc;
#pragma unroll
        for (int g = 0; g < RG; ++g) {
          const int rr = r0 + warp * RG + g;
          if (rr >= a.nrhs) break;
          int q = 0;
          if (kC) {
            part[row * a.nrhs + rr] = acc[0][g];
            continue;
          }
          if (kS) {
            part[(row + q) * a.nrhs + rr] = acc[q][g];
            ++q;
          }
          if (kD) {
            part[(row + q) * a.nrhs + rr] = acc[q][g];
            ++q;
          }
          if (kG) {
            const cplx kA = smul(kk, acc[q][g]);
            const cplx Bi = acc[q + 1][g] * (2.0 * ir);
            part[(row + q) * a.nrhs + rr] = kA * ux + Bi * uy;
            part[(row + q + 1) * a.nrhs + rr] = kA * uy - Bi * ux;
          }
        }
      }
    }
    if (!dynamic) break;
  }
}

template <int OPS, typename T, int RG, bool LOCAL = false, int W = kGrpWarps>
static cudaError_t launch_group_t(const GroupArgs& a, int grid, cudaStream_t st) {
  const size_t smem = GroupSmem<OPS, T, RG, W>::bytes(a.p);
  auto kern = k_apply_group<OPS, T, RG, LOCAL, W>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kGrpCentres * W, smem, st>>>(a);
  return cudaGetLastError();
}

#define QBX_GROUP_OPS(X, T, RG)                                          \
  switch (ops) {                                                         \
    case OPB_S: X(OPB_S, T, RG);                                         \
    case OPB_D: X(OPB_D, T, RG);                                         \
    case OPB_S | OPB_D: X(OPB_S | OPB_D, T, RG);                         \
    case OPB_S | OPB_D | OPB_G: X(OPB_S | OPB_D | OPB_G, T, RG);         \
    case OPB_C: X(OPB_C, T, RG);                                         \
    default: break;                                                      \
  }

// rg: rhs per warp 2 or 8 with four warps per CTA, or kGrpRhsWide (64 rhs
// per pass: eight warps of 8; single curves, global apply)
template <typename T, bool LOCAL = false>
static cudaError_t launch_group_any(const GroupArgs& a, int rg, int grid, cudaStream_t st) {
  const int ops = a.ops;
  if constexpr (!LOCAL) {
    if (rg == kGrpRhsWide) {
#define X(O, TT, R) return launch_group_t<O, TT, R, false, 8>(a, grid, st)
      QBX_GROUP_OPS(X, T, 8)
#undef X
      return cudaErrorInvalidValue;
    }
  }
#define X(O, TT, R) return launch_group_t<O, TT, R, LOCAL>(a, grid, st)
  if (rg == 8) {
    QBX_GROUP_OPS(X, T, 8)
  } else {
    QBX_GROUP_OPS(X, T, 2)
  }
#undef X
  return cudaErrorInvalidValue;
}

template <typename T, bool LOCAL = false>
static int group_occupancy_any(int ops, int p, int rg) {
  int n = 0;
  if constexpr (!LOCAL) {
    if (rg == kGrpRhsWide) {
#define X(O, TT, R)                                                                                               \
  cudaFuncSetAttribute(k_apply_group<O, TT, R, false, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                       (int)GroupSmem<O, TT, R, 8>::bytes(p));                                                   \
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_apply_group<O, TT, R, false, 8>, kGrpCentres * 8,          \
                                                GroupSmem<O, TT, R, 8>::bytes(p));                               \
  return n
      QBX_GROUP_OPS(X, T, 8)
#undef X
      return 0;
    }
  }
#define X(O, TT, R)                                                                                         \
  cudaFuncSetAttribute(k_apply_group<O, TT, R, LOCAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                       (int)GroupSmem<O, TT, R>::bytes(p));                                                 \
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_apply_group<O, TT, R, LOCAL>, kGrpCentres * kGrpWarps, \
                                                GroupSmem<O, TT, R>::bytes(p));                             \
  return n
  if (rg == 8) {
    QBX_GROUP_OPS(X, T, 8)
  } else {
    QBX_GROUP_OPS(X, T, 2)
  }
#undef X
  return 0;
}

template <typename T, bool LOCAL = false>
static const void* group_ptr_any(int ops, int rg) {
#define X(O, TT, R) return (const void*)k_apply_group<O, TT, R, LOCAL>
  if (rg == 8) {
    QBX_GROUP_OPS(X, T, 8)
  } else {
    QBX_GROUP_OPS(X, T, 2)
  }
#undef X
  return nullptr;
}

template <typename T>
static size_t group_smem_any(int ops, int p, int rg) {
  if (rg == kGrpRhsWide) {
#define X(O, TT, R) return GroupSmem<O, TT, R, 8>::bytes(p)
    QBX_GROUP_OPS(X, T, 8)
#undef X
    return 0;
  }
#define X(O, TT, R) return GroupSmem<O, TT, R>::bytes(p)
  if (rg == 8) {
    QBX_GROUP_OPS(X, T, 8)
  } else {
    QBX_GROUP_OPS(X, T, 2)
  }
#undef X
  return 0;
}

}  // namespace qbx
