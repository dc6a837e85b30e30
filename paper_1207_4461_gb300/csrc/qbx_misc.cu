// qbx_misc.cu -- geometry (a0), density oversampling (a1), the unfused
// coefficient formation (a4) and evaluation (a5 + a6), the split reductions
// with the jump epilogue (a7), centre assignment and diagnostics.
#include <cuda_runtime.h>
#include <stdint.h>
#include "qbx_device.cuh"
#include "qbx_internal.h"

namespace qbx {

__device__ __forceinline__ bool finite_c(cplx v) { return isfinite(v.re) && isfinite(v.im); }

// ---------------------------------------------------------------------------
// a0 Geometry (Sec. 3.3 step 4a; Sec. 3.2 n = (t_2, -t_1); Sec. 4.1 panels).
// ---------------------------------------------------------------------------
__global__ void k_geom_nodes(int n, int q, const double* t_edges, const double* gam,
                             const double* dgam, const double* wgl, double* x, double* y,
                             double* nx, double* ny, double* w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m = i / q, j = i - m * q;
  const double half = 0.5 * (t_edges[m + 1] - t_edges[m]);
  const double gx = dgam[2 * i], gy = dgam[2 * i + 1];
  const double sp = hypot(gx, gy);
  x[i] = gam[2 * i];
  y[i] = gam[2 * i + 1];
  nx[i] = gy / sp;
  ny[i] = -gx / sp;
  w[i] = wgl[j] * half * sp;
}

// h_m: sum of the panel's source weights in node order (deterministic).
__global__ void k_panel_h(int M, int q_src, const double* w, double* h) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double s = 0.0;
  for (int j = 0; j < q_src; ++j) s += w[m * q_src + j];
  h[m] = s;
}

__global__ void k_centres(int n_tgt, int q_tgt, double r_factor, int rule, const double* h, const double* tx,
                          const double* ty, const double* tnx, const double* tny, double* cx,
                          double* cy, double* cr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tgt) return;
  const double hm = h[t / q_tgt];
  const double r = rule == QBX_RADIUS_SQRT_H ? r_factor * sqrt(hm) : r_factor * hm;
  cx[t] = tx[t] - r * tnx[t];
  cy[t] = ty[t] - r * tny[t];
  cr[t] = r;
  cx[n_tgt + t] = tx[t] + r * tnx[t];
  cy[n_tgt + t] = ty[t] + r * tny[t];
  cr[n_tgt + t] = r;
}

// Radius rule QBX_RADIUS_ADMISSIBLE (a departure from Sec. 3.3 step 4a for
// corners of 90 degrees or less): each centre's radius lowered to the largest
// r whose disk holds no source node.  With d = x_s - x and c = x + sg r n,
// |d - sg r n|^2 >= r^2 reads |d|^2 - 2 sg r (d.n) >= 0: a bound
// r <= |d|^2 / (2 sg d.n) for every source with sg d.n > 0.
__global__ void k_cap_radius(int n_tgt, const double* tx, const double* ty, const double* tnx, const double* tny,
                             int n_src, const double* sx, const double* sy, double* cx, double* cy, double* cr) {
  __shared__ double bx[256], by[256];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int cc = c < 2 * n_tgt ? c : 2 * n_tgt - 1;
  const int t = cc % n_tgt;
  const double sg = cc < n_tgt ? -1.0 : 1.0;
  const double x = tx[t], y = ty[t], nx = sg * tnx[t], ny = sg * tny[t];
  double r = cr[cc];
  for (int base = 0; base < n_src; base += 256) {
    const int nt = min(256, n_src - base);
    __syncthreads();
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
      bx[i] = sx[base + i];
      by[i] = sy[base + i];
    }
    __syncthreads();
    for (int j = 0; j < nt; ++j) {
      const double dx = bx[j] - x, dy = by[j] - y;
      const double a = fma(dx, nx, dy * ny);
      if (a > 0.0) r = fmin(r, fma(dx, dx, dy * dy) / (2.0 * a));
    }
  }
  if (c < 2 * n_tgt) {
    cr[c] = r;
    cx[c] = fma(r, nx, x);
    cy[c] = fma(r, ny, y);
  }
}

// ratio = min_s |x_s - c| / r  (eq. x-c-closest)
__global__ void k_ratio(int n_ctr, const double* cx, const double* cy, const double* cr, int n_src,
                        const double* sx, const double* sy, double* ratio) {
  __shared__ double bx[256], by[256];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int cc = c < n_ctr ? c : n_ctr - 1;
  const double x = cx[cc], y = cy[cc];
  double best = INFINITY;
  for (int base = 0; base < n_src; base += 256) {
    const int nt = min(256, n_src - base);
    __syncthreads();
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
      bx[i] = sx[base + i];
      by[i] = sy[base + i];
    }
    __syncthreads();
    for (int j = 0; j < nt; ++j) {
      const double dx = bx[j] - x, dy = by[j] - y;
      best = fmin(best, fma(dx, dx, dy * dy));
    }
  }
  if (c < n_ctr) ratio[c] = sqrt(best) / cr[c];
}

cudaError_t launch_geometry(int M, int q_tgt, int q_src, const double* t_edges,
                            const double* gam_tgt, const double* dgam_tgt,
                            const double* gam_src, const double* dgam_src,
                            const double* wgl_tgt, const double* wgl_src, double r_factor, int rule,
                            const qbx_geom& g, cudaStream_t st) {
  const int n_t = M * q_tgt, n_s = M * q_src;
  k_geom_nodes<<<(n_s + 255) / 256, 256, 0, st>>>(n_s, q_src, t_edges, gam_src, dgam_src, wgl_src,
                                                 g.src_x, g.src_y, g.src_nx, g.src_ny, g.src_w);
  k_geom_nodes<<<(n_t + 255) / 256, 256, 0, st>>>(n_t, q_tgt, t_edges, gam_tgt, dgam_tgt, wgl_tgt,
                                                 g.tgt_x, g.tgt_y, g.tgt_nx, g.tgt_ny, g.tgt_w);
  k_panel_h<<<(M + 127) / 128, 128, 0, st>>>(M, q_src, g.src_w, g.panel_h);
  k_centres<<<(n_t + 255) / 256, 256, 0, st>>>(n_t, q_tgt, r_factor, rule, g.panel_h, g.tgt_x, g.tgt_y,
                                              g.tgt_nx, g.tgt_ny, g.ctr_x, g.ctr_y, g.ctr_r);
  if (rule == QBX_RADIUS_ADMISSIBLE)
    k_cap_radius<<<(2 * n_t + 255) / 256, 256, 0, st>>>(n_t, g.tgt_x, g.tgt_y, g.tgt_nx, g.tgt_ny, n_s, g.src_x,
                                                       g.src_y, g.ctr_x, g.ctr_y, g.ctr_r);
  k_ratio<<<(2 * n_t + 255) / 256, 256, 0, st>>>(2 * n_t, g.ctr_x, g.ctr_y, g.ctr_r, n_s, g.src_x,
                                                g.src_y, g.ctr_ratio);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a1 Oversampling (Sec. 3.4.2): wdens[s][r] = w_s sum_i P[j][i] dens[m q_tgt + i][r].
// ---------------------------------------------------------------------------
__global__ void k_upsample(int n_src, int q_tgt, int q_src, int nrhs, const double* P,
                           const double* w, const cplx* dens, cplx* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_src * nrhs) return;
  const int s = idx / nrhs, r = idx - s * nrhs;
  const int m = s / q_src, j = s - m * q_src;
  const double* row = P + (size_t)j * q_tgt;
  const cplx* d = dens + (size_t)m * q_tgt * nrhs + r;
  double re = 0.0, im = 0.0;
  for (int i = 0; i < q_tgt; ++i) {
    const double c = row[i];
    const cplx v = d[(size_t)i * nrhs];
    re = fma(c, v.re, re);
    im = fma(c, v.im, im);
  }
  out[idx] = cplx{w[s] * re, w[s] * im};
}

// Unit tangents t = (-n_y, n_x) of the source nodes (the R operator of
// Sec. 3.2, eq. riesz-def, takes the D kernel with t in place of n).
__global__ void k_tangents(int n, const double* nx, const double* ny, double* tx, double* ty) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  tx[i] = -ny[i];
  ty[i] = nx[i];
}

cudaError_t launch_tangents(int n, const double* nx, const double* ny, double* tx, double* ty, cudaStream_t st) {
  if (n < 1) return cudaSuccess;
  k_tangents<<<(n + 255) / 256, 256, 0, st>>>(n, nx, ny, tx, ty);
  return cudaGetLastError();
}

// grad D finish (Sec. 3.2, eq. dlpderiv): ev [n_ctr][2][nrhs] are the
// gradients of the D expansions at the targets (interior centres first for
// two sides).  Two-sided: the average; PV from one side: lim -/+ t dmu/ds / 2
// (+ exterior), t = (-n_y, n_x), dmu/ds = (sum_j Dx[i][j] mu_j) w^GL_i / w_t.
__global__ void k_grad_d_finish(int n_tgt, int q_tgt, int nsides, int side0, int limit, int nrhs,
                                const cplx* ev, const cplx* dens, const double* tnx, const double* tny,
                                const double* tw, const double* wgl, const double* Dx, cplx* out, int* status) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_tgt * nrhs) return;
  const int t = idx / nrhs, r = idx - t * nrhs;
  cplx gx{0.0, 0.0}, gy{0.0, 0.0};
  for (int sd = 0; sd < nsides; ++sd) {
    const size_t row = ((size_t)(sd * n_tgt + t) * 2) * nrhs + r;
    gx = gx + ev[row];
    gy = gy + ev[row + nrhs];
  }
  if (nsides == 2) {
    gx = 0.5 * gx;
    gy = 0.5 * gy;
  } else if (limit == QBX_LIMIT_PV) {
    const int m = t / q_tgt, i = t - m * q_tgt;
    const cplx* d = dens + (size_t)m * q_tgt * nrhs + r;
    double re = 0.0, im = 0.0;
    for (int j = 0; j < q_tgt; ++j) {
      const double c = Dx[i * q_tgt + j];
      re = fma(c, d[(size_t)j * nrhs].re, re);
      im = fma(c, d[(size_t)j * nrhs].im, im);
    }
    const double f = wgl[i] / tw[t];
    const cplx ds{re * f, im * f};
    const double sg = side0 == QBX_SIDE_EXT ? 1.0 : -1.0;
    gx = gx - (0.5 * sg * -tny[t]) * ds;
    gy = gy - (0.5 * sg * tnx[t]) * ds;
  }
  out[((size_t)t * 2) * nrhs + r] = gx;
  out[((size_t)t * 2 + 1) * nrhs + r] = gy;
  if (!(isfinite(gx.re) && isfinite(gx.im) && isfinite(gy.re) && isfinite(gy.im))) atomicOr(status, 1);
}

cudaError_t launch_grad_d_finish(int n_tgt, int q_tgt, int nsides, int side0, int limit, int nrhs, const void* ev,
                                 const void* dens, const double* tnx, const double* tny, const double* tw,
                                 const double* wgl, const double* Dx, void* out, int* status, cudaStream_t st) {
  const int n = n_tgt * nrhs;
  k_grad_d_finish<<<(n + 255) / 256, 256, 0, st>>>(n_tgt, q_tgt, nsides, side0, limit, nrhs, (const cplx*)ev,
                                                   (const cplx*)dens, tnx, tny, tw, wgl, Dx, (cplx*)out, status);
  return cudaGetLastError();
}

cudaError_t launch_upsample(int M, int q_tgt, int q_src, int nrhs, const double* interp,
                            const double* src_w, const void* dens_tgt, void* wdens,
                            cudaStream_t st) {
  const int n = M * q_src * nrhs;
  k_upsample<<<(n + 255) / 256, 256, 0, st>>>(M * q_src, q_tgt, q_src, nrhs, interp, src_w,
                                              (const cplx*)dens_tgt, (cplx*)wdens);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a7 Reduction over splits (fixed order), factor i/4, jump / average (Sec. 3.2).
// part: [nsplit][n_ctr][ncomp][nrhs]; for side TWO, centre t (interior) and
// n_tgt + t (exterior) are averaged.
// ---------------------------------------------------------------------------
__global__ void k_apply_finish(int op, int side, int limit, int n_tgt, int nsplit, int n_ctr,
                               int nrhs, int comp0, int ncomp_total, const cplx* part, const cplx* dens,
                               const double* tnx, const double* tny, cplx* out, int* status) {
  const int ncomp = op == QBX_OP_GRAD_S ? 2 : 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_tgt * ncomp * nrhs) return;
  const int t = idx / (ncomp * nrhs);
  const int rem = idx - t * ncomp * nrhs;
  const int comp = rem / nrhs, r = rem - comp * nrhs;
  const int nsides = side == QBX_SIDE_TWO ? 2 : 1;
  cplx res{0.0, 0.0};
  for (int sd = 0; sd < nsides; ++sd) {
    const int c = t + sd * n_tgt;
    cplx u{0.0, 0.0};
    for (int k = 0; k < nsplit; ++k)
      u = u + part[(((size_t)k * n_ctr + c) * ncomp_total + comp0 + comp) * nrhs + r];
    u = mul_i(0.25 * u);
    if (side != QBX_SIDE_TWO && limit == QBX_LIMIT_PV) {
      const double sg = side == QBX_SIDE_EXT ? 1.0 : -1.0;
      const cplx dv = dens[(size_t)t * nrhs + r];
      if (op == QBX_OP_D) u = u - (0.5 * sg) * dv;
      else if (op == QBX_OP_GRAD_S) u = u + (0.5 * sg * (comp == 0 ? tnx[t] : tny[t])) * dv;
    }
    res = res + u;
  }
  if (nsides == 2) res = 0.5 * res;
  out[idx] = res;
  if (!finite_c(res)) atomicOr(status, 1);
}

cudaError_t launch_apply_finish(int op, int side, int limit, int n_tgt, int nsplit, int n_ctr,
                                int nrhs, int comp0, int ncomp_total, const void* part,
                                const void* dens_tgt, const double* tgt_nx, const double* tgt_ny,
                                void* out, int* status, cudaStream_t st) {
  const int ncomp = op == QBX_OP_GRAD_S ? 2 : 1;
  const int n = n_tgt * ncomp * nrhs;
  k_apply_finish<<<(n + 255) / 256, 256, 0, st>>>(op, side, limit, n_tgt, nsplit, n_ctr, nrhs, comp0,
                                                  ncomp_total, (const cplx*)part, (const cplx*)dens_tgt,
                                                  tgt_nx, tgt_ny, (cplx*)out, status);
  return cudaGetLastError();
}

// Fused apply dispatch: real k (fitted real-argument Hankel path) or complex k.
cudaError_t launch_apply_fused(const ApplyArgs& a, cudaStream_t st) {
  if (a.eta2 > 0.0) return a.kim == 0.0 ? launch_apply_fused_local_real(a, st) : launch_apply_fused_local_cplx(a, st);
  return a.kim == 0.0 ? launch_apply_fused_real(a, st) : launch_apply_fused_cplx(a, st);
}

size_t apply_smem_bytes(int ops, bool ck, int p, int nr) {
  return ck ? apply_smem_bytes_cplx(ops, p, nr) : apply_smem_bytes_real(ops, p, nr);
}

// rhs per launch: accumulators for one operator take 8 rhs in registers,
// several operators together 4.
int apply_chunk(int ops) { return (ops == 1 || ops == 2 || ops == 4) ? 8 : 4; }

__global__ void k_far_finish(int op, double kre, double kim, int n_far, int nsplit, int nrhs,
                             const cplx* part, cplx* out, int* status) {
  const int ncomp = op == QBX_OP_GRAD_S ? 2 : 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_far * ncomp * nrhs) return;
  cplx u{0.0, 0.0};
  for (int k = 0; k < nsplit; ++k) u = u + part[(size_t)k * n_far * ncomp * nrhs + idx];
  cplx f = op == QBX_OP_S ? cplx{0.0, 0.25} : cplx{-0.25 * kim, 0.25 * kre};  // i/4 or ik/4
  if (op == QBX_OP_GRAD_S) f = -f;
  u = f * u;
  out[idx] = u;
  if (!finite_c(u)) atomicOr(status, 1);
}

cudaError_t launch_far_finish(int op, double kre, double kim, int n_far, int nsplit, int nrhs,
                              const void* part, void* out, int* status, cudaStream_t st) {
  const int ncomp = op == QBX_OP_GRAD_S ? 2 : 1;
  const int n = n_far * ncomp * nrhs;
  k_far_finish<<<(n + 255) / 256, 256, 0, st>>>(op, kre, kim, n_far, nsplit, nrhs,
                                                (const cplx*)part, (cplx*)out, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a4 Unfused coefficients (Sec. 3.3 step 4b).  One thread per centre,
// accumulators for the 2p+1 orders of `nr` rhs in shared memory.
//   S: alpha_l += wd H_l e^{-i l theta},  alpha_{-l} += wd (-1)^l H_l e^{i l theta}
//   D: alpha^D_l += wd (-1)^l (k/2) [nu F_{-l-1} - conj(nu) F_{-l+1}],
//      F_m = H_m e^{i m theta}, F_{-m} = (-1)^m H_m e^{-i m theta}
// (factor i/4 in the finishing kernel).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kFormThreads)
k_form(FormArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s_x = reinterpret_cast<double*>(smem_raw);
  double* s_y = s_x + kSrcTile;
  double* s_nx = s_y + kSrcTile;
  double* s_ny = s_nx + kSrcTile;
  const int nr = a.nr;
  cplx* s_wd = reinterpret_cast<cplx*>(s_ny + kSrcTile);        // [tile][nr]
  cplx* s_acc = s_wd + kSrcTile * nr;                          // [(2p+1)*nr][threads]
  const int tid = threadIdx.x;
  const int c = blockIdx.x * kFormThreads + tid;
  const bool active = c < a.n_ctr;
  const int cc = active ? c : a.n_ctr - 1;
  const int p = a.p, nl = 2 * p + 1;
  for (int i = 0; i < nl * nr; ++i) s_acc[i * kFormThreads + tid] = cplx{0.0, 0.0};
  const double cx = a.cx[cc], cy = a.cy[cc];
  const cplx k = cplx{a.kre, a.kim};
  const cplx hk = 0.5 * k;
  const int s_begin = blockIdx.y * a.src_per_split;
  const int s_end = min(a.src.n, s_begin + a.src_per_split);
  const cplx* wd = reinterpret_cast<const cplx*>(a.wd);
  for (int base = s_begin; base < s_end; base += kSrcTile) {
    const int nt = min(kSrcTile, s_end - base);
    __syncthreads();
    for (int i = tid; i < nt; i += kFormThreads) {
      s_x[i] = a.src.x[base + i];
      s_y[i] = a.src.y[base + i];
      s_nx[i] = a.src.nx[base + i];
      s_ny[i] = a.src.ny[base + i];
    }
    for (int i = tid; i < nt * nr; i += kFormThreads) {
      const int s = i / nr, rr = i - s * nr;
      s_wd[i] = wd[(size_t)(base + s) * a.nrhs + a.rhs0 + rr];
    }
    __syncthreads();
    if (!active) continue;
    for (int j = 0; j < nt; ++j) {
      const double dx = s_x[j] - cx, dy = s_y[j] - cy;
      const double rho2 = fma(dx, dx, dy * dy);
      const double inv = rsqrt(rho2);
      const double rho = rho2 * inv;
      const cplx e1 = cplx{dx * inv, -dy * inv};   // e^{-i theta}
      cplx H0, H1;
      cplx twoz;
      if (a.kim == 0.0) {
        const double z = a.kre * rho, invz = inv / a.kre;
        hankel01_real(z, invz, sqrt(invz), H0, H1);
        twoz = cplx{2.0 * invz, 0.0};
      } else {
        const cplx z = cplx{a.kre * rho, a.kim * rho};
        hankel01_cplx(z, H0, H1);
        twoz = 2.0 * cinv(z);
      }
      if (a.kind == QBX_OP_S) {
        cplx Hm = H0, H = H1, E = cplx{1.0, 0.0};   // E = e^{-i l theta}
        cplx s = twoz;
        for (int l = 0; l <= p; ++l) {
          const cplx Hl = (l == 0) ? H0 : H;
          const cplx Kp = Hl * E;                          // H_l e^{-i l theta}
          const cplx Km = ((l & 1) ? -1.0 : 1.0) * (Hl * conj(E));
          for (int rr = 0; rr < nr; ++rr) {
            const cplx w = s_wd[j * nr + rr];
            cplx* A = s_acc + ((size_t)(l + p) * nr + rr) * kFormThreads + tid;
            *A = *A + w * Kp;
            if (l > 0) {
              cplx* B = s_acc + ((size_t)(p - l) * nr + rr) * kFormThreads + tid;
              *B = *B + w * Km;
            }
          }
          E = E * e1;
          if (l >= 1) {
            const cplx Hn = s * H - Hm;
            Hm = H;
            H = Hn;
            s = s + twoz;
          }
        }
      } else {
        // sliding window of F_{+n}, F_{-n} for n, n-1, n-2
        const cplx nu = cplx{s_nx[j], s_ny[j]};
        const cplx nub = conj(nu);
        cplx Hm = H0, H = H1;
        cplx s = twoz;
        cplx E = cplx{1.0, 0.0};          // e^{-i n theta}
        cplx Fp0{0, 0}, Fm0{0, 0}, Fp1{0, 0}, Fm1{0, 0}, Fp2{0, 0}, Fm2{0, 0};   // index n, n-1, n-2
        for (int n = 0; n <= p + 1; ++n) {
          const cplx Hn_ = (n == 0) ? H0 : H;
          const double sg = (n & 1) ? -1.0 : 1.0;
          Fp2 = Fp1; Fm2 = Fm1; Fp1 = Fp0; Fm1 = Fm0;
          Fp0 = Hn_ * conj(E);              // F_{+n} = H_n e^{i n theta}
          Fm0 = sg * (Hn_ * E);             // F_{-n} = (-1)^n H_n e^{-i n theta}
          if (n >= 1) {
            const int l = n - 1;
            const double sl = (l & 1) ? -1.0 : 1.0;
            // alpha^D_l (l >= 0): nu F_{-l-1} - conj(nu) F_{-l+1}
            const cplx Fl1 = (l == 0) ? Fp0 : Fm2;   // F_{-l+1}: l = 0 -> F_{+1}
            const cplx kp = (sl * hk) * (nu * Fm0 - nub * Fl1);
            cplx km{0, 0};
            if (l >= 1) km = (sl * hk) * (nu * Fp2 - nub * Fp0);   // l' = -l: F_{l-1}, F_{l+1}
            for (int rr = 0; rr < nr; ++rr) {
              const cplx w = s_wd[j * nr + rr];
              cplx* A = s_acc + ((size_t)(l + p) * nr + rr) * kFormThreads + tid;
              *A = *A + w * kp;
              if (l >= 1) {
                cplx* B = s_acc + ((size_t)(p - l) * nr + rr) * kFormThreads + tid;
                *B = *B + w * km;
              }
            }
          }
          E = E * e1;
          if (n >= 1) {
            const cplx Hn = s * H - Hm;
            Hm = H;
            H = Hn;
            s = s + twoz;
          }
        }
      }
    }
  }
  if (!active) return;
  cplx* part = reinterpret_cast<cplx*>(a.part);
  for (int l = 0; l < nl; ++l)
    for (int rr = 0; rr < nr; ++rr)
      part[(((size_t)blockIdx.y * a.n_ctr + c) * nl + l) * a.nrhs + a.rhs0 + rr] =
          s_acc[((size_t)l * nr + rr) * kFormThreads + tid];
}

size_t form_smem_bytes(int p, int nr) {
  return 4 * kSrcTile * sizeof(double) + (size_t)kSrcTile * nr * 16 +
         (size_t)(2 * p + 1) * nr * kFormThreads * 16;
}

cudaError_t launch_form(const FormArgs& a, cudaStream_t st) {
  const size_t smem = form_smem_bytes(a.p, a.nr);
  cudaError_t e = cudaFuncSetAttribute(k_form, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.n_ctr + kFormThreads - 1) / kFormThreads, a.nsplit);
  k_form<<<grid, kFormThreads, smem, st>>>(a);
  return cudaGetLastError();
}

__global__ void k_form_finish(int n_ctr, int ncoef, int nsplit, int nrhs, const cplx* part,
                              cplx* alpha, int* status) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t n = (size_t)n_ctr * ncoef * nrhs;
  if (idx >= n) return;
  cplx u{0.0, 0.0};
  for (int k = 0; k < nsplit; ++k) u = u + part[(size_t)k * n + idx];
  u = mul_i(0.25 * u);
  alpha[idx] = u;
  if (!finite_c(u)) atomicOr(status, 1);
}

cudaError_t launch_form_finish(int n_ctr, int ncoef, int nsplit, int nrhs, const void* part,
                               void* alpha, int* status, cudaStream_t st) {
  const size_t n = (size_t)n_ctr * ncoef * nrhs;
  k_form_finish<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n_ctr, ncoef, nsplit, nrhs,
                                                            (const cplx*)part, (cplx*)alpha, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a5 + a6: evaluate stored coefficients (Sec. 3.3 step 4c), value or gradient
//   u = sum_l alpha_l J_l(k rho) e^{i l theta}
//   (d_x + i d_y) u = -k sum alpha_l J_{l+1} e^{i(l+1)theta},
//   (d_x - i d_y) u =  k sum alpha_l J_{l-1} e^{i(l-1)theta}.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ cplx jc(const T* J, int l) {
  const int al = l < 0 ? -l : l;
  cplx v = to_c(J[al]);
  if (l < 0 && (al & 1)) v = -v;
  return v;
}

template <typename T> __device__ __forceinline__ T make_kr(double kre, double kim, double rho);
template <> __device__ __forceinline__ double make_kr<double>(double kre, double, double rho) { return kre * rho; }
template <> __device__ __forceinline__ cplx make_kr<cplx>(double kre, double kim, double rho) {
  return cplx{kre * rho, kim * rho};
}

template <typename T>
__global__ void k_eval(EvalArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.n_eval) return;
  const int c = a.ectr ? a.ectr[e] : e;
  if (c < 0 || c >= a.n_ctr) {   // invalid centre index: NaN output, status flag
    const int nout = (a.what == QBX_GRAD ? 2 : 1) * a.nrhs;
    cplx* o = reinterpret_cast<cplx*>(a.out) + (size_t)e * nout;
    for (int i = 0; i < nout; ++i) o[i] = cplx{NAN, NAN};
    atomicOr(a.status, 2);
    return;
  }
  double x, y;
  if (a.ex) {
    x = a.ex[e];
    y = a.ey[e];
  } else {
    x = a.tx[c % a.n_tgt];
    y = a.ty[c % a.n_tgt];
  }
  const double dx = x - a.cx[c], dy = y - a.cy[c];
  const double rho = hypot(dx, dy);
  const cplx eith = rho > 0.0 ? cplx{dx / rho, dy / rho} : cplx{1.0, 0.0};
  T J[QBX_MAX_P + 2];
  const T kr = make_kr<T>(a.kre, a.kim, rho);
  if (rho > 0.0) besselj_seq<T>(kr, a.p + 1, J, 1);
  else {
    for (int l = 0; l <= a.p + 1; ++l) sc_zero(J[l]);
    sc_set(J[0], 1.0);
  }
  cplx E[QBX_MAX_P + 2];   // e^{i m theta}, m = 0..p+1
  E[0] = cplx{1.0, 0.0};
  for (int m = 1; m <= a.p + 1; ++m) E[m] = E[m - 1] * eith;
  const int p = a.p, nl = 2 * p + 1;
  const cplx k = cplx{a.kre, a.kim};
  const cplx* alpha = reinterpret_cast<const cplx*>(a.alpha) + (size_t)c * nl * a.nrhs;
  cplx* out = reinterpret_cast<cplx*>(a.out);
  for (int r = 0; r < a.nrhs; ++r) {
    if (a.what == QBX_GRAD) {
      cplx up{0, 0}, um{0, 0};
      for (int l = -p; l <= p; ++l) {
        const cplx al = alpha[(size_t)(l + p) * a.nrhs + r];
        const int mp1 = l + 1, mm1 = l - 1;
        const cplx ep = mp1 >= 0 ? E[mp1] : conj(E[-mp1]);
        const cplx em = mm1 >= 0 ? E[mm1] : conj(E[-mm1]);
        up = up + al * (jc(J, mp1) * ep);
        um = um + al * (jc(J, mm1) * em);
      }
      up = -(k * up);
      um = k * um;
      const cplx gx = 0.5 * (up + um);
      const cplx d = up - um;
      const cplx gy = cplx{0.5 * d.im, -0.5 * d.re};   // d / (2i)
      out[((size_t)e * 2 + 0) * a.nrhs + r] = gx;
      out[((size_t)e * 2 + 1) * a.nrhs + r] = gy;
    } else {
      cplx u{0, 0};
      for (int l = -p; l <= p; ++l) {
        const cplx el = l >= 0 ? E[l] : conj(E[-l]);
        u = u + alpha[(size_t)(l + p) * a.nrhs + r] * (jc(J, l) * el);
      }
      out[(size_t)e * a.nrhs + r] = u;
    }
  }
}

cudaError_t launch_eval(const EvalArgs& a, cudaStream_t st) {
  const int threads = 128;
  const int blocks = (a.n_eval + threads - 1) / threads;
  if (a.kim == 0.0) k_eval<double><<<blocks, threads, 0, st>>>(a);
  else k_eval<cplx><<<blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Centre assignment for off-surface points (smallest |x-c|/r <= 1, lowest index).
// ---------------------------------------------------------------------------
__global__ void k_assign(int n, const double* xy, int n_ctr, const double* cx, const double* cy,
                         const double* cr, int* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double x = xy[2 * e], y = xy[2 * e + 1];
  int best = -1;
  double bq = INFINITY;
  for (int c = 0; c < n_ctr; ++c) {
    const double q = hypot(x - cx[c], y - cy[c]) / cr[c];
    if (q <= 1.0 && q < bq) {
      bq = q;
      best = c;
    }
  }
  out[e] = best;
}

cudaError_t launch_assign(int n, const double* xy, int n_ctr, const double* cx, const double* cy,
                          const double* cr, int* out, cudaStream_t st) {
  k_assign<<<(n + 127) / 128, 128, 0, st>>>(n, xy, n_ctr, cx, cy, cr, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Diagnostics: the device special functions at given points.
// ---------------------------------------------------------------------------
__global__ void k_debug_hankel(const cplx* z, int n, cplx* h0, cplx* h1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const cplx zz = z[i];
  cplx a, b;
  if (zz.im == 0.0 && zz.re > 0.0) hankel01_real(zz.re, 1.0 / zz.re, sqrt(1.0 / zz.re), a, b);
  else hankel01_cplx(zz, a, b);
  h0[i] = a;
  h1[i] = b;
}

__global__ void k_debug_besselj(const cplx* z, int n, int nmax, cplx* j) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const cplx zz = z[i];
  if (zz.im == 0.0) {
    double J[QBX_MAX_P + 2];
    besselj_seq<double>(zz.re, nmax, J, 1);
    for (int l = 0; l <= nmax; ++l) j[(size_t)i * (nmax + 1) + l] = cplx{J[l], 0.0};
  } else {
    cplx J[QBX_MAX_P + 2];
    besselj_seq<cplx>(zz, nmax, J, 1);
    for (int l = 0; l <= nmax; ++l) j[(size_t)i * (nmax + 1) + l] = J[l];
  }
}

cudaError_t launch_debug_hankel(const void* z, int n, void* h0, void* h1, cudaStream_t st) {
  k_debug_hankel<<<(n + 127) / 128, 128, 0, st>>>((const cplx*)z, n, (cplx*)h0, (cplx*)h1);
  return cudaGetLastError();
}

cudaError_t launch_debug_besselj(const void* z, int n, int nmax, void* j, cudaStream_t st) {
  k_debug_besselj<<<(n + 127) / 128, 128, 0, st>>>((const cplx*)z, n, nmax, (cplx*)j);
  return cudaGetLastError();
}

}  // namespace qbx
