// qbx_internal.h -- launch descriptors shared by the library's translation
// units (host side of the kernels).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <vector>
#include "../../include/qbx.h"

namespace qbx {

struct cplx;

constexpr int kApplyThreads = 128;   // centres per CTA of the fused apply
constexpr int kSrcTile = 128;        // sources staged in shared memory per step
constexpr int kFormThreads = 64;     // centres per CTA of form_locals
constexpr int kMaxSplit = 64;        // source splits of the split reductions

struct SrcView {
  const double *x, *y, *nx, *ny;
  int n;
};

// Fused storage-free apply (a2-a6 fused) of an operator subset, one launch
// per chunk of `nr` rhs.
struct ApplyArgs {
  int ops;                // bit (1 << QBX_OP_S) | (1 << QBX_OP_D) | (1 << QBX_OP_GRAD_S)
  int p;
  double kre, kim;
  int n_ctr;              // centres in this launch
  const double *cx, *cy;  // [n_ctr]
  int n_tgt;              // target of centre c is c mod n_tgt
  const double *tx, *ty;  // [n_tgt]
  SrcView src;
  const void* wd[3];      // per operator (S, D, grad S): [n_src][nrhs] complex
  int nrhs, rhs0, nr;     // total rhs, first rhs of this chunk, chunk width
  int nsplit, src_per_split;
  void* part;             // [nsplit][n_ctr][ncomp][nrhs] complex, comps S, D, grad S (x, y)
  double eta2;            // near-only QBX: if > 0, sources with |x_s - c|^2 >= eta2 r^2 by the
                          // smooth rule at the target; otherwise (default) all through the expansion
  int near_q_tgt, near_q_src;   // > 0: near-field items first (node counts per panel); 0: plain order
  int one_w;              // 1: wd[] of every requested operator is one array and nr = 1 (weighted
                          // seeds: the density multiplies H0, H1); 0: per-pair kernel values
  const double* hk_tab;   // complex k: the amplitude table of this k's ray (launch_hk_table), or null
};
// Amplitudes B_n = H_n(z) e^{-i(z - pi/4)}, n = 0, 1, along the ray z = k rho
// (|z| >= 2) as piecewise polynomials in s = |z|^{-1/2}, in the layout of the
// real-axis table (hk_table_doubles() doubles), for Im k > 0.
int hk_table_doubles();
cudaError_t launch_hk_table(double kre, double kim, double* tab, cudaStream_t st);
cudaError_t launch_debug_hankel_ray(double kre, double kim, const double* tab, const double* rho, int n, void* h0,
                                    void* h1, cudaStream_t st);
cudaError_t launch_apply_fused(const ApplyArgs& a, cudaStream_t st);
cudaError_t launch_apply_fused_real(const ApplyArgs& a, cudaStream_t st);
cudaError_t launch_apply_fused_cplx(const ApplyArgs& a, cudaStream_t st);
cudaError_t launch_apply_fused_local_real(const ApplyArgs& a, cudaStream_t st);
cudaError_t launch_apply_fused_local_cplx(const ApplyArgs& a, cudaStream_t st);
int apply_occupancy_local(int ops, bool ck, int p, int nr, bool one_w = false);   // near-only instances
// Storage-free grad D (one rhs per launch, a.rhs0; a.wd[0] the weighted
// density): partial sums [nsplit][n_ctr][2][nrhs] of the expansion gradient
// without the factor i/4.
cudaError_t launch_grad_d_fused(const ApplyArgs& a, cudaStream_t st);
size_t grad_d_fused_smem(bool ck, int p);
int grad_d_fused_occupancy(bool ck, int p);
size_t apply_smem_bytes(int ops, bool ck, int p, int nr);
size_t apply_smem_bytes_real(int ops, int p, int nr);
size_t apply_smem_bytes_cplx(int ops, int p, int nr);
int apply_chunk(int ops);   // rhs per launch for an operator subset
int apply_occupancy_real(int ops, int p, int nr, bool one_w = false);   // resident CTAs per SM
int apply_occupancy_cplx(int ops, int p, int nr, bool one_w = false);

// Far targets: plain quadrature partial sums.
struct FarArgs {
  int op;
  double kre, kim;
  int n_far;
  const double* xy;       // [n_far][2]
  SrcView src;
  const void* wd;
  int nrhs, rhs0, nr;
  int nsplit, src_per_split;
  void* part;             // [nsplit][n_far][ncomp][nrhs]
  const double* hk_tab;   // complex k: the amplitude table of this k's ray, or null
};
cudaError_t launch_far(const FarArgs& a, cudaStream_t st);

// Unfused coefficients (a4).
struct FormArgs {
  int kind, p;
  double kre, kim;
  int n_ctr;
  const double *cx, *cy;
  SrcView src;
  const void* wd;
  int nrhs, rhs0, nr;
  int nsplit, src_per_split;
  void* part;             // [nsplit][n_ctr][2p+1][nrhs]
};
cudaError_t launch_form(const FormArgs& a, cudaStream_t st);
size_t form_smem_bytes(int p, int nr);

// Evaluation of stored coefficients (a5 + a6).
struct EvalArgs {
  int what, p;
  double kre, kim;
  int n_eval;
  const double *ex, *ey;  // targets (may be null: default on-surface)
  const int* ectr;        // centre per target (null: identity)
  const double *cx, *cy;
  int n_tgt;
  const double *tx, *ty;
  const void* alpha;      // [n_ctr][2p+1][nrhs]
  int nrhs;
  void* out;
  int n_ctr;              // centres of the side (bound for ectr)
  int* status;
};
cudaError_t launch_eval(const EvalArgs& a, cudaStream_t st);

// Reductions over splits and epilogues.
// comp0: first component of operator `op` among the ncomp_total components
// of each partial-sum row.
cudaError_t launch_apply_finish(int op, int side, int limit, int n_tgt, int nsplit, int n_ctr,
                                int nrhs, int comp0, int ncomp_total, const void* part,
                                const void* dens_tgt, const double* tgt_nx, const double* tgt_ny,
                                void* out, int* status, cudaStream_t st);
cudaError_t launch_far_finish(int op, double kre, double kim, int n_far, int nsplit, int nrhs,
                              const void* part, void* out, int* status, cudaStream_t st);
cudaError_t launch_form_finish(int n_ctr, int ncoef, int nsplit, int nrhs, const void* part,
                               void* alpha, int* status, cudaStream_t st);

// Geometry, oversampling, centre assignment.
cudaError_t launch_geometry(int M, int q_tgt, int q_src, const double* t_edges,
                            const double* gam_tgt, const double* dgam_tgt,
                            const double* gam_src, const double* dgam_src,
                            const double* wgl_tgt, const double* wgl_src, double r_factor, int rule,
                            const qbx_geom& g, cudaStream_t st);
cudaError_t launch_upsample(int M, int q_tgt, int q_src, int nrhs, const double* interp,
                            const double* src_w, const void* dens_tgt, void* wdens,
                            cudaStream_t st);
cudaError_t launch_grad_d_finish(int n_tgt, int q_tgt, int nsides, int side0, int limit, int nrhs, const void* ev,
                                 const void* dens, const double* tnx, const double* tny, const double* tw,
                                 const double* wgl, const double* Dx, void* out, int* status, cudaStream_t st);
cudaError_t launch_tangents(int n, const double* nx, const double* ny, double* tx, double* ty, cudaStream_t st);
cudaError_t launch_assign(int n, const double* xy, int n_ctr, const double* cx,
                          const double* cy, const double* cr, int* out, cudaStream_t st);
cudaError_t launch_debug_hankel(const void* z, int n, void* h0, void* h1, cudaStream_t st);
cudaError_t launch_debug_besselj(const void* z, int n, int nmax, void* j, cudaStream_t st);

// Host helpers shared by the C-ABI translation units (qbx_capi.cu).
void host_interp_matrix(int q_tgt, int q_src, std::vector<double>& M);
size_t host_align256(size_t b);
int host_choose_split(int num_sms, int n_units, int n_src, size_t bytes_per_split, size_t avail);
int host_choose_split_waves(int num_sms, int occ, int n_units, int n_src, size_t bytes_per_split,
                            size_t avail, int min_waves = 1);
int host_split_len(int n_src, int ns);
int host_fail(int code, const char* msg);   // sets qbx_last_error(), returns code
void host_plan_info(const qbx_plan* plan, int* device, int* q_tgt, int* q_src, const double** interp);
// y = A x for a column-major n x n matrix (qbx_matmul_cm); with gate, every
// kernel returns at once while *gate (device) is 0.
int matmul_cm_gated(int n, int nrhs, const qbx_c64* A, const qbx_c64* x, qbx_c64* y, void* work,
                    size_t work_bytes, const int* gate, void* stream);

}  // namespace qbx

namespace qbx {

// ---- many right-hand sides and batches: the group kernel ------------------
constexpr int kGrpCentres = 32;   // centres per CTA (one per lane)
constexpr int kGrpWarps = 4;      // warps per CTA: rhs groups in phase 2
constexpr int kGrpRhsWide = 64;   // the rg code of the eight-warp instances (64 rhs per pass)
// the group kernel's operator set of the combined field D - i eta S (OPB_C)
constexpr int kOpsCombined = 16;
constexpr int kGrpTile = 32;      // sources per shared-memory tile

// One curve of a batch (or the single curve of a many-rhs apply).
struct GroupInst {
  double kre, kim;
  int n_src, n_tgt, n_ctr;        // n_ctr: centres of the side set
  int side, nsplit, M;
  const double *sx, *sy, *snx, *sny, *sw;
  const double *cx, *cy;          // centres of the side set
  const double *tx, *ty, *tnx, *tny;
  const void* wd;                 // [n_src][nrhs] oversampled weighted density
  const void* dens;               // [n_tgt][nrhs] density on the target grid (jump terms)
  void* part;                     // [nsplit][n_ctr][ncomp][nrhs] raw sums
  void* out[3];                   // per operator (S, D, grad S) outputs, for the finish
  const double* hk_tab;           // complex k: the amplitude table of this curve's k, or null
};
// A work item: 32 centres from ctr0 of instance inst, sources [src0, src1),
// partial-sum slot `split`.
struct GroupItem {
  int inst, ctr0, split, src0, src1;
};
struct GroupArgs {
  int ops, p, nrhs;
  const GroupInst* inst;          // dynamic mode: instance table
  GroupInst inst0;                // static mode: the one instance
  int n_items;
  const GroupItem* items;         // dynamic mode: item list (longest first)
  int* counter;                   // dynamic mode: next item (zeroed before launch)
  int st_units, st_nsplit, st_split_len;   // static mode (items == nullptr): one instance
  double eta2;                    // near-only QBX (> 0): sources with |x_s - c|^2 >= eta2 r^2 by the
                                  // smooth rule at the target; 0: all through the expansion
  double cf_re, cf_im;            // ops == OPB_C: eta of the combined field D - i eta S
};
cudaError_t launch_group_real(const GroupArgs& a, int rg, int grid, cudaStream_t st);
cudaError_t launch_group_cplx(const GroupArgs& a, int rg, int grid, cudaStream_t st);
size_t group_smem_real(int ops, int p, int rg);
size_t group_smem_cplx(int ops, int p, int rg);
int group_occupancy_real(int ops, int p, int rg);
int group_occupancy_cplx(int ops, int p, int rg);
const void* group_ptr_real(int ops, int rg);
const void* group_ptr_cplx(int ops, int rg);
// near-only instances of the group kernel (GroupArgs::eta2 > 0)
cudaError_t launch_group_local(const GroupArgs& a, bool ck, int rg, int grid, cudaStream_t st);
int group_occupancy_local(int ops, bool ck, int p, int rg);
const void* group_ptr_local(int ops, bool ck, int rg);

}  // namespace qbx

namespace qbx {

// ---- adjoint (transposed sweep) -------------------------------------------
struct AdjArgs {
  int ops, p, nrhs;
  double kre, kim;
  int n_ctr, n_tgt, n_src;
  const double *cx, *cy, *tx, *ty;
  const double *sx, *sy, *snx, *sny;
  const void* gc;        // [n_ctr][nrhs] gradient carried to each centre
  void* coef;            // [n_ctr][nslots][p+2] coefficient columns (workspace)
  double* cgeo;          // [n_ctr][3] target direction and 1/r (workspace)
  int nsplit, ctr_per_split;
  void* part;            // [nsplit][n_src][1][nrhs]
  const double* hk_tab;  // complex k: the amplitude table of this k's ray, or null
};
cudaError_t launch_adjoint_real(const AdjArgs& a, cudaStream_t st);
cudaError_t launch_adjoint_cplx(const AdjArgs& a, cudaStream_t st);
void host_plan_workspace(const qbx_plan* plan, void** ws, size_t* bytes, int* num_sms, int** status);
// The plan's amplitude table for complex k (made on st when k changes), or
// null for real k.
const double* host_plan_hk_table(qbx_plan* plan, qbx_c64 k, cudaStream_t st, cudaError_t* err);

}  // namespace qbx
