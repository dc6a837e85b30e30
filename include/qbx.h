/*
 * qbx.h -- C ABI of the GB300 (sm_103a) QBX library: quadrature by expansion
 * for 2D Helmholtz layer potentials, complex FP64.
 *
 * Method: Kloeckner, Barnett, Greengard, O'Neil, "Quadrature by Expansion: a
 * new method for the evaluation of layer potentials", arXiv:1207.4461.
 *
 * Problem statement (Sec. 3.3): a closed curve Gamma, counter-clockwise, split
 * into M panels; outward normal n = (gamma'_y, -gamma'_x)/|gamma'| (Sec. 3.2);
 * a density on Gamma; a wavenumber k with Im k >= 0 (Sec. 1); an expansion
 * order p.  Return, at the panel nodes, the one-sided limit, the principal
 * value (jump subtraction) or the two-sided average of
 *   S sigma(x) = int G(x,x') sigma(x') dx'                    (Sec. 1, eq. kernelint)
 *   D mu(x)    = int dG/dn_{x'}(x,x') mu(x') dx'              (Sec. 1, eq. kernelintd)
 *   grad S sigma                                              (Sec. 3.2)
 * with G(x,x') = (i/4) H0^(1)(k|x-x'|)                        (Sec. 1, eq. helmholtz-ker),
 * and plain smooth quadrature at far (off-surface) targets.
 *
 * Conventions shared by every call:
 *  - Complex numbers are qbx_c64 {re, im}, interleaved FP64.
 *  - Unless stated "host", every pointer is a DEVICE pointer owned by the
 *    caller; the library never frees it.  Arrays are dense, row-major.
 *  - Density arrays have a right-hand-side axis: [n][nrhs].
 *  - Every compute call is asynchronous on `stream` (a cudaStream_t passed as
 *    void*, NULL = legacy default stream) and allocates nothing; only
 *    qbx_plan_create (its workspace), qbx_batch_create (the batch's arrays)
 *    and the GMRES solves (their Krylov bases, and for the assembled solve
 *    the product's split partial sums and one instantiated CUDA graph, freed
 *    before they return) allocate.
 *  - A plan is not thread-safe: calls on one plan from several host threads,
 *    or on several streams at once, must be serialised by the caller (they
 *    share the plan's workspace and its complex-k amplitude table).
 *  - Return value: QBX_OK or an error code; qbx_last_error() gives a
 *    thread-local message.  Argument errors are detected on the host before
 *    anything is launched.  Device-side conditions (non-finite values in the
 *    result) are recorded in a status word that qbx_sync_status() returns.
 *  - Grids: target nodes are the q_tgt-point Gauss-Legendre nodes of every
 *    panel (n_tgt = M q_tgt, the Nystrom unknowns); source nodes the
 *    q_src-point nodes of the same panels (n_src = M q_src), the oversampled
 *    grid of Sec. 3.4.2.
 *  - Centres: index j in [0, n_tgt) is the interior centre of target j,
 *    index n_tgt + j its exterior centre (Sec. 3.3 step 4a).
 *  - Phase convention of the coefficients:
 *      alpha_l = (i/4) sum_s w_s sigma_s H_l(k rho_s) e^{-i l theta_s},
 *      u(x)    = sum_{l=-p..p} alpha_l J_l(k rho) e^{+i l theta},
 *    i.e. the paper's eq. graf-coefficient / eq. local-exp with l -> -l
 *    (alpha^paper_{-l} = (-1)^l alpha_l); the potential is the same.
 */
#ifndef QBX_H
#define QBX_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } qbx_c64;

enum {
  QBX_OK = 0,
  QBX_EINVAL = 1,          /* bad argument (host check, nothing launched) */
  QBX_ECUDA = 2,           /* a CUDA runtime call failed */
  QBX_EINADMISSIBLE = 3,   /* reserved: strict admissibility (not raised by default) */
  QBX_ENONFINITE = 4,      /* a kernel produced a non-finite value */
  QBX_ENOCONV = 5,         /* reserved: iterative solve did not converge */
  QBX_ETIMEOUT = 6,        /* reserved: a bounded device wait ran out */
  QBX_ENOMEM = 7           /* workspace too small / allocation failed */
};

/* Operators: S sigma, D mu, grad S sigma (Sec. 1, Sec. 3.2), R sigma =
 * integral of t(x') . grad_{x'} G(x, x') sigma(x') ds (the tangential
 * dipole, Sec. 3.2 eq. riesz-def: continuous across the curve since
 * n . t = 0), and grad D mu, the target gradient of the double layer
 * (Sec. 3.2, eq. dlpderiv: PV = lim -/+ t dmu/ds / 2, + exterior), output
 * [n_tgt][2][nrhs] like grad S.  R is accepted by qbx_apply and qbx_far;
 * grad D by qbx_apply on the surface only (coefficients formed unfused,
 * a4 + a6); neither by qbx_apply_ops, the batch, the adjoints or
 * qbx_apply_static. */
enum { QBX_OP_S = 0, QBX_OP_D = 1, QBX_OP_GRAD_S = 2, QBX_OP_R = 3, QBX_OP_GRAD_D = 4 };
enum { QBX_SIDE_INT = 0, QBX_SIDE_EXT = 1, QBX_SIDE_TWO = 2 };
enum { QBX_LIMIT_ONE_SIDED = 0, QBX_LIMIT_PV = 1 };
enum { QBX_VALUE = 0, QBX_GRAD = 1 };

/* Largest supported expansion order and right-hand-side count per launch. */
#define QBX_MAX_P 40
#define QBX_MAX_Q 128

typedef struct qbx_plan qbx_plan;

/* Discretised curve.  All pointers are caller-owned device arrays of the
 * stated length; qbx_geometry fills them. */
typedef struct {
  int M, q_tgt, q_src;       /* panels, target and source nodes per panel */
  int n_tgt, n_src;          /* M*q_tgt, M*q_src */
  double *src_x, *src_y, *src_nx, *src_ny, *src_w;   /* [n_src] */
  double *tgt_x, *tgt_y, *tgt_nx, *tgt_ny, *tgt_w;   /* [n_tgt] */
  double *panel_h;                                  /* [M] panel arc length */
  double *ctr_x, *ctr_y, *ctr_r, *ctr_ratio;        /* [2*n_tgt] centres */
} qbx_geom;

/* Thread-local message describing the last error of the calling thread. */
const char *qbx_last_error(void);

/* Library ABI version (increments on incompatible changes). */
int qbx_version(void);

/* host.  q-node Gauss-Legendre rule on [-1,1] (the base smooth rule
 * of Sec. 3.1 / Sec. 4.1).  nodes, weights: host arrays of length q,
 * nodes ascending.  1 <= q <= QBX_MAX_Q, else QBX_EINVAL. */
int qbx_gauss_legendre(int q, double *nodes, double *weights);

/* Create a plan on CUDA device `device` for the grid pair (q_tgt, q_src):
 * uploads the per-panel interpolation matrix from the target to the source
 * nodes (Sec. 3.4.2), a device status word, and allocates `workspace_bytes`
 * of device workspace used by the split-source reductions (see
 * qbx_workspace_bytes) and a 29 KB buffer for the H0/H1 amplitude table of
 * the ray z = k rho, which calls with a complex k fill (on their stream)
 * when k differs from the last one.  *plan receives the handle.  Host call,
 * synchronous. */
int qbx_plan_create(qbx_plan **plan, int device, int q_tgt, int q_src, size_t workspace_bytes);
int qbx_plan_destroy(qbx_plan *plan);

/* Kernel timing (no counterpart in the paper; for measurement).  With timing
 * on, every qbx_apply / qbx_apply_ops call on the plan records two CUDA
 * events on its stream around its pair-sum launches (the fused or group
 * kernel, without oversampling and finishing); qbx_plan_kernel_ms waits for
 * the second event and returns the elapsed milliseconds of the last call.
 * QBX_EINVAL if timing is off.  Host calls. */
int qbx_plan_set_timing(qbx_plan *plan, int on);
int qbx_plan_kernel_ms(qbx_plan *plan, float *ms);

/* Work decomposition of the plan's applies (no counterpart in the paper):
 * the source-split choice aims for at least `waves` waves of the kernel's
 * resident CTAs (1..64; 1 at plan creation), so that the block scheduler
 * can even out CTAs of unequal duration.  The near-only applies and the
 * applies of one rhs of one density take at least 4 whatever the setting
 * (one density at complex k: 8).
 * Host call. */
int qbx_plan_set_min_waves(qbx_plan *plan, int waves);

/* Workspace a call needs: for qbx_apply / qbx_far / qbx_form_locals with the
 * given sizes.  n_ctr = number of centres (or far targets) processed, ncoef =
 * coefficients per centre (1 for S/D values, 2 for grad S, 2p+1 for
 * form_locals).  Host, pure function. */
size_t qbx_workspace_bytes(int n_src, int n_ctr, int ncoef, int nrhs);

/* Read (and clear) the plan's device status word: QBX_OK or QBX_ENONFINITE.
 * Synchronises `stream`. */
int qbx_sync_status(qbx_plan *plan, void *stream);

/* Geometry and centres (Sec. 3.3 steps 3-4a; Sec. 4.1).
 * Inputs (device): t_edges [M+1] panel parameter edges; gam_tgt, dgam_tgt
 * [n_tgt][2] curve point gamma(t) and derivative gamma'(t) at the q_tgt GL
 * nodes of each panel (t = (t_m + t_{m+1})/2 + (t_{m+1}-t_m)/2 xi_i, xi from
 * qbx_gauss_legendre); gam_src, dgam_src [n_src][2] likewise at the q_src
 * nodes.  g->M, q_tgt, q_src must be set (q's equal to the plan's) and all
 * output pointers valid.  Outputs: normals n = (gamma'_y,-gamma'_x)/|gamma'|,
 * weights w = w^GL (t_{m+1}-t_m)/2 |gamma'|, panel_h[m] = sum of the panel's
 * source weights, centres c = x -/+ r n with r = r_factor * panel_h (0.5 in the
 * paper, Sec. 3.3 step 3), and ctr_ratio = min_s |x_s - c| / r (>= 1 means
 * eq. x-c-closest holds for every source node).  Sets g->n_tgt, g->n_src. */
int qbx_geometry(qbx_plan *plan, qbx_geom *g, const double *t_edges,
                 const double *gam_tgt, const double *dgam_tgt,
                 const double *gam_src, const double *dgam_src,
                 double r_factor, void *stream);

/* qbx_geometry with a choice of expansion radius: QBX_RADIUS_H gives
 * r = r_factor * panel_h (as qbx_geometry), QBX_RADIUS_SQRT_H gives
 * r = r_factor * sqrt(panel_h): r refined more slowly than h, which makes
 * QBX classically convergent without source oversampling (the remarks after
 * eq. error_anal, Sec. 3.1).  QBX_RADIUS_ADMISSIBLE starts from
 * r = r_factor * panel_h and lowers each centre's radius to the largest one
 * whose disk holds no source node (|x_s - c| >= r for every s; closed form
 * r <= |d|^2 / (2 |d.n|) per source, d = x_s - x, on the centre's side of
 * the tangent): a departure from Sec. 3.3 step 4a for corners of 90 degrees
 * or less, where the r = h/2 centres of the targets next to the corner lie
 * on the opposite arm whatever the refinement; the radius then varies within
 * a panel (ctr_r holds it per centre).  QBX_EINVAL for another rule. */
enum { QBX_RADIUS_H = 0, QBX_RADIUS_SQRT_H = 1, QBX_RADIUS_ADMISSIBLE = 2 };
int qbx_geometry_rule(qbx_plan *plan, qbx_geom *g, const double *t_edges,
                      const double *gam_tgt, const double *dgam_tgt,
                      const double *gam_src, const double *dgam_src,
                      int rule, double r_factor, void *stream);

/* Source oversampling (Sec. 3.4.2): per panel, polynomial interpolation of
 * dens_tgt [n_tgt][nrhs] from the target to the source nodes, times the source
 * weight: wdens_src [n_src][nrhs] = w_s sigma(x_s). */
int qbx_upsample(qbx_plan *plan, const qbx_geom *g, const qbx_c64 *dens_tgt, int nrhs,
                 qbx_c64 *wdens_src, void *stream);

/* Expansion coefficients (Sec. 3.3 step 4b):
 *   kind QBX_OP_S: alpha_l   = (i/4) sum_s wdens_s H_l(k rho_s) e^{-i l theta_s}
 *                  (Sec. 2, eq. graf-coefficient)
 *   kind QBX_OP_D: alpha^D_l = (i/4) sum_s wdens_s n_s . grad_{x_s}[H_l(k rho_s) e^{-i l theta_s}]
 *                  (Sec. 3.2, eq. graf-coefficient-dlp)
 * for the centres of `side` (INT: n_tgt centres, EXT: n_tgt, TWO: 2 n_tgt,
 * interior first).  wdens_src [n_src][nrhs] (e.g. from qbx_upsample).
 * alpha: [n_ctr][2p+1][nrhs], index l+p.  0 <= p <= QBX_MAX_P.
 * Needs qbx_workspace_bytes(n_src, n_ctr, 2p+1, nrhs) of workspace. */
int qbx_form_locals(qbx_plan *plan, const qbx_geom *g, int kind, int side, qbx_c64 k, int p,
                    const qbx_c64 *wdens_src, int nrhs, qbx_c64 *alpha, void *stream);

/* Evaluate local expansions (Sec. 2 eq. local-exp; Sec. 3.3 step 4c) and,
 * with what = QBX_GRAD, their target gradient (Sec. 3.2).  alpha as produced
 * by qbx_form_locals for `side`.  If n_eval == 0, every centre of `side` is
 * evaluated at its own on-surface target (n_eval becomes the centre count);
 * otherwise target e at (ex[e], ey[e]) uses centre ectr[e] (index within the
 * side's centres, 0-based).  out: [n_eval][nrhs] (VALUE) or [n_eval][2][nrhs]
 * (GRAD: d/dx then d/dy).  J_l(k rho) by Miller's backward recurrence. */
int qbx_eval_locals(qbx_plan *plan, const qbx_geom *g, int side, qbx_c64 k, int p,
                    const qbx_c64 *alpha, int nrhs, int what,
                    int n_eval, const double *ex, const double *ey, const int *ectr,
                    qbx_c64 *out, void *stream);

/* The on-surface operator apply (Sec. 3.3 in full), storage-free: alpha is
 * never materialised (Sec. 3.3, remark on saving storage; Sec. 2 eq.
 * qbx-kernel G_p).  dens_tgt [n_tgt][nrhs] is the density on the target grid;
 * it is oversampled inside.  op: S, D or grad S.  side INT / EXT gives the
 * one-sided limit (limit = ONE_SIDED) or the principal value by jump
 * subtraction (limit = PV; Sec. 3.2: D: PV = lim -/+ mu/2, grad S:
 * PV = lim +/- n sigma/2, + = exterior); side TWO gives the two-sided average
 * (Sec. 3.2, eq. dlp-twosided; `limit` ignored).  out_on: [n_tgt][nrhs], or
 * [n_tgt][2][nrhs] for grad S.  If n_far > 0, x_far [n_far][2] are off-surface
 * targets evaluated by plain quadrature into out_far (same layout); the caller
 * places them outside every expansion disk (see qbx_assign_centres).
 * Needs qbx_workspace_bytes(n_src, max(n_ctr, n_far), ncomp, nrhs) of workspace
 * (ncomp = 2 for grad S, else 1); that figure includes the oversampled
 * densities. */
int qbx_apply(qbx_plan *plan, const qbx_geom *g, int op, int side, int limit, qbx_c64 k, int p,
              const qbx_c64 *dens_tgt, int nrhs, int n_far, const double *x_far,
              qbx_c64 *out_on, qbx_c64 *out_far, void *stream);

/* Several operators in one pass over the (centre, source) pairs: `ops` is a
 * non-empty subset of {S, D, grad S} as bits (1 << QBX_OP_S) | (1 << QBX_OP_D)
 * | (1 << QBX_OP_GRAD_S).  dens[op] / out[op] (host arrays of three device
 * pointers, entries of operators not in `ops` ignored) are the density and
 * output of each operator, with qbx_apply's layouts; densities may alias
 * (e.g. one density for all three).  The pair set-up (distance, H0, H1) and
 * the Hankel / Chebyshev recurrences are computed once per pair for all the
 * requested operators, which is why this is faster than separate qbx_apply
 * calls.  side / limit as in qbx_apply; no far targets.  Needs
 * qbx_workspace_bytes(n_src, n_ctr, ncomp, nrhs) with ncomp = 1 (S) + 1 (D)
 * + 2 (grad S) over the requested operators. */
#define QBX_OPS_S (1 << QBX_OP_S)
#define QBX_OPS_D (1 << QBX_OP_D)
#define QBX_OPS_GRAD_S (1 << QBX_OP_GRAD_S)
int qbx_apply_ops(qbx_plan *plan, const qbx_geom *g, int ops, int side, int limit, qbx_c64 k, int p,
                  const qbx_c64 *const dens[3], int nrhs, qbx_c64 *const out[3], void *stream);

/* The combined-field operator of the exterior Dirichlet problem without its
 * identity term (Sec. 4.2, the integral equation (1/2 I + D - i eta S) mu =
 * f): out = (D - i eta S) mu, both operators as two-sided QBX averages
 * (qbx_apply_ops with side QBX_SIDE_TWO and dens[S] = dens[D] = mu, then
 * out[D] - i eta out[S]), with the two kernel values of each (centre, source)
 * pair combined before they multiply the right-hand sides: one complex
 * multiply-add per pair and rhs instead of two.  dens, out: [n_tgt][nrhs]
 * interleaved complex, device.  eta finite, else QBX_EINVAL.  Needs
 * qbx_workspace_bytes(n_src, n_ctr, 1, nrhs). */
int qbx_apply_cfie(qbx_plan *plan, const qbx_geom *g, qbx_c64 k, qbx_c64 eta, int p, const qbx_c64 *dens,
                   int nrhs, qbx_c64 *out, void *stream);

/* Near-only QBX (the optimisation remarked in Sec. 5: direct evaluation for
 * distant interactions, QBX for near ones): as qbx_apply_ops, except that a
 * source node with |x_s - c| >= eta r_c goes through the smooth rule at the
 * centre's target (as qbx_far) instead of the expansion at c.  The result
 * differs from qbx_apply_ops by about eta^-(p+1) relative (QBX truncation of
 * the distant pairs); eta = 8 at p = 12 agrees to ~1e-13.  eta > 0, else
 * QBX_EINVAL.  Kernels as qbx_apply_ops: the group kernel for >= 16 rhs of
 * one density (S, D, S + D or all three), the fused kernel otherwise. */
int qbx_apply_local(qbx_plan *plan, const qbx_geom *g, int ops, int side, int limit, qbx_c64 k, int p,
                    double eta, const qbx_c64 *const dens[3], int nrhs, qbx_c64 *const out[3], void *stream);

/* Plain smooth quadrature at off-surface points (Sec. 1, Sec. 2):
 * S = (i/4) sum wdens H0(kd), D = (ik/4) sum wdens H1(kd) (x-x_s).n_s/d,
 * grad S = -(ik/4) sum wdens H1(kd) (x-x_s)/d.  wdens_src [n_src][nrhs],
 * x_far [n_far][2], out [n_far][nrhs] or [n_far][2][nrhs]. */
int qbx_far(qbx_plan *plan, const qbx_geom *g, int op, qbx_c64 k, const qbx_c64 *wdens_src,
            int nrhs, int n_far, const double *x_far, qbx_c64 *out, void *stream);

/* Which centre serves each off-surface point (Sec. 2: inside a disk use its
 * expansion).  Among the centres of `side` with |x - c| <= r_c, the smallest
 * |x - c|/r_c, ties to the lowest index; -1 if no disk contains x.
 * xy [n][2]; out [n] (index within the side's centres). */
int qbx_assign_centres(qbx_plan *plan, const qbx_geom *g, int side, int n, const double *xy,
                       int *out, void *stream);

/* Adjoint of the on-surface apply with respect to the density (op S or D):
 * for u = qbx_apply(sigma) = A sigma, returns gdens = A^H gout, the
 * vector-Jacobian product that reverse-mode differentiation of a loss of u
 * needs (A = (i/4) K W P with kernel values K(c, x_s) of the truncated Graf
 * sum, source weights W and the per-panel interpolation P of Sec. 3.4.2, so
 * A^H = P^T W K^H (-i/4), plus the self-adjoint jump term of a PV).  The
 * transposed sweep runs over (source, centre) pairs and recomputes the
 * Hankel recurrences; nothing of the forward apply is stored.  gout, gdens:
 * [n_tgt][nrhs] device arrays; other arguments as qbx_apply.  Uses the plan's
 * workspace. */
int qbx_apply_adjoint(qbx_plan *plan, const qbx_geom *g, int op, int side, int limit, qbx_c64 k, int p,
                      const qbx_c64 *gout, int nrhs, qbx_c64 *gdens, void *stream);

/* Shape adjoint of the on-surface S apply: for u = S sigma at the targets
 * (side INT, EXT or TWO; S is continuous, so the limit does not enter) and
 * the real functional L = Re sum_{t,r} conj(gout[t][r]) u[t][r], the
 * gradient of L with respect to the curve samples that qbx_geometry
 * consumed: gamma and gamma' at the target nodes and at the source nodes
 * (every quantity of Sec. 3.3 step 4a -- normals, weights, panel lengths,
 * radii, centres -- is differentiated; the density stays fixed on the
 * target grid as a function of the curve parameter).  With torch's complex
 * convention gout = dL/dRe u + i dL/dIm u this is the vector-Jacobian
 * product of u.  Two sweeps recompute the Hankel recurrences (centres ->
 * sources for grad_x and grad_{x_s} of the Graf sum of eq. graf-addition,
 * sources -> centres for the transposed sums); nothing is stored from the
 * forward apply.
 *   dens_tgt, gout: [n_tgt][nrhs] complex device arrays;
 *   dgam_tgt [n_tgt][2], dgam_src [n_src][2]: the gamma' samples given to
 *     qbx_geometry (device);
 *   g_gam_tgt, g_dgam_tgt [n_tgt][2], g_gam_src, g_dgam_src [n_src][2]:
 *     device outputs, overwritten (summed over the right-hand sides).
 * The geometry must have r = r_factor * panel_h (qbx_geometry, or
 * QBX_RADIUS_H): the chain through the radius uses dr/dh = r/h.
 * Uses the plan's workspace (qbx_shape_adjoint_workspace_bytes); too small
 * a workspace gives QBX_ENOMEM, bad arguments QBX_EINVAL, nothing launched. */
int qbx_apply_shape_adjoint(qbx_plan *plan, const qbx_geom *g, int side, qbx_c64 k, int p,
                            const qbx_c64 *dens_tgt, const qbx_c64 *gout, int nrhs,
                            const double *dgam_tgt, const double *dgam_src, double *g_gam_tgt,
                            double *g_dgam_tgt, double *g_gam_src, double *g_dgam_src, void *stream);

/* The same gradient for the D apply, L = Re sum conj(gout) (D mu) (any
 * limit: the PV jump term does not depend on the curve), Sec. 3.2's double
 * layer n_s . grad_{x_s} G differentiated through the source positions (the
 * second source derivatives of the Graf sum), the source normals, the
 * weights and the centres.  Same arguments, layouts, workspace and errors as
 * qbx_apply_shape_adjoint (dens_tgt is mu). */
int qbx_apply_shape_adjoint_d(qbx_plan *plan, const qbx_geom *g, int side, qbx_c64 k, int p,
                              const qbx_c64 *dens_tgt, const qbx_c64 *gout, int nrhs,
                              const double *dgam_tgt, const double *dgam_src, double *g_gam_tgt,
                              double *g_dgam_tgt, double *g_gam_src, double *g_dgam_src, void *stream);

/* Workspace for qbx_apply_shape_adjoint and qbx_apply_shape_adjoint_d with up
 * to 64 splits of each sweep (any side).  Host, pure function; 0 on bad
 * arguments. */
size_t qbx_shape_adjoint_workspace_bytes(int M, int q_tgt, int q_src, int p, int nrhs);

/* Second-kind exterior Dirichlet (sound-soft) solve, Sec. 4.2 eq.
 * dirichlet-inteq with the exterior sign and the combined-field coupling
 * alpha = -i eta:  (1/2) mu + D mu - i eta S mu = f  on Gamma, D and S as
 * two-sided averages (Sec. 3.5: two-sided averaging gives a spectrum that
 * clusters at zero), unknowns scaled by sqrt(w) (Sec. 4.2), by restarted
 * GMRES(restart) for nrhs right-hand sides f [n_tgt][nrhs] at once (every
 * system its own Krylov space; one combined-field apply per iteration,
 * qbx_apply_cfie, serves all).
 * Arnoldi by classical Gram-Schmidt with re-orthogonalisation, the Givens
 * rotations, the residual estimates, the convergence test and the
 * back-substitution all run on the device; the host waits once per restart
 * cycle (and, matrix-free, once per iteration, each a full QBX apply).  mu [n_tgt][nrhs]: initial guess in,
 * solution out.  Stops when every relative residual ||f - A mu||/||f|| (in
 * the sqrt-weighted norm, GMRES estimate) is below tol, or after maxiter
 * matvecs (QBX_ENOCONV).  iters (host, may be NULL) receives the matvec
 * count, resid (host [nrhs], may be NULL) the final relative residuals.
 * Allocates its Krylov basis ((restart+1) n_tgt nrhs complex) for the
 * duration of the call; synchronous. */
int qbx_solve_exterior_dirichlet(qbx_plan *plan, const qbx_geom *g, qbx_c64 k, qbx_c64 eta, int p,
                                 const qbx_c64 *f, int nrhs, double tol, int restart, int maxiter,
                                 qbx_c64 *mu, int *iters, double *resid, void *stream);

/* Vector kernels of the solve, also usable on their own.  Vectors are
 * [n][nrhs] complex device arrays; bases [nv][n][nrhs].
 *   qbx_vec_scale_sqrtw: out = in * sqrt(w) (inverse = 0) or in / sqrt(w).
 *   qbx_cfie_combine: y = sqrt(w) (xden/2 + dmu - i eta smu); smu may be NULL,
 *     dmu then holding (D - i eta S) mu (qbx_apply_cfie).
 *   qbx_vec_dots: out[j][r] = sum_i conj(V_j[i][r]) w[i][r], j < nv <= 65535
 *     (fixed reduction order); work needs qbx_vec_dots_work_bytes(nrhs, nv) bytes.
 *   qbx_vec_orth_update: w -= sum_j V_j h[j][r].
 *   qbx_vec_scale_cols: out[i][r] = a[r] in[i][r] (a: device [nrhs] real).
 *   qbx_vec_combine: x += sum_j V_j y[j][r]. */
int qbx_vec_scale_sqrtw(int n, int nrhs, const double *w, const qbx_c64 *in, qbx_c64 *out, int inverse,
                        void *stream);
int qbx_cfie_combine(int n, int nrhs, const double *w, const qbx_c64 *xden, const qbx_c64 *dmu,
                     const qbx_c64 *smu, qbx_c64 eta, qbx_c64 *y, void *stream);
int qbx_vec_dots(int n, int nrhs, int nv, const qbx_c64 *V, const qbx_c64 *w, qbx_c64 *work, qbx_c64 *out,
                 void *stream);
size_t qbx_vec_dots_work_bytes(int nrhs, int nv);
int qbx_vec_orth_update(int n, int nrhs, int nv, const qbx_c64 *V, const qbx_c64 *h, qbx_c64 *w, void *stream);
int qbx_vec_scale_cols(int n, int nrhs, const double *a, const qbx_c64 *in, qbx_c64 *out, void *stream);
int qbx_vec_combine(int n, int nrhs, int nv, const qbx_c64 *V, const qbx_c64 *y, qbx_c64 *x, void *stream);

/* The assembled Nystrom matrix of the same combined-field operator (Sec. 4.2;
 * Sec. 3.3 notes the discrete operator may be stored as a matrix): A~ =
 * W^{1/2} (1/2 I + D - i eta S) W^{-1/2} with D and S the two-sided
 * averages and W the target weights, n_tgt x n_tgt complex, written
 * column-major into A (entry (t, t') at A[t' n_tgt + t]; 16 n_tgt^2 bytes,
 * caller-owned device memory).  Row t holds, for both centres of target t,
 * the truncated Graf sums against every source node carried back to the
 * target grid by the per-panel interpolation.  q_tgt <= 16.  Async on
 * stream.  qbx_solve_exterior_dirichlet_assembled then runs the same GMRES
 * with one complex matrix product (qbx_matmul_cm) per iteration for all
 * right-hand sides, one Arnoldi step captured as a CUDA graph and launched
 * up to `restart` times per cycle without a host wait (steps after
 * convergence do nothing); k, eta and p are those the matrix was assembled
 * with. */
int qbx_assemble_cfie(qbx_plan *plan, const qbx_geom *g, qbx_c64 k, qbx_c64 eta, int p, qbx_c64 *A,
                      void *stream);
int qbx_solve_exterior_dirichlet_assembled(qbx_plan *plan, const qbx_geom *g, const qbx_c64 *A,
                                           const qbx_c64 *f, int nrhs, double tol, int restart, int maxiter,
                                           qbx_c64 *mu, int *iters, double *resid, void *stream);

/* y = A x for a column-major n x n complex matrix A (entry (i, j) at
 * A[j n + i]; the layout qbx_assemble_cfie writes) and nrhs vectors x, y
 * [n][nrhs] (device, caller-owned; y must not overlap A or x), in FP64 with
 * three real products per complex multiply-add (Re A Re x, Im A Im x and
 * (Re A + Im A)(Re x + Im x)).  The paper's Sec. 3.3 notes that the discrete
 * operator may be stored; this applies it.  work: device array of at least
 * qbx_matmul_cm_work_bytes(n, nrhs) bytes (split partial sums, added in a
 * fixed order: the result does not depend on timing).  Async on stream;
 * QBX_EINVAL on bad sizes or NULL pointers, QBX_ENOMEM when work is too
 * small.  qbx_matmul_cm_work_bytes queries the current device (host call). */
int qbx_matmul_cm(int n, int nrhs, const qbx_c64 *A, const qbx_c64 *x, qbx_c64 *y, void *work,
                  size_t work_bytes, void *stream);
size_t qbx_matmul_cm_work_bytes(int n, int nrhs);

/* Batched apply: many curves, each with its own panels, wavenumber and nrhs
 * densities, in one persistent launch run as a CUDA graph (the paper's cost
 * remark, Sec. 5: the work is O(N N_t) per curve; many small curves would
 * under-fill the GPU one launch at a time).  Every curve uses the same order
 * p, operator set (S, D, S+D or S+D+grad S, as QBX_OPS_* bits), side and
 * limit, and the plan's (q_tgt, q_src); geoms[i] is curve i's geometry from
 * qbx_geometry, k[i] its wavenumber (host arrays).  dens[i] (host array of
 * device pointers, [n_tgt_i][nrhs]) and out[3*i + op] (device pointers in
 * qbx_apply's layout, NULL for operators not requested) are bound at
 * creation: every qbx_batch_apply reads the current contents of dens and
 * writes out.  Work items are 32 centres of one curve against one range of
 * at most `chunk` of its sources (equal ranges per curve; the ranges' partial
 * sums are added in a fixed order), taken longest first by persistent CTAs
 * through an atomic counter; no CTA ever waits for another.
 * qbx_batch_create allocates the batch's device memory (with, for every
 * curve of complex k, the H0/H1 amplitude table of its ray z = k rho), picks
 * the chunk with the smallest predicted makespan of that schedule (a model
 * of the persistent grid), and builds and instantiates the graph
 * (synchronous); qbx_batch_apply launches the graph on `stream`. */
typedef struct qbx_batch qbx_batch;
int qbx_batch_create(qbx_batch **batch, qbx_plan *plan, int n_inst, const qbx_geom *geoms,
                     const qbx_c64 *k, int p, int ops, int side, int limit, int nrhs,
                     const qbx_c64 *const *dens, qbx_c64 *const *out);
int qbx_batch_apply(qbx_batch *batch, void *stream);
/* Read (and clear) the batch's device status word, as qbx_sync_status. */
int qbx_batch_status(qbx_batch *batch, void *stream);
/* Autotuner (no counterpart in the paper): times the whole batch (one untimed
 * and one timed graph launch on `stream`) for the model's chunk, half and
 * twice it, and for the applicable rhs groupings per warp (2 or 8), then
 * rebuilds the batch with the fastest; *rg, *chunk (may be NULL) receive the
 * choice.  Writes the outputs as an apply does.  Host call, synchronous.
 * The choice is cached in the process per (device, p, operators, side,
 * nrhs, real/complex k, and power-of-two buckets of the largest curve's
 * sources, the total pairs and the curve count); qbx_batch_create starts
 * from a cached choice when one matches. */
int qbx_batch_tune(qbx_batch *batch, void *stream, int *rg, int *chunk);
/* Near-only QBX for the whole batch (as qbx_apply_local, Sec. 5 remark):
 * eta > 0 sends every source node with |x_s - c| >= eta r_c through the
 * smooth rule at the centre's target instead of the expansion; eta = 0
 * restores the global apply.  Rebuilds the batch's graph with its current
 * configuration (host call, synchronous); eta < 0 or not finite:
 * QBX_EINVAL.  qbx_batch_tune measures the mode that is set. */
int qbx_batch_set_eta(qbx_batch *batch, double eta);
/* The batch's current configuration: rhs per warp group, sources per item,
 * work items, persistent CTAs.  Host, no device work. */
int qbx_batch_info(const qbx_batch *batch, int *rg, int *chunk, int *n_items, int *grid);
int qbx_batch_destroy(qbx_batch *batch);

/* qbx_apply without a plan, for callers that cannot allocate device memory.
 * The paper has no counterpart; this is a deployment variant of qbx_apply.
 *
 * Who needs it: qbx_apply works in a plan's workspace, and qbx_plan_create
 * calls cudaMalloc.  Code whose device memory belongs to a pooling allocator
 * cannot make raw allocations behind the pool (they fail once the pool holds
 * the memory), and latency-critical loops cannot afford cudaMalloc's implicit
 * device synchronisation.  This call allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine.
 *
 * Arguments and results are those of qbx_apply's on-surface part (no far
 * targets): same operators, sides, limits, layouts and device pointers owned
 * by the caller, asynchronous on `stream`.  The scratch (the oversampled
 * density and the per-split partial sums) is a fixed device array of
 * QBX_STATIC_SCRATCH_BYTES (32 MiB) that every GPU loading this library holds
 * until the process exits; calls whose sizes need more,
 * 16 B * (n_src*nrhs rounded up to 256 B + n_ctr*ncomp*nrhs) with
 * ncomp = 2 for grad S, fail with QBX_ENOMEM and a message naming the limit.
 *
 * The first call on each device (the current device) looks up the device
 * addresses of the fixed arrays and clears a status word on `stream`.  A call
 * whose (q_tgt, q_src) pair differs from the previous call's on that device
 * drains `stream` (cudaStreamSynchronize: earlier calls on it still read the
 * old matrix), uploads the pair's interpolation matrix on `stream` and drains
 * it again, so it returns only when the GPU has caught up.  A call with
 * Im k > 0 whose k differs from the previous complex k on that device
 * makes the amplitude table of k's ray in a fourth fixed array, on `stream`.
 * Make the first call, and any call that changes the grid pair, before a
 * stream capture.
 * Every call shares the one scratch array (and the matrix and the table),
 * which keeps the last call's contents: calls that overlap on the GPU
 * (several streams or threads on the same device) race and must be
 * serialised by the caller; calls in order on one stream do not.
 *
 * Device-side errors (a non-finite result) set the status word, which
 * qbx_apply_static_status reads. */
#define QBX_STATIC_SCRATCH_BYTES (32u << 20)
int qbx_apply_static(const qbx_geom *g, int op, int side, int limit, qbx_c64 k, int p,
                     const qbx_c64 *dens_tgt, int nrhs, qbx_c64 *out_on, void *stream);
/* The status word of qbx_apply_static on the current device: read and
 * cleared in the order of `stream` (after the calls queued on it), then
 * `stream` is synchronised.  QBX_ENONFINITE if a kernel of any call since the
 * last read produced a non-finite value, QBX_OK otherwise (also before the
 * first call on the device).  Allocates nothing. */
int qbx_apply_static_status(void *stream);

/* Diagnostics of the device special functions used by the kernels: H0, H1
 * at z[n] (complex, Im z >= 0, z != 0; the real-argument path is taken when
 * Im z == 0), and J_0..J_nmax (Miller) at z[n].  For tests. */
int qbx_debug_hankel01(const qbx_c64 *z, int n, qbx_c64 *h0, qbx_c64 *h1, void *stream);
int qbx_debug_besselj(const qbx_c64 *z, int n, int nmax, qbx_c64 *j, void *stream);
/* H0, H1 at z = k rho[i] (rho > 0, n values) as the pair kernels evaluate
 * them for this k: for Im k > 0 through the plan's amplitude table of the ray
 * z = k rho (fitted once per k) where |z| >= 2, the direct evaluation
 * otherwise; for real k the direct complex-argument evaluation.  For tests. */
int qbx_debug_hankel01_ray(qbx_plan *plan, qbx_c64 k, const double *rho, int n, qbx_c64 *h0, qbx_c64 *h1,
                           void *stream);

#ifdef __cplusplus
}
#endif
#endif /* QBX_H */
