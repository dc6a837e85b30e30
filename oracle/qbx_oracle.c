/*
 * qbx_oracle.c -- plain, slow, FP64 CPU oracle for quadrature by expansion
 * (QBX) applied to 2D Helmholtz layer potentials.
 *
 * TEST INFRASTRUCTURE ONLY.  The GPU library is checked against this file.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may build, load or call it.  It shares no code, header, table or constant
 * generator with the CUDA library, and it includes nothing from it.
 *
 * Method: Kloeckner, Barnett, Greengard, O'Neil, "Quadrature by Expansion: a
 * new method for the evaluation of layer potentials" (arXiv:1207.4461).
 *   Green's function       G(x,x') = (i/4) H0(k|x-x'|), Im k >= 0   (Sec. 1, eq. helmholtz-ker)
 *   layer potentials       S sigma, D mu                           (Sec. 1, eqs. kernelint, kernelintd)
 *   centres                c_j = x_j -/+ (h_m/2) n_j                (Sec. 3.3, step 4a)
 *   S coefficients         Graf's addition theorem                 (Sec. 2, eqs. graf-coefficient, graf-addition)
 *   D coefficients         normal derivative at the source         (Sec. 3.2, eq. graf-coefficient-dlp)
 *   evaluation             local (Bessel) expansion                (Sec. 2, eq. local-exp; Sec. 3.3 step 4c)
 *   target gradient        derivative of the local expansion       (Sec. 3.2)
 *   R (tangential dipole)  t_s . grad_{x_s} G, no jump             (Sec. 3.2, eq. riesz-def)
 *   grad D                 target gradient of the D expansion, jump
 *                          -/+ t dsigma/ds / 2                      (Sec. 3.2, eq. dlpderiv)
 *   jumps / PV / averaging                                          (Sec. 3.2, eqs. dlpjump, dlp-twosided)
 *   source oversampling    interpolate density to a finer grid      (Sec. 3.4.2)
 *   far targets            plain smooth quadrature                 (Sec. 1, Sec. 2)
 *
 * Phase convention (a reading of Sec. 2, eqs. graf-coefficient / local-exp):
 *   alpha_l = (i/4) sum_s w_s sigma_s H_l(k rho_s) e^{-i l theta_s},
 *   u(x)    = sum_{l=-p..p} alpha_l J_l(k rho) e^{+i l theta},
 * where (rho_s, theta_s), (rho, theta) are polar coordinates of x_s - c and
 * x - c.  The paper writes the same sum with l -> -l; since
 * H_{-l} = (-1)^l H_l and J_{-l} = (-1)^l J_l, alpha^paper_{-l} = (-1)^l alpha_l
 * and the potential is identical.
 *
 * Sums over sources run in source-index order.  OpenMP parallelises over
 * centres / targets only, so results are bitwise independent of the number
 * of threads.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORC_PI 3.14159265358979323846264338327950288
#define ORC_EULER_GAMMA 0.57721566490153286060651209008240243

enum { OP_S = 0, OP_D = 1, OP_GRAD_S = 2, OP_R = 3, OP_GRAD_D = 4 };
enum { SIDE_INT = 0, SIDE_EXT = 1, SIDE_TWO = 2 };
enum { LIMIT_ONE_SIDED = 0, LIMIT_PV = 1 };
enum { WHAT_VALUE = 0, WHAT_GRAD = 1 };

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre rule on [-1,1]: Newton's method on P_q, evaluated by the    */
/* three-term recurrence (n+1)P_{n+1} = (2n+1) x P_n - n P_{n-1}.             */
/* Starting guess cos(pi (i - 1/4)/(q + 1/2)).  Nodes ascending.              */
/* w_i = 2 / ((1 - x_i^2) P_q'(x_i)^2).                                       */
/* ------------------------------------------------------------------------- */
static void legendre_eval(int q, double x, double *pq, double *dpq)
{
    double p0 = 1.0, p1 = x;
    if (q == 0) { *pq = 1.0; *dpq = 0.0; return; }
    for (int n = 1; n < q; ++n) {
        double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pq = p1;
    /* P_q'(x) = q (x P_q - P_{q-1}) / (x^2 - 1) */
    *dpq = q * (x * p1 - p0) / (x * x - 1.0);
}

int orc_gauss_legendre(int q, double *nodes, double *weights)
{
    if (q < 1) return 1;
    for (int i = 1; i <= q; ++i) {
        double x = cos(ORC_PI * (i - 0.25) / (q + 0.5));
        double pq, dpq;
        for (int it = 0; it < 100; ++it) {
            legendre_eval(q, x, &pq, &dpq);
            double dx = pq / dpq;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        legendre_eval(q, x, &pq, &dpq);
        /* i = 1 is the largest node; store ascending */
        nodes[q - i] = x;
        weights[q - i] = 2.0 / ((1.0 - x * x) * dpq * dpq);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Bessel and Hankel functions of the first kind, integer order, complex z   */
/* with Im z >= 0, z != 0.                                                     */
/*   |z| <  1e-3 : ascending series (DLMF 10.2.2, 10.8.1)                      */
/*   |z| <= 25   : J_n by Miller's backward recurrence, normalised with        */
/*                 J_0 + 2 sum_k J_2k = 1 (generating function, DLMF 10.12.4   */
/*                 at t = 1); Y_0, Y_1 by Neumann series (DLMF 10.23.?, A&S   */
/*                 9.1.88 and its derivative)                                  */
/*   |z| >  25   : Hankel's asymptotic expansion (DLMF 10.17.5), truncated     */
/*                 at the smallest term                                        */
/* ------------------------------------------------------------------------- */
#define ORC_MAXN 1024

/* digamma at positive integers: psi(1) = -gamma, psi(m+1) = psi(m) + 1/m */
static double psi_int(int m)
{
    double s = -ORC_EULER_GAMMA;
    for (int j = 1; j < m; ++j) s += 1.0 / j;
    return s;
}

static void jy01_series(cplx z, cplx *j0, cplx *j1, cplx *y0, cplx *y1)
{
    cplx t = -z * z / 4.0;
    cplx lg = clog(z / 2.0);
    cplx sj0 = 0, sj1 = 0, sy0 = 0, sy1 = 0;
    cplx tk = 1.0;             /* t^k */
    double fk = 1.0, fk1 = 1.0; /* k!, (k+1)! */
    for (int k = 0; k < 40; ++k) {
        if (k > 0) { fk *= k; fk1 *= (k + 1); }
        cplx a0 = tk / (fk * fk);
        cplx a1 = tk / (fk * fk1);
        sj0 += a0;
        sj1 += a1;
        sy0 += psi_int(k + 1) * a0;
        sy1 += (psi_int(k + 1) + psi_int(k + 2)) * a1;
        if (cabs(a0) < 1e-20 * cabs(sj0) && k > 2) break;
        tk *= t;
    }
    *j0 = sj0;
    *j1 = (z / 2.0) * sj1;
    *y0 = (2.0 / ORC_PI) * lg * (*j0) - (2.0 / ORC_PI) * sy0;
    *y1 = -(2.0 / ORC_PI) / z + (2.0 / ORC_PI) * lg * (*j1) - (z / (2.0 * ORC_PI)) * sy1;
}

/* Miller: fills f[0..N] with J_0..J_N(z), N = returned start index (even). */
static int miller_j(cplx z, int nmax, cplx *f)
{
    double az = cabs(z);
    int N = nmax + 2 * (int)ceil(az) + 30;
    if (N & 1) ++N;
    if (N > ORC_MAXN - 2) N = ORC_MAXN - 2;
    f[N + 1] = 0.0;
    f[N] = 1e-30;
    for (int n = N; n >= 1; --n) {
        f[n - 1] = (2.0 * n / z) * f[n] - f[n + 1];
        if (cabs(f[n - 1]) > 1e250) {           /* rescale to avoid overflow */
            for (int m = n - 1; m <= N + 1; ++m) f[m] *= 1e-250;
        }
    }
    cplx norm = f[0];
    for (int m = 2; m <= N; m += 2) norm += 2.0 * f[m];
    for (int m = 0; m <= N; ++m) f[m] /= norm;
    return N;
}

static void jy01_miller(cplx z, cplx *j0, cplx *j1, cplx *y0, cplx *y1)
{
    cplx f[ORC_MAXN];
    int N = miller_j(z, 2, f);
    cplx lg = clog(z / 2.0) + ORC_EULER_GAMMA;
    cplx s0 = 0, s1 = 0;
    for (int k = 1; 2 * k + 1 <= N; ++k) {
        double sg = (k & 1) ? -1.0 : 1.0;     /* (-1)^k */
        s0 += sg * f[2 * k] / (double)k;
        s1 += sg * (f[2 * k - 1] - f[2 * k + 1]) / (2.0 * k);
    }
    *j0 = f[0];
    *j1 = f[1];
    *y0 = (2.0 / ORC_PI) * lg * f[0] - (4.0 / ORC_PI) * s0;
    *y1 = -(2.0 / ORC_PI) * f[0] / z + (2.0 / ORC_PI) * lg * f[1] + (4.0 / ORC_PI) * s1;
}

/* DLMF 10.17.5: H_nu(z) ~ sqrt(2/(pi z)) e^{i w} sum_k i^k a_k(nu) / z^k,
 * w = z - nu pi/2 - pi/4, a_k(nu) = prod_{j=1..k} (4 nu^2 - (2j-1)^2) / (k! 8^k). */
static cplx hankel_asymptotic(cplx z, int nu)
{
    double mu = 4.0 * nu * nu;
    cplx sum = 1.0, term = 1.0;
    double prev = 1.0;
    for (int k = 1; k < 200; ++k) {
        double a = (mu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) / (8.0 * k);
        cplx next = term * (I * a / z);
        double mag = cabs(next);
        if (mag >= prev) break;                 /* smallest term reached */
        term = next;
        sum += term;
        prev = mag;
        if (mag < 1e-18 * cabs(sum)) break;
    }
    cplx w = z - nu * ORC_PI / 2.0 - ORC_PI / 4.0;
    return csqrt(2.0 / (ORC_PI * z)) * cexp(I * w) * sum;
}

void orc_hankel01(cplx z, cplx *h0, cplx *h1)
{
    double az = cabs(z);
    if (az > 25.0) {
        *h0 = hankel_asymptotic(z, 0);
        *h1 = hankel_asymptotic(z, 1);
        return;
    }
    cplx j0, j1, y0, y1;
    if (az < 1e-3) jy01_series(z, &j0, &j1, &y0, &y1);
    else jy01_miller(z, &j0, &j1, &y0, &y1);
    *h0 = j0 + I * y0;
    *h1 = j1 + I * y1;
}

/* H_0..H_n by the upward recurrence H_{l+1} = (2l/z) H_l - H_{l-1}. */
void orc_hankel_seq(cplx z, int n, cplx *h)
{
    cplx h0, h1;
    orc_hankel01(z, &h0, &h1);
    h[0] = h0;
    if (n >= 1) h[1] = h1;
    for (int l = 1; l < n; ++l) h[l + 1] = (2.0 * l / z) * h[l] - h[l - 1];
}

/* J_0..J_n: ascending series J_l = sum_m (-1)^m (z/2)^{2m+l} / (m! (m+l)!) for
 * |z| <= 4 (DLMF 10.2.2), otherwise Miller's algorithm. */
void orc_besselj_seq(cplx z, int n, cplx *j)
{
    if (cabs(z) <= 4.0) {
        cplx hz = z / 2.0, t = -hz * hz;
        cplx hzl = 1.0;      /* (z/2)^l / l! */
        for (int l = 0; l <= n; ++l) {
            if (l > 0) hzl *= hz / (double)l;
            cplx term = hzl, sum = hzl;
            for (int m = 1; m < 200; ++m) {
                term *= t / ((double)m * (double)(m + l));
                sum += term;
                if (cabs(term) < 1e-20 * cabs(sum)) break;
            }
            j[l] = sum;
        }
        return;
    }
    cplx f[ORC_MAXN];
    miller_j(z, n, f);
    for (int l = 0; l <= n; ++l) j[l] = f[l];
}

/* Convenience for testing: H0, H1 at an array of points. */
void orc_hankel01_array(int n, const double *zin, double *h0out, double *h1out)
{
    for (int i = 0; i < n; ++i) {
        cplx z = zin[2 * i] + I * zin[2 * i + 1];
        cplx a, b;
        orc_hankel01(z, &a, &b);
        h0out[2 * i] = creal(a); h0out[2 * i + 1] = cimag(a);
        h1out[2 * i] = creal(b); h1out[2 * i + 1] = cimag(b);
    }
}

void orc_hankel_seq_array(int n, const double *zin, int nmax, double *hout)
{
    cplx h[ORC_MAXN];
    for (int i = 0; i < n; ++i) {
        cplx z = zin[2 * i] + I * zin[2 * i + 1];
        orc_hankel_seq(z, nmax, h);
        for (int l = 0; l <= nmax; ++l) {
            hout[2 * (i * (nmax + 1) + l)] = creal(h[l]);
            hout[2 * (i * (nmax + 1) + l) + 1] = cimag(h[l]);
        }
    }
}

void orc_besselj_seq_array(int n, const double *zin, int nmax, double *jout)
{
    cplx j[ORC_MAXN];
    for (int i = 0; i < n; ++i) {
        cplx z = zin[2 * i] + I * zin[2 * i + 1];
        orc_besselj_seq(z, nmax, j);
        for (int l = 0; l <= nmax; ++l) {
            jout[2 * (i * (nmax + 1) + l)] = creal(j[l]);
            jout[2 * (i * (nmax + 1) + l) + 1] = cimag(j[l]);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Geometry (Sec. 3.3 algorithm outline; Sec. 4.1 discretisation).           */
/* Panel m spans [t_m, t_{m+1}] of the curve parameter.  The caller samples   */
/* gamma and gamma' at the q-node Gauss-Legendre points of every panel.       */
/*   n = (gamma'_y, -gamma'_x)/|gamma'|   outward for a counter-clockwise      */
/*        curve (Sec. 3.2: n = (t_2, -t_1))                                   */
/*   w = w^GL (t_{m+1}-t_m)/2 |gamma'|    arc-length quadrature weight         */
/*   h_m = sum of the panel's source weights (arc length of the panel)        */
/*   r_m = r_factor h_m (Sec. 3.3 step 3: r_m = h_m/2), or with rule 1         */
/*   r_m = r_factor sqrt(h_m): r refined more slowly than h, the classically    */
/*   convergent choice of the remarks after eq. error_anal (Sec. 3.1)           */
/*   c   = x - r_m n (interior side), x + r_m n (exterior side)  (step 4a)    */
/*   rule 2 (a departure from step 4a, for corners of 90 degrees or less):   */
/*   each centre's radius r_m is lowered to the largest r whose disk holds   */
/*   no source node, |x_s - c| >= r for all s.  With d = x_s - x, the        */
/*   interior condition |d + r n|^2 >= r^2 reads |d|^2 + 2 r (d.n) >= 0, a   */
/*   bound r <= |d|^2 / (-2 d.n) for every source with d.n < 0 (exterior:   */
/*   r <= |d|^2 / (2 d.n) where d.n > 0).                                    */
/*   ratio = min_s |x_s - c| / r_m  (Graf validity, eq. x-c-closest)          */
/* Centre arrays have length 2*n_tgt: interior centres first, then exterior.  */
/* ------------------------------------------------------------------------- */
int orc_geometry(int M, int q_tgt, int q_src, const double *t_edges,
                 const double *gam_tgt, const double *dgam_tgt,
                 const double *gam_src, const double *dgam_src,
                 double r_factor, int rule,
                 double *src_x, double *src_y, double *src_nx, double *src_ny, double *src_w,
                 double *tgt_x, double *tgt_y, double *tgt_nx, double *tgt_ny, double *tgt_w,
                 double *panel_h,
                 double *ctr_x, double *ctr_y, double *ctr_r, double *ctr_ratio)
{
    double xt[ORC_MAXN], wt[ORC_MAXN], xs[ORC_MAXN], ws[ORC_MAXN];
    if (q_tgt < 1 || q_src < 1 || q_tgt > ORC_MAXN || q_src > ORC_MAXN) return 1;
    orc_gauss_legendre(q_tgt, xt, wt);
    orc_gauss_legendre(q_src, xs, ws);
    int n_tgt = M * q_tgt, n_src = M * q_src;
    for (int m = 0; m < M; ++m) {
        double half = 0.5 * (t_edges[m + 1] - t_edges[m]);
        double h = 0.0;
        for (int j = 0; j < q_src; ++j) {
            int s = m * q_src + j;
            double dx = dgam_src[2 * s], dy = dgam_src[2 * s + 1];
            double sp = sqrt(dx * dx + dy * dy);
            src_x[s] = gam_src[2 * s];
            src_y[s] = gam_src[2 * s + 1];
            src_nx[s] = dy / sp;
            src_ny[s] = -dx / sp;
            src_w[s] = ws[j] * half * sp;
            h += src_w[s];
        }
        panel_h[m] = h;
        for (int i = 0; i < q_tgt; ++i) {
            int t = m * q_tgt + i;
            double dx = dgam_tgt[2 * t], dy = dgam_tgt[2 * t + 1];
            double sp = sqrt(dx * dx + dy * dy);
            tgt_x[t] = gam_tgt[2 * t];
            tgt_y[t] = gam_tgt[2 * t + 1];
            tgt_nx[t] = dy / sp;
            tgt_ny[t] = -dx / sp;
            tgt_w[t] = wt[i] * half * sp;
            double r = rule == 1 ? r_factor * sqrt(h) : r_factor * h;
            ctr_x[t] = tgt_x[t] - r * tgt_nx[t];
            ctr_y[t] = tgt_y[t] - r * tgt_ny[t];
            ctr_r[t] = r;
            ctr_x[n_tgt + t] = tgt_x[t] + r * tgt_nx[t];
            ctr_y[n_tgt + t] = tgt_y[t] + r * tgt_ny[t];
            ctr_r[n_tgt + t] = r;
        }
    }
    if (rule == 2) {
        #pragma omp parallel for schedule(static)
        for (int c = 0; c < 2 * n_tgt; ++c) {
            int t = c % n_tgt;
            double sg = c < n_tgt ? -1.0 : 1.0;      /* c = x + sg r n */
            double r = ctr_r[c];
            for (int s = 0; s < n_src; ++s) {
                double dx = src_x[s] - tgt_x[t], dy = src_y[s] - tgt_y[t];
                double a = sg * (dx * tgt_nx[t] + dy * tgt_ny[t]);   /* -d.n interior, d.n exterior */
                if (a > 0.0) {
                    double bound = (dx * dx + dy * dy) / (2.0 * a);
                    if (bound < r) r = bound;
                }
            }
            ctr_r[c] = r;
            ctr_x[c] = tgt_x[t] + sg * r * tgt_nx[t];
            ctr_y[c] = tgt_y[t] + sg * r * tgt_ny[t];
        }
    }
    #pragma omp parallel for schedule(static)
    for (int c = 0; c < 2 * n_tgt; ++c) {
        double best = INFINITY;
        for (int s = 0; s < n_src; ++s) {
            double d = hypot(src_x[s] - ctr_x[c], src_y[s] - ctr_y[c]);
            if (d < best) best = d;
        }
        ctr_ratio[c] = best / ctr_r[c];
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Source oversampling (Sec. 3.4.2): per panel, interpolate the density from  */
/* the q_tgt target nodes to the q_src source nodes with the barycentric      */
/* Lagrange formula (second form; Berrut & Trefethen, SIAM Review 2004), then */
/* multiply by the source weights: wdens_s = w_s sigma(x_s).                  */
/* Densities are [n][nrhs] complex, row-major.                                */
/* ------------------------------------------------------------------------- */
int orc_upsample(int M, int q_tgt, int q_src, int nrhs, const double *src_w,
                 const cplx *dens_tgt, cplx *wdens_src)
{
    double xt[ORC_MAXN], wt[ORC_MAXN], xs[ORC_MAXN], ws[ORC_MAXN], lam[ORC_MAXN];
    if (q_tgt < 1 || q_src < 1 || q_tgt > ORC_MAXN || q_src > ORC_MAXN) return 1;
    orc_gauss_legendre(q_tgt, xt, wt);
    orc_gauss_legendre(q_src, xs, ws);
    for (int i = 0; i < q_tgt; ++i) {
        double pr = 1.0;
        for (int k = 0; k < q_tgt; ++k) if (k != i) pr *= (xt[i] - xt[k]);
        lam[i] = 1.0 / pr;
    }
    for (int m = 0; m < M; ++m) {
        for (int j = 0; j < q_src; ++j) {
            int s = m * q_src + j;
            int exact = -1;
            for (int i = 0; i < q_tgt; ++i) if (xs[j] == xt[i]) exact = i;
            for (int r = 0; r < nrhs; ++r) {
                cplx val;
                if (exact >= 0) {
                    val = dens_tgt[(m * q_tgt + exact) * nrhs + r];
                } else {
                    cplx num = 0.0;
                    double den = 0.0;
                    for (int i = 0; i < q_tgt; ++i) {
                        double c = lam[i] / (xs[j] - xt[i]);
                        num += c * dens_tgt[(m * q_tgt + i) * nrhs + r];
                        den += c;
                    }
                    val = num / den;
                }
                wdens_src[s * nrhs + r] = src_w[s] * val;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Expansion coefficients (Sec. 3.3 step 4b), literal double loop.            */
/*   S: alpha_l   = (i/4) sum_s wdens_s H_l(k rho_s) e^{-i l theta_s}          */
/*      (Sec. 2, eq. graf-coefficient with l -> -l)                            */
/*   D: alpha^D_l = (i/4) sum_s wdens_s  n_s . grad_{x_s} [H_l(k rho_s) e^{-i l theta_s}] */
/*      (Sec. 3.2, eq. graf-coefficient-dlp).  With F_m(y) = H_m(k|y|) e^{i m arg y}, */
/*      H_l e^{-i l theta} = (-1)^l F_{-l}, and (DLMF 10.6.2 in polar form)     */
/*      n . grad F_m = (k/2) [ nu F_{m-1} - conj(nu) F_{m+1} ],  nu = n_x + i n_y. */
/*   R: the same with the unit tangent t = (-n_y, n_x) in place of n          */
/*      (Sec. 3.2, eq. riesz-def): nu = t_x + i t_y.                           */
/* alpha is [n_ctr][2p+1][nrhs], index l + p.                                  */
/* ------------------------------------------------------------------------- */
static cplx F_m(int m, const cplx *H, double theta)
{
    int am = m < 0 ? -m : m;
    cplx h = H[am];
    if (m < 0 && (am & 1)) h = -h;           /* H_{-m} = (-1)^m H_m */
    return h * cexp(I * (double)m * theta);
}

int orc_form_locals(int kind, int n_ctr, const double *ctr_x, const double *ctr_y,
                    int n_src, const double *src_x, const double *src_y,
                    const double *src_nx, const double *src_ny,
                    const cplx *wdens, int nrhs, double kre, double kim, int p,
                    cplx *alpha)
{
    cplx k = kre + I * kim;
    if (p < 0 || p + 2 >= ORC_MAXN) return 1;
    int nl = 2 * p + 1;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int c = 0; c < n_ctr; ++c) {
        cplx H[ORC_MAXN];
        cplx *a = alpha + (size_t)c * nl * nrhs;
        for (int i = 0; i < nl * nrhs; ++i) a[i] = 0.0;
        for (int s = 0; s < n_src; ++s) {
            double dx = src_x[s] - ctr_x[c], dy = src_y[s] - ctr_y[c];
            double rho = hypot(dx, dy);
            double theta = atan2(dy, dx);
            orc_hankel_seq(k * rho, p + 1, H);
            cplx nu = (kind == OP_R) ? -src_ny[s] + I * src_nx[s] : src_nx[s] + I * src_ny[s];
            for (int l = -p; l <= p; ++l) {
                cplx kern;
                if (kind == OP_D || kind == OP_R) {
                    double sg = (l & 1) ? -1.0 : 1.0;   /* (-1)^l */
                    kern = sg * (k / 2.0) * (nu * F_m(-l - 1, H, theta) - conj(nu) * F_m(-l + 1, H, theta));
                } else {
                    int al = l < 0 ? -l : l;
                    cplx hl = H[al];
                    if (l < 0 && (al & 1)) hl = -hl;
                    kern = hl * cexp(-I * (double)l * theta);
                }
                for (int r = 0; r < nrhs; ++r)
                    a[(l + p) * nrhs + r] += (I / 4.0) * wdens[(size_t)s * nrhs + r] * kern;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Evaluation of the local expansion (Sec. 2 eq. local-exp, Sec. 3.3 step 4c) */
/*   u = sum_{l=-p..p} alpha_l J_l(k rho) e^{i l theta}                        */
/* and its target gradient (Sec. 3.2: differentiate the expansion), through    */
/*   (d_x + i d_y)[J_l e^{i l th}] = -k J_{l+1} e^{i(l+1)th}                   */
/*   (d_x - i d_y)[J_l e^{i l th}] =  k J_{l-1} e^{i(l-1)th}   (DLMF 10.6.2)   */
/* so d_x u = (U+ + U-)/2, d_y u = (U+ - U-)/(2i).                             */
/* Target e is evaluated from centre ectr[e]; out is [n_eval][nrhs] (VALUE) or */
/* [n_eval][2][nrhs] (GRAD: d_x then d_y).                                     */
/* ------------------------------------------------------------------------- */
static cplx J_signed(int l, const cplx *J)
{
    int al = l < 0 ? -l : l;
    cplx j = J[al];
    if (l < 0 && (al & 1)) j = -j;           /* J_{-l} = (-1)^l J_l */
    return j;
}

int orc_eval_locals(int n_eval, const double *ex, const double *ey, const int *ectr,
                    const double *ctr_x, const double *ctr_y,
                    const cplx *alpha, int nrhs, double kre, double kim, int p,
                    int what, cplx *out)
{
    cplx k = kre + I * kim;
    int nl = 2 * p + 1;
    if (p < 0 || p + 2 >= ORC_MAXN) return 1;
    #pragma omp parallel for schedule(static)
    for (int e = 0; e < n_eval; ++e) {
        cplx J[ORC_MAXN];
        int c = ectr[e];
        double dx = ex[e] - ctr_x[c], dy = ey[e] - ctr_y[c];
        double rho = hypot(dx, dy), theta = atan2(dy, dx);
        orc_besselj_seq(k * rho, p + 1, J);
        const cplx *a = alpha + (size_t)c * nl * nrhs;
        for (int r = 0; r < nrhs; ++r) {
            if (what == WHAT_GRAD) {
                cplx up = 0.0, um = 0.0;
                for (int l = -p; l <= p; ++l) {
                    cplx al = a[(l + p) * nrhs + r];
                    up += al * (-k) * J_signed(l + 1, J) * cexp(I * (double)(l + 1) * theta);
                    um += al * k * J_signed(l - 1, J) * cexp(I * (double)(l - 1) * theta);
                }
                out[((size_t)e * 2 + 0) * nrhs + r] = (up + um) / 2.0;
                out[((size_t)e * 2 + 1) * nrhs + r] = (up - um) / (2.0 * I);
            } else {
                cplx u = 0.0;
                for (int l = -p; l <= p; ++l)
                    u += a[(l + p) * nrhs + r] * J_signed(l, J) * cexp(I * (double)l * theta);
                out[(size_t)e * nrhs + r] = u;
            }
        }
    }
    return 0;
}

/* d sigma/ds at target node t (panel m, node i): derivative of the panel's   */
/* degree q-1 interpolant at its own node, in barycentric form,               */
/*   p'(x_i) = sum_{j != i} (lam_j / lam_i) (sigma_j - sigma_i) / (x_i - x_j), */
/* lam_j = 1 / prod_{k != j} (x_j - x_k), divided by ds/dxi = w_t / w^GL_i.   */
static cplx dsigma_ds(int q, int t, int nrhs, int r, const cplx *dens, const double *tgt_w)
{
    double x[ORC_MAXN], w[ORC_MAXN], lam[ORC_MAXN];
    orc_gauss_legendre(q, x, w);
    for (int j = 0; j < q; ++j) {
        double pr = 1.0;
        for (int k = 0; k < q; ++k) if (k != j) pr *= (x[j] - x[k]);
        lam[j] = 1.0 / pr;
    }
    int m = t / q, i = t - m * q;
    const cplx *d = dens + (size_t)m * q * nrhs + r;
    cplx acc = 0.0;
    for (int j = 0; j < q; ++j)
        if (j != i) acc += (lam[j] / lam[i]) * (d[(size_t)j * nrhs] - d[(size_t)i * nrhs]) / (x[i] - x[j]);
    return acc * w[i] / tgt_w[t];
}

/* ------------------------------------------------------------------------- */
/* Full on-surface apply, Sec. 3.3: upsample, coefficients at every centre of  */
/* the requested side(s), evaluation at the centre's own target, and the jump */
/* step 5 (Sec. 3.2):                                                          */
/*   S:      continuous, no correction                                         */
/*   D:      PV = lim_{+-} D mu  -/+ mu/2            (eq. dlpjump)             */
/*   grad S: PV = lim_{+-} grad S sigma +/- n sigma/2                          */
/*   R:      continuous (the jump is (n . t) sigma / 2 = 0; Sec. 3.2)           */
/*   grad D: PV = lim_{+-} grad D mu -/+ t dmu/ds / 2  (eq. dlpderiv), with     */
/*           dmu/ds from the derivative of the panel's interpolant at the node  */
/*           (barycentric form, Berrut & Trefethen 2004, eq. 9.4) divided by    */
/*           ds/dxi = w / w^GL                                                  */
/*   two-sided: PV = (lim_+ + lim_-)/2                (eq. dlp-twosided)        */
/* (+ = exterior side, - = interior side).  Output [n_tgt][nrhs] for S and D,  */
/* [n_tgt][2][nrhs] for grad S.  If sel != NULL only the n_sel targets sel[i]  */
/* are computed and output row i belongs to target sel[i].                      */
/* ------------------------------------------------------------------------- */
int orc_apply(int op, int side, int limit, double kre, double kim, int p,
              int M, int q_tgt, int q_src,
              const double *src_x, const double *src_y, const double *src_nx,
              const double *src_ny, const double *src_w,
              const double *tgt_x, const double *tgt_y, const double *tgt_nx,
              const double *tgt_ny, const double *tgt_w,
              const double *ctr_x, const double *ctr_y,
              const cplx *dens_tgt, int nrhs, int n_sel, const int *sel, cplx *out)
{
    int n_tgt = M * q_tgt, n_src = M * q_src, nl = 2 * p + 1;
    int grad = (op == OP_GRAD_S || op == OP_GRAD_D);
    int ncomp = grad ? 2 : 1;
    if (n_sel <= 0 || !sel) n_sel = n_tgt, sel = NULL;
    cplx *wd = malloc(sizeof(cplx) * (size_t)n_src * nrhs);
    cplx *alpha = malloc(sizeof(cplx) * (size_t)n_sel * nl * nrhs);
    cplx *val = malloc(sizeof(cplx) * (size_t)n_sel * ncomp * nrhs);
    int *ectr = malloc(sizeof(int) * (size_t)n_sel);
    double *cx = malloc(sizeof(double) * (size_t)n_sel), *cy = malloc(sizeof(double) * (size_t)n_sel);
    double *ex = malloc(sizeof(double) * (size_t)n_sel), *ey = malloc(sizeof(double) * (size_t)n_sel);
    if (!wd || !alpha || !val || !ectr || !cx || !cy || !ex || !ey) {
        free(wd); free(alpha); free(val); free(ectr); free(cx); free(cy); free(ex); free(ey);
        return 2;
    }
    orc_upsample(M, q_tgt, q_src, nrhs, src_w, dens_tgt, wd);
    for (size_t i = 0; i < (size_t)n_sel * ncomp * nrhs; ++i) out[i] = 0.0;
    int s0 = (side == SIDE_TWO) ? SIDE_INT : side;
    int s1 = (side == SIDE_TWO) ? SIDE_EXT : side;
    for (int sd = s0; sd <= s1; ++sd) {
        for (int i = 0; i < n_sel; ++i) {
            int t = sel ? sel[i] : i;
            cx[i] = ctr_x[(size_t)sd * n_tgt + t];
            cy[i] = ctr_y[(size_t)sd * n_tgt + t];
            ex[i] = tgt_x[t];
            ey[i] = tgt_y[t];
            ectr[i] = i;
        }
        orc_form_locals(op == OP_GRAD_S ? OP_S : (op == OP_GRAD_D ? OP_D : op), n_sel, cx, cy, n_src, src_x, src_y,
                        src_nx, src_ny, wd, nrhs, kre, kim, p, alpha);
        orc_eval_locals(n_sel, ex, ey, ectr, cx, cy, alpha, nrhs, kre, kim, p,
                        grad ? WHAT_GRAD : WHAT_VALUE, val);
        double sgn = (sd == SIDE_EXT) ? 1.0 : -1.0;    /* +1 exterior, -1 interior */
        for (int i = 0; i < n_sel; ++i) {
            int t = sel ? sel[i] : i;
            for (int r = 0; r < nrhs; ++r) {
                cplx dens = dens_tgt[(size_t)t * nrhs + r];
                if (grad) {
                    cplx gx = val[((size_t)i * 2 + 0) * nrhs + r];
                    cplx gy = val[((size_t)i * 2 + 1) * nrhs + r];
                    if (side != SIDE_TWO && limit == LIMIT_PV && op == OP_GRAD_S) {
                        gx += sgn * 0.5 * tgt_nx[t] * dens;
                        gy += sgn * 0.5 * tgt_ny[t] * dens;
                    }
                    if (side != SIDE_TWO && limit == LIMIT_PV && op == OP_GRAD_D) {
                        cplx ds = dsigma_ds(q_tgt, t, nrhs, r, dens_tgt, tgt_w);
                        gx -= sgn * 0.5 * (-tgt_ny[t]) * ds;     /* tangent t = (-n_y, n_x) */
                        gy -= sgn * 0.5 * tgt_nx[t] * ds;
                    }
                    if (side == SIDE_TWO) { gx *= 0.5; gy *= 0.5; }
                    out[((size_t)i * 2 + 0) * nrhs + r] += gx;
                    out[((size_t)i * 2 + 1) * nrhs + r] += gy;
                } else {
                    cplx u = val[(size_t)i * nrhs + r];
                    if (op == OP_D && side != SIDE_TWO && limit == LIMIT_PV) u -= sgn * 0.5 * dens;
                    if (side == SIDE_TWO) u *= 0.5;
                    out[(size_t)i * nrhs + r] += u;
                }
            }
        }
    }
    free(wd); free(alpha); free(val); free(ectr); free(cx); free(cy); free(ex); free(ey);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Far targets: the plain smooth quadrature rule (Sec. 1; Sec. 2 "high-       */
/* accuracy region").  With d = |x - x_s|:                                     */
/*   S      = (i/4) sum_s wdens_s H0(k d)                                      */
/*   D      = (i/4) sum_s wdens_s n_s . grad_{x_s} H0(k|x - x_s|)              */
/*          = (i k/4) sum_s wdens_s H1(k d) ((x - x_s) . n_s) / d              */
/*   grad S = (i/4) sum_s wdens_s grad_x H0(k d) = -(i k/4) sum_s wdens_s H1(k d) (x - x_s)/d */
/*   R      = as D with the unit tangent t_s = (-n_y, n_x) in place of n_s      */
/* Output [n][nrhs] or [n][2][nrhs].                                           */
/* ------------------------------------------------------------------------- */
int orc_far(int op, int n_far, const double *xy, int n_src,
            const double *src_x, const double *src_y, const double *src_nx, const double *src_ny,
            const cplx *wdens, int nrhs, double kre, double kim, cplx *out)
{
    cplx k = kre + I * kim;
    #pragma omp parallel for schedule(static)
    for (int e = 0; e < n_far; ++e) {
        int ncomp = (op == OP_GRAD_S) ? 2 : 1;
        for (int i = 0; i < ncomp * nrhs; ++i) out[(size_t)e * ncomp * nrhs + i] = 0.0;
        for (int s = 0; s < n_src; ++s) {
            double rx = xy[2 * e] - src_x[s], ry = xy[2 * e + 1] - src_y[s];
            double d = hypot(rx, ry);
            cplx h0, h1;
            orc_hankel01(k * d, &h0, &h1);
            for (int r = 0; r < nrhs; ++r) {
                cplx wdv = wdens[(size_t)s * nrhs + r];
                if (op == OP_S) {
                    out[(size_t)e * nrhs + r] += (I / 4.0) * wdv * h0;
                } else if (op == OP_D) {
                    out[(size_t)e * nrhs + r] += (I * k / 4.0) * wdv * h1 * (rx * src_nx[s] + ry * src_ny[s]) / d;
                } else if (op == OP_R) {   /* t = (-n_y, n_x) in place of n */
                    out[(size_t)e * nrhs + r] += (I * k / 4.0) * wdv * h1 * (-rx * src_ny[s] + ry * src_nx[s]) / d;
                } else {
                    out[((size_t)e * 2 + 0) * nrhs + r] += -(I * k / 4.0) * wdv * h1 * rx / d;
                    out[((size_t)e * 2 + 1) * nrhs + r] += -(I * k / 4.0) * wdv * h1 * ry / d;
                }
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Which centre serves an off-surface point (Sec. 2: a point inside a disk    */
/* uses that disk's expansion; otherwise it is in the high-accuracy region of */
/* the smooth rule).  Reading: among centres [c0, c1) with |x - c| <= r_c,     */
/* pick the smallest |x - c|/r_c, ties to the lowest index; -1 if none.        */
/* ------------------------------------------------------------------------- */
int orc_assign_centres(int n, const double *xy, int c0, int c1,
                       const double *ctr_x, const double *ctr_y, const double *ctr_r,
                       int *out)
{
    #pragma omp parallel for schedule(static)
    for (int e = 0; e < n; ++e) {
        int best = -1;
        double bestq = INFINITY;
        for (int c = c0; c < c1; ++c) {
            double q = hypot(xy[2 * e] - ctr_x[c], xy[2 * e + 1] - ctr_y[c]) / ctr_r[c];
            if (q <= 1.0 && q < bestq) { bestq = q; best = c; }
        }
        out[e] = best;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Shape derivative of the on-surface S apply, forward mode (the reference    */
/* for the reverse-mode shape adjoint).  The curve samples gamma, gamma' at   */
/* the target and source nodes move along a direction (pg, pdg) (their        */
/* derivatives with respect to a scalar eps); every quantity of orc_geometry   */
/* follows by the chain rule, with tau = gamma'/|gamma'| and R v = (v_y, -v_x):*/
/*   x'   = pg                                                                 */
/*   n'   = (R pdg - n (tau . pdg)) / |gamma'|                                 */
/*   w'   = w^GL (t_{m+1} - t_m)/2 (tau . pdg),   h_m' = sum over the panel    */
/*   r'   = r_factor h_m',   c' = x' -/+ (r' n + r n')  (interior / exterior)  */
/* The density is held fixed on the target grid as a function of the curve   */
/* parameter, so (w sigma)_s' = w_s' (P sigma)_s (P: Sec. 3.4.2 interpolation).*/
/* The S coefficients and the evaluation (Sec. 2 eqs. graf-coefficient,        */
/* local-exp; Sec. 3.3 steps 4b-4c) are differentiated term by term:           */
/*   alpha_l' = (i/4) sum_s [ (w sigma)_s' H_l                                 */
/*              + (w sigma)_s (k H_l'(k rho_s) rho_s' - i l H_l theta_s') ] e^{-il theta_s} */
/*   u'       = sum_l [ alpha_l' J_l + alpha_l (k J_l'(k rho) rho' + i l J_l theta') ] e^{il theta} */
/* with rho' = (d . d')/rho, theta' = (d_x d'_y - d_y d'_x)/rho^2 for the      */
/* vector d = x_s - c (sources) or x - c (target), and for signed orders       */
/* Z_l' = (Z_{l-1} - Z_{l+1})/2, Z = H or J (DLMF 10.6.1).  S has no jump, so  */
/* the one-sided limit and the PV agree; side TWO averages the two centres.    */
/* ndir directions at once (pg_*, pdg_*: [ndir][n][2]).  u: [n_tgt][nrhs],     */
/* du: [ndir][n_tgt][nrhs].  Returns 0, 1 on bad sizes, 2 on allocation failure.*/
/* ------------------------------------------------------------------------- */
static cplx Z_signed(int l, const cplx *Z)
{
    int al = l < 0 ? -l : l;
    cplx z = Z[al];
    if (l < 0 && (al & 1)) z = -z;           /* Z_{-l} = (-1)^l Z_l */
    return z;
}

int orc_apply_s_tangent(int side, double kre, double kim, int p, int M, int q_tgt, int q_src,
                        const double *t_edges, double r_factor,
                        const double *gam_tgt, const double *dgam_tgt,
                        const double *gam_src, const double *dgam_src, int ndir,
                        const double *pg_tgt, const double *pdg_tgt,
                        const double *pg_src, const double *pdg_src,
                        const cplx *dens_tgt, int nrhs, cplx *u, cplx *du)
{
    if (p < 0 || p + 2 >= ORC_MAXN || q_tgt < 1 || q_src < 1 || q_tgt > ORC_MAXN || q_src > ORC_MAXN ||
        M < 1 || nrhs < 1 || ndir < 1)
        return 1;
    cplx k = kre + I * kim;
    int n_tgt = M * q_tgt, n_src = M * q_src, nl = 2 * p + 1;
    size_t nd_s = (size_t)n_src, nd_t = (size_t)n_tgt, nd = (size_t)ndir;
    double *buf = malloc(sizeof(double) * (7 * nd_s + 17 * nd_t + (size_t)M));
    double *dbuf = malloc(sizeof(double) * nd * (3 * nd_s + 4 * nd_t + (size_t)M));
    cplx *psig = malloc(sizeof(cplx) * nd_s * nrhs);
    cplx *wd = malloc(sizeof(cplx) * nd_s * nrhs);
    if (!buf || !dbuf || !psig || !wd) { free(buf); free(dbuf); free(psig); free(wd); return 2; }
    double *src_x = buf, *src_y = src_x + nd_s, *src_nx = src_y + nd_s, *src_ny = src_nx + nd_s;
    double *src_w = src_ny + nd_s, *ones = src_w + nd_s, *spare = ones + nd_s;
    double *tgt_x = spare + nd_s, *tgt_y = tgt_x + nd_t, *tgt_nx = tgt_y + nd_t, *tgt_ny = tgt_nx + nd_t;
    double *tgt_w = tgt_ny + nd_t;
    double *ctr_x = tgt_w + nd_t, *ctr_y = ctr_x + 2 * nd_t, *ctr_r = ctr_y + 2 * nd_t;
    double *ctr_ratio = ctr_r + 2 * nd_t, *spare2 = ctr_ratio + 2 * nd_t;
    double *panel_h = spare2 + 4 * nd_t;
    /* per direction: d_sx, d_sy, d_sw [n_src]; d_cx, d_cy [2 n_tgt]; d_h [M] */
    double *d_sx = dbuf, *d_sy = d_sx + nd * nd_s, *d_sw = d_sy + nd * nd_s;
    double *d_cx = d_sw + nd * nd_s, *d_cy = d_cx + nd * 2 * nd_t, *d_h = d_cy + nd * 2 * nd_t;
    (void)spare; (void)spare2;
    orc_geometry(M, q_tgt, q_src, t_edges, gam_tgt, dgam_tgt, gam_src, dgam_src, r_factor, 0,
                 src_x, src_y, src_nx, src_ny, src_w, tgt_x, tgt_y, tgt_nx, tgt_ny, tgt_w,
                 panel_h, ctr_x, ctr_y, ctr_r, ctr_ratio);
    double xs[ORC_MAXN], ws[ORC_MAXN];
    orc_gauss_legendre(q_src, xs, ws);
    for (int s = 0; s < n_src; ++s) ones[s] = 1.0;
    for (int d = 0; d < ndir; ++d) {
        const double *pgs = pg_src + (size_t)d * 2 * nd_s, *pdgs = pdg_src + (size_t)d * 2 * nd_s;
        const double *pgt = pg_tgt + (size_t)d * 2 * nd_t, *pdgt = pdg_tgt + (size_t)d * 2 * nd_t;
        double *dsx = d_sx + d * nd_s, *dsy = d_sy + d * nd_s, *dsw = d_sw + d * nd_s;
        double *dcx = d_cx + d * 2 * nd_t, *dcy = d_cy + d * 2 * nd_t, *dh = d_h + (size_t)d * M;
        /* tangents of the source nodes, weights and panel lengths */
        for (int m = 0; m < M; ++m) {
            double half = 0.5 * (t_edges[m + 1] - t_edges[m]), acc = 0.0;
            for (int j = 0; j < q_src; ++j) {
                int s = m * q_src + j;
                double vx = dgam_src[2 * s], vy = dgam_src[2 * s + 1];
                double sp = sqrt(vx * vx + vy * vy);
                double tp = (vx * pdgs[2 * s] + vy * pdgs[2 * s + 1]) / sp;   /* tau . pdg */
                dsw[s] = ws[j] * half * tp;
                acc += dsw[s];
                dsx[s] = pgs[2 * s];
                dsy[s] = pgs[2 * s + 1];
            }
            dh[m] = acc;
        }
        /* tangents of the centres */
        for (int t = 0; t < n_tgt; ++t) {
            int m = t / q_tgt;
            double vx = dgam_tgt[2 * t], vy = dgam_tgt[2 * t + 1];
            double sp = sqrt(vx * vx + vy * vy);
            double px = pdgt[2 * t], py = pdgt[2 * t + 1];
            double tp = (vx * px + vy * py) / sp;
            double dnx = (py - tgt_nx[t] * tp) / sp, dny = (-px - tgt_ny[t] * tp) / sp;
            double r = ctr_r[t], dr = r_factor * dh[m];
            double ox = dr * tgt_nx[t] + r * dnx, oy = dr * tgt_ny[t] + r * dny;
            dcx[t] = pgt[2 * t] - ox;
            dcy[t] = pgt[2 * t + 1] - oy;
            dcx[n_tgt + t] = pgt[2 * t] + ox;
            dcy[n_tgt + t] = pgt[2 * t + 1] + oy;
        }
    }
    orc_upsample(M, q_tgt, q_src, nrhs, ones, dens_tgt, psig);     /* P sigma */
    for (size_t i = 0; i < nd_s * nrhs; ++i) wd[i] = src_w[i / nrhs] * psig[i];
    for (size_t i = 0; i < nd_t * nrhs; ++i) u[i] = 0.0;
    for (size_t i = 0; i < nd * nd_t * nrhs; ++i) du[i] = 0.0;
    int s0 = (side == SIDE_TWO) ? SIDE_INT : side;
    int s1 = (side == SIDE_TWO) ? SIDE_EXT : side;
    double wgt = (side == SIDE_TWO) ? 0.5 : 1.0;
    int fail = 0;
    for (int sd = s0; sd <= s1; ++sd) {
        #pragma omp parallel for schedule(dynamic, 4)
        for (int t = 0; t < n_tgt; ++t) {
            cplx H[ORC_MAXN], J[ORC_MAXN];
            cplx *al = malloc(sizeof(cplx) * (1 + nd) * (size_t)nl * nrhs);
            if (!al) {
                #pragma omp atomic write
                fail = 1;
                continue;
            }
            cplx *dal = al + (size_t)nl * nrhs;             /* [ndir][nl][nrhs] */
            for (size_t i = 0; i < (1 + nd) * (size_t)nl * nrhs; ++i) al[i] = 0.0;
            int c = sd * n_tgt + t;
            double cx = ctr_x[c], cy = ctr_y[c];
            for (int s = 0; s < n_src; ++s) {
                double dx = src_x[s] - cx, dy = src_y[s] - cy;
                double rho = hypot(dx, dy), th = atan2(dy, dx);
                orc_hankel_seq(k * rho, p + 1, H);
                for (int l = -p; l <= p; ++l) {
                    cplx hl = Z_signed(l, H);
                    cplx hd = (Z_signed(l - 1, H) - Z_signed(l + 1, H)) / 2.0;
                    cplx e = cexp(-I * (double)l * th);
                    cplx kern = hl * e;
                    for (int r = 0; r < nrhs; ++r)
                        al[(size_t)(l + p) * nrhs + r] += (I / 4.0) * wd[(size_t)s * nrhs + r] * kern;
                    for (int d = 0; d < ndir; ++d) {
                        double ddx = d_sx[d * nd_s + s] - d_cx[d * 2 * nd_t + c];
                        double ddy = d_sy[d * nd_s + s] - d_cy[d * 2 * nd_t + c];
                        double drho = (dx * ddx + dy * ddy) / rho;
                        double dth = (dx * ddy - dy * ddx) / (rho * rho);
                        cplx dkern = (k * hd * drho - I * (double)l * hl * dth) * e;
                        for (int r = 0; r < nrhs; ++r) {
                            size_t sr = (size_t)s * nrhs + r;
                            cplx dwd = d_sw[d * nd_s + s] * psig[sr];
                            dal[((size_t)d * nl + (l + p)) * nrhs + r] += (I / 4.0) * (dwd * kern + wd[sr] * dkern);
                        }
                    }
                }
            }
            double ex = tgt_x[t] - cx, ey = tgt_y[t] - cy;
            double rt = hypot(ex, ey), tht = atan2(ey, ex);
            orc_besselj_seq(k * rt, p + 1, J);
            for (int l = -p; l <= p; ++l) {
                cplx jl = Z_signed(l, J);
                cplx jd = (Z_signed(l - 1, J) - Z_signed(l + 1, J)) / 2.0;
                cplx e = cexp(I * (double)l * tht);
                for (int r = 0; r < nrhs; ++r)
                    u[(size_t)t * nrhs + r] += wgt * al[(size_t)(l + p) * nrhs + r] * jl * e;
                for (int d = 0; d < ndir; ++d) {
                    const double *pgt = pg_tgt + (size_t)d * 2 * nd_t;
                    double dex = pgt[2 * t] - d_cx[d * 2 * nd_t + c], dey = pgt[2 * t + 1] - d_cy[d * 2 * nd_t + c];
                    double drt = (ex * dex + ey * dey) / rt;
                    double dtht = (ex * dey - ey * dex) / (rt * rt);
                    cplx dfac = (k * jd * drt + I * (double)l * jl * dtht) * e;
                    for (int r = 0; r < nrhs; ++r) {
                        cplx a = al[(size_t)(l + p) * nrhs + r], da = dal[((size_t)d * nl + (l + p)) * nrhs + r];
                        du[((size_t)d * nd_t + t) * nrhs + r] += wgt * (da * jl * e + a * dfac);
                    }
                }
            }
            free(al);
        }
    }
    free(buf); free(dbuf); free(psig); free(wd);
    return fail ? 2 : 0;
}

/* ------------------------------------------------------------------------- */
/* Shape derivative of the on-surface D apply, forward mode, as               */
/* orc_apply_s_tangent: the D coefficients of orc_form_locals,                */
/*   alpha^D_l = (i/4) sum_s wdens_s (-1)^l (k/2) [nu F_{-l-1} - conj(nu) F_{-l+1}], */
/* differentiated through the source position (rho, theta of x_s - c), the    */
/* source normal nu = n_x + i n_y (n = (gamma'_y, -gamma'_x)/|gamma'|), the   */
/* weight and the centre, with dF_m = (k H_m' drho + i m H_m dtheta) e^{i m theta}, */
/* H_m' = (H_{m-1} - H_{m+1})/2; then the evaluation as for S.  The PV jump   */
/* -+ mu/2 (limit PV, one side) does not move with the curve.                 */
/* ------------------------------------------------------------------------- */
static cplx dF_m(int m, const cplx *H, double theta, cplx k, double drho, double dth)
{
    cplx hm = Z_signed(m, H);
    cplx hd = (Z_signed(m - 1, H) - Z_signed(m + 1, H)) / 2.0;
    return (k * hd * drho + I * (double)m * hm * dth) * cexp(I * (double)m * theta);
}

int orc_apply_d_tangent(int side, int limit, double kre, double kim, int p, int M, int q_tgt, int q_src,
                        const double *t_edges, double r_factor,
                        const double *gam_tgt, const double *dgam_tgt,
                        const double *gam_src, const double *dgam_src, int ndir,
                        const double *pg_tgt, const double *pdg_tgt,
                        const double *pg_src, const double *pdg_src,
                        const cplx *dens_tgt, int nrhs, cplx *u, cplx *du)
{
    if (p < 0 || p + 3 >= ORC_MAXN || q_tgt < 1 || q_src < 1 || q_tgt > ORC_MAXN || q_src > ORC_MAXN ||
        M < 1 || nrhs < 1 || ndir < 1)
        return 1;
    cplx k = kre + I * kim;
    int n_tgt = M * q_tgt, n_src = M * q_src, nl = 2 * p + 1;
    size_t nd_s = (size_t)n_src, nd_t = (size_t)n_tgt, nd = (size_t)ndir;
    double *buf = malloc(sizeof(double) * (7 * nd_s + 17 * nd_t + (size_t)M));
    double *dbuf = malloc(sizeof(double) * nd * (5 * nd_s + 4 * nd_t + (size_t)M));
    cplx *psig = malloc(sizeof(cplx) * nd_s * nrhs);
    cplx *wd = malloc(sizeof(cplx) * nd_s * nrhs);
    if (!buf || !dbuf || !psig || !wd) { free(buf); free(dbuf); free(psig); free(wd); return 2; }
    double *src_x = buf, *src_y = src_x + nd_s, *src_nx = src_y + nd_s, *src_ny = src_nx + nd_s;
    double *src_w = src_ny + nd_s, *ones = src_w + nd_s;
    double *tgt_x = ones + 2 * nd_s, *tgt_y = tgt_x + nd_t, *tgt_nx = tgt_y + nd_t, *tgt_ny = tgt_nx + nd_t;
    double *tgt_w = tgt_ny + nd_t;
    double *ctr_x = tgt_w + nd_t, *ctr_y = ctr_x + 2 * nd_t, *ctr_r = ctr_y + 2 * nd_t;
    double *ctr_ratio = ctr_r + 2 * nd_t;
    double *panel_h = ctr_ratio + 6 * nd_t;
    /* per direction: d_sx, d_sy, d_sw, d_snx, d_sny [n_src]; d_cx, d_cy [2 n_tgt]; d_h [M] */
    double *d_sx = dbuf, *d_sy = d_sx + nd * nd_s, *d_sw = d_sy + nd * nd_s;
    double *d_snx = d_sw + nd * nd_s, *d_sny = d_snx + nd * nd_s;
    double *d_cx = d_sny + nd * nd_s, *d_cy = d_cx + nd * 2 * nd_t, *d_h = d_cy + nd * 2 * nd_t;
    orc_geometry(M, q_tgt, q_src, t_edges, gam_tgt, dgam_tgt, gam_src, dgam_src, r_factor, 0,
                 src_x, src_y, src_nx, src_ny, src_w, tgt_x, tgt_y, tgt_nx, tgt_ny, tgt_w,
                 panel_h, ctr_x, ctr_y, ctr_r, ctr_ratio);
    double xs[ORC_MAXN], ws[ORC_MAXN];
    orc_gauss_legendre(q_src, xs, ws);
    for (int s = 0; s < n_src; ++s) ones[s] = 1.0;
    for (int d = 0; d < ndir; ++d) {
        const double *pgs = pg_src + (size_t)d * 2 * nd_s, *pdgs = pdg_src + (size_t)d * 2 * nd_s;
        const double *pgt = pg_tgt + (size_t)d * 2 * nd_t, *pdgt = pdg_tgt + (size_t)d * 2 * nd_t;
        double *dsx = d_sx + d * nd_s, *dsy = d_sy + d * nd_s, *dsw = d_sw + d * nd_s;
        double *dsnx = d_snx + d * nd_s, *dsny = d_sny + d * nd_s;
        double *dcx = d_cx + d * 2 * nd_t, *dcy = d_cy + d * 2 * nd_t, *dh = d_h + (size_t)d * M;
        /* tangents of the source nodes, normals, weights and panel lengths */
        for (int m = 0; m < M; ++m) {
            double half = 0.5 * (t_edges[m + 1] - t_edges[m]), acc = 0.0;
            for (int j = 0; j < q_src; ++j) {
                int s = m * q_src + j;
                double vx = dgam_src[2 * s], vy = dgam_src[2 * s + 1];
                double sp = sqrt(vx * vx + vy * vy);
                double px = pdgs[2 * s], py = pdgs[2 * s + 1];
                double tp = (vx * px + vy * py) / sp;   /* tau . pdg */
                dsw[s] = ws[j] * half * tp;
                acc += dsw[s];
                dsx[s] = pgs[2 * s];
                dsy[s] = pgs[2 * s + 1];
                dsnx[s] = (py - src_nx[s] * tp) / sp;
                dsny[s] = (-px - src_ny[s] * tp) / sp;
            }
            dh[m] = acc;
        }
        /* tangents of the centres */
        for (int t = 0; t < n_tgt; ++t) {
            int m = t / q_tgt;
            double vx = dgam_tgt[2 * t], vy = dgam_tgt[2 * t + 1];
            double sp = sqrt(vx * vx + vy * vy);
            double px = pdgt[2 * t], py = pdgt[2 * t + 1];
            double tp = (vx * px + vy * py) / sp;
            double dnx = (py - tgt_nx[t] * tp) / sp, dny = (-px - tgt_ny[t] * tp) / sp;
            double r = ctr_r[t], dr = r_factor * dh[m];
            double ox = dr * tgt_nx[t] + r * dnx, oy = dr * tgt_ny[t] + r * dny;
            dcx[t] = pgt[2 * t] - ox;
            dcy[t] = pgt[2 * t + 1] - oy;
            dcx[n_tgt + t] = pgt[2 * t] + ox;
            dcy[n_tgt + t] = pgt[2 * t + 1] + oy;
        }
    }
    orc_upsample(M, q_tgt, q_src, nrhs, ones, dens_tgt, psig);     /* P mu */
    for (size_t i = 0; i < nd_s * nrhs; ++i) wd[i] = src_w[i / nrhs] * psig[i];
    for (size_t i = 0; i < nd_t * nrhs; ++i) u[i] = 0.0;
    for (size_t i = 0; i < nd * nd_t * nrhs; ++i) du[i] = 0.0;
    int s0 = (side == SIDE_TWO) ? SIDE_INT : side;
    int s1 = (side == SIDE_TWO) ? SIDE_EXT : side;
    double wgt = (side == SIDE_TWO) ? 0.5 : 1.0;
    int fail = 0;
    for (int sd = s0; sd <= s1; ++sd) {
        #pragma omp parallel for schedule(dynamic, 4)
        for (int t = 0; t < n_tgt; ++t) {
            cplx H[ORC_MAXN], J[ORC_MAXN];
            cplx *al = malloc(sizeof(cplx) * (1 + nd) * (size_t)nl * nrhs);
            if (!al) {
                #pragma omp atomic write
                fail = 1;
                continue;
            }
            cplx *dal = al + (size_t)nl * nrhs;             /* [ndir][nl][nrhs] */
            for (size_t i = 0; i < (1 + nd) * (size_t)nl * nrhs; ++i) al[i] = 0.0;
            int c = sd * n_tgt + t;
            double cx = ctr_x[c], cy = ctr_y[c];
            for (int s = 0; s < n_src; ++s) {
                double dx = src_x[s] - cx, dy = src_y[s] - cy;
                double rho = hypot(dx, dy), th = atan2(dy, dx);
                orc_hankel_seq(k * rho, p + 2, H);
                cplx nu = src_nx[s] + I * src_ny[s];
                for (int l = -p; l <= p; ++l) {
                    double sg = (l & 1) ? -1.0 : 1.0;   /* (-1)^l */
                    cplx fa = F_m(-l - 1, H, th), fb = F_m(-l + 1, H, th);
                    cplx kern = sg * (k / 2.0) * (nu * fa - conj(nu) * fb);
                    for (int r = 0; r < nrhs; ++r)
                        al[(size_t)(l + p) * nrhs + r] += (I / 4.0) * wd[(size_t)s * nrhs + r] * kern;
                    for (int d = 0; d < ndir; ++d) {
                        double ddx = d_sx[d * nd_s + s] - d_cx[d * 2 * nd_t + c];
                        double ddy = d_sy[d * nd_s + s] - d_cy[d * 2 * nd_t + c];
                        double drho = (dx * ddx + dy * ddy) / rho;
                        double dth = (dx * ddy - dy * ddx) / (rho * rho);
                        cplx dnu = d_snx[d * nd_s + s] + I * d_sny[d * nd_s + s];
                        cplx dfa = dF_m(-l - 1, H, th, k, drho, dth), dfb = dF_m(-l + 1, H, th, k, drho, dth);
                        cplx dkern = sg * (k / 2.0) * (dnu * fa + nu * dfa - conj(dnu) * fb - conj(nu) * dfb);
                        for (int r = 0; r < nrhs; ++r) {
                            size_t sr = (size_t)s * nrhs + r;
                            cplx dwd = d_sw[d * nd_s + s] * psig[sr];
                            dal[((size_t)d * nl + (l + p)) * nrhs + r] += (I / 4.0) * (dwd * kern + wd[sr] * dkern);
                        }
                    }
                }
            }
            double ex = tgt_x[t] - cx, ey = tgt_y[t] - cy;
            double rt = hypot(ex, ey), tht = atan2(ey, ex);
            orc_besselj_seq(k * rt, p + 1, J);
            for (int l = -p; l <= p; ++l) {
                cplx jl = Z_signed(l, J);
                cplx jd = (Z_signed(l - 1, J) - Z_signed(l + 1, J)) / 2.0;
                cplx e = cexp(I * (double)l * tht);
                for (int r = 0; r < nrhs; ++r)
                    u[(size_t)t * nrhs + r] += wgt * al[(size_t)(l + p) * nrhs + r] * jl * e;
                for (int d = 0; d < ndir; ++d) {
                    const double *pgt = pg_tgt + (size_t)d * 2 * nd_t;
                    double dex = pgt[2 * t] - d_cx[d * 2 * nd_t + c], dey = pgt[2 * t + 1] - d_cy[d * 2 * nd_t + c];
                    double drt = (ex * dex + ey * dey) / rt;
                    double dtht = (ex * dey - ey * dex) / (rt * rt);
                    cplx dfac = (k * jd * drt + I * (double)l * jl * dtht) * e;
                    for (int r = 0; r < nrhs; ++r) {
                        cplx a = al[(size_t)(l + p) * nrhs + r], da = dal[((size_t)d * nl + (l + p)) * nrhs + r];
                        du[((size_t)d * nd_t + t) * nrhs + r] += wgt * (da * jl * e + a * dfac);
                    }
                }
            }
            free(al);
        }
    }
    /* PV, one side: u = lim - sg mu / 2 (sg = +1 exterior, -1 interior); no derivative */
    if (side != SIDE_TWO && limit == LIMIT_PV) {
        double sg = (side == SIDE_EXT) ? 1.0 : -1.0;
        for (size_t i = 0; i < nd_t * nrhs; ++i) u[i] -= sg * 0.5 * dens_tgt[i];
    }
    free(buf); free(dbuf); free(psig); free(wd);
    return fail ? 2 : 0;
}

/* ------------------------------------------------------------------------- */
/* Near-only QBX (the optimisation remarked in Sec. 5: direct evaluation for  */
/* distant interactions, QBX for near ones).  Reading: for the centre c of    */
/* target x_t, a source node x_s is near when |x_s - c| < eta r_c; near nodes */
/* go through the local expansion at c (form + evaluate, as orc_apply), the   */
/* others through the smooth rule at x_t itself (as orc_far).  The jumps of   */
/* orc_apply follow.  ops S, D, grad S; out as orc_apply.                    */
/* ------------------------------------------------------------------------- */
int orc_apply_local(int op, int side, int limit, double kre, double kim, int p, double eta,
                    int M, int q_tgt, int q_src,
                    const double *src_x, const double *src_y, const double *src_nx,
                    const double *src_ny, const double *src_w,
                    const double *tgt_x, const double *tgt_y, const double *tgt_nx,
                    const double *tgt_ny,
                    const double *ctr_x, const double *ctr_y, const double *ctr_r,
                    const cplx *dens_tgt, int nrhs, int n_sel, const int *sel, cplx *out)
{
    int n_tgt = M * q_tgt, n_src = M * q_src, nl = 2 * p + 1;
    int ncomp = (op == OP_GRAD_S) ? 2 : 1;
    if (op != OP_S && op != OP_D && op != OP_GRAD_S) return 1;
    if (n_sel <= 0 || !sel) n_sel = n_tgt, sel = NULL;
    cplx *wd = malloc(sizeof(cplx) * (size_t)n_src * nrhs);
    if (!wd) return 2;
    orc_upsample(M, q_tgt, q_src, nrhs, src_w, dens_tgt, wd);
    for (size_t i = 0; i < (size_t)n_sel * ncomp * nrhs; ++i) out[i] = 0.0;
    int s0 = (side == SIDE_TWO) ? SIDE_INT : side;
    int s1 = (side == SIDE_TWO) ? SIDE_EXT : side;
    cplx k = kre + I * kim;
    int fail = 0;
    for (int sd = s0; sd <= s1; ++sd) {
        double sgn = (sd == SIDE_EXT) ? 1.0 : -1.0;
        #pragma omp parallel for schedule(dynamic, 4)
        for (int i = 0; i < n_sel; ++i) {
            int t = sel ? sel[i] : i;
            size_t c = (size_t)sd * n_tgt + t;
            double cx = ctr_x[c], cy = ctr_y[c], lim = eta * ctr_r[c];
            /* near sources, compacted */
            double *nx_ = malloc(sizeof(double) * 4 * (size_t)n_src);
            cplx *nwd = malloc(sizeof(cplx) * (size_t)n_src * nrhs);
            cplx *al = malloc(sizeof(cplx) * (size_t)nl * nrhs);
            cplx val[2 * 64];
            if (!nx_ || !nwd || !al || nrhs > 64) {
                free(nx_); free(nwd); free(al);
                #pragma omp atomic write
                fail = 1;
                continue;
            }
            double *ny_ = nx_ + n_src, *nnx = ny_ + n_src, *nny = nnx + n_src;
            int nn = 0;
            cplx far[2 * 64];
            for (int q = 0; q < ncomp * nrhs; ++q) far[q] = 0.0;
            for (int s = 0; s < n_src; ++s) {
                if (hypot(src_x[s] - cx, src_y[s] - cy) < lim) {
                    nx_[nn] = src_x[s]; ny_[nn] = src_y[s]; nnx[nn] = src_nx[s]; nny[nn] = src_ny[s];
                    for (int r = 0; r < nrhs; ++r) nwd[(size_t)nn * nrhs + r] = wd[(size_t)s * nrhs + r];
                    ++nn;
                } else {   /* smooth rule at the target */
                    double rx = tgt_x[t] - src_x[s], ry = tgt_y[t] - src_y[s];
                    double d = hypot(rx, ry);
                    cplx h0, h1;
                    orc_hankel01(k * d, &h0, &h1);
                    for (int r = 0; r < nrhs; ++r) {
                        cplx w = wd[(size_t)s * nrhs + r];
                        if (op == OP_S) far[r] += (I / 4.0) * w * h0;
                        else if (op == OP_D) far[r] += (I * k / 4.0) * w * h1 * (rx * src_nx[s] + ry * src_ny[s]) / d;
                        else {
                            far[r] += -(I * k / 4.0) * w * h1 * rx / d;
                            far[nrhs + r] += -(I * k / 4.0) * w * h1 * ry / d;
                        }
                    }
                }
            }
            double ccx[1] = {cx}, ccy[1] = {cy}, ex[1] = {tgt_x[t]}, ey[1] = {tgt_y[t]};
            int ec[1] = {0};
            orc_form_locals(op == OP_D ? OP_D : OP_S, 1, ccx, ccy, nn, nx_, ny_, nnx, nny, nwd, nrhs, kre, kim, p, al);
            orc_eval_locals(1, ex, ey, ec, ccx, ccy, al, nrhs, kre, kim, p,
                            op == OP_GRAD_S ? WHAT_GRAD : WHAT_VALUE, val);
            for (int r = 0; r < nrhs; ++r) {
                cplx dens = dens_tgt[(size_t)t * nrhs + r];
                if (op == OP_GRAD_S) {
                    cplx gx = val[r] + far[r], gy = val[nrhs + r] + far[nrhs + r];
                    if (side != SIDE_TWO && limit == LIMIT_PV) {
                        gx += sgn * 0.5 * tgt_nx[t] * dens;
                        gy += sgn * 0.5 * tgt_ny[t] * dens;
                    }
                    if (side == SIDE_TWO) { gx *= 0.5; gy *= 0.5; }
                    out[((size_t)i * 2 + 0) * nrhs + r] += gx;
                    out[((size_t)i * 2 + 1) * nrhs + r] += gy;
                } else {
                    cplx u = val[r] + far[r];
                    if (op == OP_D && side != SIDE_TWO && limit == LIMIT_PV) u -= sgn * 0.5 * dens;
                    if (side == SIDE_TWO) u *= 0.5;
                    out[(size_t)i * nrhs + r] += u;
                }
            }
            free(nx_); free(nwd); free(al);
        }
    }
    free(wd);
    return fail ? 2 : 0;
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
