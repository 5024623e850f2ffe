/*
 * sac_oracle.c -- plain, slow FP64 CPU oracle for face-staggered
 * susceptibility artifact correction (SAC) of EPI-MRI, after Macdonald &
 * Ruthotto, "Efficient Numerical Optimization for Susceptibility Artifact
 * Correction of EPI-MRI" (arXiv 1607.00531).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library: every quantity below is
 * recomputed here from the paper's definitions.
 *
 * Contents (each function names the passage it follows):
 *   - continuous image model by 1D linear interpolation       (Sec. 3)
 *   - residual r(b), Jacobian J_r, distance D                 (Sec. 3, Eq. D)
 *   - regulariser S, penalty P, phi, phi', phi''               (Sec. 3, Eqs. S, P, dphi)
 *   - gradients / (GN-)Hessian products                       (Sec. 3, Eqs. dJ, dJGN)
 *   - primal active-set QP with Schur-complement solves       (Sec. 4.2, Eqs. qp, schurasqp)
 *   - ADMM b-step (SQP), z-step (DCT), u-step, stopping       (Sec. 4.2, Eqs. admmStep1-3, dctdiag, admmStop)
 *   - block-Jacobi preconditioner and inexact GN-PCG          (Sec. 4.1, Eqs. Pblock, GNstep, inexactGNsolve, stopping1-3)
 *   - image restriction, field prolongation, coarse-to-fine ADMM (Sec. 4.4)
 *
 * Readings where the paper is silent or garbled (interpolation at the
 * boundary, units of b, the D1^T in the b-step gradient and in grad P, gamma
 * in P_block, the step form of the QP, the active-set start, the number of SQP
 * passes, the DCT type, the line search) are each stated at the place they
 * are used.  One option serves the
 * comparison with single-precision kernels only: with knot32 the position at
 * which the image model is evaluated is formed in FP32 as they form it (the
 * model's interval is an integer decided in floating point), all else FP64.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Grid                                                                      */
/* ------------------------------------------------------------------------ */

/* A grid of M[0] x M[1] x M[2] cells (M[2] = 1 in 2D) with the field b on
   the faces normal to the phase-encoding (PE) axis `pe` (Sec. 3, "b on the
   x1-faces").  Arrays are row-major over (axis0, axis1, axis2); face arrays
   carry M[pe]+1 entries along the PE axis. */
typedef struct {
    int nd, pe;
    long M[3], F[3];
    double h[3];
    double hd;                    /* cell volume h1*h2(*h3) */
    long n_outer, mpe, n_inner;   /* line view: (outer, PE, inner) */
    long nf, nc;                  /* number of faces / cells */
} grid_t;

/* Parameters.  Field order must match oracle/__init__.py. */
typedef struct {
    double alpha, beta, gamma, rho;
    double eps_abs, eps_rel;
    double eta, eps_obj, eps_iter, eps_grad, gn_rel_grad;
    int max_iter, n_sqp, max_pcg, precond, max_gn, nthreads;
    int adapt_rho;                /* 0 fixed rho, 1 adaptive, 2 adaptive with lower bound */
    double rho_min, rho_tau, rho_mu;
    int knot32;                   /* 1: interpolation positions formed in FP32 (see line_cells) */
} ref_params;

enum { REF_OK = 0, REF_NOTCONV = 1, REF_EINVAL = -1, REF_EINFEASIBLE = -4, REF_ELSFAIL = -7 };

static int make_grid(int nd, const int* m, const double* h, int pe, grid_t* g) {
    if (nd != 2 && nd != 3) return REF_EINVAL;
    if (pe < 0 || pe >= nd) return REF_EINVAL;
    g->nd = nd; g->pe = pe; g->hd = 1.0;
    for (int a = 0; a < 3; ++a) {
        g->M[a] = (a < nd) ? m[a] : 1;
        g->h[a] = (a < nd) ? h[a] : 1.0;
        if (g->M[a] < 1 || !(g->h[a] > 0)) return REF_EINVAL;
        if (a < nd) g->hd *= g->h[a];
        g->F[a] = g->M[a] + (a == pe ? 1 : 0);
    }
    g->mpe = g->M[pe];
    g->n_outer = 1; g->n_inner = 1;
    for (int a = 0; a < pe; ++a) g->n_outer *= g->M[a];
    for (int a = pe + 1; a < 3; ++a) g->n_inner *= g->M[a];
    g->nf = g->F[0] * g->F[1] * g->F[2];
    g->nc = g->M[0] * g->M[1] * g->M[2];
    return REF_OK;
}

static long n_lines(const grid_t* g) { return g->n_outer * g->n_inner; }
/* first face / first cell of line l, and the stride along PE */
static long line_face0(const grid_t* g, long l) {
    long o = l / g->n_inner, n = l % g->n_inner;
    return o * (g->mpe + 1) * g->n_inner + n;
}
static long line_cell0(const grid_t* g, long l) {
    long o = l / g->n_inner, n = l % g->n_inner;
    return o * g->mpe * g->n_inner + n;
}

/* nthreads > 0: that many OpenMP threads; 0: all the host's processors */
static void set_threads(const ref_params* p) {
#ifdef _OPENMP
    if (p) omp_set_num_threads(p->nthreads > 0 ? p->nthreads : omp_get_num_procs());
#else
    (void)p;
#endif
}

int ref_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Penalty function phi and its derivatives (Sec. 3, Eqs. P and dphi)        */
/* ------------------------------------------------------------------------ */

double ref_phi(double x) {
    if (!(fabs(x) < 1.0)) return INFINITY;
    return x * x * x * x / (1.0 - x * x);
}
double ref_dphi(double x) {
    double s = 1.0 - x * x;
    return (4.0 * x * x * x - 2.0 * x * x * x * x * x) / (s * s);
}
double ref_d2phi(double x) {
    double s = 1.0 - x * x;
    double x2 = x * x;
    return 2.0 * x2 * (x2 * x2 - 3.0 * x2 + 6.0) / (s * s * s);
}

/* ------------------------------------------------------------------------ */
/* Continuous image model (Sec. 3: "a continuous image model is built from   */
/* discrete data by using interpolation").                                   */
/*                                                                           */
/* Reading: 1D linear interpolation along the PE line of the cell-centred    */
/* samples I[k] at x_k = (k + 1/2) h.  In index units t = x/h - 1/2 the      */
/* model passes through (k, I[k]) for k = 0..m-1 and through zero at k = -1  */
/* and k = m (compact support); it is zero outside [-1, m].  The slope is    */
/* that of the interval [floor(t), floor(t)+1] (right interval at a knot).   */
/* Returns the value and dI/dt (index units).                                */
/* ------------------------------------------------------------------------ */
static void interp_line(const double* I, long stride, long m, double t, double* v, double* dv) {
    double fl = floor(t);
    if (!(fl >= -1.0) || !(fl <= (double)(m - 1))) { *v = 0.0; *dv = 0.0; return; }
    long k = (long)fl;
    double f = t - fl;
    double left = (k >= 0) ? I[k * stride] : 0.0;
    double right = (k + 1 <= m - 1) ? I[(k + 1) * stride] : 0.0;
    *v = (1.0 - f) * left + f * right;
    *dv = right - left;
}

/* Per-cell quantities of one line at the field values bl[0..m] (stride sb):
   averaging A1 (Eq. A) and short difference D1 (Eq. D1), the residual
   r = I1(x + A b)(1 + D1 b) - I2(x - A b)(1 - D1 b) (Sec. 3, residual of Eq. D),
   and the two nonzeros of row j of the Jacobian J_r (Sec. 3, "The Jacobian of
   the residual"):  Jd[j] = dr_j/db_j, Ju[j] = dr_j/db_{j+1}. */
typedef struct { double r, d, Jd, Ju; } cellq;

static void line_cells(const grid_t* g, const double* I1, const double* I2, long cstride,
                       const double* bl, long sb, cellq* q, int knot32) {
    long m = g->mpe;
    double h = g->h[g->pe];
    for (long j = 0; j < m; ++j) {
        double b0 = bl[j * sb], b1 = bl[(j + 1) * sb];
        double a = 0.5 * (b0 + b1);       /* A1 b: displacement at the cell centre */
        double d = (b1 - b0) / h;         /* D1 b: derivative along PE */
        double t1 = (double)j + a / h, t2 = (double)j - a / h;
        if (knot32) {
            /* The interval of the piecewise-linear model (an integer) is decided
               by a floating-point position; its slope jumps at the knots, so a
               position that rounds across one changes the Jacobian, not just
               its last digits.  For comparison with single-precision kernels the
               position is formed as they form it: A1 b and 1/h rounded to FP32,
               then one fused multiply-add with the cell index. */
            const float af = 0.5f * ((float)b0 + (float)b1);
            const float invh = (float)(1.0 / h);
            t1 = (double)fmaf(af, invh, (float)j);
            t2 = (double)fmaf(-af, invh, (float)j);
        }
        double v1, s1, v2, s2;
        interp_line(I1, cstride, m, t1, &v1, &s1);   /* I_v(x + A b)  */
        interp_line(I2, cstride, m, t2, &v2, &s2);   /* I_-v(x - A b) */
        double g1 = s1 / h, g2 = s2 / h;  /* spatial derivatives d/dx */
        q[j].r = v1 * (1.0 + d) - v2 * (1.0 - d);
        q[j].d = d;
        /* J_r = diag(dI_v (1+D1b)) A1 + diag(I_v) D1 + diag(dI_-v (1-D1b)) A1 + diag(I_-v) D1 */
        double p = 0.5 * (g1 * (1.0 + d) + g2 * (1.0 - d));
        double qq = (v1 + v2) / h;
        q[j].Jd = p - qq;
        q[j].Ju = p + qq;
    }
}

/* ------------------------------------------------------------------------ */
/* Regulariser pieces: D_a^T D_a along every axis (Sec. 3, Eqs. S and d2d3). */
/* ------------------------------------------------------------------------ */

static long face_index(const grid_t* g, long i0, long i1, long i2) {
    return (i0 * g->F[1] + i1) * g->F[2] + i2;
}

/* out += s * D_a^T D_a v for axis a (short differences between neighbouring
   faces along a with spacing h_a; Neumann at the ends). */
static void add_DtD_axis(const grid_t* g, int a, double s, const double* v, double* out) {
    if (g->F[a] < 2) return;
    double ih2 = 1.0 / (g->h[a] * g->h[a]);
    long st = (a == 0) ? g->F[1] * g->F[2] : (a == 1) ? g->F[2] : 1;
    for (long i0 = 0; i0 < g->F[0]; ++i0)
        for (long i1 = 0; i1 < g->F[1]; ++i1)
            for (long i2 = 0; i2 < g->F[2]; ++i2) {
                long ia = (a == 0) ? i0 : (a == 1) ? i1 : i2;
                long f = face_index(g, i0, i1, i2);
                double acc = 0.0;
                if (ia > 0) acc += (v[f] - v[f - st]);
                if (ia < g->F[a] - 1) acc += (v[f] - v[f + st]);
                out[f] += s * ih2 * acc;
            }
}

/* sum over axis a of ((v_{i+e_a} - v_i)/h_a)^2 = ||D_a v||^2 */
static double sq_Dv_axis(const grid_t* g, int a, const double* v) {
    if (g->F[a] < 2) return 0.0;
    long st = (a == 0) ? g->F[1] * g->F[2] : (a == 1) ? g->F[2] : 1;
    double acc = 0.0;
    for (long i0 = 0; i0 < g->F[0]; ++i0)
        for (long i1 = 0; i1 < g->F[1]; ++i1)
            for (long i2 = 0; i2 < g->F[2]; ++i2) {
                long ia = (a == 0) ? i0 : (a == 1) ? i1 : i2;
                if (ia >= g->F[a] - 1) continue;
                long f = face_index(g, i0, i1, i2);
                double d = (v[f + st] - v[f]) / g->h[a];
                acc += d * d;
            }
    return acc;
}

/* number of neighbours of face f along axis a (for M = diag(D2^T D2 + D3^T D3)) */
static int n_nbr(const grid_t* g, int a, long ia) {
    if (g->F[a] < 2) return 0;
    return (ia > 0) + (ia < g->F[a] - 1);
}

/* ------------------------------------------------------------------------ */
/* Objective J = D + alpha S + P (Sec. 3, Eqs. D, S, P, discprob, JGN)      */
/* ------------------------------------------------------------------------ */

/* out[0..3] = {J, D, S, P}.  P uses beta; P = +inf when some |D1 b| >= 1 and
   beta > 0 (phi is +inf outside (-1, 1)). */
int ref_objective(int nd, const int* m, const double* h, int pe, const ref_params* prm,
                  const double* I1, const double* I2, const double* b, double* out) {
    grid_t g;
    int st = make_grid(nd, m, h, pe, &g);
    if (st) return st;
    set_threads(prm);
    long L = n_lines(&g);
    double* partD = (double*)calloc((size_t)L, sizeof(double));
    double* partP = (double*)calloc((size_t)L, sizeof(double));
    double* partS1 = (double*)calloc((size_t)L, sizeof(double));
#pragma omp parallel
    {
        cellq* q = (cellq*)malloc(sizeof(cellq) * (size_t)g.mpe);
#pragma omp for schedule(static)
        for (long l = 0; l < L; ++l) {
            line_cells(&g, I1 + line_cell0(&g, l), I2 + line_cell0(&g, l), g.n_inner,
                       b + line_face0(&g, l), g.n_inner, q, prm->knot32);
            double sD = 0.0, sP = 0.0, sS = 0.0;
            for (long j = 0; j < g.mpe; ++j) {
                sD += q[j].r * q[j].r;
                sS += q[j].d * q[j].d;
                if (prm->beta > 0) sP += ref_phi(q[j].d);
            }
            partD[l] = sD; partP[l] = sP; partS1[l] = sS;
        }
        free(q);
    }
    double sD = 0.0, sP = 0.0, sS1 = 0.0;
    for (long l = 0; l < L; ++l) { sD += partD[l]; sP += partP[l]; sS1 += partS1[l]; }
    free(partD); free(partP); free(partS1);
    double sS = sS1;
    for (int a = 0; a < 3; ++a)
        if (a != g.pe) sS += sq_Dv_axis(&g, a, b);
    double D = 0.5 * g.hd * sD;
    double S = 0.5 * g.hd * sS;
    double P = (prm->beta > 0) ? prm->beta * g.hd * sP : 0.0;
    out[0] = D + prm->alpha * S + P;
    out[1] = D; out[2] = S; out[3] = P;
    return REF_OK;
}

/* residual r(b) per cell (cell-array layout) */
int ref_residual(int nd, const int* m, const double* h, int pe,
                 const double* I1, const double* I2, const double* b, double* r) {
    grid_t g;
    int st = make_grid(nd, m, h, pe, &g);
    if (st) return st;
    long L = n_lines(&g);
#pragma omp parallel
    {
        cellq* q = (cellq*)malloc(sizeof(cellq) * (size_t)g.mpe);
#pragma omp for schedule(static)
        for (long l = 0; l < L; ++l) {
            long c0 = line_cell0(&g, l);
            line_cells(&g, I1 + c0, I2 + c0, g.n_inner, b + line_face0(&g, l), g.n_inner, q, 0);
            for (long j = 0; j < g.mpe; ++j) r[c0 + j * g.n_inner] = q[j].r;
        }
        free(q);
    }
    return REF_OK;
}

/* Gradient of J_GN = D + alpha S + P:
   grad D = h^d J_r^T r, grad S = h^d sum_a D_a^T D_a b,
   grad P = beta h^d D1^T phi'(D1 b)  (reading of the garbled D1 in Sec. 3). */
int ref_gradient(int nd, const int* m, const double* h, int pe, const ref_params* prm,
                 const double* I1, const double* I2, const double* b, double* grad) {
    grid_t g;
    int st = make_grid(nd, m, h, pe, &g);
    if (st) return st;
    set_threads(prm);
    long L = n_lines(&g);
    double hpe = g.h[g.pe];
    memset(grad, 0, sizeof(double) * (size_t)g.nf);
#pragma omp parallel
    {
        cellq* q = (cellq*)malloc(sizeof(cellq) * (size_t)g.mpe);
#pragma omp for schedule(static)
        for (long l = 0; l < L; ++l) {
            long f0 = line_face0(&g, l), c0 = line_cell0(&g, l), s = g.n_inner;
            line_cells(&g, I1 + c0, I2 + c0, s, b + f0, s, q, prm->knot32);
            for (long i = 0; i <= g.mpe; ++i) {
                double gi = 0.0;
                if (i > 0) gi += q[i - 1].Ju * q[i - 1].r;
                if (i < g.mpe) gi += q[i].Jd * q[i].r;
                gi *= g.hd;
                if (prm->beta > 0) {
                    double t = 0.0;
                    if (i > 0) t += ref_dphi(q[i - 1].d);
                    if (i < g.mpe) t -= ref_dphi(q[i].d);
                    gi += prm->beta * g.hd * t / hpe;
                }
                grad[f0 + i * s] = gi;
            }
        }
        free(q);
    }
    for (int a = 0; a < 3; ++a) add_DtD_axis(&g, a, prm->alpha * g.hd, b, grad);
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* Hessian pieces applied to a vector (Sec. 3 and Sec. 4.1)                  */
/*   op 0: H_D v = h^d J_r^T J_r v                                           */
/*   op 1: grad^2 S v = h^d sum_a D_a^T D_a v                                */
/*   op 2: D1^T D1 v                                                         */
/*   op 3: D_a^T D_a v for the first non-PE axis (the paper's D2)            */
/*   op 4: grad^2 P v = beta h^d D1^T diag(phi''(D1 b)) D1 v                 */
/*   op 5: H_JGN v = H_D v + alpha grad^2 S v + grad^2 P v + gamma v         */
/*   op 6: P_block v = [H_D + alpha h^d (D1^T D1 + M) + grad^2 P + gamma I] v */
/*   op 7: D_a^T D_a v for the second non-PE axis (the paper's D3)           */
/*   op 8: M v, M = diag(D2^T D2 + D3^T D3)                                  */
/* ------------------------------------------------------------------------ */

static void other_axes(const grid_t* g, int* a1, int* a2) {
    int k = 0, ax[2] = {0, 0};
    for (int a = 0; a < 3; ++a) if (a != g->pe) ax[k++] = a;
    *a1 = ax[0]; *a2 = ax[1];
}

static double M_diag(const grid_t* g, long f) {
    long i2 = f % g->F[2], i1 = (f / g->F[2]) % g->F[1], i0 = f / (g->F[1] * g->F[2]);
    long ia[3] = {i0, i1, i2};
    double s = 0.0;
    for (int a = 0; a < 3; ++a)
        if (a != g->pe) s += n_nbr(g, a, ia[a]) / (g->h[a] * g->h[a]);
    return s;
}

int ref_apply(int nd, const int* m, const double* h, int pe, const ref_params* prm, int op,
              const double* I1, const double* I2, const double* b, const double* v, double* out) {
    grid_t g;
    int st = make_grid(nd, m, h, pe, &g);
    if (st) return st;
    set_threads(prm);
    memset(out, 0, sizeof(double) * (size_t)g.nf);
    int a1, a2;
    other_axes(&g, &a1, &a2);
    double hpe = g.h[g.pe];
    if (op == 1) { for (int a = 0; a < 3; ++a) add_DtD_axis(&g, a, g.hd, v, out); return REF_OK; }
    if (op == 2) { add_DtD_axis(&g, g.pe, 1.0, v, out); return REF_OK; }
    if (op == 3) { add_DtD_axis(&g, a1, 1.0, v, out); return REF_OK; }
    if (op == 7) { add_DtD_axis(&g, a2, 1.0, v, out); return REF_OK; }
    if (op == 8) { for (long f = 0; f < g.nf; ++f) out[f] = M_diag(&g, f) * v[f]; return REF_OK; }
    if (op != 0 && op != 4 && op != 5 && op != 6) return REF_EINVAL;
    int want_D = (op == 0 || op == 5 || op == 6);
    int want_P = (op == 4 || op == 5 || op == 6) && prm->beta > 0;
    long L = n_lines(&g);
#pragma omp parallel
    {
        cellq* q = (cellq*)malloc(sizeof(cellq) * (size_t)g.mpe);
        double* w = (double*)malloc(sizeof(double) * (size_t)g.mpe);
        double* e = (double*)malloc(sizeof(double) * (size_t)g.mpe);
#pragma omp for schedule(static)
        for (long l = 0; l < L; ++l) {
            long f0 = line_face0(&g, l), c0 = line_cell0(&g, l), s = g.n_inner;
            line_cells(&g, I1 + c0, I2 + c0, s, b + f0, s, q, prm->knot32);
            for (long j = 0; j < g.mpe; ++j) {
                w[j] = q[j].Jd * v[f0 + j * s] + q[j].Ju * v[f0 + (j + 1) * s];   /* J_r v */
                e[j] = (v[f0 + (j + 1) * s] - v[f0 + j * s]) / hpe;               /* D1 v */
            }
            for (long i = 0; i <= g.mpe; ++i) {
                double acc = 0.0;
                if (want_D) {
                    double t = 0.0;
                    if (i > 0) t += q[i - 1].Ju * w[i - 1];
                    if (i < g.mpe) t += q[i].Jd * w[i];
                    acc += g.hd * t;
                }
                if (want_P) {
                    double t = 0.0;
                    if (i > 0) t += ref_d2phi(q[i - 1].d) * e[i - 1];
                    if (i < g.mpe) t -= ref_d2phi(q[i].d) * e[i];
                    acc += prm->beta * g.hd * t / hpe;
                }
                out[f0 + i * s] += acc;
            }
        }
        free(q); free(w); free(e);
    }
    if (op == 5) {
        for (int a = 0; a < 3; ++a) add_DtD_axis(&g, a, prm->alpha * g.hd, v, out);
        for (long f = 0; f < g.nf; ++f) out[f] += prm->gamma * v[f];
    }
    if (op == 6) {
        add_DtD_axis(&g, g.pe, prm->alpha * g.hd, v, out);
        for (long f = 0; f < g.nf; ++f) out[f] += (prm->alpha * g.hd * M_diag(&g, f) + prm->gamma) * v[f];
    }
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* Symmetric tridiagonal solve (Thomas algorithm, no pivoting: the systems   */
/* here are symmetric positive definite).  off[i] couples unknowns i, i+1.   */
/* ------------------------------------------------------------------------ */
static void thomas(long n, const double* dg, const double* off, const double* rhs, double* x, double* cp) {
    double beta = dg[0];
    x[0] = rhs[0] / beta;
    if (n > 1) cp[0] = off[0] / beta;
    for (long i = 1; i < n; ++i) {
        beta = dg[i] - off[i - 1] * cp[i - 1];
        x[i] = (rhs[i] - off[i - 1] * x[i - 1]) / beta;
        if (i < n - 1) cp[i] = off[i] / beta;
    }
    for (long i = n - 2; i >= 0; --i) x[i] -= cp[i] * x[i + 1];
}

/* dense Cholesky solve of the q x q SPD system S y = r (in place in S) */
static void chol_solve(long q, double* S, double* y) {
    for (long j = 0; j < q; ++j) {
        double s = S[j * q + j];
        for (long k = 0; k < j; ++k) s -= S[j * q + k] * S[j * q + k];
        S[j * q + j] = sqrt(s);
        for (long i = j + 1; i < q; ++i) {
            double t = S[i * q + j];
            for (long k = 0; k < j; ++k) t -= S[i * q + k] * S[j * q + k];
            S[i * q + j] = t / S[j * q + j];
        }
    }
    for (long i = 0; i < q; ++i) {
        double t = y[i];
        for (long k = 0; k < i; ++k) t -= S[i * q + k] * y[k];
        y[i] = t / S[i * q + i];
    }
    for (long i = q - 1; i >= 0; --i) {
        double t = y[i];
        for (long k = i + 1; k < q; ++k) t -= S[k * q + i] * y[k];
        y[i] = t / S[i * q + i];
    }
}

/* ------------------------------------------------------------------------ */
/* Per-line QP by the primal active-set method (Sec. 4.2, Eqs. qp and       */
/* schurasqp; Nocedal & Wright, Ch. 16).                                     */
/*                                                                           */
/*   min_x 1/2 x^T G x + c^T x   s.t.  A x >= d,                             */
/*                                                                           */
/* with G symmetric tridiagonal (diagonal Gd[0..m], off-diagonal Go[0..m-1]) */
/* and the rows of A the short differences D1 and -D1 of one line.  Step     */
/* form (reading): x is the SQP step from the current feasible b^k whose     */
/* cell derivatives are dk[j]; row "lower j" is (x_{j+1}-x_j)/h >= -1-dk[j], */
/* row "upper j" is -(x_{j+1}-x_j)/h >= -1+dk[j].                            */
/*                                                                           */
/* Start: x = 0 (feasible because b^k is), empty working set.  Each pass     */
/* solves the equality-constrained QP on the working set through the Schur   */
/* complement:                                                               */
/*   lambda = -(A_I G^-1 A_I^T)^-1 (A_I G^-1 g - h),  p = G^-1(A_I^T lambda + g) */
/* with g = -c - G x, h = d_I - A_I x.  Then (paper's three cases):          */
/*   p = 0, lambda >= 0       -> x is the solution;                          */
/*   p = 0, some lambda < 0   -> drop the constraint with the most negative  */
/*                               lambda (lowest cell on a tie);              */
/*   p != 0                   -> step t = min(1, blocking ratios); if t < 1  */
/*                               add every constraint that blocks at t.      */
/* "p = 0" holds exactly when the previous pass took its full step (x then   */
/* minimises the QP on the working set); that pass's p is not recomputed to  */
/* be compared with zero.  At most 4(m+1) passes; returns the pass count, or */
/* -1 when the cap is reached (x is then feasible but not optimal).          */
/* ------------------------------------------------------------------------ */
int ref_line_qp(long m, double h, const double* Gd, const double* Go, const double* c,
                const double* dk, double* x, int* n_active_out) {
    long n = m + 1;
    /* working set: for each cell j, 0 = free, -1 = lower active (D1 b' = -1),
       +1 = upper active (D1 b' = +1) */
    int* act = (int*)calloc((size_t)m, sizeof(int));
    long* W = (long*)malloc(sizeof(long) * (size_t)(m > 0 ? m : 1));
    double* Y = (double*)malloc(sizeof(double) * (size_t)(n * (m > 0 ? m : 1)));
    double* S = (double*)malloc(sizeof(double) * (size_t)((m > 0 ? m : 1) * (m > 0 ? m : 1)));
    double* lam = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double* gvec = (double*)malloc(sizeof(double) * (size_t)n);
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    double* p = (double*)malloc(sizeof(double) * (size_t)n);
    double* col = (double*)malloc(sizeof(double) * (size_t)n);
    double* cp = (double*)malloc(sizeof(double) * (size_t)n);
    for (long i = 0; i < n; ++i) x[i] = 0.0;
    int at_min = 0, passes = 0, result = -1;
    long cap = 4 * n;
    for (long it = 0; it < cap; ++it) {
        ++passes;
        long q = 0;
        for (long j = 0; j < m; ++j) if (act[j]) W[q++] = j;
        if (at_min && q == 0) { result = passes; break; }
        /* g = -c - G x */
        for (long i = 0; i < n; ++i) {
            double Gx = Gd[i] * x[i];
            if (i > 0) Gx += Go[i - 1] * x[i - 1];
            if (i < m) Gx += Go[i] * x[i + 1];
            gvec[i] = -c[i] - Gx;
        }
        thomas(n, Gd, Go, gvec, w, cp);                 /* w = G^-1 g */
        /* Y(:,k) = G^-1 a_k for the active rows a_k = sigma_k (e_{j+1}-e_j)/h,
           sigma = +1 for a lower row, -1 for an upper row */
        for (long k = 0; k < q; ++k) {
            long j = W[k];
            double sg = (act[j] < 0) ? 1.0 : -1.0;
            for (long i = 0; i < n; ++i) col[i] = 0.0;
            col[j] = -sg / h; col[j + 1] = sg / h;
            thomas(n, Gd, Go, col, Y + k * n, cp);
        }
        /* Schur complement S = A_I G^-1 A_I^T and rhs = A_I w - h_I */
        for (long k = 0; k < q; ++k) {
            long j = W[k];
            double sg = (act[j] < 0) ? 1.0 : -1.0;
            for (long l = 0; l < q; ++l)
                S[k * q + l] = sg * (Y[l * n + j + 1] - Y[l * n + j]) / h;
            double Ax = sg * (x[j + 1] - x[j]) / h;
            double dI = (act[j] < 0) ? (-1.0 - dk[j]) : (-1.0 + dk[j]);
            double Aw = sg * (w[j + 1] - w[j]) / h;
            lam[k] = Aw - (dI - Ax);
        }
        if (q > 0) chol_solve(q, S, lam);
        for (long k = 0; k < q; ++k) lam[k] = -lam[k];
        if (at_min) {
            /* p = 0: optimality test on the multipliers */
            long worst = -1;
            double wl = 0.0;
            for (long k = 0; k < q; ++k)
                if (lam[k] < wl) { wl = lam[k]; worst = k; }
            if (worst < 0) { result = passes; break; }
            act[W[worst]] = 0;
            at_min = 0;
            continue;
        }
        /* p = G^-1 (A_I^T lambda + g) = w + Y lambda */
        for (long i = 0; i < n; ++i) {
            double t = w[i];
            for (long k = 0; k < q; ++k) t += Y[k * n + i] * lam[k];
            p[i] = t;
        }
        /* ratio test over the constraints outside the working set */
        double tau = 1.0;
        for (long j = 0; j < m; ++j) {
            if (act[j]) continue;
            double dcur = dk[j] + (x[j + 1] - x[j]) / h;
            double dp = (p[j + 1] - p[j]) / h;
            double tj = INFINITY;
            if (dp < 0) tj = (-1.0 - dcur) / dp;
            else if (dp > 0) tj = (1.0 - dcur) / dp;
            if (tj < tau) tau = tj;
        }
        if (tau < 0) tau = 0;   /* rounding guard: never step backwards */
        int blocked = (tau < 1.0);
        if (blocked) {
            for (long j = 0; j < m; ++j) {
                if (act[j]) continue;
                double dcur = dk[j] + (x[j + 1] - x[j]) / h;
                double dp = (p[j + 1] - p[j]) / h;
                double tj = INFINITY;
                if (dp < 0) tj = (-1.0 - dcur) / dp;
                else if (dp > 0) tj = (1.0 - dcur) / dp;
                if (tj <= tau) act[j] = (dp < 0) ? -1 : 1;
            }
        }
        for (long i = 0; i < n; ++i) x[i] += tau * p[i];
        at_min = !blocked;
    }
    if (n_active_out) {
        int na = 0;
        for (long j = 0; j < m; ++j) na += (act[j] != 0);
        *n_active_out = na;
    }
    free(act); free(W); free(Y); free(S); free(lam); free(gvec); free(w); free(p); free(col); free(cp);
    return result;
}

/* ------------------------------------------------------------------------ */
/* ADMM b-step (Sec. 4.2, Eq. admmStep1): per line, n_sqp SQP passes.  Each  */
/* pass linearises at the current b and solves the QP above with             */
/*   c = grad D(b) + alpha h^d D1^T D1 b + rho h^d (b - z + u)               */
/*   G = H_D(b) + alpha h^d D1^T D1 + rho h^d I                              */
/* (reading: the printed "alpha h^3 D1 b" is the gradient alpha h^3 D1^T D1 b */
/* of the alpha-part of f), then takes the full step b <- b + x (no SQP      */
/* line search: reading).                                                    */
/* stats[0] = number of lines whose QP hit its pass cap,                     */
/* stats[1] = total number of active constraints at the end,                 */
/* stats[2] = total QP passes.                                               */
/* ------------------------------------------------------------------------ */
int ref_bstep(int nd, const int* m, const double* h, int pe, const ref_params* prm,
              const double* I1, const double* I2, const double* b_in, const double* z,
              const double* u, double* b_out, long* stats) {
    grid_t g;
    int st = make_grid(nd, m, h, pe, &g);
    if (st) return st;
    set_threads(prm);
    long L = n_lines(&g), mp = g.mpe, n = mp + 1;
    double hpe = g.h[g.pe], hd = g.hd;
    long capped = 0, nact = 0, npass = 0;
    if (b_out != b_in) memcpy(b_out, b_in, sizeof(double) * (size_t)g.nf);
#pragma omp parallel reduction(+:capped, nact, npass)
    {
        cellq* q = (cellq*)malloc(sizeof(cellq) * (size_t)mp);
        double* bl = (double*)malloc(sizeof(double) * (size_t)n);
        double* Gd = (double*)malloc(sizeof(double) * (size_t)n);
        double* Go = (double*)malloc(sizeof(double) * (size_t)n);
        double* c = (double*)malloc(sizeof(double) * (size_t)n);
        double* dk = (double*)malloc(sizeof(double) * (size_t)mp);
        double* x = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(dynamic, 16)
        for (long l = 0; l < L; ++l) {
            long f0 = line_face0(&g, l), c0 = line_cell0(&g, l), s = g.n_inner;
            for (long i = 0; i < n; ++i) bl[i] = b_out[f0 + i * s];
            for (int it = 0; it < prm->n_sqp; ++it) {
                line_cells(&g, I1 + c0, I2 + c0, s, bl, 1, q, prm->knot32);
                for (long i = 0; i < n; ++i) {
                    double Jup = (i > 0) ? q[i - 1].Ju : 0.0, rup = (i > 0) ? q[i - 1].r : 0.0;
                    double Jdn = (i < mp) ? q[i].Jd : 0.0, rdn = (i < mp) ? q[i].r : 0.0;
                    double dup = (i > 0) ? q[i - 1].d : 0.0, ddn = (i < mp) ? q[i].d : 0.0;
                    double nadj = (double)((i > 0) + (i < mp));
                    Gd[i] = hd * (Jup * Jup + Jdn * Jdn) + prm->alpha * hd * nadj / (hpe * hpe) + prm->rho * hd;
                    c[i] = hd * (Jup * rup + Jdn * rdn)                      /* grad D */
                         + prm->alpha * hd * (dup - ddn) / hpe                 /* alpha h^d D1^T D1 b */
                         + prm->rho * hd * (bl[i] - z[f0 + i * s] + u[f0 + i * s]);
                    if (i < mp) Go[i] = hd * q[i].Jd * q[i].Ju - prm->alpha * hd / (hpe * hpe);
                }
                for (long j = 0; j < mp; ++j) dk[j] = q[j].d;
                int na = 0;
                int res = ref_line_qp(mp, hpe, Gd, Go, c, dk, x, &na);
                if (res < 0) capped += 1; else npass += res;
                if (it == prm->n_sqp - 1) nact += na;
                for (long i = 0; i < n; ++i) bl[i] += x[i];
            }
            for (long i = 0; i < n; ++i) b_out[f0 + i * s] = bl[i];
        }
        free(q); free(bl); free(Gd); free(Go); free(c); free(dk); free(x);
    }
    if (stats) { stats[0] = capped; stats[1] = nact; stats[2] = npass; }
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* DCT diagonalisation of the cross-line Laplacian (Sec. 4.2, Eq. dctdiag).  */
/* Reading: C(m) is the orthonormal DCT-II, C[k][j] = s_k cos(pi k (2j+1)/(2m)), */
/* s_0 = sqrt(1/m), s_k = sqrt(2/m); it diagonalises the Neumann             */
/* D~(m,h)^T D~(m,h) with eigenvalues lambda_k = 4/h^2 sin^2(pi k/(2m)).     */
/* ------------------------------------------------------------------------ */
void ref_dct_matrix(long m, double* C) {
    for (long k = 0; k < m; ++k) {
        double s = (k == 0) ? sqrt(1.0 / (double)m) : sqrt(2.0 / (double)m);
        for (long j = 0; j < m; ++j) {
            long num = (k * (2 * j + 1)) % (4 * m);   /* exact reduction of the angle */
            C[k * m + j] = s * cos(M_PI * (double)num / (2.0 * (double)m));
        }
    }
}

void ref_dct_eigs(long m, double h, double* lam) {
    for (long k = 0; k < m; ++k) {
        double s = sin(M_PI * (double)k / (2.0 * (double)m));
        lam[k] = 4.0 / (h * h) * s * s;
    }
}

/* w <- C w (or C^T w) along axis a of a face array */
static void dct_along(const grid_t* g, int a, const double* C, int transpose, double* w) {
    long len = g->F[a];
    if (len < 2) return;
    long st = (a == 0) ? g->F[1] * g->F[2] : (a == 1) ? g->F[2] : 1;
    long nlines = g->nf / len;
#pragma omp parallel
    {
        double* tin = (double*)malloc(sizeof(double) * (size_t)len);
        double* tout = (double*)malloc(sizeof(double) * (size_t)len);
#pragma omp for schedule(static)
        for (long t = 0; t < nlines; ++t) {
            long base = (t / st) * st * len + (t % st);
            for (long j = 0; j < len; ++j) tin[j] = w[base + j * st];
            for (long k = 0; k < len; ++k) {
                double acc = 0.0;
                for (long j = 0; j < len; ++j)
                    acc += (transpose ? C[j * len + k] : C[k * len + j]) * tin[j];
                tout[k] = acc;
            }
            for (long k = 0; k < len; ++k) w[base + k * st] = tout[k];
        }
        free(tin); free(tout);
    }
}

/* ADMM z-step (Sec. 4.2, Eq. admmStep2): z = Gt^{-1} rho h^d (b + u) with
   Gt = alpha h^d (D2^T D2 + D3^T D3) + rho h^d I = C^T (alpha h^d Lambda + rho h^d) C,
   i.e. z = C^T diag(rho / (alpha Lambda + rho)) C (b + u), the 2D DCT C taken
   over the non-PE axes of every PE-face slab. */
int ref_zstep(int nd, const int* m, const double* h, int pe, const ref_params* prm,
              const double* b, const double* u, double* z) {
    grid_t g;
    int st = make_grid(nd, m, h, pe, &g);
    if (st) return st;
    set_threads(prm);
    int ax[2];
    other_axes(&g, &ax[0], &ax[1]);
    double* C[2] = {NULL, NULL};
    double* lam[2] = {NULL, NULL};
    for (int k = 0; k < 2; ++k) {
        long len = g.F[ax[k]];
        C[k] = (double*)malloc(sizeof(double) * (size_t)(len * len));
        lam[k] = (double*)malloc(sizeof(double) * (size_t)len);
        ref_dct_matrix(len, C[k]);
        ref_dct_eigs(len, g.h[ax[k]], lam[k]);
        if (len < 2) lam[k][0] = 0.0;
    }
    for (long f = 0; f < g.nf; ++f) z[f] = b[f] + u[f];
    dct_along(&g, ax[0], C[0], 0, z);
    dct_along(&g, ax[1], C[1], 0, z);
    for (long f = 0; f < g.nf; ++f) {
        long i2 = f % g.F[2], i1 = (f / g.F[2]) % g.F[1], i0 = f / (g.F[1] * g.F[2]);
        long ia[3] = {i0, i1, i2};
        double L = lam[0][ia[ax[0]]] + lam[1][ia[ax[1]]];
        z[f] *= prm->rho / (prm->alpha * L + prm->rho);
    }
    dct_along(&g, ax[1], C[1], 1, z);
    dct_along(&g, ax[0], C[0], 1, z);
    for (int k = 0; k < 2; ++k) { free(C[k]); free(lam[k]); }
    return REF_OK;
}

static double norm2(long n, const double* v) {
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += v[i] * v[i];
    return sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* Corrected images and image similarity (Sec. 6, comparison of the 3D       */
/* results: SSD and NCC between the transformed blip-up and blip-down data). */
/*                                                                           */
/* The transformed images are the two terms of the residual of Eq. D:       */
/*   T1 = I_v(x + A b) .* (1 + D1 b),   T2 = I_-v(x - A b) .* (1 - D1 b).     */
/* Readings (the paper cites the measures without formulas):                 */
/*   SSD(b) = h^d / 2 |T1 - T2|^2 (the sum-of-squared-differences distance,  */
/*            the same value as D(b) of Eq. D);                              */
/*   NCC(b) = <T1, T2>^2 / (|T1|^2 |T2|^2), in [0, 1] with 1 optimal.        */
/* out[0] = SSD, out[1] = NCC; T1, T2 (cell arrays) may be NULL.            */
/* ------------------------------------------------------------------------ */
int ref_corrected(int nd, const int* m, const double* h, int pe, const double* I1, const double* I2,
                  const double* b, double* T1, double* T2, double* out) {
    grid_t g;
    int st = make_grid(nd, m, h, pe, &g);
    if (st) return st;
    long L = n_lines(&g);
    double hp = g.h[g.pe];
    double s_dd = 0.0, s_12 = 0.0, s_11 = 0.0, s_22 = 0.0;
    for (long l = 0; l < L; ++l) {
        long c0 = line_cell0(&g, l), f0 = line_face0(&g, l);
        for (long j = 0; j < g.mpe; ++j) {
            double b0 = b[f0 + j * g.n_inner], b1 = b[f0 + (j + 1) * g.n_inner];
            double a = 0.5 * (b0 + b1);       /* A1 b */
            double d = (b1 - b0) / hp;        /* D1 b */
            double v1, s1, v2, s2;
            interp_line(I1 + c0, g.n_inner, g.mpe, (double)j + a / hp, &v1, &s1);
            interp_line(I2 + c0, g.n_inner, g.mpe, (double)j - a / hp, &v2, &s2);
            double t1 = v1 * (1.0 + d), t2 = v2 * (1.0 - d);
            if (T1) T1[c0 + j * g.n_inner] = t1;
            if (T2) T2[c0 + j * g.n_inner] = t2;
            s_dd += (t1 - t2) * (t1 - t2);
            s_12 += t1 * t2;
            s_11 += t1 * t1;
            s_22 += t2 * t2;
        }
    }
    out[0] = 0.5 * g.hd * s_dd;
    out[1] = (s_11 > 0.0 && s_22 > 0.0) ? (s_12 * s_12) / (s_11 * s_22) : 0.0;
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* Multilevel strategy (Sec. 4.4): a coarse-to-fine sequence of grids, each  */
/* coarse grid with twice the spacing along every axis.  The paper defers    */
/* the transfer operators to the image registration literature; readings:   */
/*   restriction of an image: the mean of the 2^d fine cells of a coarse     */
/*     cell;                                                                 */
/*   prolongation of b (faces along the PE axis, cells across it): linear   */
/*     interpolation in every axis at the fine positions, i.e. along the PE  */
/*     axis fine face 2k = coarse face k and fine face 2k+1 = the mean of    */
/*     coarse faces k and k+1; across it fine cell 2j = 3/4 coarse cell j +  */
/*     1/4 cell j-1 and fine cell 2j+1 = 3/4 cell j + 1/4 cell j+1, the      */
/*     outside neighbour of a boundary cell replaced by the cell itself.     */
/* With these, D1 of the prolongated field repeats the coarse D1 (and is a   */
/* convex combination of coarse values across the PE axis), so a feasible    */
/* coarse field stays feasible.  m are the FINE cells (every axis even).     */
/* ------------------------------------------------------------------------ */
int ref_restrict(int nd, const int* m, const double* I, double* Ic) {
    if (nd != 2 && nd != 3) return REF_EINVAL;
    long M[3] = {m[0], m[1], nd == 3 ? m[2] : 1};
    for (int a = 0; a < nd; ++a)
        if (M[a] % 2) return REF_EINVAL;
    long C[3] = {M[0] / 2, M[1] / 2, nd == 3 ? M[2] / 2 : 1};
    double w = 1.0 / (nd == 3 ? 8.0 : 4.0);
    for (long i = 0; i < C[0]; ++i)
        for (long j = 0; j < C[1]; ++j)
            for (long k = 0; k < C[2]; ++k) {
                double s = 0.0;
                for (int di = 0; di < 2; ++di)
                    for (int dj = 0; dj < 2; ++dj)
                        for (int dk = 0; dk < (nd == 3 ? 2 : 1); ++dk)
                            s += I[((2 * i + di) * M[1] + (2 * j + dj)) * M[2] + (nd == 3 ? 2 * k + dk : 0)];
                Ic[(i * C[1] + j) * C[2] + k] = w * s;
            }
    return REF_OK;
}

/* 1D prolongation weights of fine index f along an axis of the coarse
   length n (faces along PE when face != 0): at most two coarse indices. */
static int prolong_1d(long f, long n, int face, long* idx, double* wt) {
    if (face) {
        if (f % 2 == 0) { idx[0] = f / 2; wt[0] = 1.0; return 1; }
        idx[0] = (f - 1) / 2; idx[1] = (f + 1) / 2; wt[0] = wt[1] = 0.5;
        return 2;
    }
    long j = f / 2, o = (f % 2 == 0) ? j - 1 : j + 1;
    if (o < 0) o = 0;
    if (o > n - 1) o = n - 1;
    idx[0] = j; wt[0] = 0.75;
    idx[1] = o; wt[1] = 0.25;
    return 2;
}

/* bf (fine faces) = P bc (coarse faces); m are the FINE cells */
int ref_prolong(int nd, const int* m, int pe, const double* bc, double* bf) {
    if (nd != 2 && nd != 3) return REF_EINVAL;
    if (pe < 0 || pe >= nd) return REF_EINVAL;
    long M[3] = {m[0], m[1], nd == 3 ? m[2] : 1};
    for (int a = 0; a < nd; ++a)
        if (M[a] % 2) return REF_EINVAL;
    long Cc[3], Ff[3], Fc[3];
    for (int a = 0; a < 3; ++a) {
        long c = (a < nd) ? M[a] / 2 : 1;
        Cc[a] = c;
        Fc[a] = c + (a == pe ? 1 : 0);
        Ff[a] = M[a] + (a == pe ? 1 : 0);
    }
    for (long i = 0; i < Ff[0]; ++i)
        for (long j = 0; j < Ff[1]; ++j)
            for (long k = 0; k < Ff[2]; ++k) {
                long ix[3][2];
                double wx[3][2];
                int nx[3];
                long f[3] = {i, j, k};
                for (int a = 0; a < 3; ++a) {
                    if (a >= nd) { nx[a] = 1; ix[a][0] = 0; wx[a][0] = 1.0; continue; }
                    nx[a] = prolong_1d(f[a], Cc[a], a == pe, ix[a], wx[a]);
                }
                double s = 0.0;
                for (int p = 0; p < nx[0]; ++p)
                    for (int q = 0; q < nx[1]; ++q)
                        for (int r = 0; r < nx[2]; ++r)
                            s += wx[0][p] * wx[1][q] * wx[2][r] * bc[(ix[0][p] * Fc[1] + ix[1][q]) * Fc[2] + ix[2][r]];
                bf[(i * Ff[1] + j) * Ff[2] + k] = s;
            }
    return REF_OK;
}

/* max |D1 b| over all cells (feasibility of b for the constraint set C) */
double ref_max_abs_d1(int nd, const int* m, const double* h, int pe, const double* b) {
    grid_t g;
    if (make_grid(nd, m, h, pe, &g)) return NAN;
    double mx = 0.0, hpe = g.h[g.pe];
    long L = n_lines(&g);
    for (long l = 0; l < L; ++l) {
        long f0 = line_face0(&g, l), s = g.n_inner;
        for (long j = 0; j < g.mpe; ++j) {
            double d = fabs(b[f0 + (j + 1) * s] - b[f0 + j * s]) / hpe;
            if (d > mx) mx = d;
        }
    }
    return mx;
}

/* ------------------------------------------------------------------------ */
/* ADMM (Sec. 4.2, Eqs. admmStep1-3 and admmStop).                           */
/* b: in b^0 (feasible), out final b.  z, u: in z^0, u^0, out final.         */
/* Stopping: r_pri = ||b^{k+1} - z^{k+1}||, r_dual = rho h^d ||z^k - z^{k+1}||, */
/*   eps_pri  = sqrt(n) eps_abs + eps_rel max(||b^{k+1}||, ||z^{k+1}||)       */
/*   eps_dual = sqrt(n) eps_abs + eps_rel rho h^d ||u^{k+1}||                */
/* (reading: the k+1 iterates, as in Boyd et al. (3.12)).                    */
/* hist (optional): 6 doubles per iteration:                                 */
/*   r_pri, r_dual, eps_pri, eps_dual, rho, J(b^{k+1}).                      */
/*                                                                           */
/* Augmentation parameter (Sec. 4.3, last paragraph; Sec. 6, ADMM            */
/* performance): fixed, or the adaptive choice of Boyd et al. (varying       */
/* penalty parameter), or that choice kept above a lower bound rho_min.      */
/* Readings (the paper gives no formula): after an iteration that did not    */
/* stop, rho <- tau rho when r_pri > mu r_dual, rho <- rho / tau when        */
/* r_dual > mu r_pri (with the bound: not when rho / tau < rho_min, rho then */
/* stays), else unchanged; tau = 1.3 (the factor between consecutive rho in  */
/* the paper's figure), mu = 10 (Boyd's usual value).  On a change the       */
/* scaled dual is rescaled, u <- u rho_old / rho_new, so that y = rho u is   */
/* unchanged.                                                                */
/* info[0] = iterations, info[1] = converged flag, info[2] = capped QPs.     */
/* ------------------------------------------------------------------------ */
static int admm_run(int nd, const int* m, const double* h, int pe, const ref_params* prm,
                    const double* I1, const double* I2, double* b, double* z, double* u,
                    double* hist, long* info, double* rho_final);

int ref_admm(int nd, const int* m, const double* h, int pe, const ref_params* prm,
             const double* I1, const double* I2, double* b, double* z, double* u,
             double* hist, long* info) {
    return admm_run(nd, m, h, pe, prm, I1, I2, b, z, u, hist, info, NULL);
}

/* The iteration of ref_admm; rho_final (optional) receives the augmentation
   parameter after the last iteration (adapted once more when that iteration
   did not stop). */
static int admm_run(int nd, const int* m, const double* h, int pe, const ref_params* prm,
                    const double* I1, const double* I2, double* b, double* z, double* u,
                    double* hist, long* info, double* rho_final) {
    grid_t g;
    int st = make_grid(nd, m, h, pe, &g);
    if (st) return st;
    if (ref_max_abs_d1(nd, m, h, pe, b) > 1.0) return REF_EINFEASIBLE;
    long n = g.nf;
    double* zold = (double*)malloc(sizeof(double) * (size_t)n);
    double* tmp = (double*)malloc(sizeof(double) * (size_t)n);
    long capped_total = 0;
    int conv = 0;
    long k;
    ref_params pk = *prm;   /* pk.rho: the current augmentation parameter */
    for (k = 0; k < prm->max_iter; ++k) {
        long stats[3];
        ref_bstep(nd, m, h, pe, &pk, I1, I2, b, z, u, b, stats);
        capped_total += stats[0];
        memcpy(zold, z, sizeof(double) * (size_t)n);
        ref_zstep(nd, m, h, pe, &pk, b, u, z);
        for (long f = 0; f < n; ++f) u[f] += b[f] - z[f];
        for (long f = 0; f < n; ++f) tmp[f] = b[f] - z[f];
        double rpri = norm2(n, tmp);
        for (long f = 0; f < n; ++f) tmp[f] = z[f] - zold[f];
        double rdual = pk.rho * g.hd * norm2(n, tmp);
        double nb = norm2(n, b), nz = norm2(n, z), nu = norm2(n, u);
        double epri = sqrt((double)n) * prm->eps_abs + prm->eps_rel * (nb > nz ? nb : nz);
        double edual = sqrt((double)n) * prm->eps_abs + prm->eps_rel * pk.rho * g.hd * nu;
        if (hist) {
            double obj[4];
            ref_objective(nd, m, h, pe, &pk, I1, I2, b, obj);
            double* hk = hist + 6 * k;
            hk[0] = rpri; hk[1] = rdual; hk[2] = epri; hk[3] = edual; hk[4] = pk.rho; hk[5] = obj[0];
        }
        if (rpri <= epri && rdual <= edual) { conv = 1; ++k; break; }
        if (prm->adapt_rho) {
            double rnew = pk.rho;
            if (rpri > prm->rho_mu * rdual) {
                rnew = pk.rho * prm->rho_tau;
            } else if (rdual > prm->rho_mu * rpri) {
                rnew = pk.rho / prm->rho_tau;
                if (prm->adapt_rho == 2 && rnew < prm->rho_min) rnew = pk.rho;
            }
            if (rnew != pk.rho) {
                for (long f = 0; f < n; ++f) u[f] *= pk.rho / rnew;
                pk.rho = rnew;
            }
        }
    }
    free(zold); free(tmp);
    if (info) { info[0] = k; info[1] = conv; info[2] = capped_total; }
    if (rho_final) *rho_final = pk.rho;
    return conv ? REF_OK : REF_NOTCONV;
}

/* ------------------------------------------------------------------------ */
/* Coarse-to-fine ADMM (Sec. 4.4, multilevel strategy).  The images are      */
/* restricted level by level (ref_restrict); ADMM runs from b = 0 on the     */
/* coarsest grid; every finer level starts from the third initialisation    */
/* strategy, b0 = z0 = (P b + P z) / 2 and u0 = 0, with P = ref_prolong.      */
/* Readings: z is not constrained, so when the average leaves |D1 b| <= 1    */
/* the start is P b (feasible with b); a start still outside by rounding is  */
/* scaled back onto the set; the augmentation parameter carries from level   */
/* to level (the value after the coarser level's last iteration).            */
/* m, h: the finest grid (each coarser level halves m and doubles h; every   */
/* axis must halve evenly).  Out: b, z, u on the finest grid; per level,     */
/* coarsest first, iters[l], conv[l] and the carried rho_lvl[l]; hist        */
/* (optional) the finest level's history as in ref_admm.                    */
/* ------------------------------------------------------------------------ */
int ref_multilevel_admm(int nd, const int* m, const double* h, int pe, const ref_params* prm, int levels,
                        const double* I1, const double* I2, double* b, double* z, double* u,
                        long* iters, int* conv, double* rho_lvl, double* hist) {
    if (levels < 1 || levels > 12 || (nd != 2 && nd != 3)) return REF_EINVAL;
    int M[12][3];
    double H[12][3];
    double* A[12];
    double* B[12];
    for (int a = 0; a < 3; ++a) {
        M[0][a] = (a < nd) ? m[a] : 1;
        H[0][a] = (a < nd) ? h[a] : 1.0;
    }
    for (int l = 1; l < levels; ++l)
        for (int a = 0; a < 3; ++a) {
            if (a < nd && (M[l - 1][a] % 2 || M[l - 1][a] < 2)) return REF_EINVAL;
            M[l][a] = (a < nd) ? M[l - 1][a] / 2 : 1;
            H[l][a] = (a < nd) ? 2.0 * H[l - 1][a] : 1.0;
        }
    A[0] = (double*)I1;
    B[0] = (double*)I2;
    for (int l = 1; l < levels; ++l) {
        size_t nc = (size_t)M[l][0] * M[l][1] * M[l][2];
        A[l] = (double*)malloc(sizeof(double) * nc);
        B[l] = (double*)malloc(sizeof(double) * nc);
        ref_restrict(nd, M[l - 1], A[l - 1], A[l]);
        ref_restrict(nd, M[l - 1], B[l - 1], B[l]);
    }
    double rho = prm->rho;
    double *bc = NULL, *zc = NULL;
    int st = REF_OK;
    for (int l = levels - 1; l >= 0; --l) {
        size_t nf = (size_t)(M[l][0] + (pe == 0)) * (M[l][1] + (pe == 1)) * (M[l][2] + (pe == 2));
        double* bl = (l == 0) ? b : (double*)malloc(sizeof(double) * nf);
        double* zl = (l == 0) ? z : (double*)malloc(sizeof(double) * nf);
        double* ul = (l == 0) ? u : (double*)malloc(sizeof(double) * nf);
        if (!bc) {
            memset(bl, 0, sizeof(double) * nf);
        } else {
            /* the third strategy's start */
            ref_prolong(nd, M[l], pe, bc, bl);
            ref_prolong(nd, M[l], pe, zc, zl);
            for (size_t f = 0; f < nf; ++f) zl[f] = 0.5 * (bl[f] + zl[f]);
            if (ref_max_abs_d1(nd, M[l], H[l], pe, zl) <= 1.0) memcpy(bl, zl, sizeof(double) * nf);
            double mx = ref_max_abs_d1(nd, M[l], H[l], pe, bl);
            if (mx > 1.0)
                for (size_t f = 0; f < nf; ++f) bl[f] /= mx;
            free(bc); free(zc);
        }
        memcpy(zl, bl, sizeof(double) * nf);
        memset(ul, 0, sizeof(double) * nf);
        ref_params pl = *prm;
        pl.rho = rho;
        long info[3];
        int r = admm_run(nd, M[l], H[l], pe, &pl, A[l], B[l], bl, zl, ul, l == 0 ? hist : NULL, info, &rho);
        if (r < 0 && st == REF_OK) st = r;
        iters[levels - 1 - l] = info[0];
        conv[levels - 1 - l] = (int)info[1];
        rho_lvl[levels - 1 - l] = rho;
        if (l > 0) {
            free(ul);
            bc = bl;
            zc = zl;
        }
    }
    for (int l = 1; l < levels; ++l) { free(A[l]); free(B[l]); }
    return st;
}

/* ------------------------------------------------------------------------ */
/* GN-PCG (Sec. 4.1)                                                         */
/* ------------------------------------------------------------------------ */

/* Block-Jacobi preconditioner solve (Sec. 4.1, Eq. Pblock): per line the    */
/* tridiagonal block of                                                      */
/*   P_block = H_D + alpha h^d (D1^T D1 + M) + grad^2 P + gamma I            */
/* (reading: the printed formula lacks h^3 and gamma; with them P_block is   */
/* exactly the block diagonal of H_JGN).  precond: 0 none, 1 Jacobi          */
/* (diag(H_JGN)), 2 block-Jacobi.                                            */
int ref_precond_solve(int nd, const int* m, const double* h, int pe, const ref_params* prm,
                      const double* I1, const double* I2, const double* b,
                      const double* rhs, double* out) {
    grid_t g;
    int st = make_grid(nd, m, h, pe, &g);
    if (st) return st;
    set_threads(prm);
    if (prm->precond == 0) { memcpy(out, rhs, sizeof(double) * (size_t)g.nf); return REF_OK; }
    long L = n_lines(&g), mp = g.mpe, n = mp + 1;
    double hpe = g.h[g.pe], hd = g.hd, a = prm->alpha, be = prm->beta;
#pragma omp parallel
    {
        cellq* q = (cellq*)malloc(sizeof(cellq) * (size_t)mp);
        double* Gd = (double*)malloc(sizeof(double) * (size_t)n);
        double* Go = (double*)malloc(sizeof(double) * (size_t)n);
        double* r = (double*)malloc(sizeof(double) * (size_t)n);
        double* x = (double*)malloc(sizeof(double) * (size_t)n);
        double* cp = (double*)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(static)
        for (long l = 0; l < L; ++l) {
            long f0 = line_face0(&g, l), c0 = line_cell0(&g, l), s = g.n_inner;
            line_cells(&g, I1 + c0, I2 + c0, s, b + f0, s, q, prm->knot32);
            for (long i = 0; i < n; ++i) {
                double Jup = (i > 0) ? q[i - 1].Ju : 0.0, Jdn = (i < mp) ? q[i].Jd : 0.0;
                double nadj = (double)((i > 0) + (i < mp));
                double pp = 0.0;
                if (be > 0) {
                    if (i > 0) pp += ref_d2phi(q[i - 1].d);
                    if (i < mp) pp += ref_d2phi(q[i].d);
                }
                /* diagonal of H_JGN; block-Jacobi swaps the full cross-line
                   Laplacian for its diagonal M */
                Gd[i] = hd * (Jup * Jup + Jdn * Jdn) + a * hd * nadj / (hpe * hpe)
                      + be * hd * pp / (hpe * hpe) + a * hd * M_diag(&g, f0 + i * s) + prm->gamma;
                if (i < mp) {
                    double pj = (be > 0) ? ref_d2phi(q[i].d) : 0.0;
                    Go[i] = hd * q[i].Jd * q[i].Ju - a * hd / (hpe * hpe) - be * hd * pj / (hpe * hpe);
                }
                r[i] = rhs[f0 + i * s];
            }
            if (prm->precond == 1) {
                for (long i = 0; i < n; ++i) x[i] = r[i] / Gd[i];
            } else {
                thomas(n, Gd, Go, r, x, cp);
            }
            for (long i = 0; i < n; ++i) out[f0 + i * s] = x[i];
        }
        free(q); free(Gd); free(Go); free(r); free(x); free(cp);
    }
    return REF_OK;
}

static double dot(long n, const double* a, const double* b) {
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* PCG on H_JGN(b) d = -grad (Sec. 4.1, Eq. inexactGNsolve): stop when
   ||grad + H d|| <= eta ||grad|| or after max_pcg iterations.  Starts at d = 0.
   Returns the iteration count; *relres = final relative residual. */
int ref_pcg(int nd, const int* m, const double* h, int pe, const ref_params* prm,
            const double* I1, const double* I2, const double* b, const double* grad,
            double* d, double* relres) {
    grid_t g;
    int st = make_grid(nd, m, h, pe, &g);
    if (st) return st;
    long n = g.nf;
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    double* zz = (double*)malloc(sizeof(double) * (size_t)n);
    double* p = (double*)malloc(sizeof(double) * (size_t)n);
    double* q = (double*)malloc(sizeof(double) * (size_t)n);
    for (long i = 0; i < n; ++i) { d[i] = 0.0; r[i] = -grad[i]; }
    double g0 = norm2(n, grad);
    double rel = 1.0;
    int it = 0;
    if (g0 > 0) {
        ref_precond_solve(nd, m, h, pe, prm, I1, I2, b, r, zz);
        memcpy(p, zz, sizeof(double) * (size_t)n);
        double rz = dot(n, r, zz);
        for (it = 0; it < prm->max_pcg;) {
            ref_apply(nd, m, h, pe, prm, 5, I1, I2, b, p, q);
            double al = rz / dot(n, p, q);
            for (long i = 0; i < n; ++i) { d[i] += al * p[i]; r[i] -= al * q[i]; }
            ++it;
            rel = norm2(n, r) / g0;
            if (rel <= prm->eta) break;
            ref_precond_solve(nd, m, h, pe, prm, I1, I2, b, r, zz);
            double rz2 = dot(n, r, zz);
            double be = rz2 / rz;
            rz = rz2;
            for (long i = 0; i < n; ++i) p[i] = zz[i] + be * p[i];
        }
    } else {
        rel = 0.0;
    }
    free(r); free(zz); free(p); free(q);
    if (relres) *relres = rel;
    return it;
}

/* Inexact Gauss-Newton with PCG (Sec. 4.1, Eqs. inexactGNstep and
   inexactGNsolve).  Step size (reading of "Wolfe conditions"): Armijo
   backtracking with c1 = 1e-4, halving, at most 10 trials; a trial point with
   J_GN = inf (some |D1 b| >= 1 when beta > 0) is rejected.  Stopping: if
   gn_rel_grad > 0, stop when ||grad J_GN|| <= gn_rel_grad ||grad J_GN(b^0)||;
   otherwise the three tests of Eqs. stopping1-3 with J_GN(0).  At most max_gn
   iterations.  hist (optional): 5 doubles per iteration:
   J_GN, ||grad J_GN||, PCG iterations, PCG relative residual, step length.
   info[0] = iterations, info[1] = converged flag, info[2] = total PCG its. */
int ref_gnpcg(int nd, const int* m, const double* h, int pe, const ref_params* prm,
              const double* I1, const double* I2, double* b, double* hist, long* info,
              double* J_out, double* gnorm_out) {
    grid_t g;
    int st = make_grid(nd, m, h, pe, &g);
    if (st) return st;
    long n = g.nf;
    double obj[4];
    double* grad = (double*)malloc(sizeof(double) * (size_t)n);
    double* d = (double*)malloc(sizeof(double) * (size_t)n);
    double* bt = (double*)malloc(sizeof(double) * (size_t)n);
    double* zero = (double*)calloc((size_t)n, sizeof(double));
    ref_objective(nd, m, h, pe, prm, I1, I2, zero, obj);
    double J0 = obj[0];
    ref_objective(nd, m, h, pe, prm, I1, I2, b, obj);
    double Jk = obj[0];
    int status = REF_NOTCONV;
    if (!isfinite(Jk)) { status = REF_EINFEASIBLE; }
    ref_gradient(nd, m, h, pe, prm, I1, I2, b, grad);
    double gk = norm2(n, grad), g0 = gk;
    long k = 0, pcg_total = 0;
    int conv = 0;
    if (status != REF_EINFEASIBLE) {
        for (k = 0; k < prm->max_gn;) {
            double relres = 0.0;
            int pits = ref_pcg(nd, m, h, pe, prm, I1, I2, b, grad, d, &relres);
            pcg_total += pits;
            double slope = dot(n, grad, d);
            double lam = 1.0, Jt = INFINITY;
            int ok = 0;
            for (int t = 0; t < 10; ++t) {
                for (long i = 0; i < n; ++i) bt[i] = b[i] + lam * d[i];
                ref_objective(nd, m, h, pe, prm, I1, I2, bt, obj);
                Jt = obj[0];
                if (isfinite(Jt) && Jt <= Jk + 1e-4 * lam * slope) { ok = 1; break; }
                lam *= 0.5;
            }
            if (!ok) { status = REF_ELSFAIL; break; }
            double dstep = 0.0, nbk = norm2(n, b);
            for (long i = 0; i < n; ++i) { double s = bt[i] - b[i]; dstep += s * s; }
            dstep = sqrt(dstep);
            memcpy(b, bt, sizeof(double) * (size_t)n);
            double Jprev = Jk;
            Jk = Jt;
            ref_gradient(nd, m, h, pe, prm, I1, I2, b, grad);
            gk = norm2(n, grad);
            if (hist) {
                double* hk = hist + 5 * k;
                hk[0] = Jk; hk[1] = gk; hk[2] = (double)pits; hk[3] = relres; hk[4] = lam;
            }
            ++k;
            if (prm->gn_rel_grad > 0) {
                if (gk <= prm->gn_rel_grad * g0) { conv = 1; break; }
            } else {
                int c1 = fabs(Jk - Jprev) <= prm->eps_obj * (1.0 + fabs(J0));
                int c2 = dstep <= prm->eps_iter * (1.0 + nbk);
                int c3 = gk <= prm->eps_grad * (1.0 + fabs(J0));
                if (c1 && c2 && c3) { conv = 1; break; }
            }
        }
        if (conv) status = REF_OK;
    }
    if (info) { info[0] = k; info[1] = conv; info[2] = pcg_total; }
    if (J_out) *J_out = Jk;
    if (gnorm_out) *gnorm_out = gk;
    free(grad); free(d); free(bt); free(zero);
    return status;
}
