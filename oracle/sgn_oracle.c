/*
 * Oracle for the split-form SBP semi-discretization of the 2D hyperbolized
 * Serre-Green-Naghdi equations (arXiv 2601.02540).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * CPU restatement of what the GPU library computes.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header or constant with the CUDA library.
 *
 * The same source is compiled twice:
 *   - with `real` = double           -> liboracle.so       (the reference values)
 *   - with `real` = double _Complex  -> liboracle_cplx.so  (complex-step
 *     directional derivatives, i.e. the tangent-linear model: every function
 *     below is a rational function of the state and the bathymetry, so
 *     Im f(x + i*eps*d) / eps = f'(x) d to rounding for tiny eps).
 * Build flags: -O2 -ffp-contract=off (no fused multiply-add), so every
 * expression is evaluated exactly as written, left to right.  The loops over
 * rows and nodes of the RHS and of RK4 carry OpenMP pragmas: a third build
 * with -fopenmp (liboracle_omp.so) runs them on all host cores for the timed
 * CPU baseline; every iteration is independent, so its results are those of
 * the plain build bit for bit.
 *
 * Layout: a state q holds five planes h, u, v, w, eta (in that order), each
 * plane nx*ny values with x fastest: q[f*nx*ny + j*nx + i].  The bathymetry b
 * is one plane.  Node i sits at x_i = xmin + i*dx, j at y_j = ymin + j*dy.
 *
 * Citations are to the paper's sections and equations:
 *   Sec. 4.1, eq. (sd_periodic_2D_SGN)      periodic semi-discretization
 *   Sec. 4.2, eq. (semi_2D)                 reflecting semi-discretization (SATs)
 *   Remark "Concrete SBP operators and SATs" (rem:concrete_sbp) operators, M, SATs
 *   Thm. 4.1 proof, eq. (splitcondition)    energy E and its derivatives
 *   Sec. 6, eq. (initialization)            eta = h and the initial w
 *   Sec. 6 (time integration)               adaptive third-order FSAL pair
 */
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef ORC_COMPLEX
#include <complex.h>
typedef double _Complex real;
#define ORC(name) orcc_##name
#else
typedef double real;
#define ORC(name) orc_##name
#endif

enum { BC_PERIODIC = 0, BC_REFLECTING = 1 };

/* Planted-mistake hooks for the mutation test.  They exist only in the build
 * made with -DORC_MUTABLE (never the reference build), where the test selects
 * one mistake at a time to show that the pins detect it:
 *   orc_mut_f/orc_mut_k/orc_mut_kind: term k of field f dropped (kind 0),
 *       sign-flipped (1) or halved (2);
 *   orc_mut_op: 1 one-sided boundary row with 1/(2dx), 2 periodic wrap
 *       missing at the last node, 3 SAT weight 1/dx, 4 SAT sign flipped in y,
 *       5 trapezoid end weights missing in M; in the rounding-error scale
 *       (orc_rhs_scale): 6 interior rows of |D| with 1/d instead of 1/(2d),
 *       7 one-sided rows of |D| with 1/(2d) instead of 1/d, 8 the factor
 *       (1 - eta/h) counted as 2 (1 + |eta/h|), 9 |sum of terms| instead of
 *       the sum of |terms|, 10 the u, v, w values not divided by |h|. */
#ifdef ORC_MUTABLE
int orc_mut_f = -1, orc_mut_k = -1, orc_mut_kind = 0, orc_mut_op = 0;
#define MUT_OP(n) (orc_mut_op == (n))
#else
#define MUT_OP(n) 0
#endif
enum { F_H = 0, F_U = 1, F_V = 2, F_W = 3, F_ETA = 4, NFIELD = 5 };

typedef struct {
    int nx, ny;
    double xmin, xmax, ymin, ymax;
    int bc;
    double g, lambda;
} orc_grid;

/* Grid spacing.  Periodic: nx nodes cover [xmin, xmax) and x_max is the image
 * of x_min; reflecting: both end points are nodes (Remark rem:concrete_sbp,
 * and the nodal grid of Sec. 2.2). */
void ORC(spacing)(const orc_grid* G, double* dx, double* dy)
{
    if (G->bc == BC_PERIODIC) {
        *dx = (G->xmax - G->xmin) / G->nx;
        *dy = (G->ymax - G->ymin) / G->ny;
    } else {
        *dx = (G->xmax - G->xmin) / (G->nx - 1);
        *dy = (G->ymax - G->ymin) / (G->ny - 1);
    }
}

/* Diagonal of the 1D mass matrix M (Remark rem:concrete_sbp):
 * periodic dx*diag(1,...,1); reflecting dx*diag(1/2,1,...,1,1/2). */
static double mass_1d(int bc, int i, int n, double d)
{
    if (MUT_OP(5)) return d;
    if (bc == BC_REFLECTING && (i == 0 || i == n - 1)) return 0.5 * d;
    return d;
}

/* 2D mass matrix M = M_x (x) M_y, entry for node (i, j). */
double ORC(mass_weight)(const orc_grid* G, int i, int j)
{
    double dx, dy;
    ORC(spacing)(G, &dx, &dy);
    return mass_1d(G->bc, i, G->nx, dx) * mass_1d(G->bc, j, G->ny, dy);
}

/* First-derivative SBP operator along one direction of a 1D line of n values
 * spaced s apart in memory (Remark rem:concrete_sbp).
 * Periodic: (f[k+1] - f[k-1]) / (2 d), indices modulo n.
 * Reflecting: the same central stencil in the interior, and the one-sided
 * rows (f[1] - f[0]) / d at k = 0 and (f[n-1] - f[n-2]) / d at k = n-1. */
static void sbp_line(int bc, int n, double d, const real* f, long s, real* out)
{
    for (int k = 0; k < n; k++) {
        real val;
        if (bc == BC_PERIODIC) {
            int kp = (k + 1) % n;
            int km = (k - 1 + n) % n;
            if (MUT_OP(2) && k == n - 1) kp = k;
            val = (f[kp * s] - f[km * s]) / (2.0 * d);
        } else if (k == 0) {
            val = (f[1 * s] - f[0]) / d;
            if (MUT_OP(1)) val = (f[1 * s] - f[0]) / (2.0 * d);
        } else if (k == n - 1) {
            val = (f[(n - 1) * s] - f[(n - 2) * s]) / d;
        } else {
            val = (f[(k + 1) * s] - f[(k - 1) * s]) / (2.0 * d);
        }
        out[k * s] = val;
    }
}

/* D_x = D (x) I: the 1D operator applied along every row (fixed j). */
void ORC(dx_apply)(const orc_grid* G, const real* f, real* out)
{
    double dx, dy;
    ORC(spacing)(G, &dx, &dy);
#pragma omp parallel for
    for (int j = 0; j < G->ny; j++)
        sbp_line(G->bc, G->nx, dx, f + (long)j * G->nx, 1, out + (long)j * G->nx);
}

/* D_y = I (x) D: the 1D operator applied along every column (fixed i). */
void ORC(dy_apply)(const orc_grid* G, const real* f, real* out)
{
    double dx, dy;
    ORC(spacing)(G, &dx, &dy);
#pragma omp parallel for
    for (int i = 0; i < G->nx; i++)
        sbp_line(G->bc, G->ny, dy, f + i, G->nx, out + i);
}

#ifndef ORC_COMPLEX
/* |D| |f| along one line: the SBP operator with each entry replaced by its
 * absolute value, applied to |f|, i.e. the magnitude of the two operands each
 * difference subtracts.  Used only for the rounding-error scale. */
static void sbp_line_abs(int bc, int n, double d, const real* f, long s, real* out)
{
    for (int k = 0; k < n; k++) {
        real val;
        const double ci = MUT_OP(6) ? 1.0 / d : 1.0 / (2.0 * d);   /* central rows */
        const double cb = MUT_OP(7) ? 1.0 / (2.0 * d) : 1.0 / d;   /* one-sided rows */
        if (bc == BC_PERIODIC) {
            int kp = (k + 1) % n;
            int km = (k - 1 + n) % n;
            val = (fabs(f[kp * s]) + fabs(f[km * s])) * ci;
        } else if (k == 0) {
            val = (fabs(f[1 * s]) + fabs(f[0])) * cb;
        } else if (k == n - 1) {
            val = (fabs(f[(n - 1) * s]) + fabs(f[(n - 2) * s])) * cb;
        } else {
            val = (fabs(f[(k + 1) * s]) + fabs(f[(k - 1) * s])) * ci;
        }
        out[k * s] = val;
    }
}
#endif

/* Derivatives needed by the right-hand side: the twelve D_x and twelve D_y
 * operands of eqs. (sd_periodic_2D_SGN) / (semi_2D), each as a full plane. */
enum {
    P_H, P_U, P_V, P_W, P_ETA, P_B,
    P_HS,      /* h (h + b)     */
    P_UU,      /* u^2           */
    P_VV,      /* v^2           */
    P_HU,      /* h u           */
    P_HV,      /* h v           */
    P_HUV,     /* h u v         */
    P_HUW,     /* h u w         */
    P_HVW,     /* h v w         */
    P_E2H,     /* eta^2 / h     */
    NPROD
};

typedef struct {
    long n;
    real* dx[NPROD];
    real* dy[NPROD];
    real* buf;
} derivs;

/* absval = 1 (real build only): |D| |product| instead of D product. */
static int derivs_compute(const orc_grid* G, const real* b, const real* q, derivs* D, int absval)
{
    long n = (long)G->nx * G->ny;
    D->n = n;
    D->buf = (real*)malloc(sizeof(real) * n * (2 * NPROD + 1));
    if (!D->buf) return -1;
    real* prod = D->buf + 2 * NPROD * n;
    const real* h = q + F_H * n;
    const real* u = q + F_U * n;
    const real* v = q + F_V * n;
    const real* w = q + F_W * n;
    const real* eta = q + F_ETA * n;
    for (int p = 0; p < NPROD; p++) {
        D->dx[p] = D->buf + (2 * p) * n;
        D->dy[p] = D->buf + (2 * p + 1) * n;
#pragma omp parallel for
        for (long c = 0; c < n; c++) {
            real val;
            switch (p) {
            case P_H:   val = h[c]; break;
            case P_U:   val = u[c]; break;
            case P_V:   val = v[c]; break;
            case P_W:   val = w[c]; break;
            case P_ETA: val = eta[c]; break;
            case P_B:   val = b[c]; break;
            case P_HS:  val = h[c] * (h[c] + b[c]); break;
            case P_UU:  val = u[c] * u[c]; break;
            case P_VV:  val = v[c] * v[c]; break;
            case P_HU:  val = h[c] * u[c]; break;
            case P_HV:  val = h[c] * v[c]; break;
            case P_HUV: val = h[c] * u[c] * v[c]; break;
            case P_HUW: val = h[c] * u[c] * w[c]; break;
            case P_HVW: val = h[c] * v[c] * w[c]; break;
            default:    val = eta[c] * eta[c] / h[c]; break; /* P_E2H */
            }
            prod[c] = val;
        }
#ifndef ORC_COMPLEX
        if (absval) {
            double dx, dy;
            ORC(spacing)(G, &dx, &dy);
            for (int j = 0; j < G->ny; j++)
                sbp_line_abs(G->bc, G->nx, dx, prod + (long)j * G->nx, 1, D->dx[p] + (long)j * G->nx);
            for (int i = 0; i < G->nx; i++)
                sbp_line_abs(G->bc, G->ny, dy, prod + i, G->nx, D->dy[p] + i);
            continue;
        }
#endif
        (void)absval;
        ORC(dx_apply)(G, prod, D->dx[p]);
        ORC(dy_apply)(G, prod, D->dy[p]);
    }
    return 0;
}

/* The individual terms of each equation at one node, in the order printed in
 * eqs. (sd_periodic_2D_SGN) / (semi_2D).  For h, u, v, w the terms are those
 * of the left-hand side (the time derivative moved aside); the caller combines
 * them.  Returned counts: nt[f] terms for field f. */
#define MAXTERMS 16
typedef struct {
    int nt[NFIELD];
    real t[NFIELD][MAXTERMS];
} node_terms;

static void terms_at(const orc_grid* G, const real* b, const real* q, const derivs* D,
                     long c, int i, int j, node_terms* T)
{
    const long n = D->n;
    const double g = G->g, lam = G->lambda;
    const real h = q[F_H * n + c], u = q[F_U * n + c], v = q[F_V * n + c];
    const real w = q[F_W * n + c], eta = q[F_ETA * n + c], bb = b[c];
    (void)bb;
#define DX(p) (D->dx[p][c])
#define DY(p) (D->dy[p][c])
    int k;

    /* h equation: h_t + u D_x h + h D_x u + v D_y h + h D_y v - SAT = 0 */
    k = 0;
    T->t[F_H][k++] = u * DX(P_H);
    T->t[F_H][k++] = h * DX(P_U);
    T->t[F_H][k++] = v * DY(P_H);
    T->t[F_H][k++] = h * DY(P_V);
    if (G->bc == BC_REFLECTING) {
        /* -M^{-1} R^T B N_x R (h u) - M^{-1} R^T B N_y R (h v), evaluated as in
         * Remark rem:concrete_sbp; corners receive both contributions. */
        double dx, dy;
        ORC(spacing)(G, &dx, &dy);
        real satx = 0.0, saty = 0.0;
        if (MUT_OP(3)) dx = 2.0 * dx;
        if (MUT_OP(4)) dy = -dy;
        if (i == 0) satx = -(2.0 / dx) * (h * u);
        if (i == G->nx - 1) satx = (2.0 / dx) * (h * u);
        if (j == 0) saty = -(2.0 / dy) * (h * v);
        if (j == G->ny - 1) saty = (2.0 / dy) * (h * v);
        T->t[F_H][k++] = -satx;
        T->t[F_H][k++] = -saty;
    }
    T->nt[F_H] = k;

    /* h u_t + [these terms] = 0 */
    k = 0;
    T->t[F_U][k++] = g * DX(P_HS);
    T->t[F_U][k++] = -g * (h + bb) * DX(P_H);
    T->t[F_U][k++] = 0.5 * h * DX(P_UU);
    T->t[F_U][k++] = -0.5 * (u * u) * DX(P_H);
    T->t[F_U][k++] = 0.5 * u * DX(P_HU);
    T->t[F_U][k++] = -0.5 * (h * u) * DX(P_U);
    T->t[F_U][k++] = 0.5 * DY(P_HUV);
    T->t[F_U][k++] = -0.5 * (u * v) * DY(P_H);
    T->t[F_U][k++] = 0.5 * (h * v) * DY(P_U);
    T->t[F_U][k++] = -0.5 * (h * u) * DY(P_V);
    T->t[F_U][k++] = (lam / 6.0) * (eta * eta / (h * h)) * DX(P_H);
    T->t[F_U][k++] = (lam / 3.0) * DX(P_ETA);
    T->t[F_U][k++] = -(lam / 3.0) * (eta / h) * DX(P_ETA);
    T->t[F_U][k++] = -(lam / 6.0) * DX(P_E2H);
    T->t[F_U][k++] = (lam / 2.0) * (1.0 - eta / h) * DX(P_B);
    T->nt[F_U] = k;

    /* h v_t + [these terms] = 0 */
    k = 0;
    T->t[F_V][k++] = g * DY(P_HS);
    T->t[F_V][k++] = -g * (h + bb) * DY(P_H);
    T->t[F_V][k++] = 0.5 * h * DY(P_VV);
    T->t[F_V][k++] = -0.5 * (v * v) * DY(P_H);
    T->t[F_V][k++] = 0.5 * v * DY(P_HV);
    T->t[F_V][k++] = -0.5 * (h * v) * DY(P_V);
    T->t[F_V][k++] = 0.5 * DX(P_HUV);
    T->t[F_V][k++] = -0.5 * (u * v) * DX(P_H);
    T->t[F_V][k++] = 0.5 * (h * u) * DX(P_V);
    T->t[F_V][k++] = -0.5 * (h * v) * DX(P_U);
    T->t[F_V][k++] = (lam / 6.0) * (eta * eta / (h * h)) * DY(P_H);
    T->t[F_V][k++] = (lam / 3.0) * DY(P_ETA);
    T->t[F_V][k++] = -(lam / 3.0) * (eta / h) * DY(P_ETA);
    T->t[F_V][k++] = -(lam / 6.0) * DY(P_E2H);
    T->t[F_V][k++] = (lam / 2.0) * (1.0 - eta / h) * DY(P_B);
    T->nt[F_V] = k;

    /* h w_t + [these terms] = lambda (1 - eta/h); the source is stored as the
     * last term with its sign flipped so that all terms share one convention. */
    k = 0;
    T->t[F_W][k++] = 0.5 * DX(P_HUW);
    T->t[F_W][k++] = 0.5 * (h * u) * DX(P_W);
    T->t[F_W][k++] = -0.5 * (u * w) * DX(P_H);
    T->t[F_W][k++] = -0.5 * (h * w) * DX(P_U);
    T->t[F_W][k++] = 0.5 * DY(P_HVW);
    T->t[F_W][k++] = 0.5 * (h * v) * DY(P_W);
    T->t[F_W][k++] = -0.5 * (v * w) * DY(P_H);
    T->t[F_W][k++] = -0.5 * (h * w) * DY(P_V);
    T->t[F_W][k++] = -lam * (1.0 - eta / h);
    T->nt[F_W] = k;

    /* eta_t + [these terms] = 0, with the source w stored as -w */
    k = 0;
    T->t[F_ETA][k++] = u * DX(P_ETA);
    T->t[F_ETA][k++] = v * DY(P_ETA);
    T->t[F_ETA][k++] = 1.5 * u * DX(P_B);
    T->t[F_ETA][k++] = 1.5 * v * DY(P_B);
    T->t[F_ETA][k++] = -w;
    T->nt[F_ETA] = k;
#undef DX
#undef DY
#ifdef ORC_MUTABLE
    if (orc_mut_f >= 0 && orc_mut_k < T->nt[orc_mut_f]) {
        real* tm = &T->t[orc_mut_f][orc_mut_k];
        *tm = orc_mut_kind == 0 ? 0.0 : (orc_mut_kind == 1 ? -*tm : 0.5 * *tm);
    }
#endif
}

/* Right-hand side dq/dt of eq. (sd_periodic_2D_SGN) (periodic) or eq.
 * (semi_2D) (reflecting).  The h and eta equations give the time derivative
 * directly; the u, v, w equations give h times it, so their sums are divided
 * by h.  Returns 0, or -1 when out of memory. */
int ORC(rhs)(const orc_grid* G, const real* b, const real* q, real* dq)
{
    derivs D;
    if (derivs_compute(G, b, q, &D, 0)) return -1;
    const long n = D.n;
#pragma omp parallel for
    for (int j = 0; j < G->ny; j++)
        for (int i = 0; i < G->nx; i++) {
            long c = (long)j * G->nx + i;
            node_terms T;
            terms_at(G, b, q, &D, c, i, j, &T);
            const real h = q[F_H * n + c];
            for (int f = 0; f < NFIELD; f++) {
                real s = 0.0;
                for (int k = 0; k < T.nt[f]; k++) s = s + T.t[f][k];
                real val = -s;
                if (f == F_U || f == F_V || f == F_W) val = val / h;
                dq[f * n + c] = val;
            }
        }
    free(D.buf);
    return 0;
}

#ifndef ORC_COMPLEX
/* Rounding-error scale of each RHS value (forward error bound): every term
 * coef * D f is replaced by |coef| * |D| |f| (the size of the operands the
 * difference subtracts, not the size of the difference), pointwise terms by
 * their absolute value, and the factor (1 - eta/h) by 1 + |eta/h| (it is itself
 * a difference of two O(1) numbers); the terms are then summed (and divided by
 * |h| where the RHS is).  Any evaluation of the RHS in a precision with unit
 * round-off u carries an error of a small multiple of u times this scale, so
 * the parity tolerances are stated with it. */
int orc_rhs_scale(const orc_grid* G, const real* b, const real* q, real* scale)
{
    derivs D;
    if (derivs_compute(G, b, q, &D, 1)) return -1;
    const long n = D.n;
    for (int j = 0; j < G->ny; j++)
        for (int i = 0; i < G->nx; i++) {
            long c = (long)j * G->nx + i;
            node_terms T;
            terms_at(G, b, q, &D, c, i, j, &T);
            const real h = q[F_H * n + c];
            /* The factor (1 - eta/h) in the last term of the u and v
             * equations and in the source of the w equation is itself a
             * difference of two O(1) numbers: its rounding error scales with
             * 1 + |eta/h|, not with its (possibly tiny) value. */
            const real rho = fabs(q[F_ETA * n + c] / h);
            const real one_rho = MUT_OP(8) ? 2.0 * (1.0 + rho) : 1.0 + rho;
            T.t[F_U][14] = (G->lambda / 2.0) * one_rho * D.dx[P_B][c];
            T.t[F_V][14] = (G->lambda / 2.0) * one_rho * D.dy[P_B][c];
            T.t[F_W][8] = G->lambda * one_rho;
            for (int f = 0; f < NFIELD; f++) {
                real s = 0.0;
                for (int k = 0; k < T.nt[f]; k++) s += MUT_OP(9) ? T.t[f][k] : fabs(T.t[f][k]);
                if (MUT_OP(9)) s = fabs(s);
                if ((f == F_U || f == F_V || f == F_W) && !MUT_OP(10)) s = s / fabs(h);
                scale[f * n + c] = s;
            }
        }
    free(D.buf);
    return 0;
}
#endif

/* Initialization of the auxiliary variables, eq. (initialization):
 * eta = h, w = -h (D_x u + D_y v) + 3/2 (u D_x b + v D_y b). */
int ORC(init_aux)(const orc_grid* G, const real* b, real* q)
{
    const long n = (long)G->nx * G->ny;
    real* tmp = (real*)malloc(sizeof(real) * n * 4);
    if (!tmp) return -1;
    real *dxu = tmp, *dyv = tmp + n, *dxb = tmp + 2 * n, *dyb = tmp + 3 * n;
    ORC(dx_apply)(G, q + F_U * n, dxu);
    ORC(dy_apply)(G, q + F_V * n, dyv);
    ORC(dx_apply)(G, b, dxb);
    ORC(dy_apply)(G, b, dyb);
    for (long c = 0; c < n; c++) {
        const real h = q[F_H * n + c], u = q[F_U * n + c], v = q[F_V * n + c];
        q[F_ETA * n + c] = h;
        q[F_W * n + c] = -h * (dxu[c] + dyv[c]) + 1.5 * (u * dxb[c] + v * dyb[c]);
    }
    free(tmp);
    return 0;
}

/* Classical fourth-order Runge-Kutta, fixed step dt, nsteps steps, in place:
 * k1 = f(q), k2 = f(q + dt/2 k1), k3 = f(q + dt/2 k2), k4 = f(q + dt k3),
 * q <- q + dt/6 (k1 + 2 k2 + 2 k3 + k4). */
int ORC(rk4)(const orc_grid* G, const real* b, real* q, double dt, int nsteps)
{
    const long m = (long)NFIELD * G->nx * G->ny;
    real* buf = (real*)malloc(sizeof(real) * m * 5);
    if (!buf) return -1;
    real *k1 = buf, *k2 = buf + m, *k3 = buf + 2 * m, *k4 = buf + 3 * m, *y = buf + 4 * m;
    int rc = 0;
    for (int s = 0; s < nsteps && rc == 0; s++) {
        rc |= ORC(rhs)(G, b, q, k1);
#pragma omp parallel for
        for (long c = 0; c < m; c++) y[c] = q[c] + (dt / 2.0) * k1[c];
        rc |= ORC(rhs)(G, b, y, k2);
#pragma omp parallel for
        for (long c = 0; c < m; c++) y[c] = q[c] + (dt / 2.0) * k2[c];
        rc |= ORC(rhs)(G, b, y, k3);
#pragma omp parallel for
        for (long c = 0; c < m; c++) y[c] = q[c] + dt * k3[c];
        rc |= ORC(rhs)(G, b, y, k4);
#pragma omp parallel for
        for (long c = 0; c < m; c++)
            q[c] = q[c] + (dt / 6.0) * (k1[c] + 2.0 * k2[c] + 2.0 * k3[c] + k4[c]);
    }
    free(buf);
    return rc;
}

/* Pointwise energy of Thm. 4.1:
 * E = h ((u^2 + v^2)/2 + w^2/6 + g/2 (h + 2 b) + lambda/6 (eta/h - 1)^2). */
static real energy_density(double g, double lam, real h, real u, real v, real w, real eta, real b)
{
    real r = eta / h - 1.0;
    return h * ((u * u + v * v) / 2.0 + w * w / 6.0 + (g / 2.0) * (h + 2.0 * b) + (lam / 6.0) * r * r);
}

/* Total energy 1^T M E (plain left-to-right sum; the complex build gives its
 * directional derivative by complex step).  Result written to *out. */
void ORC(energy_total)(const orc_grid* G, const real* b, const real* q, real* out)
{
    const long n = (long)G->nx * G->ny;
    real s = 0.0;
    for (int j = 0; j < G->ny; j++)
        for (int i = 0; i < G->nx; i++) {
            long c = (long)j * G->nx + i;
            real e = energy_density(G->g, G->lambda, q[F_H * n + c], q[F_U * n + c], q[F_V * n + c],
                                    q[F_W * n + c], q[F_ETA * n + c], b[c]);
            s += ORC(mass_weight)(G, i, j) * e;
        }
    *out = s;
}

/* Gauge recording and gauge-misfit loss for the inversion problem: run nsteps
 * RK4 steps from q0 (copied), and every `every` steps read h at `ng` gauge
 * nodes (flat node indices).  record: writes them to out[(k-1)*ng + g];
 * loss: returns sum over k, g of (h - obs)^2. */
int ORC(gauge_run)(const orc_grid* G, const real* b, const real* q0, double dt, int nsteps,
                   int every, int ng, const long* gauge, const double* obs, real* out, real* loss)
{
    const long m = (long)NFIELD * G->nx * G->ny;
    real* q = (real*)malloc(sizeof(real) * m);
    if (!q) return -1;
    memcpy(q, q0, sizeof(real) * m);
    real acc = 0.0;
    int rc = 0;
    for (int k = 1; every * k <= nsteps && rc == 0; k++) {
        rc |= ORC(rk4)(G, b, q, dt, every);
        for (int gi = 0; gi < ng; gi++) {
            real hv = q[F_H * (long)G->nx * G->ny + gauge[gi]];
            if (out) out[(long)(k - 1) * ng + gi] = hv;
            if (obs) {
                real d = hv - obs[(long)(k - 1) * ng + gi];
                acc += d * d;
            }
        }
    }
    if (loss) *loss = acc;
    free(q);
    return rc;
}

/* Energy rate along a direction d: sum over nodes of M * (d_q E . d), with the
 * derivatives of E listed after eq. (splitcondition):
 *   dE/dh = u^2/2 + v^2/2 + w^2/6 + g h + g b + lambda/6 (1 - eta^2/h^2),
 *   dE/du = h u,  dE/dv = h v,  dE/dw = h w / 3,  dE/deta = -lambda/3 (1 - eta/h).
 * Plain left-to-right sum; result written to *out. */
void ORC(energy_rate)(const orc_grid* G, const real* b, const real* q, const real* d, real* out)
{
    const long n = (long)G->nx * G->ny;
    const double g = G->g, lam = G->lambda;
    real s = 0.0;
    for (int j = 0; j < G->ny; j++)
        for (int i = 0; i < G->nx; i++) {
            long c = (long)j * G->nx + i;
            real h = q[F_H * n + c], u = q[F_U * n + c], v = q[F_V * n + c];
            real w = q[F_W * n + c], eta = q[F_ETA * n + c], bb = b[c];
            real dEh = 0.5 * u * u + 0.5 * v * v + w * w / 6.0 + g * h + g * bb
                     + (lam / 6.0) * (1.0 - eta * eta / (h * h));
            real r = dEh * d[F_H * n + c] + (h * u) * d[F_U * n + c] + (h * v) * d[F_V * n + c]
                   + (h * w / 3.0) * d[F_W * n + c] - (lam / 3.0) * (1.0 - eta / h) * d[F_ETA * n + c];
            s += ORC(mass_weight)(G, i, j) * r;
        }
    *out = s;
}

#ifndef ORC_COMPLEX
/* Neumaier-compensated running sum. */
typedef struct { double s, c; } csum;
static void csum_add(csum* a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

/* Diagnostics (Thm. 4.1 / 4.2 and eq. (splitcondition)), compensated sums:
 *   out[0] = 1^T M h                            total mass
 *   out[1] = 1^T M E                            total energy
 *   out[2] = 1^T M E',  E' = E + g b^2 / 2      the same energy shifted by a
 *            time-independent constant: h(u^2+v^2)/2 + h w^2/6 + g/2 (h+b)^2
 *            + lambda h/6 (eta/h - 1)^2
 *   out[3] = <d_q E, dq/dt>_M                   semi-discrete energy rate
 *   out[4] = sum M sum_k |d_{q_k} E| * scale_k  magnitude scale of out[3]
 *            (scale_k = orc_rhs_scale), bounding its rounding error. */
int orc_diagnostics(const orc_grid* G, const double* b, const double* q, double* out)
{
    const long n = (long)G->nx * G->ny;
    double* dq = (double*)malloc(sizeof(double) * n * NFIELD * 2);
    if (!dq) return -1;
    double* sc = dq + n * NFIELD;
    if (orc_rhs(G, b, q, dq) || orc_rhs_scale(G, b, q, sc)) { free(dq); return -1; }
    const double g = G->g, lam = G->lambda;
    csum mass = {0, 0}, en = {0, 0}, en2 = {0, 0}, rate = {0, 0}, rsc = {0, 0};
    for (int j = 0; j < G->ny; j++)
        for (int i = 0; i < G->nx; i++) {
            long c = (long)j * G->nx + i;
            double M = orc_mass_weight(G, i, j);
            double h = q[F_H * n + c], u = q[F_U * n + c], v = q[F_V * n + c];
            double w = q[F_W * n + c], eta = q[F_ETA * n + c], bb = b[c];
            double rho = eta / h;
            csum_add(&mass, M * h);
            csum_add(&en, M * energy_density(g, lam, h, u, v, w, eta, bb));
            double e2 = h * (u * u + v * v) / 2.0 + h * w * w / 6.0 + (g / 2.0) * (h + bb) * (h + bb)
                      + (lam / 6.0) * h * (rho - 1.0) * (rho - 1.0);
            csum_add(&en2, M * e2);
            /* derivatives of E, as listed after eq. (splitcondition) */
            double dEh = 0.5 * u * u + 0.5 * v * v + w * w / 6.0 + g * h + g * bb
                       + (lam / 6.0) * (1.0 - eta * eta / (h * h));
            double dEu = h * u, dEv = h * v, dEw = h * w / 3.0;
            double dEeta = -(lam / 3.0) * (1.0 - eta / h);
            double r = dEh * dq[F_H * n + c] + dEu * dq[F_U * n + c] + dEv * dq[F_V * n + c]
                     + dEw * dq[F_W * n + c] + dEeta * dq[F_ETA * n + c];
            csum_add(&rate, M * r);
            double s = fabs(dEh) * sc[F_H * n + c] + fabs(dEu) * sc[F_U * n + c]
                     + fabs(dEv) * sc[F_V * n + c] + fabs(dEw) * sc[F_W * n + c]
                     + fabs(dEeta) * sc[F_ETA * n + c];
            csum_add(&rsc, M * s);
        }
    out[0] = mass.s + mass.c;
    out[1] = en.s + en.c;
    out[2] = en2.s + en2.c;
    out[3] = rate.s + rate.c;
    out[4] = rsc.s + rsc.c;
    free(dq);
    return 0;
}
#endif

/* ---- Adaptive time stepping (Sec. 6) -------------------------------------
 * The paper integrates the semi-discretization with an explicit third-order
 * Runge-Kutta pair that has the first-same-as-last (FSAL) property, an
 * embedded error estimator and automatic step-size control, with relative and
 * absolute tolerances 1e-6; it does not print the pair's coefficients.  The
 * pair restated here is the third-order FSAL pair of Bogacki and Shampine
 * (1989) with its embedded second-order solution:
 *   k1 = f(q_n)                      (the k4 of the previous accepted step)
 *   k2 = f(q_n + dt (1/2) k1)
 *   k3 = f(q_n + dt (3/4) k2)
 *   q_{n+1} = q_n + dt (2/9 k1 + 1/3 k2 + 4/9 k3)
 *   k4 = f(q_{n+1})
 *   qhat_{n+1} = q_n + dt (7/24 k1 + 1/4 k2 + 1/3 k3 + 1/8 k4)
 *   e = q_{n+1} - qhat_{n+1} = dt sum_i (b_i - bhat_i) k_i
 * Error of an attempt (root-mean-square over all 5 nx ny values):
 *   err = sqrt( mean( (e / (atol + rtol max(|q_n|, |q_{n+1}|)))^2 ) ).
 * Control: accept when err <= 1; the next step size is
 *   dt * min(QMAX, max(QMIN, SAFETY err^(-1/3)))     (QMAX when err = 0)
 * with SAFETY = 0.9, QMIN = 0.2, QMAX = 10; a rejected attempt is retried
 * from q_n (k1 is kept).  A step that would pass t_end is cut to land on it. */
#ifndef ORC_COMPLEX
static const double BS_B[4] = {2.0 / 9.0, 1.0 / 3.0, 4.0 / 9.0, 0.0};
static const double BS_BHAT[4] = {7.0 / 24.0, 1.0 / 4.0, 1.0 / 3.0, 1.0 / 8.0};
#define BS_SAFETY 0.9
#define BS_QMIN 0.2
#define BS_QMAX 10.0

/* One attempt of size dt from q (with k1 = f(q)): writes q1 = q_{n+1},
 * k4 = f(q1) and the error vector e; returns err (or -1 on failure).
 * work holds 3 * m values. */
static double bs3_attempt(const orc_grid* G, const double* b, const double* q, const double* k1,
                          double dt, double rtol, double atol, double* q1, double* k4, double* e,
                          double* work)
{
    const long m = (long)NFIELD * G->nx * G->ny;
    double *k2 = work, *k3 = work + m, *y = work + 2 * m;
    for (long c = 0; c < m; c++) y[c] = q[c] + dt * (0.5 * k1[c]);
    if (orc_rhs(G, b, y, k2)) return -1.0;
    for (long c = 0; c < m; c++) y[c] = q[c] + dt * (0.75 * k2[c]);
    if (orc_rhs(G, b, y, k3)) return -1.0;
    for (long c = 0; c < m; c++)
        q1[c] = q[c] + dt * (BS_B[0] * k1[c] + BS_B[1] * k2[c] + BS_B[2] * k3[c]);
    if (orc_rhs(G, b, q1, k4)) return -1.0;
    double s = 0.0;
    for (long c = 0; c < m; c++) {
        e[c] = dt * ((BS_B[0] - BS_BHAT[0]) * k1[c] + (BS_B[1] - BS_BHAT[1]) * k2[c]
                     + (BS_B[2] - BS_BHAT[2]) * k3[c] + (BS_B[3] - BS_BHAT[3]) * k4[c]);
        double sc = atol + rtol * fmax(fabs(q[c]), fabs(q1[c]));
        double r = e[c] / sc;
        s += r * r;
    }
    return sqrt(s / (double)m);
}

/* Fixed step size dt for nsteps steps (every step accepted), in place.  If
 * e_last is not NULL it receives the error vector e of the last step. */
int orc_bs3_fixed(const orc_grid* G, const double* b, double* q, double dt, int nsteps, double* e_last)
{
    const long m = (long)NFIELD * G->nx * G->ny;
    double* buf = (double*)malloc(sizeof(double) * m * 7);
    if (!buf) return -1;
    double *k1 = buf, *k4 = buf + m, *q1 = buf + 2 * m, *e = buf + 3 * m, *work = buf + 4 * m;
    int rc = orc_rhs(G, b, q, k1);
    for (int n = 0; n < nsteps && rc == 0; n++) {
        if (bs3_attempt(G, b, q, k1, dt, 1.0, 1.0, q1, k4, e, work) < 0.0) { rc = -1; break; }
        memcpy(q, q1, sizeof(double) * m);
        memcpy(k1, k4, sizeof(double) * m);
        if (e_last) memcpy(e_last, e, sizeof(double) * m);
    }
    free(buf);
    return rc;
}

/* Adaptive integration of q (in place) from t0 to t_end, first attempt dt0,
 * at most max_attempts attempts.  hist (if not NULL) receives per attempt
 * {dt, err, accepted}.  stats: {accepted, rejected, t reached, next dt}.
 * Returns the number of attempts, or -1 on failure. */
int orc_rk_adaptive(const orc_grid* G, const double* b, double* q, double t0, double t_end,
                    double dt0, double rtol, double atol, int max_attempts, double* hist, double* stats)
{
    const long m = (long)NFIELD * G->nx * G->ny;
    double* buf = (double*)malloc(sizeof(double) * m * 7);
    if (!buf) return -1;
    double *k1 = buf, *k4 = buf + m, *q1 = buf + 2 * m, *e = buf + 3 * m, *work = buf + 4 * m;
    if (orc_rhs(G, b, q, k1)) { free(buf); return -1; }
    double t = t0, dt = dt0;
    int acc = 0, rej = 0, n = 0;
    while (t < t_end && n < max_attempts) {
        const int last = dt >= t_end - t;
        const double h = last ? t_end - t : dt;
        const double err = bs3_attempt(G, b, q, k1, h, rtol, atol, q1, k4, e, work);
        if (err < 0.0) { free(buf); return -1; }
        const int ok = err <= 1.0;
        const double fac = err == 0.0 ? BS_QMAX
                                      : fmin(BS_QMAX, fmax(BS_QMIN, BS_SAFETY * pow(err, -1.0 / 3.0)));
        if (hist) {
            hist[3 * n] = h;
            hist[3 * n + 1] = err;
            hist[3 * n + 2] = ok;
        }
        if (ok) {
            memcpy(q, q1, sizeof(double) * m);
            memcpy(k1, k4, sizeof(double) * m);
            t = last ? t_end : t + h;
            acc++;
        } else {
            rej++;
        }
        dt = h * fac;
        n++;
    }
    stats[0] = acc;
    stats[1] = rej;
    stats[2] = t;
    stats[3] = dt;
    free(buf);
    return n;
}

/* ---- The five-stage third-order FSAL pair (Sec. 6) ------------------------
 * Sec. 6 integrates with an explicit third-order, five-stage Runge-Kutta
 * method with the FSAL property and an embedded error estimator, optimized
 * for stability-limited discretizations of hyperbolic problems; the paper
 * does not print its coefficients.  The pair below has exactly these
 * properties; its coefficients were constructed to them here:
 *  - stability polynomial R(z) = 1 + z + z^2/2 + z^3/6 + 0.0324 z^4 + 0.006 z^5
 *    (|R(iy)| <= 1 for |y| <= 3.8798: the central SBP operators give an
 *    imaginary spectrum; classical RK4 reaches 2.83 with four stages);
 *  - Butcher matrix of the two-register form a_ij = b_j for j < i - 1, with
 *    a21 = 0.3464, a32 = 0.5544, a43 = 0.3078 and a54, b1..b5 the solution of
 *    the four third-order conditions and the two stability coefficients;
 *  - embedded weights bhat over k1..k5 and k6 = f(q_{n+1}) (FSAL), order 2,
 *    with bhat3..bhat6 = 0.103, 0.1816, 0.1978, 0.2406 and bhat1, bhat2 from
 *    the two order conditions.
 * One attempt of size dt from q_n (k1 = f(q_n)):
 *   k_i = f(q_n + dt sum_{j<i} a_ij k_j),  i = 2..5
 *   q_{n+1} = q_n + dt sum_i b_i k_i,  k6 = f(q_{n+1})
 *   e = dt sum_{i<=6} (b_i - bhat_i) k_i     (b6 = 0)
 * err = sqrt(mean((e / (atol + rtol max(|q_n|, |q_{n+1}|)))^2)), accepted
 * when err <= 1.  Step size (PI control in digital-filter form, Soederlind
 * 2003, with the limiter of Soederlind and Wang 2006), rho(x) = 1 + atan(x - 1),
 * eps = 0.9 / max(err, 1e-10) (the controller aims at err = 0.9), K = 3:
 *   accepted:  dt_next = dt rho(eps^(B1/K) eps_prev^(B2/K)), B1 = 0.7, B2 = -0.4
 *              (the stabilized PI control of Gustafsson, with exponents
 *              0.7/K and 0.4/K as in Hairer, Noersett and Wanner, Solving
 *              Ordinary Differential Equations I, Sec. II.4),
 *              eps_prev the value of the previous accepted attempt (1 before
 *              the first);
 *   rejected:  dt_next = dt rho(eps^(1/K)) (the elementary controller), and the
 *              attempt is retried from q_n with dt_next (k1 kept).
 * A step that would pass t_end is cut to land on it. */
static const double P5_A[5][5] = {
    {0.0, 0.0, 0.0, 0.0, 0.0},
    {0.3464, 0.0, 0.0, 0.0, 0.0},
    {-0.077114705798502101362, 0.5544, 0.0, 0.0, 0.0},
    {-0.077114705798502101362, 0.51296293729322573879, 0.3078, 0.0, 0.0},
    {-0.077114705798502101362, 0.51296293729322573879, -0.53636230691175187515,
     0.25084211224332113157, 0.0}};
static const double P5_B[5] = {-0.077114705798502101362, 0.51296293729322573879,
                               -0.53636230691175187515, 0.69586264419699749322,
                               0.40465143122003074449};
static const double P5_BHAT[6] = {0.14576960111557976478, 0.13123039888442023522, 0.103, 0.1816,
                                  0.1978, 0.2406};
#define P5_B1 0.7
#define P5_B2 (-0.4)
#define P5_K 3.0
#define P5_ERR_FLOOR 1e-10
#define P5_SAFETY 0.9

/* The coefficients above, for the tests: A (25, row-major), b (5), bhat (6). */
void orc_p5_tableau(double* A, double* b, double* bhat)
{
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) A[5 * i + j] = P5_A[i][j];
    for (int i = 0; i < 5; i++) b[i] = P5_B[i];
    for (int i = 0; i < 6; i++) bhat[i] = P5_BHAT[i];
}

/* One attempt: writes q1 = q_{n+1}, k6 = f(q1) and e; returns err, or -1.
 * k holds 5 slopes (k[0] = k1 = f(q) on entry), y one stage state. */
static double p5_attempt(const orc_grid* G, const double* b, const double* q, double* const k[5],
                         double dt, double rtol, double atol, double* q1, double* k6, double* e,
                         double* y)
{
    const long m = (long)NFIELD * G->nx * G->ny;
    for (int i = 1; i < 5; i++) {
        for (long c = 0; c < m; c++) {
            double s = 0.0;
            for (int j = 0; j < i; j++) s += P5_A[i][j] * k[j][c];
            y[c] = q[c] + dt * s;
        }
        if (orc_rhs(G, b, y, k[i])) return -1.0;
    }
    for (long c = 0; c < m; c++) {
        double s = 0.0;
        for (int j = 0; j < 5; j++) s += P5_B[j] * k[j][c];
        q1[c] = q[c] + dt * s;
    }
    if (orc_rhs(G, b, q1, k6)) return -1.0;
    double sum = 0.0;
    for (long c = 0; c < m; c++) {
        double s = 0.0;
        for (int j = 0; j < 5; j++) s += (P5_B[j] - P5_BHAT[j]) * k[j][c];
        s += (0.0 - P5_BHAT[5]) * k6[c];
        e[c] = dt * s;
        double sc = atol + rtol * fmax(fabs(q[c]), fabs(q1[c]));
        double r = e[c] / sc;
        sum += r * r;
    }
    return sqrt(sum / (double)m);
}

/* nsteps fixed steps of the five-stage pair (every step accepted); e_last
 * (may be NULL) receives the error vector of the last step. */
int orc_p5_fixed(const orc_grid* G, const double* b, double* q, double dt, int nsteps, double* e_last)
{
    const long m = (long)NFIELD * G->nx * G->ny;
    double* buf = (double*)malloc(sizeof(double) * m * 9);
    if (!buf) return -1;
    double* k[5] = {buf, buf + m, buf + 2 * m, buf + 3 * m, buf + 4 * m};
    double *k6 = buf + 5 * m, *q1 = buf + 6 * m, *e = buf + 7 * m, *y = buf + 8 * m;
    int rc = orc_rhs(G, b, q, k[0]) ? -1 : 0;
    for (int s = 0; s < nsteps && rc == 0; s++) {
        if (p5_attempt(G, b, q, k, dt, 1.0, 1.0, q1, k6, e, y) < 0.0) { rc = -1; break; }
        memcpy(q, q1, sizeof(double) * m);
        memcpy(k[0], k6, sizeof(double) * m);
        if (e_last) memcpy(e_last, e, sizeof(double) * m);
    }
    free(buf);
    return rc;
}

/* Adaptive integration with the five-stage pair and the PI controller above;
 * arguments and results as orc_rk_adaptive. */
int orc_p5_adaptive(const orc_grid* G, const double* b, double* q, double t0, double t_end,
                    double dt0, double rtol, double atol, int max_attempts, double* hist, double* stats)
{
    const long m = (long)NFIELD * G->nx * G->ny;
    double* buf = (double*)malloc(sizeof(double) * m * 9);
    if (!buf) return -1;
    double* k[5] = {buf, buf + m, buf + 2 * m, buf + 3 * m, buf + 4 * m};
    double *k6 = buf + 5 * m, *q1 = buf + 6 * m, *e = buf + 7 * m, *y = buf + 8 * m;
    if (orc_rhs(G, b, q, k[0])) { free(buf); return -1; }
    double t = t0, dt = dt0, eps_prev = 1.0;
    int acc = 0, rej = 0, n = 0;
    while (t < t_end && n < max_attempts) {
        const int last = dt >= t_end - t;
        const double h = last ? t_end - t : dt;
        const double err = p5_attempt(G, b, q, k, h, rtol, atol, q1, k6, e, y);
        if (err < 0.0) { free(buf); return -1; }
        const int ok = err <= 1.0;
        const double eps = P5_SAFETY / fmax(err, P5_ERR_FLOOR);
        const double x = ok ? pow(eps, P5_B1 / P5_K) * pow(eps_prev, P5_B2 / P5_K) : pow(eps, 1.0 / P5_K);
        const double fac = 1.0 + atan(x - 1.0);
        if (hist) {
            hist[3 * n] = h;
            hist[3 * n + 1] = err;
            hist[3 * n + 2] = ok;
        }
        if (ok) {
            memcpy(q, q1, sizeof(double) * m);
            memcpy(k[0], k6, sizeof(double) * m);
            t = last ? t_end : t + h;
            eps_prev = eps;
            acc++;
        } else {
            rej++;
        }
        dt = h * fac;
        n++;
    }
    stats[0] = acc;
    stats[1] = rej;
    stats[2] = t;
    stats[3] = dt;
    free(buf);
    return n;
}
#endif

/* ---- Relaxation Runge-Kutta (Sec. 7, named there as future work) ----------
 * Standard explicit Runge-Kutta methods do not conserve the energy of Thm.
 * 4.1 / 4.2 in the fully discrete scheme (Sec. 6, energy conservation).  The
 * relaxation approach (Ketcheson 2019; Ranocha et al. 2020) scales the RK
 * update d = q_{n+1}^{RK} - q_n by a factor gamma_n chosen so that
 *     E(q_n + gamma_n d) = E(q_n)          (1^T M E, Thm. 4.1)
 * and advances time by gamma_n dt: q_{n+1} = q_n + gamma_n d,
 * t_{n+1} = t_n + gamma_n dt (the relaxed step keeps the order of the RK
 * method).  gamma_n is the root near 1 (gamma = 0 is the trivial root).
 * Here: classical RK4 for d; the root by bisection on [1/2, 3/2] of
 *     r(gamma) = sum over nodes of M (E_node(q_n + gamma d) - E_node(q_n))
 * (compensated sum), to a bracket of 4 ulp or 200 halvings. */
#ifndef ORC_COMPLEX
static double energy_change(const orc_grid* G, const double* b, const double* q, const double* d,
                            double gam)
{
    const long n = (long)G->nx * G->ny;
    csum acc = {0.0, 0.0};
    for (int j = 0; j < G->ny; j++)
        for (int i = 0; i < G->nx; i++) {
            long c = (long)j * G->nx + i;
            double e0 = energy_density(G->g, G->lambda, q[F_H * n + c], q[F_U * n + c], q[F_V * n + c],
                                       q[F_W * n + c], q[F_ETA * n + c], b[c]);
            double e1 = energy_density(G->g, G->lambda, q[F_H * n + c] + gam * d[F_H * n + c],
                                       q[F_U * n + c] + gam * d[F_U * n + c],
                                       q[F_V * n + c] + gam * d[F_V * n + c],
                                       q[F_W * n + c] + gam * d[F_W * n + c],
                                       q[F_ETA * n + c] + gam * d[F_ETA * n + c], b[c]);
            csum_add(&acc, orc_mass_weight(G, i, j) * (e1 - e0));
        }
    return acc.s + acc.c;
}

/* nsteps relaxed RK4 steps of nominal size dt, in place.  gammas (may be
 * NULL) receives gamma_n per step; *t_out the time reached from 0.  Returns
 * 0, -1 on allocation failure, -2 if r does not change sign on [1/2, 3/2]. */
int orc_rrk4(const orc_grid* G, const double* b, double* q, double dt, int nsteps, double* gammas,
             double* t_out)
{
    const long m = (long)NFIELD * G->nx * G->ny;
    double* q1 = (double*)malloc(sizeof(double) * m * 2);
    if (!q1) return -1;
    double* d = q1 + m;
    double t = 0.0;
    int rc = 0;
    for (int s = 0; s < nsteps && rc == 0; s++) {
        memcpy(q1, q, sizeof(double) * m);
        if (orc_rk4(G, b, q1, dt, 1)) { rc = -1; break; }
        for (long c = 0; c < m; c++) d[c] = q1[c] - q[c];
        double lo = 0.5, hi = 1.5;
        double rlo = energy_change(G, b, q, d, lo), rhi = energy_change(G, b, q, d, hi);
        if (!(rlo * rhi < 0.0)) { rc = -2; break; }
        for (int it = 0; it < 200 && hi - lo > 4.0 * 2.220446049250313e-16 * hi; it++) {
            double mid = 0.5 * (lo + hi);
            double rm = energy_change(G, b, q, d, mid);
            if (rm == 0.0) { lo = hi = mid; break; }
            if ((rm < 0.0) == (rlo < 0.0)) { lo = mid; rlo = rm; }
            else hi = mid;
        }
        double gam = 0.5 * (lo + hi);
        for (long c = 0; c < m; c++) q[c] = q[c] + gam * d[c];
        t += gam * dt;
        if (gammas) gammas[s] = gam;
    }
    if (t_out) *t_out = t;
    free(q1);
    return rc;
}
#endif

/* ---- Relaxation zones (Sec. 6, the wave-tank experiments) ----------------
 * Zones of width wx at both x-ends (and wy at both y-ends) absorb outgoing
 * waves: every equation gets the source -sigma (q - q0), q0 the rest state,
 * with sigma rising quadratically from 0 at the inner edge of a zone to smax
 * at the domain boundary:  sigma_x = smax ((wx - d_x) / wx)^2 for d_x < wx,
 * d_x = min(x - xmin, xmax - x) (0 outside), likewise in y; corners take
 * sigma_x + sigma_y.  Width 0 disables a direction. */
#ifndef ORC_COMPLEX
double orc_sponge_sigma(const orc_grid* G, int i, int j, double wx, double wy, double smax)
{
    double dx, dy;
    orc_spacing(G, &dx, &dy);
    const double x = G->xmin + i * dx, y = G->ymin + j * dy;
    double s = 0.0;
    if (wx > 0.0) {
        double d = fmin(x - G->xmin, G->xmax - x);
        if (d < wx) s += smax * ((wx - d) / wx) * ((wx - d) / wx);
    }
    if (wy > 0.0) {
        double d = fmin(y - G->ymin, G->ymax - y);
        if (d < wy) s += smax * ((wy - d) / wy) * ((wy - d) / wy);
    }
    return s;
}

static int rhs_sponge(const orc_grid* G, const double* b, const double* y, const double* q0, double wx,
                      double wy, double smax, double* k)
{
    if (orc_rhs(G, b, y, k)) return -1;
    const long n = (long)G->nx * G->ny;
    for (int j = 0; j < G->ny; j++)
        for (int i = 0; i < G->nx; i++) {
            const double sg = orc_sponge_sigma(G, i, j, wx, wy, smax);
            const long c = (long)j * G->nx + i;
            for (int f = 0; f < NFIELD; f++) k[f * n + c] -= sg * (y[f * n + c] - q0[f * n + c]);
        }
    return 0;
}

/* Classical RK4 (as orc_rk4) of q' = RHS(q) - sigma (q - q0), in place. */
int orc_rk4_sponge(const orc_grid* G, const double* b, double* q, double dt, int nsteps, const double* q0,
                   double wx, double wy, double smax)
{
    const long m = (long)NFIELD * G->nx * G->ny;
    double* buf = (double*)malloc(sizeof(double) * m * 5);
    if (!buf) return -1;
    double *k1 = buf, *k2 = buf + m, *k3 = buf + 2 * m, *k4 = buf + 3 * m, *y = buf + 4 * m;
    int rc = 0;
    for (int s = 0; s < nsteps && rc == 0; s++) {
        rc |= rhs_sponge(G, b, q, q0, wx, wy, smax, k1);
        for (long c = 0; c < m; c++) y[c] = q[c] + (dt / 2.0) * k1[c];
        rc |= rhs_sponge(G, b, y, q0, wx, wy, smax, k2);
        for (long c = 0; c < m; c++) y[c] = q[c] + (dt / 2.0) * k2[c];
        rc |= rhs_sponge(G, b, y, q0, wx, wy, smax, k3);
        for (long c = 0; c < m; c++) y[c] = q[c] + dt * k3[c];
        rc |= rhs_sponge(G, b, y, q0, wx, wy, smax, k4);
        for (long c = 0; c < m; c++)
            q[c] = q[c] + (dt / 6.0) * (k1[c] + 2.0 * k2[c] + 2.0 * k3[c] + k4[c]);
    }
    free(buf);
    return rc;
}
#endif
