/*
 * FastLSQ FP64 CPU oracle.  TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this library.  The GPU product path never calls it, and it shares no code,
 * header, table or constant with the CUDA sources: it is an independent,
 * plain, slow restatement of the method in double precision (no blocking, no
 * fusion, no BLAS), written so that each step can be checked against the paper
 * by eye.
 *
 * Notation: the paper writes N for the number of features and M for the number
 * of collocation rows (A is M x N, Sec. 2.3, eq. linear_system).  Here they are
 * n_feat and n_rows.  All matrices are column-major with a leading dimension.
 *
 * Pins (what fixes each function independently of itself) are listed in the
 * header comment of every function and exercised by tests/test_oracle_*.py.
 * Parity status: every function below is pinned; none is "parity unpinned".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Features and their derivatives (Sec. 2.1 eq. approximation; Sec. 2.2 eq.   */
/* cyclic).                                                                   */
/* ------------------------------------------------------------------------- */

/* Phi_s of eq. cyclic: Phi_0 = sin, Phi_1 = cos, Phi_2 = -sin, Phi_3 = -cos. */
static double orc_phase(int s, double z)
{
    switch (s & 3) {
    case 0: return sin(z);
    case 1: return cos(z);
    case 2: return -sin(z);
    default: return -cos(z);
    }
}

/* Symbolic derivative of one feature, one axis at a time (chain rule of
 * Sec. 2.2): the feature is carried as the pair (multiplier c, phase index s)
 * meaning c * Phi_s(W.x + b).  d/dx_k maps (c, s) -> (c * W_k, s + 1), so that
 * after applying the multi-index alpha the pair is (prod_k W_k^alpha_k,
 * |alpha| mod 4), which is eq. cyclic. */
static void orc_term_derivative(const int *alpha, int d, const double *Wj,
                                double *c_out, int *s_out)
{
    double c = 1.0;
    int s = 0;
    for (int k = 0; k < d; ++k)
        for (int r = 0; r < alpha[k]; ++r) {
            c *= Wj[k];
            s += 1;
        }
    *c_out = c;
    *s_out = s & 3;
}

/* z_ij = W_j . x_i + b_j  (argument of the feature, eq. approximation). */
static double orc_arg(const double *xi, const double *Wj, double bj, int d)
{
    double z = bj;
    for (int k = 0; k < d; ++k) z += Wj[k] * xi[k];
    return z;
}

/*
 * Operator matrix block (Sec. 2.3 eq. linear_system; Alg. 1 steps 3-4):
 *
 *   A[i + j*ldA] = row_weight * scale * sum_t (coef[t] + coef_pt[t][i]) * D^{alpha_t} phi_j(x_i)
 *
 * phi_j(x) = sin(W_j.x + b_j), scale is the 1/sqrt(n_feat) of eq. approximation,
 * row_weight is the boundary penalty lambda for boundary blocks (1 for PDE rows).
 * alpha is [n_terms][d] row-major, W is [n_feat][d] row-major, x is [n_rows][d]
 * row-major.  coef_pt (may be NULL) is [n_terms][n_rows]: a per-point addition
 * to term t's coefficient, which is how the Newton Jacobian's N'(u_i) phi_j term
 * (Sec. 2.4 eq. newton) enters with alpha = 0.
 *
 * Pins: closed forms of Corollary 1 (Laplacian, biharmonic, advection), central
 * finite differences of phi_j written independently in the tests, W = 0 and
 * d = 1 special cases.
 */
void orc_assemble(const double *x, long n_rows, int d,
                  int n_terms, const int *alpha, const double *coef,
                  const double *coef_pt, double row_weight,
                  const double *W, const double *b, long n_feat, double scale,
                  double *A, long ldA)
{
    for (long j = 0; j < n_feat; ++j) {
        const double *Wj = W + j * d;
        for (long i = 0; i < n_rows; ++i) {
            const double *xi = x + i * d;
            double z = orc_arg(xi, Wj, b[j], d);
            double acc = 0.0;
            for (int t = 0; t < n_terms; ++t) {
                double c;
                int s;
                orc_term_derivative(alpha + t * d, d, Wj, &c, &s);
                double ct = coef[t];
                if (coef_pt) ct += coef_pt[(long)t * n_rows + i];
                acc += ct * c * orc_phase(s, z);
            }
            A[i + j * ldA] = row_weight * scale * acc;
        }
    }
}

/* u(x_i) = scale * sum_j beta_j sin(W_j.x_i + b_j)  (eq. approximation). */
void orc_eval_u(const double *x, long n, int d, const double *W, const double *b,
                long n_feat, double scale, const double *beta, double *u)
{
    for (long i = 0; i < n; ++i) {
        double acc = 0.0;
        for (long j = 0; j < n_feat; ++j)
            acc += beta[j] * sin(orc_arg(x + i * d, W + j * d, b[j], d));
        u[i] = scale * acc;
    }
}

/* ------------------------------------------------------------------------- */
/* Dense least squares by Householder QR (Sec. 2.3: "via QR or SVD").         */
/* ------------------------------------------------------------------------- */

/*
 * Unblocked Householder QR in place (m >= n).  Column j is reduced by
 * H_j = I - tau_j v v^T with v = [1; A(j+1:m, j)], LAPACK's convention for the
 * reflector sign: beta = -sign(a_jj) * ||A(j:m, j)||, so that H_j A(j:m, j) =
 * beta e_1 without cancellation.  On exit R is in the upper triangle and the
 * reflector tails below it.
 *
 * Pins: A = QR and Q^T Q = I to rounding (tests rebuild Q from the reflectors
 * with plain numpy), agreement with LAPACK's least-squares solve on tiny
 * well-conditioned systems, and exact recovery of beta_0 from b = A beta_0.
 */
void orc_qr(double *A, long m, long n, long lda, double *tau)
{
    for (long j = 0; j < n; ++j) {
        double *col = A + j * lda;
        double alpha = col[j];
        double ss = 0.0;
        for (long i = j + 1; i < m; ++i) ss += col[i] * col[i];
        if (ss == 0.0) {            /* nothing below the diagonal: H = I */
            tau[j] = 0.0;
            continue;
        }
        double norm = sqrt(alpha * alpha + ss);
        double beta = (alpha >= 0.0) ? -norm : norm;
        tau[j] = (beta - alpha) / beta;
        double inv = 1.0 / (alpha - beta);
        for (long i = j + 1; i < m; ++i) col[i] *= inv;
        col[j] = beta;
        /* apply H_j to the columns on its right: a <- a - tau v (v^T a) */
        for (long c = j + 1; c < n; ++c) {
            double *ac = A + c * lda;
            double w = ac[j];
            for (long i = j + 1; i < m; ++i) w += col[i] * ac[i];
            w *= tau[j];
            ac[j] -= w;
            for (long i = j + 1; i < m; ++i) ac[i] -= w * col[i];
        }
    }
}

/* y <- Q^T y for the reflectors stored by orc_qr (applied H_0 first). */
void orc_apply_qt(const double *QR, long m, long n, long lda, const double *tau,
                  double *y, int nrhs, long ldy)
{
    for (int r = 0; r < nrhs; ++r) {
        double *yr = y + (long)r * ldy;
        for (long j = 0; j < n; ++j) {
            const double *v = QR + j * lda;
            double w = yr[j];
            for (long i = j + 1; i < m; ++i) w += v[i] * yr[i];
            w *= tau[j];
            yr[j] -= w;
            for (long i = j + 1; i < m; ++i) yr[i] -= w * v[i];
        }
    }
}

/* Solve R x = y (upper triangle of QR, n x n) by back substitution. */
void orc_backsolve(const double *QR, long n, long lda, double *y)
{
    for (long i = n - 1; i >= 0; --i) {
        double acc = y[i];
        for (long c = i + 1; c < n; ++c) acc -= QR[i + c * lda] * y[c];
        y[i] = acc / QR[i + i * lda];
    }
}

/* Solve R^T x = y (forward substitution with the transpose of R). */
void orc_forwardsolve_rt(const double *QR, long n, long lda, double *y)
{
    for (long i = 0; i < n; ++i) {
        double acc = y[i];
        for (long c = 0; c < i; ++c) acc -= QR[c + i * lda] * y[c];
        y[i] = acc / QR[i + i * lda];
    }
}

/* Build the Tikhonov-augmented matrix [A; sqrt(mu) I] ((m + n) x n when mu > 0,
 * else a copy of A) as used for the regularised solves of Sec. 2.4 and the
 * inverse-problem forward map beta = (A^T A + mu I)^{-1} A^T f of Sec. 3.8. */
static double *orc_augment(const double *A, long m, long n, long lda, double mu,
                           long *m_aug)
{
    long ma = (mu > 0.0) ? m + n : m;
    double *Aa = (double *)calloc((size_t)ma * (size_t)n, sizeof(double));
    if (!Aa) return NULL;
    for (long j = 0; j < n; ++j) {
        memcpy(Aa + j * ma, A + j * lda, (size_t)m * sizeof(double));
        if (mu > 0.0) Aa[m + j + j * ma] = sqrt(mu);
    }
    *m_aug = ma;
    return Aa;
}

/*
 * beta = argmin ||A beta - rhs||^2 + mu ||beta||^2 for nrhs right-hand sides
 * (rhs is m x nrhs, beta is n x nrhs, both column-major with ld m and n).
 * Returns 0, or -2 on allocation failure.
 */
int orc_lstsq(const double *A, long m, long n, long lda, double mu,
              const double *rhs, int nrhs, double *beta)
{
    long ma;
    double *Aa = orc_augment(A, m, n, lda, mu, &ma);
    double *tau = (double *)malloc((size_t)n * sizeof(double));
    double *y = (double *)calloc((size_t)ma * (size_t)nrhs, sizeof(double));
    if (!Aa || !tau || !y) { free(Aa); free(tau); free(y); return -2; }
    for (int r = 0; r < nrhs; ++r)
        memcpy(y + (long)r * ma, rhs + (long)r * m, (size_t)m * sizeof(double));
    orc_qr(Aa, ma, n, ma, tau);
    orc_apply_qt(Aa, ma, n, ma, tau, y, nrhs, ma);
    for (int r = 0; r < nrhs; ++r) {
        orc_backsolve(Aa, n, ma, y + (long)r * ma);
        memcpy(beta + (long)r * n, y + (long)r * ma, (size_t)n * sizeof(double));
    }
    free(Aa); free(tau); free(y);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Manufactured problems and sources (Sec. 3.1: errors are measured against   */
/* known solutions on an independent test set).  The expressions below are    */
/* hand-derived; tests pin each source f = L[u*] by finite differences of u*. */
/* ------------------------------------------------------------------------- */

enum {
    ORC_POISSON_1D = 1,    /* -u'' = f on [0,1]; u* = sin(2 pi x) + 0.5 sin(6 pi x)            */
    ORC_HELMHOLTZ_2D = 2,  /* Lap u + k^2 u = f on [0,1]^2; params[0] = k;                      */
                           /* u* = sin(pi x) sin(2 pi y) + 0.3 cos(3 pi x + pi y)               */
    ORC_POISSON_5D = 3,    /* -Lap u = f on [0,1]^5; u* = sum_k sin(pi x_k) + prod_k x_k        */
    ORC_BRATU_2D = 4,      /* Lap u + lam e^u = 0, u = 0 on the boundary (no closed form)       */
    ORC_GAUSS_SOURCE_2D = 5, /* -Lap u = s(x; theta), u = 0 on the boundary; params = theta     */
    /* the cubic Newton problems of Sec. 3.3 ("u^3 term"; the equations are this reading):    */
    /* u* = sin(pi x) sin(pi y) + x y / 2 on [0,1]^2, Dirichlet data u* on the boundary        */
    ORC_NLPOISSON_2D = 6,  /* -Lap u + lam u^3 = f; params[0] = lam                              */
    ORC_NLHELMHOLTZ_2D = 7, /* Lap u + k^2 u + lam u^3 = f; params = (k, lam)                    */
    /* the 1-D Newton problems of Sec. 3.3 in true solver mode (f = 0), each with a kink   */
    /* that solves the equation exactly on the real line, Dirichlet data u* at x = 0, 1:  */
    ORC_ALLEN_CAHN_1D = 8, /* eps u'' + u - u^3 = 0; params[0] = eps;                          */
                           /* u* = tanh((x - 1/2) / sqrt(2 eps))                                */
    ORC_BURGERS_1D = 9,    /* u u' - nu u'' = 0; params[0] = nu; u* = -tanh((x - 1/2) / (2 nu))  */
    /* the variable-coefficient form of Sec. 3.8 (div(nu grad u), expanded as             */
    /* nu Lap u + grad nu . grad u), with a manufactured u*:                              */
    ORC_VARCOEF_2D = 10    /* div(nu grad u) = f on [0,1]^2, nu = 1 + a (x^2 + y^2/2),           */
                           /* params[0] = a; u* = sin(pi x) sin(2 pi y) + x y                    */
};

/* The variable coefficient of problem 10 (comp = -1) or its derivative along x_comp. */
void orc_problem_coef(int prob, int comp, const double *x, long n, int d, const double *params,
                      double *out)
{
    for (long i = 0; i < n; ++i) {
        const double *p = x + i * d;
        double v = 0.0;
        if (prob == ORC_VARCOEF_2D) {
            const double a = params[0];
            if (comp < 0) v = 1.0 + a * (p[0] * p[0] + 0.5 * p[1] * p[1]);
            else if (comp == 0) v = 2.0 * a * p[0];
            else if (comp == 1) v = a * p[1];
        }
        out[i] = v;
    }
}

/* s(x; theta) = sum_k a_k exp(-|x - c_k|^2 / (2 w_k^2)), theta_k = (c_kx, c_ky, w_k, a_k). */
static double orc_gauss(const double *x, const double *theta, int n_src)
{
    double s = 0.0;
    for (int k = 0; k < n_src; ++k) {
        const double *th = theta + 4 * k;
        double dx = x[0] - th[0], dy = x[1] - th[1];
        s += th[3] * exp(-(dx * dx + dy * dy) / (2.0 * th[2] * th[2]));
    }
    return s;
}

/* Exact solution u*(x) (0 for problems without a closed form). */
void orc_problem_exact(int prob, const double *x, long n, int d,
                       const double *params, double *u)
{
    const double pi = M_PI;
    for (long i = 0; i < n; ++i) {
        const double *p = x + i * d;
        double v = 0.0;
        if (prob == ORC_POISSON_1D) {
            v = sin(2 * pi * p[0]) + 0.5 * sin(6 * pi * p[0]);
        } else if (prob == ORC_HELMHOLTZ_2D) {
            v = sin(pi * p[0]) * sin(2 * pi * p[1]) + 0.3 * cos(3 * pi * p[0] + pi * p[1]);
        } else if (prob == ORC_POISSON_5D) {
            double sum = 0.0, prod = 1.0;
            for (int k = 0; k < d; ++k) { sum += sin(pi * p[k]); prod *= p[k]; }
            v = sum + prod;
        } else if (prob == ORC_NLPOISSON_2D || prob == ORC_NLHELMHOLTZ_2D) {
            v = sin(pi * p[0]) * sin(pi * p[1]) + 0.5 * p[0] * p[1];
        } else if (prob == ORC_ALLEN_CAHN_1D) {
            /* u = tanh(k s): u'' = -2 k^2 u (1 - u^2), so eps u'' + u - u^3 = 0 at k^2 = 1/(2 eps) */
            v = tanh((p[0] - 0.5) / sqrt(2.0 * params[0]));
        } else if (prob == ORC_BURGERS_1D) {
            /* u = -tanh(k s): u u' = k tanh sech^2 and nu u'' = 2 nu k^2 tanh sech^2, equal at k = 1/(2 nu) */
            v = -tanh((p[0] - 0.5) / (2.0 * params[0]));
        } else if (prob == ORC_VARCOEF_2D) {
            v = sin(pi * p[0]) * sin(2 * pi * p[1]) + p[0] * p[1];
        }
        u[i] = v;
    }
}

/* Source term f(x) of the interior equation. */
void orc_problem_source(int prob, const double *x, long n, int d,
                        const double *params, int n_params, double *f)
{
    const double pi = M_PI;
    for (long i = 0; i < n; ++i) {
        const double *p = x + i * d;
        double v = 0.0;
        if (prob == ORC_POISSON_1D) {
            /* -(d^2/dx^2) of u*: (2 pi)^2 sin(2 pi x) + 0.5 (6 pi)^2 sin(6 pi x) */
            v = 4 * pi * pi * sin(2 * pi * p[0]) + 18 * pi * pi * sin(6 * pi * p[0]);
        } else if (prob == ORC_HELMHOLTZ_2D) {
            double k2 = params[0] * params[0];
            /* Lap of sin(pi x) sin(2 pi y) is -5 pi^2 times it; of cos(3 pi x + pi y) is -10 pi^2 times it */
            v = (k2 - 5 * pi * pi) * sin(pi * p[0]) * sin(2 * pi * p[1])
              + 0.3 * (k2 - 10 * pi * pi) * cos(3 * pi * p[0] + pi * p[1]);
        } else if (prob == ORC_POISSON_5D) {
            /* prod_k x_k is harmonic, so only the sine sum contributes */
            double sum = 0.0;
            for (int k = 0; k < d; ++k) sum += sin(pi * p[k]);
            v = pi * pi * sum;
        } else if (prob == ORC_GAUSS_SOURCE_2D) {
            v = orc_gauss(p, params, n_params / 4);
        } else if (prob == ORC_NLPOISSON_2D || prob == ORC_NLHELMHOLTZ_2D) {
            /* Lap of sin(pi x) sin(pi y) is -2 pi^2 times it; x y is harmonic */
            double s = sin(pi * p[0]) * sin(pi * p[1]);
            double u = s + 0.5 * p[0] * p[1];
            if (prob == ORC_NLPOISSON_2D)
                v = 2 * pi * pi * s + params[0] * u * u * u;
            else
                v = -2 * pi * pi * s + params[0] * params[0] * u + params[1] * u * u * u;
        } else if (prob == ORC_VARCOEF_2D) {
            /* nu Lap u* + grad nu . grad u*, with Lap u* = -5 pi^2 sin(pi x) sin(2 pi y) (x y is
             * harmonic) and grad u* = (pi cos(pi x) sin(2 pi y) + y, 2 pi sin(pi x) cos(2 pi y) + x) */
            double a = params[0];
            double s = sin(pi * p[0]) * sin(2 * pi * p[1]);
            double nu = 1.0 + a * (p[0] * p[0] + 0.5 * p[1] * p[1]);
            double ux = pi * cos(pi * p[0]) * sin(2 * pi * p[1]) + p[1];
            double uy = 2 * pi * sin(pi * p[0]) * cos(2 * pi * p[1]) + p[0];
            v = nu * (-5 * pi * pi * s) + 2.0 * a * p[0] * ux + a * p[1] * uy;
        }
        f[i] = v;
    }
}

/* dL/dtheta = sum_i w_i ds(x_i; theta)/dtheta for the Gaussian source, with
 * ds/dc_kx = a_k e_k (x - c_kx) / w_k^2, ds/dc_ky likewise,
 * ds/dw_k = a_k e_k |x - c_k|^2 / w_k^3, ds/da_k = e_k. */
void orc_gauss_source_grad(const double *x, long n, const double *theta, int n_src,
                           const double *w, double *dtheta)
{
    for (int q = 0; q < 4 * n_src; ++q) dtheta[q] = 0.0;
    for (long i = 0; i < n; ++i) {
        const double *p = x + 2 * i;
        for (int k = 0; k < n_src; ++k) {
            const double *th = theta + 4 * k;
            double dx = p[0] - th[0], dy = p[1] - th[1];
            double r2 = dx * dx + dy * dy, w2 = th[2] * th[2];
            double e = exp(-r2 / (2.0 * w2));
            dtheta[4 * k + 0] += w[i] * th[3] * e * dx / w2;
            dtheta[4 * k + 1] += w[i] * th[3] * e * dy / w2;
            dtheta[4 * k + 2] += w[i] * th[3] * e * r2 / (w2 * th[2]);
            dtheta[4 * k + 3] += w[i] * e;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Newton-Raphson for L[u] + N[u] = f (Sec. 2.4, eq. newton).                 */
/* ------------------------------------------------------------------------- */

/* N(u) = lam e^u, lam u^3, or (Burgers) lam u du/dx_0, the advection term along the first
 * coordinate. */
enum { ORC_NL_NONE = 0, ORC_NL_EXP = 1, ORC_NL_CUBIC = 2, ORC_NL_BURGERS = 3 };

static double orc_nl(int kind, double lam, double u, double ux)
{
    if (kind == ORC_NL_EXP) return lam * exp(u);
    if (kind == ORC_NL_CUBIC) return lam * u * u * u;
    if (kind == ORC_NL_BURGERS) return lam * u * ux;
    return 0.0;
}

/* Derivative of N in the direction phi: c0 phi + c1 d(phi)/dx_0. */
static void orc_nl_prime(int kind, double lam, double u, double ux, double *c0, double *c1)
{
    *c0 = 0.0;
    *c1 = 0.0;
    if (kind == ORC_NL_EXP) *c0 = lam * exp(u);
    if (kind == ORC_NL_CUBIC) *c0 = 3.0 * lam * u * u;
    if (kind == ORC_NL_BURGERS) { *c0 = lam * ux; *c1 = lam * u; }
}

static void orc_matvec(const double *M, long m, long n, const double *v, double *out)
{
    for (long i = 0; i < m; ++i) out[i] = 0.0;
    for (long j = 0; j < n; ++j)
        for (long i = 0; i < m; ++i) out[i] += M[i + j * m] * v[j];
}

/* Residual R(beta): interior rows L[u] + N(u) - f, then boundary rows
 * bc_weight * (u - g).  Also returns u at every collocation row. */
static double orc_newton_residual(const double *HL, const double *Hi, const double *Hb,
                                  const double *Hd, long n_int, long n_bc, long n, int nl_kind,
                                  double nl_lam, double bc_weight, const double *f,
                                  const double *g, const double *beta, double *R, double *u_rows,
                                  double *ux, double *tmp)
{
    double rr = 0.0;
    orc_matvec(HL, n_int, n, beta, tmp);          /* L[u] at interior points */
    orc_matvec(Hi, n_int, n, beta, u_rows);       /* u at interior points    */
    orc_matvec(Hb, n_bc, n, beta, u_rows + n_int); /* u at boundary points    */
    if (Hd) orc_matvec(Hd, n_int, n, beta, ux);   /* du/dx_0 at interior points */
    for (long i = 0; i < n_int; ++i) {
        R[i] = tmp[i] + orc_nl(nl_kind, nl_lam, u_rows[i], Hd ? ux[i] : 0.0) - f[i];
        rr += R[i] * R[i];
    }
    for (long i = 0; i < n_bc; ++i) {
        R[n_int + i] = bc_weight * (u_rows[n_int + i] - g[i]);
        rr += R[n_int + i] * R[n_int + i];
    }
    return rr;
}

/*
 * Newton-Raphson with the refinements of Sec. 2.4:
 *   J_ij = L[phi_j](x_i) + N'(u_i) phi_j(x_i) on interior rows (for Burgers, N = lam u u_x,
 *   the derivative lam u_x(x_i) phi_j(x_i) + lam u(x_i) d(phi_j)/dx_0(x_i)), bc_weight
 *   phi_j on boundary rows; delta = argmin ||J delta + R||^2 + mu ||delta||^2 (Tikhonov);
 *   backtracking on the residual norm with the Armijo-type test
 *   ||R(beta + a delta)||^2 <= (1 - 2 c a) ||R(beta)||^2, halving a at most
 *   max_halvings times; stop when ||a J_u delta|| / ||u_new|| <= tol, the change of
 *   u at the collocation rows relative to u (solution-level test).
 * Warm start (solving the linear part first) is the caller's: pass its beta in.
 *
 * x_int [n_int][d], x_bc [n_bc][d]; the interior linear operator is given by
 * (n_terms, alpha, coef); the boundary operator is Dirichlet.  beta is in/out.
 * res_hist receives ||R|| before each iteration and after the last (max_iter+1).
 * Returns 0 converged, 1 max_iter reached, 2 line search failed, -2 no memory.
 *
 * Pins: for Bratu, an independent second-order finite-difference Newton solve
 * (tests); for a linear problem (N = 0) one step equals the linear solve; for the
 * problems with a closed-form solution, convergence to it (tests).
 */
int orc_newton(const double *x_int, long n_int, const double *x_bc, long n_bc, int d,
               int n_terms, const int *alpha, const double *coef,
               int nl_kind, double nl_lam, double bc_weight,
               const double *f, const double *g,
               const double *W, const double *b, long n_feat, double scale,
               double mu, int max_iter, double tol, double armijo_c, int max_halvings,
               double *beta, int *iters_out, double *res_hist)
{
    long n = n_feat, m = n_int + n_bc;
    int zero_alpha[16] = {0}, dx0_alpha[16] = {1};
    double one = 1.0;
    const int burgers = (nl_kind == ORC_NL_BURGERS);
    double *HL = malloc(sizeof(double) * n_int * n);
    double *Hd = burgers ? malloc(sizeof(double) * n_int * n) : NULL;
    double *ux = calloc(n_int + 1, sizeof(double));
    double *uxn = calloc(n_int + 1, sizeof(double));
    double *Hi = malloc(sizeof(double) * n_int * n);
    double *Hb = malloc(sizeof(double) * n_bc * n);
    double *J = malloc(sizeof(double) * m * n);
    double *R = malloc(sizeof(double) * m);
    double *Rn = malloc(sizeof(double) * m);
    double *u = malloc(sizeof(double) * m);
    double *un = malloc(sizeof(double) * m);
    double *tmp = malloc(sizeof(double) * (n_int + 1));
    double *delta = malloc(sizeof(double) * n);
    double *bt = malloc(sizeof(double) * n);
    int status = 1, it = 0;
    if (!HL || !Hi || !Hb || !J || !R || !Rn || !u || !un || !tmp || !delta || !bt || !ux || !uxn ||
        (burgers && !Hd) || d > 16) {
        status = -2;
        goto done;
    }
    orc_assemble(x_int, n_int, d, n_terms, alpha, coef, NULL, 1.0, W, b, n, scale, HL, n_int);
    orc_assemble(x_int, n_int, d, 1, zero_alpha, &one, NULL, 1.0, W, b, n, scale, Hi, n_int);
    orc_assemble(x_bc, n_bc, d, 1, zero_alpha, &one, NULL, 1.0, W, b, n, scale, Hb, n_bc);
    if (burgers) orc_assemble(x_int, n_int, d, 1, dx0_alpha, &one, NULL, 1.0, W, b, n, scale, Hd, n_int);

    double rr = orc_newton_residual(HL, Hi, Hb, Hd, n_int, n_bc, n, nl_kind, nl_lam, bc_weight,
                                    f, g, beta, R, u, ux, tmp);
    for (it = 0; it < max_iter; ++it) {
        if (res_hist) res_hist[it] = sqrt(rr);
        /* Jacobian, eq. newton */
        for (long j = 0; j < n; ++j) {
            for (long i = 0; i < n_int; ++i) {
                double c0, c1;
                orc_nl_prime(nl_kind, nl_lam, u[i], ux[i], &c0, &c1);
                J[i + j * m] = HL[i + j * n_int] + c0 * Hi[i + j * n_int];
                if (burgers) J[i + j * m] += c1 * Hd[i + j * n_int];
            }
            for (long i = 0; i < n_bc; ++i)
                J[n_int + i + j * m] = bc_weight * Hb[i + j * n_bc];
        }
        for (long i = 0; i < m; ++i) Rn[i] = -R[i];
        if (orc_lstsq(J, m, n, m, mu, Rn, 1, delta) != 0) { status = -2; goto done; }
        /* backtracking line search on ||R|| */
        double a = 1.0, rr_new = 0.0;
        int accepted = 0;
        for (int h = 0; h <= max_halvings; ++h) {
            for (long j = 0; j < n; ++j) bt[j] = beta[j] + a * delta[j];
            rr_new = orc_newton_residual(HL, Hi, Hb, Hd, n_int, n_bc, n, nl_kind, nl_lam,
                                         bc_weight, f, g, bt, Rn, un, uxn, tmp);
            if (rr_new <= (1.0 - 2.0 * armijo_c * a) * rr) { accepted = 1; break; }
            a *= 0.5;
        }
        if (!accepted) { status = 2; break; }
        /* solution-level stopping test at the collocation rows */
        double du2 = 0.0, u2 = 0.0;
        for (long i = 0; i < m; ++i) {
            double du = un[i] - u[i];
            du2 += du * du;
            u2 += un[i] * un[i];
        }
        memcpy(beta, bt, sizeof(double) * n);
        memcpy(R, Rn, sizeof(double) * m);
        memcpy(u, un, sizeof(double) * m);
        memcpy(ux, uxn, sizeof(double) * n_int);
        rr = rr_new;
        if (sqrt(du2) <= tol * sqrt(u2)) { status = 0; ++it; break; }
    }
    if (res_hist) res_hist[it] = sqrt(rr);
done:
    if (iters_out) *iters_out = it;
    free(HL); free(Hd); free(ux); free(uxn); free(Hi); free(Hb); free(J); free(R); free(Rn);
    free(u); free(un);
    free(tmp); free(delta); free(bt);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Differentiable solve and its adjoint (Sec. 2.5; Sec. 3.8 inverse heat      */
/* source: beta = (A^T A + mu I)^{-1} A^T f with a pre-factored matrix).      */
/* ------------------------------------------------------------------------- */

/*
 * Forward: QR of [A; sqrt(mu) I] (R^T R = A^T A + mu I), beta = R^{-1} Q^T [f; 0],
 * sensor values u_s = Hs beta, loss = mean_s (u_s - y_s)^2.
 * Adjoint: grad_beta = Hs^T dL/du_s, v = R^{-1} R^{-T} grad_beta (the two
 * triangular solves), dL/df = A v, and r = f - A beta for coefficient gradients.
 * A is m x n (lda), Hs is ns x n (ldh).  Outputs beta (n), u_s (ns), loss,
 * v (n), grad_rhs (m), resid (m).  Returns 0 or -2.
 *
 * Pins: central finite differences (h = 1e-6) of the loss through this same
 * forward map, in the tests.
 */
int orc_inverse_adjoint(const double *A, long m, long n, long lda, double mu,
                        const double *rhs, const double *Hs, long ns, long ldh,
                        const double *y_obs, double *beta, double *u_s, double *loss,
                        double *v, double *grad_rhs, double *resid)
{
    long ma;
    double *Aa = orc_augment(A, m, n, lda, mu, &ma);
    double *tau = malloc(sizeof(double) * n);
    double *y = calloc((size_t)ma, sizeof(double));
    if (!Aa || !tau || !y) { free(Aa); free(tau); free(y); return -2; }
    memcpy(y, rhs, sizeof(double) * m);
    orc_qr(Aa, ma, n, ma, tau);
    orc_apply_qt(Aa, ma, n, ma, tau, y, 1, ma);
    orc_backsolve(Aa, n, ma, y);
    memcpy(beta, y, sizeof(double) * n);
    double l = 0.0;
    for (long s = 0; s < ns; ++s) {
        double acc = 0.0;
        for (long j = 0; j < n; ++j) acc += Hs[s + j * ldh] * beta[j];
        u_s[s] = acc;
        l += (acc - y_obs[s]) * (acc - y_obs[s]);
    }
    *loss = l / (double)ns;
    for (long j = 0; j < n; ++j) {
        double acc = 0.0;
        for (long s = 0; s < ns; ++s) acc += Hs[s + j * ldh] * 2.0 * (u_s[s] - y_obs[s]) / (double)ns;
        v[j] = acc;
    }
    orc_forwardsolve_rt(Aa, n, ma, v);   /* R^{-T} grad_beta */
    orc_backsolve(Aa, n, ma, v);         /* R^{-1} (...)     */
    for (long i = 0; i < m; ++i) {
        double av = 0.0, ab = 0.0;
        for (long j = 0; j < n; ++j) {
            av += A[i + j * lda] * v[j];
            ab += A[i + j * lda] * beta[j];
        }
        grad_rhs[i] = av;
        resid[i] = rhs[i] - ab;
    }
    free(Aa); free(tau); free(y);
    return 0;
}

/*
 * Gradient of the loss with respect to the coefficient c_t of one operator term
 * on the interior rows: with r = f - A beta and v as above,
 *   dL/dc_t = sum_ij (r_i v_j - (A v)_i beta_j) dA_ij/dc_t,
 * and dA_ij/dc_t = scale * D^{alpha_t} phi_j(x_i) (from differentiating the
 * normal equations (A^T A + mu I) beta = A^T f).  x_int holds the rows the term
 * acts on; r and Av are their entries.
 */
double orc_term_coef_grad(const double *x_int, long n_int, int d, const int *alpha_t,
                          const double *W, const double *b, long n_feat, double scale,
                          const double *r, const double *Av, const double *v,
                          const double *beta)
{
    double one = 1.0, g = 0.0;
    double *At = malloc(sizeof(double) * n_int * n_feat);
    if (!At) return NAN;
    orc_assemble(x_int, n_int, d, 1, alpha_t, &one, NULL, 1.0, W, b, n_feat, scale, At, n_int);
    for (long j = 0; j < n_feat; ++j)
        for (long i = 0; i < n_int; ++i)
            g += At[i + j * n_int] * (r[i] * v[j] - Av[i] * beta[j]);
    free(At);
    return g;
}

/* ------------------------------------------------------------------------- */
/* Learnable bandwidth (App. "Learnable Bandwidth via Reparameterisation",    */
/* Alg. 2): the gradient of a loss with respect to the feature weights W and  */
/* biases b through the exact inner solve.                                    */
/* ------------------------------------------------------------------------- */

/*
 * dA_ij/dW_jk for the block A_ij = row_weight * scale * sum_t coef_t D^{alpha_t} phi_j(x_i):
 * each term is coef_t * prod_l W_jl^alpha_tl * Phi_{|alpha_t|}(z) (eq. cyclic), so by the
 * product rule
 *   d/dW_jk = coef_t * [alpha_tk W_jk^(alpha_tk - 1) prod_{l != k} W_jl^alpha_tl Phi_{|alpha_t|}(z)
 *                       + prod_l W_jl^alpha_tl * x_ik * Phi_{|alpha_t| + 1}(z)],
 * and d/db_j replaces x_ik by 1 in the second part and drops the first.
 *
 * Weights of the bilinear form (differentiating the normal equations
 * (A^T A + mu I) beta = A^T rhs, r = rhs - A beta, v = (A^T A + mu I)^{-1} g):
 *   w_ij = r_i (c_v v_j + c_rb beta_j) + c_av (A v)_i beta_j.
 * A loss that sees A only through beta, with grad_beta = g, takes (c_v, c_rb, c_av) =
 * (1, 0, -1) (as orc_term_coef_grad).  The outer loss ||A beta - rhs||^2 of Alg. 2 has
 * grad_beta = -2 A^T r = -2 mu beta and an explicit dependence on A (-2 r_i beta_j): with
 * v = (A^T A + mu I)^{-1} beta it takes (c_v, c_rb, c_av) = (-2 mu, -2, 2 mu).  v and Av
 * may be NULL (their terms dropped).
 *   gW[j*d + k] += sum_i w_ij dA_ij/dW_jk,    gb[j] += sum_i w_ij dA_ij/db_j.
 */
void orc_weight_grad(const double *x, long n_rows, int d, int n_terms, const int *alpha,
                     const double *coef, double row_weight, const double *W, const double *b,
                     long n_feat, double scale, const double *r, const double *beta,
                     const double *v, const double *Av, double c_v, double c_rb, double c_av,
                     double *gW, double *gb)
{
    for (long j = 0; j < n_feat; ++j) {
        const double *Wj = W + j * d;
        for (long i = 0; i < n_rows; ++i) {
            const double *xi = x + i * d;
            double wij = r[i] * ((v ? c_v * v[j] : 0.0) + c_rb * beta[j]);
            if (Av) wij += c_av * Av[i] * beta[j];
            double z = orc_arg(xi, Wj, b[j], d);
            for (int t = 0; t < n_terms; ++t) {
                const int *at = alpha + t * d;
                double c;
                int s;
                orc_term_derivative(at, d, Wj, &c, &s);
                double f = wij * row_weight * scale * coef[t];
                double phase_next = orc_phase((s + 1) & 3, z);
                gb[j] += f * c * phase_next;
                for (int k = 0; k < d; ++k) {
                    /* product-rule factor of W_jk: alpha_tk W_jk^(alpha_tk - 1) prod_{l != k} */
                    double dc = 0.0;
                    if (at[k] > 0) {
                        dc = (double)at[k];
                        for (int l = 0; l < d; ++l) {
                            int p = (l == k) ? at[l] - 1 : at[l];
                            for (int q = 0; q < p; ++q) dc *= Wj[l];
                        }
                    }
                    gW[j * d + k] += f * (dc * orc_phase(s, z) + c * xi[k] * phase_next);
                }
            }
        }
    }
}
