/*
 * Statistical equilibrium (Eq. 2) of the oracle (test infrastructure only):
 * Jacobi (ALI) update with the diagonal of the Lambda operator (Sec. 2, Sec. 5).
 *
 * Unknowns per voxel are multipolar components of the line source function,
 * S^K_Q, proportional to rho^K_Q of the upper level (lower level J = 0,
 * unpolarized, so the line absorption is unpolarized).
 *
 * Two-level atom, CRD, no stimulated emission:
 *   S^K_Q - i (1-eps) Gamma_u sum_Q' K^K_QQ'(B) S^K_Q' = (1-eps) w^(K) J^K_Q + eps B delta_K0 delta_Q0
 * with Gamma_u = |B| / bcrit and K^K_QQ' the matrix of the angular momentum
 * component along the field direction (theta_B, chi_B). The S^K_Q follow the
 * convention of J^K_Q (they are the complex conjugates of the atomic rho^K_Q):
 * the atom precesses counterclockwise about B (Lande factor > 0), which in this
 * convention is the factor -i (HANLE_SENSE below) of the magnetic term.
 *   K_QQ = Q cos(theta_B),
 *   K_Q,Q-1 = 1/2 sin(theta_B) e^{+i chi_B} sqrt((K+Q)(K-Q+1)),
 *   K_Q,Q+1 = 1/2 sin(theta_B) e^{-i chi_B} sqrt((K-Q)(K+Q+1)).
 * Jacobi step: S^0_0 is updated implicitly with Lambda-bar*,
 *   S00 <- S00 + [(1-eps) J00 + eps B - S00] / [1 - (1-eps) Lambda-bar*],
 * the K = 2 components explicitly from the current J^2_Q (5x5 Hanle solve).
 */
#include <math.h>
#include <stddef.h>
#include "or_common.h"
#include <complex.h>
#undef I
#define IU _Complex_I

/* sign of the magnetic term of the equation above (see the header) */
#define HANLE_SENSE (-1.0)

/* M = 1 + i gamma K for K = 2 (rows and columns Q = -2..2) for the field (bx, by, bz) */
static void hanle_matrix(double gamma, double bx, double by, double bz, double complex M[5][5])
{
    const int K = 2;
    double b = sqrt(bx * bx + by * by + bz * bz);
    double ct = b > 0 ? bz / b : 1.0;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double chib = (bx == 0.0 && by == 0.0) ? 0.0 : atan2(by, bx);
    for (int a = 0; a < 5; a++) {
        int Q = a - 2;
        for (int c = 0; c < 5; c++) {
            int Qp = c - 2;
            double complex k = 0.0;
            if (Qp == Q) k = Q * ct;
            else if (Qp == Q - 1) k = 0.5 * st * cexp(IU * chib) * sqrt((double)(K + Q) * (K - Q + 1));
            else if (Qp == Q + 1) k = 0.5 * st * cexp(-IU * chib) * sqrt((double)(K - Q) * (K + Q + 1));
            M[a][c] = (a == c ? 1.0 : 0.0) + IU * gamma * k;
        }
    }
}

/* real layout (X00, X20, Re X21, Im X21, Re X22, Im X22) -> complex X_Q, Q = -2..2,
   using X_{-Q} = (-1)^Q conj(X_Q) */
static void to_complex(const double *r6, double complex x[5])
{
    double complex xq[3] = {r6[1], r6[2] + IU * r6[3], r6[4] + IU * r6[5]};
    for (int a = 0; a < 5; a++) {
        int Q = a - 2;
        x[a] = Q >= 0 ? xq[Q] : ((Q % 2) ? -1.0 : 1.0) * conj(xq[-Q]);
    }
}

/* solve sum_Q' (delta_QQ' + i gamma K_QQ') S_Q' = rhs_Q for K = 2; rhs6 and s6 in the
   real layout (X00, X20, Re X21, Im X21, Re X22, Im X22); entry 0 is ignored/zeroed */
int or_hanle_solve(double gamma, double bx, double by, double bz, const double *rhs6, double *s6)
{
    double complex M[5][5], r[5], x[5];
    hanle_matrix(gamma, bx, by, bz, M);
    to_complex(rhs6, r);
    /* complex Gaussian elimination with partial pivoting */
    for (int c = 0; c < 5; c++) {
        int piv = c;
        for (int a = c + 1; a < 5; a++) if (cabs(M[a][c]) > cabs(M[piv][c])) piv = a;
        if (cabs(M[piv][c]) == 0.0) return -1;
        if (piv != c) {
            for (int q = 0; q < 5; q++) { double complex t = M[c][q]; M[c][q] = M[piv][q]; M[piv][q] = t; }
            double complex t = r[c]; r[c] = r[piv]; r[piv] = t;
        }
        for (int a = c + 1; a < 5; a++) {
            double complex f = M[a][c] / M[c][c];
            for (int q = c; q < 5; q++) M[a][q] -= f * M[c][q];
            r[a] -= f * r[c];
        }
    }
    for (int a = 4; a >= 0; a--) {
        double complex s = r[a];
        for (int q = a + 1; q < 5; q++) s -= M[a][q] * x[q];
        x[a] = s / M[a][a];
    }
    s6[0] = 0.0;
    s6[1] = creal(x[2]);
    s6[2] = creal(x[3]); s6[3] = cimag(x[3]);
    s6[4] = creal(x[4]); s6[5] = cimag(x[4]);
    return 0;
}

/*
 * The statistical-equilibrium operator of the two-level atom written as
 * A(S) = f (Eq. 2 as L rho = f): per voxel
 *   A(S)^0_0 = S^0_0 - (1-eps) J^0_0,
 *   A(S)^2_Q = S^2_Q - i (1-eps) Gamma_u sum_Q' K_QQ' S^2_Q' - (1-eps) J^2_Q,
 * with J = J[S] from the formal solution and f = eps B delta_K0 delta_Q0.
 * out = A(S) (nvox * nl, the layout of rho).
 */
int or_see_apply(const or_problem *p, const double *jkq, const double *rho, double *out)
{
    long nv = (long)p->nx * p->ny * p->nz;
    for (long v = 0; v < nv; v++) {
        double e = p->eps[v];
        if (p->model == OR_MODEL_UNPOL) {
            out[v] = rho[v] - (1.0 - e) * jkq[v];
            continue;
        }
        const double *s = rho + 6 * v, *J = jkq + 6 * v;
        double *o = out + 6 * v;
        double bx = p->bx[v], by = p->by[v], bz = p->bz[v];
        double gamma = HANLE_SENSE * (1.0 - e) * sqrt(bx * bx + by * by + bz * bz) / p->bcrit;
        double complex M[5][5], x[5];
        hanle_matrix(gamma, bx, by, bz, M);
        to_complex(s, x);
        double complex y[5];
        for (int a = 0; a < 5; a++) {
            y[a] = 0.0;
            for (int c = 0; c < 5; c++) y[a] += M[a][c] * x[c];
        }
        o[0] = s[0] - (1.0 - e) * J[0];
        o[1] = creal(y[2]) - (1.0 - e) * J[1];
        o[2] = creal(y[3]) - (1.0 - e) * J[2];
        o[3] = cimag(y[3]) - (1.0 - e) * J[3];
        o[4] = creal(y[4]) - (1.0 - e) * J[4];
        o[5] = cimag(y[4]) - (1.0 - e) * J[5];
    }
    return 0;
}

/*
 * Jacobi (ALI) update of A(S) = src for a general per-voxel right-hand side src
 * (nvox * nl, the layout of rho): the update of or_see_update with eps B
 * replaced by src^0_0 and src^2_Q added to (1-eps) J^2_Q. src = NULL is the
 * two-level problem itself (src = eps B delta_K0 delta_Q0). The coarse-grid
 * problems of the multigrid method have this form (Sec. 5.1).
 */
int or_see_update_src(const or_problem *p, const double *jkq, const double *lstar, const double *src, double *rho,
                      double *max_change)
{
    long nv = (long)p->nx * p->ny * p->nz;
    int nl = or_nl(p->model);
    double mc = 0.0;
    for (long v = 0; v < nv; v++) {
        double e = p->eps[v];
        double f0 = src ? src[v * nl] : e * p->bpl[v];
        if (p->model == OR_MODEL_UNPOL) {
            double S = rho[v];
            double dS = ((1.0 - e) * jkq[v] + f0 - S) / (1.0 - (1.0 - e) * lstar[v]);
            double ch = fabs(dS) / fabs(S);
            if (ch > mc || ch != ch) mc = ch;
            rho[v] = S + dS;
        } else {
            double *s = rho + 6 * v;
            const double *J = jkq + 6 * v;
            double S00 = s[0];
            double dS = ((1.0 - e) * J[0] + f0 - S00) / (1.0 - (1.0 - e) * lstar[v]);
            double S00n = S00 + dS;
            double rhs[6], s2[6];
            for (int c = 0; c < 6; c++) rhs[c] = (1.0 - e) * J[c] + (src && c > 0 ? src[v * nl + c] : 0.0);
            double gamma = HANLE_SENSE * (1.0 - e) *
                           sqrt(p->bx[v] * p->bx[v] + p->by[v] * p->by[v] + p->bz[v] * p->bz[v]) / p->bcrit;
            if (or_hanle_solve(gamma, p->bx[v], p->by[v], p->bz[v], rhs, s2) != 0) return -3;
            double ch = fabs(dS) / fabs(S00);
            if (ch > mc || ch != ch) mc = ch;
            for (int c = 1; c < 6; c++) {
                double d = fabs(s2[c] / S00n - s[c] / S00);
                if (d > mc || d != d) mc = d;
            }
            s[0] = S00n;
            for (int c = 1; c < 6; c++) s[c] = s2[c];
        }
    }
    if (max_change) *max_change = mc;
    return 0;
}

int or_see_update(const or_problem *p, const double *jkq, const double *lstar, double *rho, double *max_change)
{
    return or_see_update_src(p, jkq, lstar, NULL, rho, max_change);
}

/* ------------------------------------------------------------------------
 * Reverse mode of the Jacobi update (differentiation through iterations).
 * ------------------------------------------------------------------------ */

/* The K = 2 map S^2 -> M S^2 (M = 1 + i gamma K) as a real 5x5 matrix on the
   layout (S20, Re S21, Im S21, Re S22, Im S22): column c is the image of the
   c-th real unit vector. */
static void hanle_real(double gamma, double bx, double by, double bz, double R[5][5])
{
    double complex M[5][5];
    hanle_matrix(gamma, bx, by, bz, M);
    for (int c = 0; c < 5; c++) {
        double u[6] = {0, 0, 0, 0, 0, 0};
        u[1 + c] = 1.0;
        double complex x[5], y[5];
        to_complex(u, x);
        for (int a = 0; a < 5; a++) {
            y[a] = 0.0;
            for (int q = 0; q < 5; q++) y[a] += M[a][q] * x[q];
        }
        R[0][c] = creal(y[2]);
        R[1][c] = creal(y[3]); R[2][c] = cimag(y[3]);
        R[3][c] = creal(y[4]); R[4][c] = cimag(y[4]);
    }
}

/* solve A x = b (5x5, partial pivoting); A and b are overwritten */
static int solve5(double A[5][5], double *b, double *x)
{
    for (int c = 0; c < 5; c++) {
        int piv = c;
        for (int r = c + 1; r < 5; r++) if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return -1;
        if (piv != c) {
            for (int q = 0; q < 5; q++) { double t = A[c][q]; A[c][q] = A[piv][q]; A[piv][q] = t; }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < 5; r++) {
            double f = A[r][c] / A[c][c];
            for (int q = c; q < 5; q++) A[r][q] -= f * A[c][q];
            b[r] -= f * b[c];
        }
    }
    for (int r = 4; r >= 0; r--) {
        double t = b[r];
        for (int q = r + 1; q < 5; q++) t -= A[r][q] * x[q];
        x[r] = t / A[r][r];
    }
    return 0;
}

/*
 * Reverse mode of or_see_update_src for one iteration (src as there: NULL is
 * eps B delta_K0; its K = 2 part must be 0). Inputs: the unknowns before the
 * update rho, J and Lambda-bar* computed from them, and g = dL/d(rho after the
 * update). Outputs (overwritten):
 *   g_rho   dL/drho through the update's explicit dependence on rho (S^0_0),
 *   g_jkq   dL/dJ^K_Q,  g_lstar  dL/dLambda-bar*,
 *   g_eb    dL/d(eps B), or dL/dsrc^0_0 (the thermal emission term),
 *   g_b     dL/dB (3 x nvox, added for the polarized model: the Hanle term).
 * S00' = S00 + ((1-eps) J00 + eps B - S00) / D, D = 1 - (1-eps) Lambda*;
 * S2' = M(B)^-1 (1-eps) J2 with M affine in B: M = 1 + HANLE_SENSE (1-eps)/bcrit sum_c B_c N_c.
 */
int or_see_update_vjp(const or_problem *p, const double *jkq, const double *lstar, const double *src,
                      const double *rho, const double *g, double *g_rho, double *g_jkq, double *g_lstar,
                      double *g_eb, double *g_b)
{
    long nv = (long)p->nx * p->ny * p->nz;
    int nl = or_nl(p->model), nj = or_nj(p->model);
    for (long v = 0; v < nv; v++) {
        double e = p->eps[v], B = p->bpl[v];
        const double *s = rho + nl * v, *J = jkq + nj * v, *gv = g + nl * v;
        double D = 1.0 - (1.0 - e) * lstar[v];
        double num = (1.0 - e) * J[0] + (src ? src[nl * v] : e * B) - s[0];
        for (int c = 0; c < nl; c++) g_rho[nl * v + c] = 0.0;
        for (int c = 0; c < nj; c++) g_jkq[nj * v + c] = 0.0;
        g_rho[nl * v] = gv[0] * (1.0 - 1.0 / D);
        g_jkq[nj * v] = gv[0] * (1.0 - e) / D;
        g_eb[v] = gv[0] / D;
        g_lstar[v] = gv[0] * num * (1.0 - e) / (D * D);
        if (p->model == OR_MODEL_UNPOL) continue;
        double bx = p->bx[v], by = p->by[v], bz = p->bz[v];
        double gamma = HANLE_SENSE * (1.0 - e) * sqrt(bx * bx + by * by + bz * bz) / p->bcrit;
        double R[5][5], Rt[5][5], rhs[6], s2[6], z[5], b5[5];
        hanle_real(gamma, bx, by, bz, R);
        for (int c = 0; c < 6; c++) rhs[c] = (1.0 - e) * J[c];
        if (or_hanle_solve(gamma, bx, by, bz, rhs, s2) != 0) return -3;
        for (int a = 0; a < 5; a++) for (int c = 0; c < 5; c++) Rt[a][c] = R[c][a];
        for (int a = 0; a < 5; a++) b5[a] = gv[1 + a];
        if (solve5(Rt, b5, z) != 0) return -3;
        for (int a = 0; a < 5; a++) g_jkq[nj * v + 1 + a] = (1.0 - e) * z[a];
        /* dM/dB_c = HANLE_SENSE (1-eps)/bcrit N_c, N_c = M(unit field along c, gamma 1) - 1;
           dS2' = -M^-1 dM S2' */
        double unit[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        for (int c = 0; c < 3; c++) {
            double N[5][5];
            hanle_real(1.0, unit[c][0], unit[c][1], unit[c][2], N);
            double acc = 0.0;
            for (int a = 0; a < 5; a++)
                for (int q = 0; q < 5; q++) acc += z[a] * (N[a][q] - (a == q ? 1.0 : 0.0)) * s2[1 + q];
            g_b[c * nv + v] += -HANLE_SENSE * (1.0 - e) / p->bcrit * acc;
        }
    }
    return 0;
}

