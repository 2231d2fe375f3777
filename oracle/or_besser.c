/*
 * BESSER formal solver of the oracle (test infrastructure only).
 * Sec. 3.2 (control points, steps 1-9), Sec. 3.3 (Eqs. 7-13, Table 1).
 */
#include <math.h>
#include "or_common.h"

/* Table 1 Taylor expansions (Horner form), used below the thresholds the
   table gives for double precision: omega_M 0.14, omega_O and omega_C 0.18. */
static double series_omega_m(double t)
{
    return (t*(t*(t*(t*(t*(t*((140.0-18.0*t)*t-945.0)+5400.0)-25200.0)+90720.0)-226800.0)+302400.0))/907200.0;
}
static double series_omega_o(double t)
{
    return (t*(t*(t*(t*(t*(t*((10.0-t)*t-90.0)+720.0)-5040.0)+30240.0)-151200.0)+604800.0))/1814400.0;
}
static double series_omega_c(double t)
{
    return (t*(t*(t*(t*(t*(t*((35.0-4.0*t)*t-270.0)+1800.0)-10080.0)+45360.0)-151200.0)+302400.0))/907200.0;
}
/* psi' expansions are not printed in the paper. They are the Taylor series of
   the closed forms of Sec. 3.3 to t^8:
   psi'_M = sum_{n>=2} (-1)^n (n-1) t^(n-1) / n!,  psi'_O = sum_{n>=2} (-1)^n t^(n-1) / n!. */
static double series_psi(double t, int which)
{
    double r = 0.0, f = 1.0;       /* f = n! */
    double tp = 1.0;               /* t^(n-1) */
    for (int n = 1; n <= 9; n++) {
        f *= n;
        if (n >= 2) {
            double a = (which == 0 ? (n - 1.0) : 1.0) / f;
            r += ((n % 2 == 0) ? a : -a) * tp;
        }
        tp *= t;
    }
    return r;
}

void or_coeffs(double t, double c[6])
{
    double e = exp(-t);
    c[0] = e;
    if (t < 0.1) {
        c[1] = series_psi(t, 0);
        c[2] = series_psi(t, 1);
    } else {
        c[1] = (1.0 - e * (1.0 + t)) / t;          /* psi'_M */
        c[2] = (e + t - 1.0) / t;                  /* psi'_O */
    }
    double t2 = t * t;
    c[3] = t < 0.14 ? series_omega_m(t) : (2.0 - e * (t2 + 2.0 * t + 2.0)) / t2;   /* Eq. 10 */
    c[4] = t < 0.18 ? series_omega_o(t) : 1.0 - 2.0 * (e + t - 1.0) / t2;          /* Eq. 11 */
    c[5] = t < 0.18 ? series_omega_c(t) : 2.0 * (t - 2.0 + e * (t + 2.0)) / t2;    /* Eq. 12 */
    OR_FLOPS(30);
}

static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

/*
 * Upwind control point c_M of the quadratic Bezier spline on MO (Sec. 3.2,
 * steps 1-9). h_M = tau_MO, h_P = tau_OP. Without a downwind point the
 * interpolation on MO is linear, c_M = (y_M + y_O)/2. DELOPAR is the
 * parabola through M, O, P (step 4 without the overshoot checks).
 */
double or_control_point(double yM, double yO, double yP, double hM, double hP, int has_p, int method)
{
    if (!has_p) { OR_FLOPS(2); return 0.5 * (yM + yO); }
    double dM = (yO - yM) / hM;                          /* step 1 */
    double dP = (yP - yO) / hP;
    OR_FLOPS(4);
    if (method == OR_DELOPAR) {
        double yp = (hM * dP + hP * dM) / (hM + hP);
        OR_FLOPS(9);
        return yO - 0.5 * hM * yp;
    }
    OR_FLOPS(1);
    if (dM * dP <= 0.0) return yO;                       /* step 2 */
    double yp = (hM * dP + hP * dM) / (hM + hP);         /* step 3, Eq. 6 */
    double cM = yO - 0.5 * hM * yp;                      /* step 4 */
    double cP = yO + 0.5 * hP * yp;
    OR_FLOPS(11);
    if (cM < dmin(yM, yO) || cM > dmax(yM, yO))          /* step 5 */
        return yM;                                       /* step 6 */
    if (cP < dmin(yO, yP) || cP > dmax(yO, yP))          /* step 7 */
        cP = yP;
    yp = (cP - yO) / (0.5 * hP);                         /* step 8 */
    OR_FLOPS(6);
    return yO - 0.5 * hM * yp;                           /* step 9 */
}

/* One-ray unpolarized solution on optical-depth nodes tau[0..n-1] (increasing
   along the propagation direction), boundary intensity I0 at node 0. */
int or_solve_1d(int n, const double *tau, const double *S, double I0, int method, double *I)
{
    if (n < 1) return -1;
    I[0] = I0;
    for (int i = 1; i < n; i++) {
        double hM = tau[i] - tau[i - 1];
        int has_p = i + 1 < n;
        double hP = has_p ? tau[i + 1] - tau[i] : 0.0;
        double c[6];
        or_coeffs(hM, c);
        double cM = or_control_point(S[i - 1], S[i], has_p ? S[i + 1] : 0.0, hM, hP, has_p, method);
        I[i] = c[0] * I[i - 1] + c[3] * S[i - 1] + c[4] * S[i] + c[5] * cM;
    }
    return 0;
}

/* normalized propagation matrix K' = K/eta_I - 1 (Sec. 3.1) from the seven
   elements (eta_I, eta_Q, eta_U, eta_V, rho_Q, rho_U, rho_V) */
static void kprime(const double *eta, double kp[4][4])
{
    double a = 1.0 / eta[0];
    double q = eta[1] * a, u = eta[2] * a, v = eta[3] * a;
    double rq = eta[4] * a, ru = eta[5] * a, rv = eta[6] * a;
    double K[4][4] = {{0, q, u, v}, {q, 0, rv, -ru}, {u, -rv, 0, rq}, {v, ru, -rq, 0}};
    for (int r = 0; r < 4; r++) for (int s = 0; s < 4; s++) kp[r][s] = K[r][s];
    OR_FLOPS(7);
}

/* solve A x = b (n x n) by Gaussian elimination with partial pivoting */
static int gauss_solve(int n, double A[4][4], double *b, double *x)
{
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++) if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return -1;
        if (piv != c) {
            for (int s = 0; s < n; s++) { double t = A[c][s]; A[c][s] = A[piv][s]; A[piv][s] = t; }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; r++) {
            double f = A[r][c] / A[c][c];
            for (int s = c; s < n; s++) A[r][s] -= f * A[c][s];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = b[r];
        for (int q = r + 1; q < n; q++) s -= A[r][q] * x[q];
        x[r] = s / A[r][r];
    }
    return 0;
}

/*
 * One BESSER step at point O (Eqs. 7-13):
 *   kappa^-1 I_O = [e^-tau 1 - psi'_M K'_M] I_M + w_M S_M + w_O S_O + w_C c_M,
 *   kappa^-1 = 1 + psi'_O K'_O,
 * with S = eps/eta_I, tau_MO = (eta_M + eta_O)/2 * ds_M and
 * tau_OP = (eta_O + eta_P)/2 * ds_P (trapezoid along the segments).
 * Lambda* = w_O + w_C c_M(0,1,0): the paper's w_O + w_C (Eq. 13) where a
 * downwind point exists, w_O + w_C/2 on the last plane of a sweep.
 */
int or_step(int ns, const double *IM, const double *etaM, const double *epsM,
            const double *etaO, const double *epsO, double etaP_I, const double *epsP,
            double dsM, double dsP, int has_p, int method, double *IO, double *lstar)
{
    double SM[4], SO[4], SP[4] = {0, 0, 0, 0};
    for (int s = 0; s < ns; s++) {
        SM[s] = epsM[s] / etaM[0];
        SO[s] = epsO[s] / etaO[0];
        if (has_p) SP[s] = epsP[s] / etaP_I;
    }
    OR_FLOPS(3 * ns);
    double tauMO = 0.5 * (etaM[0] + etaO[0]) * dsM;
    double tauOP = has_p ? 0.5 * (etaO[0] + etaP_I) * dsP : 0.0;
    OR_FLOPS(6);
    double c[6];
    or_coeffs(tauMO, c);
    double cM[4];
    for (int s = 0; s < ns; s++)
        cM[s] = or_control_point(SM[s], SO[s], SP[s], tauMO, tauOP, has_p, method);
    double rhs[4];
    if (ns == 1) {
        IO[0] = c[0] * IM[0] + c[3] * SM[0] + c[4] * SO[0] + c[5] * cM[0];
        OR_FLOPS(7);
    } else {
        double kM[4][4], kO[4][4], A[4][4];
        kprime(etaM, kM);
        kprime(etaO, kO);
        for (int r = 0; r < 4; r++) {
            double acc = c[0] * IM[r];
            for (int s = 0; s < 4; s++) acc -= c[1] * kM[r][s] * IM[s];
            rhs[r] = acc + c[3] * SM[r] + c[4] * SO[r] + c[5] * cM[r];
            for (int s = 0; s < 4; s++) A[r][s] = (r == s ? 1.0 : 0.0) + c[2] * kO[r][s];
        }
        /* 4x4: rhs 4*(1 + 4*2 + 6) ; A 4*4*2 ; elimination ~ 2n^3/3 + 2n^2 */
        OR_FLOPS(60 + 32 + 75);
        if (gauss_solve(4, A, rhs, IO) != 0) return -1;
    }
    /* impulse response of the control point: S_M = S_P = 0, S_O = 1 */
    double cM1;
    if (method == OR_BESSER) {
        cM1 = has_p ? 1.0 : 0.5;
    } else {
        int on = or_count_on;
        or_count_on = 0;
        cM1 = or_control_point(0.0, 1.0, 0.0, tauMO, tauOP, has_p, method);
        or_count_on = on;
    }
    *lstar = c[4] + c[5] * cM1;
    OR_FLOPS(2);
    return 0;
}
