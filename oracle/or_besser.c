/*
 * BESSER formal solver of the oracle (test infrastructure only).
 * Sec. 3.2 (control points, steps 1-9), Sec. 3.3 (Eqs. 7-14, Table 1).
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
    c[3] = t < 0.14 ? series_omega_m(t) : (2.0 - e * (t2 + 2.0 * t + 2.0)) / t2;   /* Eq. 11 */
    c[4] = t < 0.18 ? series_omega_o(t) : 1.0 - 2.0 * (e + t - 1.0) / t2;          /* Eq. 12 */
    c[5] = t < 0.18 ? series_omega_c(t) : 2.0 * (t - 2.0 + e * (t + 2.0)) / t2;    /* Eq. 13 */
    OR_FLOPS(30);
}

static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

/*
 * Upwind control point c_M of the quadratic Bezier spline on MO (Sec. 3.2,
 * steps 1-9). h_M = tau_MO, h_P = tau_OP. Without a downwind point the
 * interpolation on MO is linear, c_M = (y_M + y_O)/2. DELOPAR is the
 * parabola through M, O, P (step 4 without the overshoot checks). The linear
 * method is the Bezier curve with c_M at the midpoint (a straight line).
 * BEZIER_FB takes the derivative at O from the weighted harmonic mean of the
 * two one-sided slopes (Fritsch & Butland 1984; 0 where they differ in sign),
 * and CBEZIER adds the upwind overshoot test of steps 5-6.
 */
double or_control_point(double yM, double yO, double yP, double hM, double hP, int has_p, int method)
{
    if (!has_p || method == OR_LINEAR) { OR_FLOPS(2); OR_BRANCH(4); return 0.5 * (yM + yO); }
    double dM = (yO - yM) / hM;                          /* step 1 */
    double dP = (yP - yO) / hP;
    OR_FLOPS(4);
    if (method == OR_DELOPAR) {
        double yp = (hM * dP + hP * dM) / (hM + hP);
        OR_FLOPS(9);
        return yO - 0.5 * hM * yp;
    }
    if (method == OR_BEZIER_FB || method == OR_CBEZIER) {
        if (dM * dP <= 0.0) return yO;
        /* 1/y'_O = alpha/d_M + (1 - alpha)/d_P, alpha = (1 + h_P/(h_M + h_P))/3 */
        double alpha = (1.0 + hP / (hM + hP)) / 3.0;
        double yp = dM * dP / (alpha * dP + (1.0 - alpha) * dM);
        double cM = yO - 0.5 * hM * yp;
        OR_FLOPS(12);
        if (method == OR_CBEZIER && (cM < dmin(yM, yO) || cM > dmax(yM, yO))) return yM;
        return cM;
    }
    OR_FLOPS(1);
    if (dM * dP <= 0.0) { OR_BRANCH(0); return yO; }     /* step 2 */
    double yp = (hM * dP + hP * dM) / (hM + hP);         /* step 3, Eq. 6 */
    double cM = yO - 0.5 * hM * yp;                      /* step 4 */
    double cP = yO + 0.5 * hP * yp;
    OR_FLOPS(11);
    if (cM < dmin(yM, yO) || cM > dmax(yM, yO)) {        /* step 5 */
        OR_BRANCH(1);
        return yM;                                       /* step 6 */
    }
    int clip = cP < dmin(yO, yP) || cP > dmax(yO, yP);   /* step 7 */
    if (clip) cP = yP;
    OR_BRANCH(clip ? 2 : 3);
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
        if (method == OR_LINEAR) {
            /* S linear on MO: I_O = e I_M + psi'_M S_M + psi'_O S_O (Sec. 3.3) */
            I[i] = c[0] * I[i - 1] + c[1] * S[i - 1] + c[2] * S[i];
            continue;
        }
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
 * One BESSER step at point O (Eqs. 7-14):
 *   kappa^-1 I_O = [e^-tau 1 - psi'_M K'_M] I_M + w_M S_M + w_O S_O + w_C c_M,
 *   kappa^-1 = 1 + psi'_O K'_O,
 * with S = eps/eta_I, tau_MO = (eta_M + eta_O)/2 * ds_M and
 * tau_OP = (eta_O + eta_P)/2 * ds_P (trapezoid along the segments).
 * Lambda* = w_O + w_C c_M(0,1,0): the paper's w_O + w_C (Eq. 14) where a
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

/* ------------------------------------------------------------------------
 * Reverse mode of the step (adjoint sweep of the emergent Stokes vector).
 * ------------------------------------------------------------------------ */

/* d/dt of (e^-t, psi'_M, psi'_O, w_M, w_O, w_C), differentiating the closed
   forms of Eqs. 9-13 and writing the result through the coefficients
   themselves:
     de = -e,               dpsi'_M = e - psi'_M/t,   dpsi'_O = psi'_M/t,
     dw_M = e - 2 w_M/t,    dw_O = w_C/t,             dw_C = 2 (psi'_M - w_C)/t.
   In these forms the cancellation is at most a factor of a few for every
   t > 0, so the derivatives are as accurate as the coefficients. */
void or_coeffs_deriv(double t, const double c[6], double dc[6])
{
    dc[0] = -c[0];
    dc[1] = c[0] - c[1] / t;
    dc[2] = c[1] / t;
    dc[3] = c[0] - 2.0 * c[3] / t;
    dc[4] = c[5] / t;
    dc[5] = 2.0 * (c[1] - c[5]) / t;
}

/* Gradient of the control point (or_control_point) with respect to
   (y_M, y_O, y_P, h_M, h_P), times gc, on the branch the control point takes:
   reverse mode through steps 1-9 in the opposite order. */
void or_control_point_vjp(double yM, double yO, double yP, double hM, double hP, int has_p, int method,
                          double gc, double g[5])
{
    for (int i = 0; i < 5; i++) g[i] = 0.0;
    if (!has_p) { g[0] = 0.5 * gc; g[1] = 0.5 * gc; return; }
    double dM = (yO - yM) / hM, dP = (yP - yO) / hP;
    double s = hM + hP;
    double yp = (hM * dP + hP * dM) / s;
    double g_yp;
    if (method == OR_DELOPAR) {
        /* c = y_O - h_M y'_O / 2 */
        g[1] += gc;
        g[3] += -0.5 * yp * gc;
        g_yp = -0.5 * hM * gc;
    } else {
        if (dM * dP <= 0.0) { g[1] = gc; return; }                      /* step 2 */
        double cM = yO - 0.5 * hM * yp, cP = yO + 0.5 * hP * yp;
        if (cM < dmin(yM, yO) || cM > dmax(yM, yO)) { g[0] = gc; return; }   /* step 6 */
        int clip = cP < dmin(yO, yP) || cP > dmax(yO, yP);               /* step 7 */
        double cPv = clip ? yP : cP;
        double yp2 = (cPv - yO) / (0.5 * hP);
        /* step 9: c = y_O - h_M yp2 / 2 */
        g[1] += gc;
        g[3] += -0.5 * yp2 * gc;
        double g_yp2 = -0.5 * hM * gc;
        /* step 8: yp2 = 2 (c_P - y_O) / h_P */
        double g_cP = 2.0 * g_yp2 / hP;
        g[1] -= 2.0 * g_yp2 / hP;
        g[4] -= 2.0 * (cPv - yO) / (hP * hP) * g_yp2;
        if (clip) { g[2] += g_cP; return; }
        /* step 4: c_P = y_O + h_P y'_O / 2 */
        g[1] += g_cP;
        g[4] += 0.5 * yp * g_cP;
        g_yp = 0.5 * hP * g_cP;
    }
    /* step 3 (Eq. 6): y'_O = (h_M d_P + h_P d_M) / (h_M + h_P) */
    g[3] += (dP - yp) / s * g_yp;
    g[4] += (dM - yp) / s * g_yp;
    double g_dP = hM / s * g_yp, g_dM = hP / s * g_yp;
    /* step 1 */
    g[1] += g_dM / hM;
    g[0] -= g_dM / hM;
    g[3] -= dM / hM * g_dM;
    g[2] += g_dP / hP;
    g[1] -= g_dP / hP;
    g[4] -= dP / hP * g_dP;
}

/* gradient of K' (kprime) with respect to the seven propagation-matrix elements, added to g_eta */
static void kprime_vjp(const double *eta, double gK[4][4], double *g_eta)
{
    double a = 1.0 / eta[0];
    double gx[7];
    gx[1] = gK[0][1] + gK[1][0];       /* eta_Q */
    gx[2] = gK[0][2] + gK[2][0];       /* eta_U */
    gx[3] = gK[0][3] + gK[3][0];       /* eta_V */
    gx[4] = gK[2][3] - gK[3][2];       /* rho_Q */
    gx[5] = gK[3][1] - gK[1][3];       /* rho_U */
    gx[6] = gK[1][2] - gK[2][1];       /* rho_V */
    for (int i = 1; i < 7; i++) {
        g_eta[i] += gx[i] * a;
        g_eta[0] -= gx[i] * eta[i] * a * a;
    }
}

/*
 * Reverse mode of or_step: given gIO = dL/dI_O, the gradients with respect
 * to I_M, the interpolated propagation matrix and emissivity at M, the node
 * values at O and the interpolated eta_I and emissivity at P (all outputs are
 * overwritten). kappa^-1 I_O = rhs gives d rhs = kappa^-T gIO and
 * d(kappa^-1) = -d rhs I_O^T; the rest follows the forward step backwards.
 */
int or_step_vjp(int ns, const double *IM, const double *etaM, const double *epsM,
                const double *etaO, const double *epsO, double etaP_I, const double *epsP,
                double dsM, double dsP, int has_p, int method, const double *gIO,
                double *gIM, double *g_etaM, double *g_epsM, double *g_etaO, double *g_epsO,
                double *g_etaP, double *g_epsP)
{
    double SM[4], SO[4], SP[4] = {0, 0, 0, 0};
    for (int s = 0; s < ns; s++) {
        SM[s] = epsM[s] / etaM[0];
        SO[s] = epsO[s] / etaO[0];
        if (has_p) SP[s] = epsP[s] / etaP_I;
    }
    double tauMO = 0.5 * (etaM[0] + etaO[0]) * dsM;
    double tauOP = has_p ? 0.5 * (etaO[0] + etaP_I) * dsP : 0.0;
    double c[6];
    or_coeffs(tauMO, c);
    double cM[4];
    for (int s = 0; s < ns; s++) cM[s] = or_control_point(SM[s], SO[s], SP[s], tauMO, tauOP, has_p, method);

    double g_c[6] = {0, 0, 0, 0, 0, 0}, g_SM[4] = {0, 0, 0, 0}, g_SO[4] = {0, 0, 0, 0};
    double g_SP[4] = {0, 0, 0, 0}, g_cM[4] = {0, 0, 0, 0};
    for (int s = 0; s < ns; s++) { gIM[s] = 0.0; g_epsM[s] = 0.0; g_epsO[s] = 0.0; g_epsP[s] = 0.0; }
    for (int q = 0; q < 7; q++) { g_etaM[q] = 0.0; g_etaO[q] = 0.0; }
    *g_etaP = 0.0;
    if (ns == 1) {
        /* I_O = e I_M + w_M S_M + w_O S_O + w_C c_M */
        double g = gIO[0];
        g_c[0] = g * IM[0]; gIM[0] = g * c[0];
        g_c[3] = g * SM[0]; g_SM[0] = g * c[3];
        g_c[4] = g * SO[0]; g_SO[0] = g * c[4];
        g_c[5] = g * cM[0]; g_cM[0] = g * c[5];
    } else {
        double kM[4][4], kO[4][4], A[4][4], At[4][4], rhs[4], IO[4], g_rhs[4], b[4];
        kprime(etaM, kM);
        kprime(etaO, kO);
        for (int r = 0; r < 4; r++) {
            double acc = c[0] * IM[r];
            for (int s = 0; s < 4; s++) acc -= c[1] * kM[r][s] * IM[s];
            rhs[r] = acc + c[3] * SM[r] + c[4] * SO[r] + c[5] * cM[r];
            for (int s = 0; s < 4; s++) A[r][s] = (r == s ? 1.0 : 0.0) + c[2] * kO[r][s];
        }
        for (int r = 0; r < 4; r++)
            for (int s = 0; s < 4; s++) At[r][s] = A[s][r];
        double Ac[4][4];
        for (int r = 0; r < 4; r++) { b[r] = rhs[r]; for (int s = 0; s < 4; s++) Ac[r][s] = A[r][s]; }
        if (gauss_solve(4, Ac, b, IO) != 0) return -1;
        for (int r = 0; r < 4; r++) b[r] = gIO[r];
        if (gauss_solve(4, At, b, g_rhs) != 0) return -1;
        double g_kM[4][4], g_kO[4][4];
        for (int r = 0; r < 4; r++)
            for (int s = 0; s < 4; s++) {
                double gA = -g_rhs[r] * IO[s];
                g_c[2] += gA * kO[r][s];
                g_kO[r][s] = c[2] * gA;
                g_kM[r][s] = 0.0;
            }
        for (int r = 0; r < 4; r++) {
            g_c[0] += g_rhs[r] * IM[r];
            gIM[r] += c[0] * g_rhs[r];
            for (int s = 0; s < 4; s++) {
                g_c[1] -= g_rhs[r] * kM[r][s] * IM[s];
                g_kM[r][s] -= g_rhs[r] * c[1] * IM[s];
                gIM[s] -= g_rhs[r] * c[1] * kM[r][s];
            }
            g_c[3] += g_rhs[r] * SM[r]; g_SM[r] += c[3] * g_rhs[r];
            g_c[4] += g_rhs[r] * SO[r]; g_SO[r] += c[4] * g_rhs[r];
            g_c[5] += g_rhs[r] * cM[r]; g_cM[r] += c[5] * g_rhs[r];
        }
        kprime_vjp(etaM, g_kM, g_etaM);
        kprime_vjp(etaO, g_kO, g_etaO);
    }
    double g_hM = 0.0, g_hP = 0.0;
    for (int s = 0; s < ns; s++) {
        double g5[5];
        or_control_point_vjp(SM[s], SO[s], SP[s], tauMO, tauOP, has_p, method, g_cM[s], g5);
        g_SM[s] += g5[0]; g_SO[s] += g5[1]; g_SP[s] += g5[2];
        g_hM += g5[3]; g_hP += g5[4];
    }
    double dc[6];
    or_coeffs_deriv(tauMO, c, dc);
    for (int i = 0; i < 6; i++) g_hM += g_c[i] * dc[i];
    g_etaM[0] += 0.5 * dsM * g_hM;
    g_etaO[0] += 0.5 * dsM * g_hM;
    if (has_p) {
        g_etaO[0] += 0.5 * dsP * g_hP;
        *g_etaP += 0.5 * dsP * g_hP;
    }
    for (int s = 0; s < ns; s++) {
        g_epsM[s] += g_SM[s] / etaM[0];
        g_etaM[0] -= g_SM[s] * SM[s] / etaM[0];
        g_epsO[s] += g_SO[s] / etaO[0];
        g_etaO[0] -= g_SO[s] * SO[s] / etaO[0];
        if (has_p) {
            g_epsP[s] += g_SP[s] / etaP_I;
            *g_etaP -= g_SP[s] * SP[s] / etaP_I;
        }
    }
    return 0;
}
