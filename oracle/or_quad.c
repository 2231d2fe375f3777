/*
 * Quadratures of the oracle (test infrastructure only).
 *
 * Angles: Gauss-Legendre inclinations per hemisphere and equally weighted
 * (trapezoid on a periodic interval) azimuths, the product rule of App. A
 * (Gauss inclinations x trapezoid azimuths per octant). Azimuths sit at the
 * interval midpoints chi_a = (a+1/2) 2pi/Nchi.
 * Frequencies: uniform grid on [-x_max, x_max] with trapezoid weights.
 */
#include <math.h>
#include <stdlib.h>
#include "or_common.h"

int or_count_on = 0;
long long or_count = 0;
void or_flops_reset(int enable) { or_count_on = enable; or_count = 0; }
long long or_flops_get(void) { return or_count; }
int or_sig_on = 0;
unsigned long long or_sig = 14695981039346656037ULL;
void or_branch_sig_reset(int enable) { or_sig_on = enable; or_sig = 14695981039346656037ULL; }
unsigned long long or_branch_sig_get(void) { return or_sig; }

int or_nl(int model) { return model == OR_MODEL_UNPOL ? 1 : 6; }
int or_ns(int model) { return model == OR_MODEL_UNPOL ? 1 : 4; }
int or_nj(int model) { return model == OR_MODEL_UNPOL ? 1 : 6; }
int or_nray(const or_problem *p) { return 2 * p->n_mu * p->n_chi; }

/* Gauss-Legendre nodes and weights on (0,1): Newton iteration on P_n(2x-1),
   the three-term Legendre recurrence gives P_n and P_{n-1}. */
int or_gauss_legendre01(int n, double *x, double *w)
{
    if (n < 1) return -1;
    for (int i = 0; i < n; i++) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double pn = 0, pn1 = 0, dp = 1;
        for (int it = 0; it < 200; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            pn = (n == 1) ? z : p1;
            pn1 = (n == 1) ? 1.0 : p0;
            dp = n * (z * pn - pn1) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-15) break;
        }
        {   /* derivative at the converged root */
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            pn = (n == 1) ? z : p1;
            pn1 = (n == 1) ? 1.0 : p0;
            dp = n * (z * pn - pn1) / (z * z - 1.0);
        }
        /* root i is descending in z; store ascending in x = (1+z)/2 */
        x[n - 1 - i] = 0.5 * (1.0 + z);
        w[n - 1 - i] = 0.5 * 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* Ray m = ((h*n_mu) + i)*n_chi + a; h = 0 upward (mu > 0), h = 1 downward.
   Weights include 1/(4 pi): sum_m w_m = 1. */
int or_rays(const or_problem *p, double *mu, double *chi, double *w)
{
    int nm = p->n_mu, nc = p->n_chi;
    double *xg = (double *)malloc(sizeof(double) * nm), *wg = (double *)malloc(sizeof(double) * nm);
    if (!xg || !wg) { free(xg); free(wg); return -2; }
    or_gauss_legendre01(nm, xg, wg);
    for (int h = 0; h < 2; h++)
        for (int i = 0; i < nm; i++)
            for (int a = 0; a < nc; a++) {
                int m = (h * nm + i) * nc + a;
                mu[m] = h == 0 ? xg[i] : -xg[i];
                chi[m] = (a + 0.5) * 2.0 * M_PI / nc;
                w[m] = 0.5 * wg[i] / nc;
            }
    free(xg); free(wg);
    return 0;
}

int or_freqs(int n_nu, double x_max, double *x, double *w)
{
    if (n_nu < 1) return -1;
    if (n_nu == 1) { x[0] = 0.0; w[0] = 1.0; return 0; }
    double dx = 2.0 * x_max / (n_nu - 1);
    for (int j = 0; j < n_nu; j++) {
        x[j] = -x_max + j * dx;
        w[j] = (j == 0 || j == n_nu - 1) ? 0.5 * dx : dx;
    }
    return 0;
}

/*
 * T^K_Q(i, Omega) for K = 0, 2 and i = I, Q, U (Eq. 1; the irreducible
 * spherical tensors of LL04 Table 5.6), reference angle gamma = 0: the
 * polarization reference direction e_a lies in the plane of Omega and the
 * z axis, e_a = d(Omega)/d(theta), e_b = z x Omega / |z x Omega|.
 * Output t[i*6 + c], c = (T^0_0, T^2_0, Re T^2_1, Im T^2_1, Re T^2_2, Im T^2_2);
 * components Q < 0 follow from T^K_{-Q} = (-1)^Q conj(T^K_Q).
 */
void or_tkq(double mu, double chi, double t[18])
{
    double st2 = 1.0 - mu * mu;
    double st = sqrt(st2 > 0 ? st2 : 0.0);
    double r3 = sqrt(3.0), r2 = sqrt(2.0);
    double c1 = cos(chi), s1 = sin(chi), c2 = cos(2 * chi), s2 = sin(2 * chi);
    /* Stokes I */
    t[0] = 1.0;
    t[1] = (3.0 * mu * mu - 1.0) / (2.0 * r2);
    t[2] = -0.5 * r3 * mu * st * c1;
    t[3] = -0.5 * r3 * mu * st * s1;
    t[4] = 0.25 * r3 * st2 * c2;
    t[5] = 0.25 * r3 * st2 * s2;
    /* Stokes Q */
    t[6] = 0.0;
    t[7] = -3.0 / (2.0 * r2) * st2;
    t[8] = -0.5 * r3 * mu * st * c1;
    t[9] = -0.5 * r3 * mu * st * s1;
    t[10] = -0.25 * r3 * (1.0 + mu * mu) * c2;
    t[11] = -0.25 * r3 * (1.0 + mu * mu) * s2;
    /* Stokes U */
    t[12] = 0.0;
    t[13] = 0.0;
    t[14] = 0.5 * r3 * st * s1;
    t[15] = -0.5 * r3 * st * c1;
    t[16] = 0.5 * r3 * mu * s2;
    t[17] = -0.5 * r3 * mu * c2;
}
