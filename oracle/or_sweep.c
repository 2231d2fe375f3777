/*
 * 3D short-characteristics formal solution of the oracle (test infrastructure only).
 *
 * Sec. 3.1: for each ray direction the grid is swept in topological order;
 * the upwind point M and downwind point P of the short characteristic through
 * grid point O lie on the neighbouring horizontal planes, where the
 * transfer coefficients (emission and absorption) and the upwind Stokes
 * vector are interpolated bilinearly from the 4 surrounding nodes, or
 * biquadratically from 9 (per axis the quadratic through the nearest node and
 * its two neighbours). The grid is periodic in x and y. Bottom boundary (rays with mu > 0): I = (B, 0, 0, 0);
 * top boundary (mu < 0): I = 0; Lambda* = 0 on the boundary plane.
 * Sec. 4.2: directions in the outer loop, frequencies in the inner loop; the
 * line profile is renormalized per direction on the frequency quadrature.
 * Eq. 1: J^K_Q = sum_p sum_m w_m T^K_Q(p, Omega_m) sum_j wt_j I_p(nu_j, Omega_m).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "or_common.h"

typedef struct {
    double mu, chi, w;
    double ox, oy, oz;     /* unit direction */
    double t[18];          /* T^K_Q(i, Omega) */
    double t1[3];          /* T^1_Q(V, Omega): (T10, Re T11, Im T11) */
} or_ray;

static void make_ray(double mu, double chi, double w, or_ray *r)
{
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    r->mu = mu; r->chi = chi; r->w = w;
    r->ox = st * cos(chi); r->oy = st * sin(chi); r->oz = mu;
    or_tkq(mu, chi, r->t);
    /* T^1_Q(V, Omega) = sqrt(3/2) Omega_Q, the spherical components of the direction:
       Omega_0 = Omega_z, Omega_{+1} = -(Omega_x + i Omega_y)/sqrt(2) */
    r->t1[0] = sqrt(1.5) * r->oz;
    r->t1[1] = -sqrt(0.75) * r->ox;
    r->t1[2] = -sqrt(0.75) * r->oy;
}

/* node coefficients at an interpolation corner: each node's coefficients are
   computed once per (ray, frequency) in the algorithm; the oracle recomputes
   them per corner, which the flop count leaves out */
static void node_coeffs(const or_problem *p, const double *rho, long v, const or_ray *r, double x,
                        double eta[7], double eps[4]);
static void corner_coeffs(const or_problem *p, const double *rho, long v, const or_ray *r, double x,
                          double eta[7], double eps[4])
{
    int on = or_count_on;
    or_count_on = 0;
    node_coeffs(p, rho, v, r, x, eta, eps);
    or_count_on = on;
}

static long vox(const or_problem *p, int i, int j, int k) { return ((long)k * p->ny + j) * p->nx + i; }

/* Doppler shift (Doppler widths) of the profile seen along the ray: the
   vertical velocity projected on Omega. */
static double shift(const or_problem *p, long v, const or_ray *r) { return p->vel ? p->vel[v] * r->oz : 0.0; }

/* Emission source vector S_i(Omega) = sum_KQ (-1)^Q T^K_Q(i,Omega) S^K_{-Q}
   = S00 T00 + S20 T20 + 2 Re(T21 conj S21) + 2 Re(T22 conj S22)   (i = I, Q, U) */
static double angular_source(const double *t6, const double *s)
{
    return t6[0] * s[0] + t6[1] * s[1] + 2.0 * (t6[2] * s[2] + t6[3] * s[3]) + 2.0 * (t6[4] * s[4] + t6[5] * s[5]);
}

/* sum_Q (-1)^Q T^1_Q S^1_{-Q} = T10 S10 + 2 Re(T11 conj S11) (rank-1 tensors, S^1_-Q = -conj S^1_Q) */
static double angular1(const double *t1, const double *s)
{
    return t1[0] * s[0] + 2.0 * (t1[1] * s[1] + t1[2] * s[2]);
}

/*
 * Transfer coefficients at a grid node for ray r and reduced frequency x:
 *   eta_I = chi exp(-(x - s)^2)    (line-centre opacity times the Gaussian profile shape)
 * Unpolarized two-level atom: eps_I = eta_I S.
 * Polarized two-level atom (Jl = 0 -> Ju = 1, w^(2) = 1): eps_i = eta_I S_i(Omega), i = I, Q, U;
 * weak-field Zeeman: eta_V = -gbar zeta (B.Omega) d(eta_I)/dx = 2 gbar zeta (x - s)(B.Omega) eta_I,
 * eps_V = S^0_0 eta_V; rho_Q = rho_U = rho_V = 0. With dichroism multipoles D^2_Q (the
 * atomic polarization of the lower level of a multilevel line, p->dich), eta_i = eta_I
 * [delta_i0 + sum_Q (-1)^Q T^2_Q(i, Omega) D^2_-Q] for i = I, Q, U (eta_V and the
 * emissivities stay relative to eta_I = chi phi); otherwise eta_Q = eta_U = 0.
 */
static void node_coeffs(const or_problem *p, const double *rho, long v, const or_ray *r, double x,
                        double eta[7], double eps[4])
{
    double xs = x - shift(p, v, r);
    double etaI = p->chi[v] * exp(-xs * xs);
    for (int q = 0; q < 7; q++) eta[q] = 0.0;
    eta[0] = etaI;
    OR_FLOPS(5);
    if (p->model == OR_MODEL_UNPOL) {
        eps[0] = etaI * rho[v];
        OR_FLOPS(1);
        return;
    }
    if (p->kexpl) {
        /* explicit medium: K'/eta_I and S given per voxel (a general propagation matrix) */
        long nv = (long)p->nx * p->ny * p->nz;
        for (int q = 1; q < 7; q++) eta[q] = etaI * p->kexpl[(q - 1) * nv + v];
        for (int i = 0; i < 4; i++) eps[i] = etaI * p->sexpl[i * nv + v];
        OR_FLOPS(10);
        return;
    }
    const double *s = rho + 6 * v;
    double bpar = p->bx[v] * r->ox + p->by[v] * r->oy + p->bz[v] * r->oz;
    eta[3] = 2.0 * p->gbar * p->zeta * xs * bpar * etaI;
    for (int i = 0; i < 3; i++) eps[i] = etaI * angular_source(r->t + 6 * i, s);
    eps[3] = s[0] * eta[3];
    OR_FLOPS(5 + 5 + 3 * 12 + 1);
    if (p->orient) eps[3] += etaI * angular1(r->t1, p->orient + 3 * v);
    if (p->dich1) eta[3] += etaI * angular1(r->t1, p->dich1 + 3 * v);
    if (p->dich) {
        const double *d = p->dich + 5 * v;
        const double d6[6] = {1.0, d[0], d[1], d[2], d[3], d[4]};
        for (int i = 0; i < 3; i++) eta[i] = etaI * angular_source(r->t + 6 * i, d6);
    }
}

/* bilinear interpolation weights on a periodic plane at cell coordinates (xc, yc) */
static void bilinear(const or_problem *p, double xc, double yc, int ii[4], int jj[4], double w[4])
{
    double fx0 = floor(xc), fy0 = floor(yc);
    double fx = xc - fx0, fy = yc - fy0;
    long i0 = (long)fx0, j0 = (long)fy0;
    int ia = (int)(((i0 % p->nx) + p->nx) % p->nx), ja = (int)(((j0 % p->ny) + p->ny) % p->ny);
    int ib = (ia + 1) % p->nx, jb = (ja + 1) % p->ny;
    ii[0] = ia; jj[0] = ja; w[0] = (1 - fx) * (1 - fy);
    ii[1] = ib; jj[1] = ja; w[1] = fx * (1 - fy);
    ii[2] = ia; jj[2] = jb; w[2] = (1 - fx) * fy;
    ii[3] = ib; jj[3] = jb; w[3] = fx * fy;
}

/* biquadratic interpolation weights on a periodic plane at cell coordinates (xc, yc):
   per axis the Lagrange quadratic through the nearest node n and n - 1, n + 1,
   evaluated at the offset f = xc - n in [-1/2, 1/2) */
static void biquadratic(const or_problem *p, double xc, double yc, int ii[9], int jj[9], double w[9])
{
    double nxn = floor(xc + 0.5), nyn = floor(yc + 0.5);
    double fx = xc - nxn, fy = yc - nyn;
    double wx[3] = {0.5 * fx * (fx - 1.0), (1.0 - fx) * (1.0 + fx), 0.5 * fx * (fx + 1.0)};
    double wy[3] = {0.5 * fy * (fy - 1.0), (1.0 - fy) * (1.0 + fy), 0.5 * fy * (fy + 1.0)};
    long i0 = (long)nxn, j0 = (long)nyn;
    for (int b = 0; b < 3; b++)
        for (int a = 0; a < 3; a++) {
            int c = 3 * b + a;
            ii[c] = (int)((((i0 + a - 1) % p->nx) + p->nx) % p->nx);
            jj[c] = (int)((((j0 + b - 1) % p->ny) + p->ny) % p->ny);
            w[c] = wx[a] * wy[b];
        }
}

int or_interp_weights(const or_problem *p, double xc, double yc, int order, int *ii, int *jj, double *w)
{
    if (order == 2) {
        biquadratic(p, xc, yc, ii, jj, w);
        return 9;
    }
    bilinear(p, xc, yc, ii, jj, w);
    return 4;
}

/* the bilinear stencil of a point on the first cell face that the short characteristic
   through node (i, j) crosses between planes k (fraction 0) and k2 (fraction 1), the
   horizontal offset over that layer being (fx, fy) cells with |fx| or |fy| above 1 (a
   vertical face): s = 1/max(|fx|, |fy|) of the layer, the face x = x_(i + sgn fx) when
   |fx| >= |fy| (offset fy s along y, between rows j and j + sgn fy), else y = y_(j + sgn fy);
   nodes (ii, jj, kk) with weights w; returns the fraction s */
static double face_stencil(const or_problem *p, int i, int j, int k, int k2, double fx, double fy,
                           int ii[4], int jj[4], int kk[4], double w[4])
{
    const int nx = p->nx, ny = p->ny;
    const double ax = fabs(fx), ay = fabs(fy);
    const double s = 1.0 / (ax >= ay ? ax : ay);
    const int sx = fx > 0 ? 1 : (fx < 0 ? -1 : 0), sy = fy > 0 ? 1 : (fy < 0 ? -1 : 0);
    int i0, j0, i1, j1;                 /* the two nodes along the face's horizontal direction */
    double g;                           /* weight of the second one */
    if (ax >= ay) {
        i0 = i1 = i + sx;
        j0 = j;
        j1 = j + (sy != 0 ? sy : 1);
        g = ay * s;
    } else {
        j0 = j1 = j + sy;
        i0 = i;
        i1 = i + (sx != 0 ? sx : 1);
        g = ax * s;
    }
    i0 = ((i0 % nx) + nx) % nx; i1 = ((i1 % nx) + nx) % nx;
    j0 = ((j0 % ny) + ny) % ny; j1 = ((j1 % ny) + ny) % ny;
    ii[0] = i0; jj[0] = j0; kk[0] = k;  w[0] = (1.0 - g) * (1.0 - s);
    ii[1] = i1; jj[1] = j1; kk[1] = k;  w[1] = g * (1.0 - s);
    ii[2] = i0; jj[2] = j0; kk[2] = k2; w[2] = (1.0 - g) * s;
    ii[3] = i1; jj[3] = j1; kk[3] = k2; w[3] = g * s;
    return s;
}

/* plane k of a sweep whose upwind or downwind characteristic meets a vertical face
   (sc_faces = 1): every point from the face stencils (or the plane stencil where the
   offset stays within one cell), the points of the plane in the upwind order, the pass
   repeated until no intensity changes by more than 1e-15 of the plane's largest
   (the upwind face's upper nodes are points of this plane; the periodic wrap closes
   their chain on itself) */
static int sweep_plane_faces(const or_problem *p, const double *rho, const or_ray *r, double x, double *I,
                             double *lstar, int k, int ku, int kd, int has_p, double dsM, double dsP)
{
    const int ns = or_ns(p->model), nx = p->nx, ny = p->ny;
    const double dx = p->lx / nx, dy = p->ly / ny;
    /* horizontal offsets (cells) from O to the upwind plane (backwards) and the downwind plane */
    const double fxM = -dsM * r->ox / dx, fyM = -dsM * r->oy / dy;
    const double fxP = dsP * r->ox / dx, fyP = dsP * r->oy / dy;
    const int vertM = fabs(fxM) > 1.0 || fabs(fyM) > 1.0;
    const int vertP = has_p && (fabs(fxP) > 1.0 || fabs(fyP) > 1.0);
    /* upwind order: a point depends on its neighbours towards the upwind offset */
    const int di = fxM < 0 ? 1 : -1, dj = fyM < 0 ? 1 : -1;
    for (int pass = 0; pass < 100000; pass++) {
        double change = 0.0, big = 0.0;
        for (int jn = 0; jn < ny; jn++)
            for (int in = 0; in < nx; in++) {
                const int i = di > 0 ? in : nx - 1 - in, j = dj > 0 ? jn : ny - 1 - jn;
                const long v = vox(p, i, j, k);
                int ii[9], jj[9], kk[9];
                double w[9];
                double etaM[7] = {0}, epsM[4] = {0}, IM[4] = {0};
                double sM = 1.0;
                int nc;
                if (vertM) {
                    sM = face_stencil(p, i, j, k, ku, fxM, fyM, ii, jj, kk, w);
                    nc = 4;
                } else {
                    nc = or_interp_weights(p, i + fxM, j + fyM, 1, ii, jj, w);
                    for (int c = 0; c < nc; c++) kk[c] = ku;
                }
                for (int c = 0; c < nc; c++) {
                    const long u = vox(p, ii[c], jj[c], kk[c]);
                    double e7[7], e4[4];
                    corner_coeffs(p, rho, u, r, x, e7, e4);
                    for (int q = 0; q < 7; q++) etaM[q] += w[c] * e7[q];
                    for (int s = 0; s < ns; s++) { epsM[s] += w[c] * e4[s]; IM[s] += w[c] * I[u * ns + s]; }
                }
                double etaO[7], epsO[4];
                node_coeffs(p, rho, v, r, x, etaO, epsO);
                double etaP = 0.0, epsP[4] = {0}, sP = 1.0;
                if (has_p) {
                    if (vertP) {
                        sP = face_stencil(p, i, j, k, kd, fxP, fyP, ii, jj, kk, w);
                        nc = 4;
                    } else {
                        nc = or_interp_weights(p, i + fxP, j + fyP, 1, ii, jj, w);
                        for (int c = 0; c < nc; c++) kk[c] = kd;
                    }
                    for (int c = 0; c < nc; c++) {
                        const long u = vox(p, ii[c], jj[c], kk[c]);
                        double e7[7], e4[4];
                        corner_coeffs(p, rho, u, r, x, e7, e4);
                        etaP += w[c] * e7[0];
                        for (int s = 0; s < ns; s++) epsP[s] += w[c] * e4[s];
                    }
                }
                double Io[4], lo;
                if (or_step(ns, IM, etaM, epsM, etaO, epsO, etaP, epsP, sM * dsM, sP * dsP, has_p, p->method, Io,
                            &lo) != 0)
                    return -3;
                for (int s = 0; s < ns; s++) {
                    change = fmax(change, fabs(Io[s] - I[v * ns + s]));
                    big = fmax(big, fabs(Io[s]));
                    I[v * ns + s] = Io[s];
                }
                lstar[v] = lo;
            }
        if (!vertM || change <= 1e-15 * big) return 0;
    }
    return -4;
}

/* one (ray, frequency) sweep; I (nvox*ns) and lstar (nvox) are outputs */
static int sweep(const or_problem *p, const double *rho, const or_ray *r, double x, double *I, double *lstar)
{
    int ns = or_ns(p->model);
    int nx = p->nx, ny = p->ny, nz = p->nz;
    double dx = p->lx / nx, dy = p->ly / ny;
    int up = r->mu > 0;
    for (int ks = 0; ks < nz; ks++) {
        int k = up ? ks : nz - 1 - ks;
        if (ks == 0) {
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    long v = vox(p, i, j, k);
                    for (int s = 0; s < ns; s++) I[v * ns + s] = 0.0;
                    if (up) I[v * ns] = p->bpl[v];
                    lstar[v] = 0.0;
                }
            continue;
        }
        int ku = up ? k - 1 : k + 1;
        int has_p = ks + 1 < nz;
        int kd = up ? k + 1 : k - 1;
        double amu = fabs(r->mu);
        double dsM = fabs(p->z[k] - p->z[ku]) / amu;
        double dsP = has_p ? fabs(p->z[kd] - p->z[k]) / amu : 0.0;
        const int order = p->interp == 2 ? 2 : 1;
        if (p->sc_faces && (fabs(dsM * r->ox / dx) > 1.0 || fabs(dsM * r->oy / dy) > 1.0 ||
                            (has_p && (fabs(dsP * r->ox / dx) > 1.0 || fabs(dsP * r->oy / dy) > 1.0)))) {
            for (long v = vox(p, 0, 0, k); v < vox(p, 0, 0, k) + (long)nx * ny; v++)
                for (int s = 0; s < ns; s++) I[v * ns + s] = 0.0;
            int rc = sweep_plane_faces(p, rho, r, x, I, lstar, k, ku, kd, has_p, dsM, dsP);
            if (rc) return rc;
            continue;
        }
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long v = vox(p, i, j, k);
                int ii[9], jj[9];
                double w[9];
                double etaM[7] = {0}, epsM[4] = {0}, IM[4] = {0};
                int nc = or_interp_weights(p, i - dsM * r->ox / dx, j - dsM * r->oy / dy, order, ii, jj, w);
                for (int c = 0; c < nc; c++) {
                    long u = vox(p, ii[c], jj[c], ku);
                    double e7[7], e4[4];
                    corner_coeffs(p, rho, u, r, x, e7, e4);
                    for (int q = 0; q < 7; q++) etaM[q] += w[c] * e7[q];
                    for (int s = 0; s < ns; s++) { epsM[s] += w[c] * e4[s]; IM[s] += w[c] * I[u * ns + s]; }
                }
                OR_FLOPS(4 * 2 * (2 + 2 * ns));   /* eta_I, eta_V, eps, I at 4 corners */
                double etaO[7], epsO[4];
                node_coeffs(p, rho, v, r, x, etaO, epsO);
                double etaP = 0.0, epsP[4] = {0};
                if (has_p) {
                    nc = or_interp_weights(p, i + dsP * r->ox / dx, j + dsP * r->oy / dy, order, ii, jj, w);
                    for (int c = 0; c < nc; c++) {
                        long u = vox(p, ii[c], jj[c], kd);
                        double e7[7], e4[4];
                        corner_coeffs(p, rho, u, r, x, e7, e4);
                        etaP += w[c] * e7[0];
                        for (int s = 0; s < ns; s++) epsP[s] += w[c] * e4[s];
                    }
                    OR_FLOPS(4 * 2 * (1 + ns));
                }
                double lo;
                if (or_step(ns, IM, etaM, epsM, etaO, epsO, etaP, epsP, dsM, dsP, has_p, p->method,
                            I + v * ns, &lo) != 0)
                    return -3;
                lstar[v] = lo;
            }
    }
    return 0;
}

static int check(const or_problem *p)
{
    if (!p || p->nx < 1 || p->ny < 1 || p->nz < 2 || p->n_mu < 1 || p->n_chi < 1 || p->n_nu < 1) return -1;
    if (p->model != OR_MODEL_UNPOL && p->model != OR_MODEL_HANLE) return -1;
    if (p->model == OR_MODEL_HANLE && (!p->bx || !p->by || !p->bz)) return -1;
    if (p->interp < 0 || p->interp > 2) return -1;
    if (p->sc_faces != 0 && p->sc_faces != 1) return -1;
    if (p->sc_faces && p->interp == 2) return -1;         /* vertical faces: bilinear stencils */
    return 0;
}

int or_sweep_ray(const or_problem *p, const double *rho, int m, int j, double *I, double *lstar)
{
    if (check(p)) return -1;
    int nr = or_nray(p);
    if (m < 0 || m >= nr || j < 0 || j >= p->n_nu) return -1;
    double *mu = malloc(sizeof(double) * nr), *ch = malloc(sizeof(double) * nr), *w = malloc(sizeof(double) * nr);
    double *xf = malloc(sizeof(double) * p->n_nu), *wf = malloc(sizeof(double) * p->n_nu);
    or_rays(p, mu, ch, w);
    or_freqs(p->n_nu, p->x_max, xf, wf);
    or_ray r;
    make_ray(mu[m], ch[m], w[m], &r);
    int rc = sweep(p, rho, &r, xf[j], I, lstar);
    free(mu); free(ch); free(w); free(xf); free(wf);
    return rc;
}

int or_formal_solve_part(const or_problem *p, const double *rho, int m0, int m1, int j0, int j1,
                         double *jkq, double *lstar)
{
    if (check(p)) return -1;
    int ns = or_ns(p->model), nj = or_nj(p->model), nr = or_nray(p), nn = p->n_nu;
    long nv = (long)p->nx * p->ny * p->nz;
    if (m0 < 0 || m1 > nr || m0 > m1 || j0 < 0 || j1 > nn || j0 > j1) return -1;
    double *mu = malloc(sizeof(double) * nr), *ch = malloc(sizeof(double) * nr), *w = malloc(sizeof(double) * nr);
    double *xf = malloc(sizeof(double) * nn), *wf = malloc(sizeof(double) * nn);
    double *I = malloc(sizeof(double) * nv * ns), *lo = malloc(sizeof(double) * nv);
    double *norm = malloc(sizeof(double) * nv);
    if (!mu || !ch || !w || !xf || !wf || !I || !lo || !norm) return -2;
    or_rays(p, mu, ch, w);
    or_freqs(nn, p->x_max, xf, wf);
    memset(jkq, 0, sizeof(double) * nv * nj);
    memset(lstar, 0, sizeof(double) * nv);
    if (p->j1) memset(p->j1, 0, sizeof(double) * nv * 3);
    int rc = 0;
    for (int m = m0; m < m1 && rc == 0; m++) {                 /* directions: outer loop */
        or_ray r;
        make_ray(mu[m], ch[m], w[m], &r);
        /* profile normalization on the frequency quadrature, per voxel and direction */
        for (long v = 0; v < nv; v++) {
            double s = shift(p, v, &r), sum = 0.0;
            for (int j = 0; j < nn; j++) sum += wf[j] * exp(-(xf[j] - s) * (xf[j] - s)) / sqrt(M_PI);
            norm[v] = sum;
        }
        for (int j = j0; j < j1 && rc == 0; j++) {             /* frequencies: inner loop */
            rc = sweep(p, rho, &r, xf[j], I, lo);
            for (long v = 0; v < nv; v++) {
                double xs = xf[j] - shift(p, v, &r);
                double wt = r.w * wf[j] * exp(-xs * xs) / sqrt(M_PI) / norm[v];
                const double *Iv = I + v * ns;
                if (p->model == OR_MODEL_UNPOL) {
                    jkq[v] += wt * Iv[0];
                    OR_FLOPS(2);
                } else {
                    for (int c = 0; c < 6; c++)
                        jkq[v * 6 + c] += wt * (r.t[c] * Iv[0] + r.t[6 + c] * Iv[1] + r.t[12 + c] * Iv[2]);
                    OR_FLOPS(6 * 7);
                    if (p->j1)
                        for (int c = 0; c < 3; c++) p->j1[v * 3 + c] += wt * r.t1[c] * Iv[3];
                }
                lstar[v] += wt * lo[v];
                OR_FLOPS(2 + 7);   /* Lambda* accumulation; weight (profile and normalization) */
            }
        }
    }
    free(mu); free(ch); free(w); free(xf); free(wf); free(I); free(lo); free(norm);
    return rc;
}

int or_formal_solve(const or_problem *p, const double *rho, double *jkq, double *lstar)
{
    if (check(p)) return -1;
    return or_formal_solve_part(p, rho, 0, or_nray(p), 0, p->n_nu, jkq, lstar);
}

int or_emergent(const or_problem *p, const double *rho, int ndir, const double *mu, const double *chi, double *out)
{
    if (check(p)) return -1;
    int ns = or_ns(p->model), nn = p->n_nu;
    long nv = (long)p->nx * p->ny * p->nz, nxy = (long)p->nx * p->ny;
    double *xf = malloc(sizeof(double) * nn), *wf = malloc(sizeof(double) * nn);
    double *I = malloc(sizeof(double) * nv * ns), *lo = malloc(sizeof(double) * nv);
    if (!xf || !wf || !I || !lo) return -2;
    or_freqs(nn, p->x_max, xf, wf);
    int rc = 0;
    for (int d = 0; d < ndir && rc == 0; d++) {
        if (!(mu[d] > 0.0 && mu[d] <= 1.0)) { rc = -1; break; }
        or_ray r;
        make_ray(mu[d], chi[d], 0.0, &r);
        for (int j = 0; j < nn && rc == 0; j++) {
            rc = sweep(p, rho, &r, xf[j], I, lo);
            const double *top = I + (long)(p->nz - 1) * nxy * ns;
            memcpy(out + ((long)d * nn + j) * nxy * ns, top, sizeof(double) * nxy * ns);
        }
    }
    free(xf); free(wf); free(I); free(lo);
    return rc;
}

/* ------------------------------------------------------------------------
 * Adjoint of the emergent Stokes vector (reverse-mode sweep).
 *
 * Parameters per voxel: chi (line-centre opacity), e = chi S^0_0 (emission
 * scale; the multipoles S^K_Q = rho^K_Q scale as e/chi with their ratios to
 * S^0_0 held fixed) and B = (Bx, By, Bz). With phi = exp(-(x - s)^2) and
 * beta = 2 gbar zeta, the node coefficients are
 *   eta_I = chi phi,           eta_V = beta (x - s)(B.Omega) chi phi,
 *   eps_i = e phi S_i/S^0_0,   eps_V = beta (x - s)(B.Omega) e phi
 * (unpolarized atom: eps_I = e phi). The boundary intensity at the bottom is
 * the Planck function, not a parameter.
 * ------------------------------------------------------------------------ */
/* add the parameter gradients of node v given dL/d(eta 7 elements) and dL/d(eps) at frequency x */
static void node_vjp(const or_problem *p, const double *rho, long v, const or_ray *r, double x,
                     const double *g_eta, const double *g_eps, double *g_chi, double *g_e, double *g_b)
{
    long nv = (long)p->nx * p->ny * p->nz;
    double xs = x - shift(p, v, r);
    double phi = exp(-xs * xs);
    if (p->model == OR_MODEL_UNPOL) {
        g_chi[v] += phi * g_eta[0];
        g_e[v] += phi * g_eps[0];
        return;
    }
    const double *s = rho + 6 * v;
    double beta = 2.0 * p->gbar * p->zeta;
    double bpar = p->bx[v] * r->ox + p->by[v] * r->oy + p->bz[v] * r->oz;
    double chi = p->chi[v], e = chi * s[0];
    g_chi[v] += phi * g_eta[0] + beta * xs * bpar * phi * g_eta[3];
    double ge = beta * xs * bpar * phi * g_eps[3];
    for (int i = 0; i < 3; i++) ge += phi * angular_source(r->t + 6 * i, s) / s[0] * g_eps[i];
    g_e[v] += ge;
    double gb = beta * xs * phi * (chi * g_eta[3] + e * g_eps[3]);
    g_b[v] += gb * r->ox;
    g_b[nv + v] += gb * r->oy;
    g_b[2 * nv + v] += gb * r->oz;
}

int or_emergent_vjp(const or_problem *p, const double *rho, int ndir, const double *mu, const double *chi,
                    const double *gout, double *g_chi, double *g_e, double *g_b)
{
    if (p && (p->interp == 2 || p->kexpl)) return -1;   /* reverse mode: bilinear, two-level media only */
    if (check(p)) return -1;
    if (p->model != OR_MODEL_UNPOL && !g_b) return -1;
    int ns = or_ns(p->model), nn = p->n_nu;
    int nx = p->nx, ny = p->ny, nz = p->nz;
    long nv = (long)nx * ny * nz, nxy = (long)nx * ny;
    double dx = p->lx / nx, dy = p->ly / ny;
    double *xf = malloc(sizeof(double) * nn), *wf = malloc(sizeof(double) * nn);
    double *I = malloc(sizeof(double) * nv * ns), *lo = malloc(sizeof(double) * nv);
    double *lam = malloc(sizeof(double) * nv * ns);
    if (!xf || !wf || !I || !lo || !lam) return -2;
    or_freqs(nn, p->x_max, xf, wf);
    memset(g_chi, 0, sizeof(double) * nv);
    memset(g_e, 0, sizeof(double) * nv);
    if (g_b) memset(g_b, 0, sizeof(double) * 3 * nv);
    int rc = 0;
    for (int d = 0; d < ndir && rc == 0; d++) {
        if (!(mu[d] > 0.0 && mu[d] <= 1.0)) { rc = -1; break; }
        or_ray r;
        make_ray(mu[d], chi[d], 0.0, &r);
        double amu = fabs(r.mu);
        for (int jf = 0; jf < nn && rc == 0; jf++) {
            double x = xf[jf];
            rc = sweep(p, rho, &r, x, I, lo);                    /* forward: I on every plane */
            memset(lam, 0, sizeof(double) * nv * ns);
            memcpy(lam + (long)(nz - 1) * nxy * ns, gout + ((long)d * nn + jf) * nxy * ns, sizeof(double) * nxy * ns);
            for (int k = nz - 1; k >= 1 && rc == 0; k--) {       /* planes in reverse sweep order */
                int ku = k - 1, kd = k + 1, has_p = k + 1 < nz;
                double dsM = fabs(p->z[k] - p->z[ku]) / amu;
                double dsP = has_p ? fabs(p->z[kd] - p->z[k]) / amu : 0.0;
                for (int j = 0; j < ny; j++)
                    for (int i = 0; i < nx; i++) {
                        long v = vox(p, i, j, k);
                        int iM[4], jM[4], iP[4], jP[4];
                        double wM[4], wP[4];
                        double etaM[7] = {0}, epsM[4] = {0}, IM[4] = {0};
                        bilinear(p, i - dsM * r.ox / dx, j - dsM * r.oy / dy, iM, jM, wM);
                        for (int c = 0; c < 4; c++) {
                            long u = vox(p, iM[c], jM[c], ku);
                            double e7[7], e4[4];
                            node_coeffs(p, rho, u, &r, x, e7, e4);
                            for (int q = 0; q < 7; q++) etaM[q] += wM[c] * e7[q];
                            for (int s = 0; s < ns; s++) { epsM[s] += wM[c] * e4[s]; IM[s] += wM[c] * I[u * ns + s]; }
                        }
                        double etaO[7], epsO[4];
                        node_coeffs(p, rho, v, &r, x, etaO, epsO);
                        double etaP = 0.0, epsP[4] = {0};
                        if (has_p) {
                            bilinear(p, i + dsP * r.ox / dx, j + dsP * r.oy / dy, iP, jP, wP);
                            for (int c = 0; c < 4; c++) {
                                long u = vox(p, iP[c], jP[c], kd);
                                double e7[7], e4[4];
                                node_coeffs(p, rho, u, &r, x, e7, e4);
                                etaP += wP[c] * e7[0];
                                for (int s = 0; s < ns; s++) epsP[s] += wP[c] * e4[s];
                            }
                        }
                        double gIM[4], gEM[7], gSM[4], gEO[7], gSO[4], gEP, gSP[4];
                        if (or_step_vjp(ns, IM, etaM, epsM, etaO, epsO, etaP, epsP, dsM, dsP, has_p, p->method,
                                        lam + v * ns, gIM, gEM, gSM, gEO, gSO, &gEP, gSP) != 0) {
                            rc = -3;
                            break;
                        }
                        /* transposed bilinear interpolation at M: scatter to the 4 upwind nodes */
                        for (int c = 0; c < 4; c++) {
                            long u = vox(p, iM[c], jM[c], ku);
                            double ge7[7], ge4[4];
                            for (int s = 0; s < ns; s++) lam[u * ns + s] += wM[c] * gIM[s];
                            for (int q = 0; q < 7; q++) ge7[q] = wM[c] * gEM[q];
                            for (int s = 0; s < ns; s++) ge4[s] = wM[c] * gSM[s];
                            node_vjp(p, rho, u, &r, x, ge7, ge4, g_chi, g_e, g_b);
                        }
                        node_vjp(p, rho, v, &r, x, gEO, gSO, g_chi, g_e, g_b);
                        if (has_p)
                            for (int c = 0; c < 4; c++) {
                                long u = vox(p, iP[c], jP[c], kd);
                                double ge7[7] = {wP[c] * gEP, 0, 0, 0, 0, 0, 0}, ge4[4];
                                for (int s = 0; s < ns; s++) ge4[s] = wP[c] * gSP[s];
                                node_vjp(p, rho, u, &r, x, ge7, ge4, g_chi, g_e, g_b);
                            }
                    }
            }
        }
    }
    free(xf); free(wf); free(I); free(lo); free(lam);
    return rc;
}

/* ------------------------------------------------------------------------
 * Reverse mode in the unknowns rho (differentiation through iterations):
 * node coefficients as functions of chi, rho and B (eps_i = chi phi S_i(rho),
 * eps_V = S00 eta_V), and the J^K_Q / Lambda-bar* sums of a formal solution.
 * ------------------------------------------------------------------------ */

/* add dL/dchi (at fixed rho), dL/drho and dL/dB of node v from dL/d(eta 7) and dL/d(eps) */
static void node_vjp_rho(const or_problem *p, const double *rho, long v, const or_ray *r, double x,
                         const double *g_eta, const double *g_eps, double *g_chi, double *g_rho, double *g_b)
{
    long nv = (long)p->nx * p->ny * p->nz;
    double xs = x - shift(p, v, r);
    double phi = exp(-xs * xs);
    double chi = p->chi[v], etaI = chi * phi;
    if (p->model == OR_MODEL_UNPOL) {
        g_chi[v] += phi * g_eta[0] + phi * rho[v] * g_eps[0];
        g_rho[v] += etaI * g_eps[0];
        return;
    }
    const double *s = rho + 6 * v;
    double beta = 2.0 * p->gbar * p->zeta;
    double bpar = p->bx[v] * r->ox + p->by[v] * r->oy + p->bz[v] * r->oz;
    double etaV = beta * xs * bpar * etaI;
    double gc = phi * g_eta[0] + beta * xs * bpar * phi * (g_eta[3] + s[0] * g_eps[3]);
    for (int i = 0; i < 3; i++) {
        const double *t = r->t + 6 * i;
        gc += phi * angular_source(t, s) * g_eps[i];
        double gS = etaI * g_eps[i];
        g_rho[6 * v + 0] += gS * t[0];
        g_rho[6 * v + 1] += gS * t[1];
        for (int c = 2; c < 6; c++) g_rho[6 * v + c] += gS * 2.0 * t[c];
    }
    g_rho[6 * v + 0] += etaV * g_eps[3];
    g_chi[v] += gc;
    double gb = beta * xs * phi * chi * (g_eta[3] + s[0] * g_eps[3]);
    g_b[v] += gb * r->ox;
    g_b[nv + v] += gb * r->oy;
    g_b[2 * nv + v] += gb * r->oz;
}

/* one (ray, frequency) reverse sweep: lam (nv*ns) holds dL/dI seeded by the caller or by
   the injections (J weights wj per voxel and Lambda* weights wl per voxel, both may be NULL) */
static int reverse_sweep(const or_problem *p, const double *rho, const or_ray *r, double x, const double *I,
                         double *lam, const double *gj_dir, const double *wj, const double *wl,
                         double *g_chi, double *g_rho, double *g_b)
{
    int ns = or_ns(p->model);
    int nx = p->nx, ny = p->ny, nz = p->nz;
    double dx = p->lx / nx, dy = p->ly / ny, amu = fabs(r->mu);
    int up = r->mu > 0;
    for (int ks = nz - 1; ks >= 1; ks--) {
        int k = up ? ks : nz - 1 - ks;
        int ku = up ? k - 1 : k + 1, kd = up ? k + 1 : k - 1, has_p = ks + 1 < nz;
        double dsM = fabs(p->z[k] - p->z[ku]) / amu;
        double dsP = has_p ? fabs(p->z[kd] - p->z[k]) / amu : 0.0;
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long v = vox(p, i, j, k);
                /* dL/dI_O from J^K_Q = sum w T I (injection) */
                if (wj)
                    for (int q = 0; q < (ns == 1 ? 1 : 3); q++) lam[v * ns + q] += wj[v] * gj_dir[v * 3 + q];
                int iM[4], jM[4], iP[4], jP[4];
                double wM[4], wP[4];
                double etaM[7] = {0}, epsM[4] = {0}, IM[4] = {0};
                bilinear(p, i - dsM * r->ox / dx, j - dsM * r->oy / dy, iM, jM, wM);
                for (int c = 0; c < 4; c++) {
                    long u = vox(p, iM[c], jM[c], ku);
                    double e7[7], e4[4];
                    node_coeffs(p, rho, u, r, x, e7, e4);
                    for (int q = 0; q < 7; q++) etaM[q] += wM[c] * e7[q];
                    for (int q = 0; q < ns; q++) { epsM[q] += wM[c] * e4[q]; IM[q] += wM[c] * I[u * ns + q]; }
                }
                double etaO[7], epsO[4];
                node_coeffs(p, rho, v, r, x, etaO, epsO);
                double etaP = 0.0, epsP[4] = {0};
                if (has_p) {
                    bilinear(p, i + dsP * r->ox / dx, j + dsP * r->oy / dy, iP, jP, wP);
                    for (int c = 0; c < 4; c++) {
                        long u = vox(p, iP[c], jP[c], kd);
                        double e7[7], e4[4];
                        node_coeffs(p, rho, u, r, x, e7, e4);
                        etaP += wP[c] * e7[0];
                        for (int q = 0; q < ns; q++) epsP[q] += wP[c] * e4[q];
                    }
                }
                double gIM[4], gEM[7], gSM[4], gEO[7], gSO[4], gEP, gSP[4];
                if (or_step_vjp(ns, IM, etaM, epsM, etaO, epsO, etaP, epsP, dsM, dsP, has_p, p->method,
                                lam + v * ns, gIM, gEM, gSM, gEO, gSO, &gEP, gSP) != 0)
                    return -3;
                if (wl && wl[v] != 0.0) {
                    /* Lambda* = w_O + w_C c_M(0,1,0) of the step depends on tau_MO only (BESSER) */
                    double tau = 0.5 * (etaM[0] + etaO[0]) * dsM, c[6], dc[6];
                    or_coeffs(tau, c);
                    or_coeffs_deriv(tau, c, dc);
                    double gt = wl[v] * (dc[4] + (has_p ? 1.0 : 0.5) * dc[5]);
                    gEM[0] += 0.5 * dsM * gt;
                    gEO[0] += 0.5 * dsM * gt;
                }
                for (int c = 0; c < 4; c++) {
                    long u = vox(p, iM[c], jM[c], ku);
                    double ge7[7], ge4[4];
                    for (int q = 0; q < ns; q++) lam[u * ns + q] += wM[c] * gIM[q];
                    for (int q = 0; q < 7; q++) ge7[q] = wM[c] * gEM[q];
                    for (int q = 0; q < ns; q++) ge4[q] = wM[c] * gSM[q];
                    node_vjp_rho(p, rho, u, r, x, ge7, ge4, g_chi, g_rho, g_b);
                }
                node_vjp_rho(p, rho, v, r, x, gEO, gSO, g_chi, g_rho, g_b);
                if (has_p)
                    for (int c = 0; c < 4; c++) {
                        long u = vox(p, iP[c], jP[c], kd);
                        double ge7[7] = {wP[c] * gEP, 0, 0, 0, 0, 0, 0}, ge4[4];
                        for (int q = 0; q < ns; q++) ge4[q] = wP[c] * gSP[q];
                        node_vjp_rho(p, rho, u, r, x, ge7, ge4, g_chi, g_rho, g_b);
                    }
            }
    }
    return 0;
}

/*
 * Gradients of L = sum g_jkq J^K_Q + sum g_lstar Lambda-bar* (J and Lambda-bar*
 * of or_formal_solve at rho) with respect to chi (at fixed rho), rho and B;
 * ADDED to g_chi (nvox), g_rho (nvox*nl) and g_b (3*nvox; ignored for the
 * unpolarized model). BESSER only.
 */
int or_jkq_vjp(const or_problem *p, const double *rho, const double *g_jkq, const double *g_lstar,
               double *g_chi, double *g_rho, double *g_b)
{
    if (p && (p->interp == 2 || p->kexpl)) return -1;   /* reverse mode: bilinear, two-level media only */
    if (check(p) || p->method != OR_BESSER) return -1;
    int ns = or_ns(p->model), nj = or_nj(p->model), nr = or_nray(p), nn = p->n_nu;
    long nv = (long)p->nx * p->ny * p->nz;
    double *mu = malloc(sizeof(double) * nr), *ch = malloc(sizeof(double) * nr), *w = malloc(sizeof(double) * nr);
    double *xf = malloc(sizeof(double) * nn), *wf = malloc(sizeof(double) * nn);
    double *I = malloc(sizeof(double) * nv * ns), *lo = malloc(sizeof(double) * nv), *lam = malloc(sizeof(double) * nv * ns);
    double *norm = malloc(sizeof(double) * nv), *wj = malloc(sizeof(double) * nv), *wl = malloc(sizeof(double) * nv);
    double *gdir = malloc(sizeof(double) * nv * 3);
    if (!mu || !ch || !w || !xf || !wf || !I || !lo || !lam || !norm || !wj || !wl || !gdir) return -2;
    or_rays(p, mu, ch, w);
    or_freqs(nn, p->x_max, xf, wf);
    int rc = 0;
    for (int m = 0; m < nr && rc == 0; m++) {
        or_ray r;
        make_ray(mu[m], ch[m], w[m], &r);
        for (long v = 0; v < nv; v++) {
            double s = shift(p, v, &r), sum = 0.0;
            for (int j = 0; j < nn; j++) sum += wf[j] * exp(-(xf[j] - s) * (xf[j] - s)) / sqrt(M_PI);
            norm[v] = sum;
            /* dL/dI_p per unit weight: sum_c T^K_Q(p, Omega) g_J^K_Q */
            for (int q = 0; q < 3; q++) {
                double a = 0.0;
                if (p->model == OR_MODEL_UNPOL) { if (q == 0) a = g_jkq[v]; }
                else for (int c = 0; c < 6; c++) a += r.t[6 * q + c] * g_jkq[v * nj + c];
                gdir[v * 3 + q] = a;
            }
        }
        for (int j = 0; j < nn && rc == 0; j++) {
            rc = sweep(p, rho, &r, xf[j], I, lo);
            if (rc) break;
            for (long v = 0; v < nv; v++) {
                double xs = xf[j] - shift(p, v, &r);
                double wt = r.w * wf[j] * exp(-xs * xs) / sqrt(M_PI) / norm[v];
                wj[v] = wt;
                wl[v] = wt * g_lstar[v];
            }
            memset(lam, 0, sizeof(double) * nv * ns);
            rc = reverse_sweep(p, rho, &r, xf[j], I, lam, gdir, wj, wl, g_chi, g_rho, g_b);
        }
    }
    free(mu); free(ch); free(w); free(xf); free(wf); free(I); free(lo); free(lam);
    free(norm); free(wj); free(wl); free(gdir);
    return rc;
}

/* adjoint of or_emergent in the unknowns: dL/dchi (fixed rho), dL/drho, dL/dB (overwritten) */
int or_emergent_vjp_rho(const or_problem *p, const double *rho, int ndir, const double *mu, const double *chi,
                        const double *gout, double *g_chi, double *g_rho, double *g_b)
{
    if (p && (p->interp == 2 || p->kexpl)) return -1;   /* reverse mode: bilinear, two-level media only */
    if (check(p)) return -1;
    int ns = or_ns(p->model), nn = p->n_nu, nl = or_nl(p->model);
    long nv = (long)p->nx * p->ny * p->nz, nxy = (long)p->nx * p->ny;
    double *xf = malloc(sizeof(double) * nn), *wf = malloc(sizeof(double) * nn);
    double *I = malloc(sizeof(double) * nv * ns), *lo = malloc(sizeof(double) * nv);
    double *lam = malloc(sizeof(double) * nv * ns);
    if (!xf || !wf || !I || !lo || !lam) return -2;
    or_freqs(nn, p->x_max, xf, wf);
    memset(g_chi, 0, sizeof(double) * nv);
    memset(g_rho, 0, sizeof(double) * nv * nl);
    if (g_b) memset(g_b, 0, sizeof(double) * 3 * nv);
    int rc = 0;
    for (int d = 0; d < ndir && rc == 0; d++) {
        if (!(mu[d] > 0.0 && mu[d] <= 1.0)) { rc = -1; break; }
        or_ray r;
        make_ray(mu[d], chi[d], 0.0, &r);
        for (int jf = 0; jf < nn && rc == 0; jf++) {
            rc = sweep(p, rho, &r, xf[jf], I, lo);
            if (rc) break;
            memset(lam, 0, sizeof(double) * nv * ns);
            memcpy(lam + (long)(p->nz - 1) * nxy * ns, gout + ((long)d * nn + jf) * nxy * ns, sizeof(double) * nxy * ns);
            rc = reverse_sweep(p, rho, &r, xf[jf], I, lam, NULL, NULL, NULL, g_chi, g_rho, g_b);
        }
    }
    free(xf); free(wf); free(I); free(lo); free(lam);
    return rc;
}

