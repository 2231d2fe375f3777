/*
 * Plain FP64 CPU oracle of the PORTA formal-solver hot path
 * (Stepan & Trujillo Bueno 2013, arXiv:1307.4217).
 *
 * TEST INFRASTRUCTURE ONLY. This code exists so that tests, the smoke check
 * and the CPU-baseline leg of the benchmark can check the CUDA library against
 * a slow, obviously correct restatement of the paper. The product path never
 * calls it, and it shares no code, header or table with the CUDA library.
 *
 * Everything is double precision, single threaded, with loops in the order
 * the paper gives (directions outer, frequencies inner, Sec. 4.2; grid planes
 * in topological order, Sec. 3.1).
 *
 * Voxel index: v = (k*ny + j)*nx + i, i along x, j along y, k along z (k = 0
 * is the bottom plane).
 */
#ifndef PORTA_ORACLE_H
#define PORTA_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_MODEL_UNPOL = 0,   /* two-level atom, Stokes I only (non-LTE problem of the 1st kind) */
       OR_MODEL_HANLE = 1 }; /* two-level atom Jl=0 -> Ju=1, rho^K_Q K=0,2, Hanle + weak-field Zeeman */

/* formal solvers of the upwind interval MO (Sec. 3.2; the family compared on the
   sigmoid benchmark of Sec. 3.4): BESSER; DELOPAR (the parabola through M, O, P:
   the standard parabolic short characteristics for Stokes I); linear SC; quadratic
   Bezier with the Fritsch-Butland derivative at O, without (BEZIER_FB) and with
   (CBEZIER) the c_M overshoot correction */
enum { OR_BESSER = 0, OR_DELOPAR = 1, OR_LINEAR = 2, OR_BEZIER_FB = 3, OR_CBEZIER = 4 };

typedef struct {
    int nx, ny, nz;
    double lx, ly;            /* horizontal periods (km); spacing lx/nx, ly/ny */
    const double *z;          /* nz heights (km), strictly increasing */
    int model;
    /* per-voxel atmosphere (nvox doubles each; bx..bz may be NULL for the unpolarized model) */
    const double *chi;        /* line-centre opacity (1/km) */
    const double *eps;        /* collisional destruction probability */
    const double *bpl;        /* Planck function */
    const double *vel;        /* vertical velocity in Doppler widths */
    const double *bx, *by, *bz; /* magnetic field (G) */
    double zeta;              /* Zeeman splitting per gauss, Doppler widths */
    double gbar;              /* effective Lande factor */
    double bcrit;             /* Hanle critical field (G): Gamma_u = |B|/bcrit */
    int n_mu, n_chi, n_nu;    /* inclinations per hemisphere, azimuths, frequencies */
    double x_max;             /* frequency grid covers [-x_max, x_max] Doppler widths */
    int method;               /* OR_BESSER, OR_DELOPAR, OR_LINEAR, OR_BEZIER_FB or OR_CBEZIER */
    /* polarized model, optional (NULL: none): dichroism multipoles per voxel,
       5 doubles (D20, Re D21, Im D21, Re D22, Im D22): eta_i = chi phi
       [delta_i0 + sum_Q (-1)^Q T^2_Q(i, Omega) D^2_-Q], i = I, Q, U */
    const double *dich;
    /* interpolation at M and P (Sec. 3.1): 0 or 1 bilinear (4 nodes), 2 biquadratic
       (9 nodes: per axis the quadratic through the nearest node and its two neighbours) */
    int interp;
    /* explicit medium (polarized model, optional; NULL: none): per voxel the
       propagation matrix over eta_I, (eta_Q, eta_U, eta_V, rho_Q, rho_U, rho_V)/eta_I
       (kexpl, 6 x nvox), and the source vector (S_I, S_Q, S_U, S_V) (sexpl, 4 x nvox),
       both independent of direction and frequency; eta_I = chi phi(x - s) */
    const double *kexpl, *sexpl;
    /* orientation (K = 1) terms of a polarized line (optional; NULL: none), 3 doubles per
       voxel in the layout (X10, Re X11, Im X11): the emission multipoles S^1_Q
       (orient: eps_V += eta_I sum_Q (-1)^Q T^1_Q(V, Omega) S^1_-Q) and the dichroism
       multipoles D^1_Q (dich1: eta_V += eta_I sum_Q (-1)^Q T^1_Q(V, Omega) D^1_-Q);
       j1 (output, or_formal_solve_part): J^1_Q = sum_m w_m T^1_Q(V, Omega_m) Vbar, zeroed first */
    const double *orient, *dich1;
    double *j1;
    /* where the short characteristic of a point meets the grid (Sec. 3.1): 0 on the
       horizontal plane of the next upwind / downwind layer (the sheared-frame sweep,
       offsets of any length); 1 on the first cell face it crosses, a vertical face
       (x or y = const) when the horizontal offset over the layer exceeds one cell:
       bilinear in the face's horizontal coordinate and in height between the two
       planes, the upwind face's upper nodes lying on the point's own plane, whose
       intensities the plane then determines jointly (periodic in x and y: solved by
       sweeps in the upwind order repeated to convergence). Forward sweeps only. */
    int sc_faces;
} or_problem;

/* the periodic interpolation stencil of the sweep at cell coordinates (xc, yc) of a
   plane (node (i, j) at (i, j)): order 1 bilinear (4 nodes), 2 biquadratic (9 nodes);
   ii, jj, w receive the nodes and weights, the return value is their number */
int or_interp_weights(const or_problem *p, double xc, double yc, int order, int *ii, int *jj, double *w);

/* number of unknowns per voxel (rho), Stokes parameters, radiation-field components */
int or_nl(int model);
int or_ns(int model);
int or_nj(int model);
int or_nray(const or_problem *p);

/* ---- quadratures (Sec. 4.2 and App. A: Gauss inclinations, trapezoid azimuths/frequencies) ---- */
int or_gauss_legendre01(int n, double *x, double *w);
int or_rays(const or_problem *p, double *mu, double *chi, double *w);
int or_freqs(int n_nu, double x_max, double *x, double *w);

/* ---- spherical tensors T^K_Q(i, Omega), K = 0, 2, i = I, Q, U (Eq. 1; LL04 Tab. 5.6, gamma = 0)
   t[i*6 + c], c = (T00, T20, Re T21, Im T21, Re T22, Im T22) ---- */
void or_tkq(double mu, double chi, double t[18]);

/* ---- BESSER coefficients and control point (Sec. 3.2, 3.3) ---- */
void or_coeffs(double tau, double c[6]);   /* e^-tau, psi'_M, psi'_O, omega_M, omega_O, omega_C */
double or_control_point(double yM, double yO, double yP, double hM, double hP, int has_p, int method);
/* one-ray unpolarized formal solution on a grid of optical depths (Sec. 3.4) */
int or_solve_1d(int n, const double *tau, const double *S, double I0, int method, double *Iout);
/* one 4x4 (or scalar) BESSER-DELO step (Eq. 7). eta*: 7 propagation-matrix elements
   (eta_I, eta_Q, eta_U, eta_V, rho_Q, rho_U, rho_V); eps*: ns emissivities. */
int or_step(int ns, const double *IM, const double *etaM, const double *epsM,
            const double *etaO, const double *epsO, double etaP_I, const double *epsP,
            double dsM, double dsP, int has_p, int method, double *IO, double *lstar);

/* ---- SEE (Eq. 2) for the two supported atoms ---- */
int or_hanle_solve(double gamma, double bx, double by, double bz, const double *rhs6, double *s6);
int or_see_update(const or_problem *p, const double *jkq, const double *lstar,
                  double *rho, double *max_change);
/* A(S) of the SEE written as A(S) = f (f = eps B delta_K0), and the Jacobi update of
   A(S) = src for a general per-voxel src (NULL: the two-level problem itself) */
int or_see_apply(const or_problem *p, const double *jkq, const double *rho, double *out);
int or_see_update_src(const or_problem *p, const double *jkq, const double *lstar, const double *src,
                      double *rho, double *max_change);
/* reverse mode of or_see_update_src (src NULL: eps B): from g = dL/d(rho after) to dL/drho (explicit
   part), dL/dJ^K_Q, dL/dLambda-bar*, dL/d(src^0_0) and (added to g_b, 3 x nvox) dL/dB of the Hanle term */
int or_see_update_vjp(const or_problem *p, const double *jkq, const double *lstar, const double *src,
                      const double *rho, const double *g, double *g_rho, double *g_jkq, double *g_lstar,
                      double *g_eb, double *g_b);

/* ---- 3D short-characteristics formal solution ---- */
/* one ray m, one frequency j, full grid: I (nvox*ns) and Lambda* (nvox) */
int or_sweep_ray(const or_problem *p, const double *rho, int m, int j, double *Iout, double *lstar);
/* all rays and frequencies: J^K_Q (nvox*nj) and Lambda-bar* (nvox) */
int or_formal_solve(const or_problem *p, const double *rho, double *jkq, double *lstar);
/* subset of rays [m0, m1) and frequencies [j0, j1): same outputs, partial sums */
int or_formal_solve_part(const or_problem *p, const double *rho, int m0, int m1, int j0, int j1,
                         double *jkq, double *lstar);
/* emergent Stokes at the top plane for ndir outgoing directions (mu > 0): out[d][j][y][x][ns] */
int or_emergent(const or_problem *p, const double *rho, int ndir, const double *mu,
                const double *chi, double *out);

/* adjoint of or_emergent: gradients of L = sum gout * out with respect to per-voxel chi,
   e = chi S^0_0 (ratios S^K_Q / S^0_0 fixed) and B (g_b: 3 x nvox, may be NULL for the
   unpolarized model); gout has the layout of out */
int or_emergent_vjp(const or_problem *p, const double *rho, int ndir, const double *mu,
                    const double *chi, const double *gout, double *g_chi, double *g_e, double *g_b);
/* reverse mode in the unknowns: dL/dchi at fixed rho, dL/drho, dL/dB of the J^K_Q / Lambda-bar* of a
   formal solution (added to the outputs) and of the emergent Stokes vector (overwritten) */
int or_jkq_vjp(const or_problem *p, const double *rho, const double *g_jkq, const double *g_lstar,
               double *g_chi, double *g_rho, double *g_b);
int or_emergent_vjp_rho(const or_problem *p, const double *rho, int ndir, const double *mu, const double *chi,
                        const double *gout, double *g_chi, double *g_rho, double *g_b);
/* reverse mode of the step coefficients, control point and step (derivatives for the adjoint) */
void or_coeffs_deriv(double tau, const double c[6], double dc[6]);
void or_control_point_vjp(double yM, double yO, double yP, double hM, double hP, int has_p, int method,
                          double gc, double g[5]);
int or_step_vjp(int ns, const double *IM, const double *etaM, const double *epsM,
                const double *etaO, const double *epsO, double etaP_I, const double *epsP,
                double dsM, double dsP, int has_p, int method, const double *gIO,
                double *gIM, double *g_etaM, double *g_epsM, double *g_etaO, double *g_epsO,
                double *g_etaP, double *g_epsP);

/* flop counter for one update (counted once per voxel.ray.frequency) */
void or_flops_reset(int enable);
long long or_flops_get(void);
/* branch signature of the control points evaluated while recording (test support) */
void or_branch_sig_reset(int enable);
unsigned long long or_branch_sig_get(void);

#ifdef __cplusplus
}
#endif
#endif
