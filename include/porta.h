/*
 * porta.h -- C ABI of the GB300 (sm_103a) formal-solver library for 3D
 * non-LTE polarized radiative transfer with the short-characteristics BESSER
 * method of Stepan & Trujillo Bueno (2013, "PORTA", arXiv:1307.4217).
 *
 * What the library computes (one Jacobi iteration of the non-LTE problem):
 *   porta_formal_solve    -- Sec. 3: for every ray direction and frequency the
 *                            grid is swept in topological order; at each point O
 *                            the Stokes vector follows from the BESSER-DELO step
 *                            (Eq. 7) between the upwind point M and O, with the
 *                            transfer coefficients and I_M interpolated bilinearly
 *                            on the neighbouring horizontal planes. The
 *                            frequency-integrated Stokes parameters and Lambda*
 *                            (Eq. 14) are reduced on the fly per ray.
 *   porta_accumulate_jkq  -- Eq. 1: J^K_Q = sum_p sum_m w_m T^K_Q(p, Omega_m)
 *                            sum_nu wt_nu I_p, and the angle- and profile-averaged
 *                            Lambda-bar*, summed in FP64 in a fixed order.
 *   porta_see_update      -- Eq. 2 with the Jacobi (ALI) step of Sec. 5: the
 *                            per-voxel statistical-equilibrium solve for the
 *                            multipolar components of the source function, in FP64,
 *                            and the maximum relative change (Sec. 5.3, R_c).
 *   porta_emergent_stokes -- Sec. 1: emergent Stokes profiles at the top of the
 *                            box for arbitrary outgoing lines of sight.
 *
 * Atomic models (Sec. 2; physics of LL04 Ch. 10 for a two-level atom):
 *   PORTA_MODEL_TWOLEVEL_UNPOL  unpolarized two-level atom, CRD, Stokes I only.
 *     Unknown per voxel (NL = 1): the line source function S.
 *     Radiation field per voxel (NJ = 1): J-bar.
 *   PORTA_MODEL_TWOLEVEL_HANLE  two-level atom Jl = 0 -> Ju = 1, CRD, Stokes IQUV,
 *     scattering polarization, Hanle effect and weak-field longitudinal Zeeman
 *     effect (eta_V, eps_V). Unknowns per voxel (NL = 6): the multipolar source
 *     function components (S^0_0, S^2_0, Re S^2_1, Im S^2_1, Re S^2_2, Im S^2_2),
 *     proportional to rho^K_Q of the upper level. Radiation field (NJ = 6): the
 *     same six real components of J^K_Q.
 *
 * Conventions
 *   * Voxel index v = (k*ny + j)*nx + i; k = 0 is the bottom plane; the grid is
 *     periodic in x and y (Sec. 4.2, "following the strategy of Auer et al.").
 *   * Per-voxel arrays are nvox = nx*ny*nz doubles; rho is nvox*NL doubles with
 *     the NL components of a voxel contiguous; J^K_Q output is nvox*NJ doubles.
 *   * Rays: 2*n_mu*n_chi directions; ray m = ((h*n_mu) + i)*n_chi + a with h = 0
 *     for mu > 0 (upward), h = 1 downward; Gauss-Legendre inclinations per
 *     hemisphere, azimuths chi_a = (a + 1/2) 2 pi / n_chi, weights summing to 1.
 *   * Frequencies: n_nu nodes uniformly spaced on [-x_max, x_max] Doppler widths,
 *     trapezoid weights, Gaussian profile renormalized per voxel and direction
 *     on this quadrature (Sec. 4.2).
 *   * Boundary conditions: I = (B, 0, 0, 0) entering at the bottom, I = 0
 *     entering at the top.
 *   * Memory: the library owns all device memory it allocates (in porta_create
 *     and porta_set_atmosphere) and frees it in porta_destroy. Inputs are
 *     copied; callers keep ownership of their buffers. Arguments named `where`
 *     say whether a caller pointer is host (PORTA_HOST) or device
 *     (PORTA_DEVICE) memory.
 *   * Streams: every call enqueues on the stream given to porta_set_stream
 *     (default: the legacy default stream). Calls that return host data
 *     synchronize that stream.
 *   * Errors: every int-returning function returns PORTA_OK (0) or a negative
 *     status; porta_last_error gives a message. Invalid arguments are rejected
 *     before anything is launched. A context is not thread-safe.
 */
#ifndef PORTA_H
#define PORTA_H

#ifdef __cplusplus
extern "C" {
#endif

#define PORTA_OK        0
#define PORTA_EINVAL   -1   /* invalid argument (shape, pointer, value, NaN input) */
#define PORTA_ENOMEM   -2   /* device or host allocation failed */
#define PORTA_ECUDA    -3   /* CUDA runtime error */
#define PORTA_ESTATE   -4   /* call order: a required input has not been set */
#define PORTA_ENOTCONV -5   /* an iteration did not reach its tolerance within its iteration cap */
#define PORTA_EKERNEL  -7   /* a kernel reported a failure (error word set) */
#define PORTA_ESCRATCH -8   /* problem too large for the fixed scratch of porta_formal_solve_noalloc */

/* size of the fixed device scratch array used by porta_formal_solve_noalloc */
#define PORTA_NOALLOC_SCRATCH_BYTES (32u << 20)
/* largest number of height levels porta_formal_solve_noalloc accepts (the heights
   are passed to the device by value, inside a kernel argument block) */
#define PORTA_NOALLOC_MAX_NZ 1024

#define PORTA_MODEL_TWOLEVEL_UNPOL 0
#define PORTA_MODEL_TWOLEVEL_HANLE 1

#define PORTA_FP64 0        /* sweeps in FP64 ("plain" form) */
#define PORTA_FP32 1        /* sweeps in FP32; SEE, J^K_Q sums and residual in FP64 */

#define PORTA_HOST   0
#define PORTA_DEVICE 1

typedef struct porta_ctx porta_ctx;

/* Cartesian grid (App. A): nz heights z (host pointer, strictly increasing,
   same length unit as lx, ly); horizontal spacing lx/nx, ly/ny. */
typedef struct {
    int nx, ny, nz;
    double lx, ly;
    const double *z;
} porta_grid;

/* Atomic model. zeta: Zeeman splitting per gauss in Doppler widths; gbar:
   effective Lande factor; bcrit: Hanle critical field in gauss, so that the
   upper-level Hanle parameter is Gamma_u = |B| / bcrit (the atom precesses
   counterclockwise about B, as for a positive Lande factor). */
typedef struct {
    int model;
    double zeta, gbar, bcrit;
} porta_atom;

/* Quadratures: n_mu Gauss inclinations per hemisphere, n_chi azimuths,
   n_nu frequencies on [-x_max, x_max]. */
typedef struct {
    int n_mu, n_chi, n_nu;
    double x_max;
} porta_quad;

/* Options. precision: PORTA_FP64 or PORTA_FP32. cluster and nu_group select
   the sweep decomposition (CTAs per ray cluster, frequencies per pass); 0
   lets the library choose. */
typedef struct {
    int precision;
    int cluster;
    int nu_group;
} porta_opts;

/* Per-voxel atmosphere (nvox doubles each): chi = line-centre opacity per unit
   length, eps = collisional destruction probability, bpl = Planck function,
   vel = vertical velocity in Doppler widths (its projection on the ray shifts
   the profile), bx, by, bz = magnetic field in gauss (NULL for the unpolarized
   model). */
typedef struct {
    const double *chi, *eps, *bpl, *vel, *bx, *by, *bz;
} porta_atmos;

/* Measured arithmetic peak (TFLOP/s) of the current GPU for the roofline of
   the formal solver: kind 0 = FP32 fused multiply-add (FFMA), 1 = packed FP32
   FMA on float2 pairs (FFMA2), 2 = FP64 FMA (DFMA). Kernels of independent FMA
   chains (8 per thread, 64 warps per SM) are launched back to back for about
   `seconds` seconds of device time (CUDA events); *tflops receives the best
   launch (2 flops per FMA), *total_ms (may be NULL) the device time spent.
   Allocates a few MB of device memory for the results and frees it.
   The paper has no counterpart. */
int porta_fma_peak(int kind, double seconds, double *tflops, double *total_ms);

/* Diagnostic: the BESSER-DELO step of Eq. 7 with a general propagation
   matrix (all seven elements eta_I, eta_Q, eta_U, eta_V, rho_Q, rho_U, rho_V
   at M and O; kappa^-1 = 1 + psi'_O K'_O of Eq. 8 solved in full) evaluated on
   the GPU in the given precision, for n cases. in (host): [n][34] =
   I_M (4), eta_M (7), eps_M (4), eta_O (7), eps_O (4), eta_P,I (1), eps_P (4),
   ds_M, ds_P, has_p (nonzero: a downwind point exists); out (host): [n][5] =
   I_O (4), Lambda*. tau_MO = (eta_I,M + eta_I,O) ds_M / 2 and likewise for OP
   (trapezoid), S = eps / eta_I. The two-level sweeps run the specializations of
   this step for their propagation matrices (I-V coupling, or the arrow form of
   dichroism). PORTA_EINVAL for non-finite inputs or non-positive eta_I, ds. */
int porta_eval_step(int precision, int n, const double *in, double *out);

/* An explicit medium for the emergent Stokes profiles (porta_emergent_stokes) and
   the J^K_Q formal solution:
   the propagation matrix of Eqs. 7-8 with all seven elements, given per voxel as
   kexpl[k][v] = (eta_Q, eta_U, eta_V, rho_Q, rho_U, rho_V)[k] / eta_I (k = 0..5)
   and the source vector sexpl[i][v] = S_i (i = I, Q, U, V), both independent of
   direction and frequency; eta_I = chi phi(x - v mu) from the atmosphere. The
   emergent sweep then interpolates eta_I (1, K'/eta_I) and eta_I S bilinearly at M
   and P and takes the BESSER-DELO step with kappa^-1 = 1 + psi'_O K'_O solved in full
   (the general step of porta_eval_step). Arrays of nvox doubles each, host or
   device (where); the library keeps a copy. NULL for either clears the medium
   (the two-level physics of the unknowns again). Polarized two-level single-box
   contexts with bilinear interpolation only (PORTA_EINVAL otherwise). While an
   explicit medium is set, porta_formal_solve sweeps it with the global-memory sweep
   of porta_set_global_sweep (the same seven-element step) and porta_accumulate_jkq
   returns its J^K_Q and Lambda-bar*; the reverse-mode calls and porta_probe_ray
   return PORTA_EINVAL. */
int porta_set_explicit_medium(porta_ctx *c, const double *kexpl, const double *sexpl, int where);

/* Interpolation of the transfer coefficients and of the upwind Stokes vector at
   the points M and P (Sec. 3.1, where both are offered): order 1 bilinear from
   the 4 surrounding nodes (the default), order 2 biquadratic from the 9 nodes
   around the nearest one (per horizontal axis the quadratic through the
   nearest node and its two neighbours; periodic). The biquadratic stencils run
   in the general sweep, whose strips then need at least two rows per CTA
   (cluster sizes up to ny/2); they can overshoot where the atmosphere changes
   abruptly (no clamping, as in the oracle). Changing the order returns the
   launch shape to porta_opts' choice (an autotuned shape is dropped) and
   drops any captured iteration graph. PORTA_EINVAL for another order, for order 2 on a
   multilevel context (its lines carry dichroism, which the biquadratic sweep
   has not) or with ny < 2. The reverse-mode calls (porta_emergent_vjp,
   porta_iterate_vjp) accept bilinear interpolation only. */
int porta_set_interpolation(porta_ctx *c, int order);

/* Where the short characteristics of the J^K_Q formal solution end (Sec. 3.1:
   M and P may lie on a vertical plane of the grid). on = 0 (the default): on the
   horizontal plane of the next layer, at offsets of any length (the sheared-frame
   sweeps). on = 1: on the first cell face crossed -- where a ray's horizontal offset
   over a layer, (f_x, f_y) cells, exceeds one cell, on the vertical face x = x_(i +
   sgn f_x) (|f_x| >= |f_y|) or y = y_(j + sgn f_y) at the fraction 1/max(|f_x|, |f_y|)
   of the layer, the face point's quantities bilinear in the face's horizontal
   coordinate and in height. The upwind face's upper nodes are points of the same
   plane; with the periodic boundaries (Sec. 4.2) each such plane is solved jointly,
   by passes over its lines in the upwind order repeated until no intensity changes
   by more than 1e-15 (FP64) or 2e-7 (FP32) of the plane's largest, or until the
   change, within 8 times that and no longer halving per pass, has reached the
   rounding floor (where (1 - s)^n <= 1/4 over the plane's n lines); the face points'
   Lambda* is their own term (Eq. 14). One CTA per (box, ray, frequency group), the
   planes in order, each box with its own cell size; the groups' partial sums are
   added in group order into the per-ray partial sums of the general sweep;
   porta_emergent_stokes then sweeps its lines of sight the same way. Two-level
   contexts (one box or several) and the line boxes of multilevel contexts, the
   polarized ones with their dichroism and orientation terms and the Stokes-V
   integrals (porta_ml_formal_solve and the iterations); bilinear stencils only,
   not with an explicit medium (PORTA_EINVAL); the reverse-mode calls and
   porta_probe_ray reject it. A plane still changing after
   1e5 passes is reported as PORTA_ENOTCONV by the synchronizing calls that read the
   sums (porta_accumulate_jkq to host). Drops any captured iteration graph. */
int porta_set_sc_faces(porta_ctx *c, int on);

/* The J^K_Q formal solution (and the emergent profiles) by the global-memory sweep
   of porta_set_sc_faces in the plane placement (Sec. 3.1: M and P on the
   neighbouring horizontal planes at any offset, bilinear and periodic; the same
   discretization as the shared-memory sweeps), its work planes in device memory
   instead of a shared-memory ring: on = 1 asks for it; a context whose planes are
   too wide for every shared-memory launch shape (e.g. the FP64 polarized atom on
   128-wide planes) takes it by itself on its first formal solution, and on = 0
   lets it check again. Bilinear stencils only, not with an explicit medium
   (PORTA_EINVAL); the reverse-mode calls and porta_probe_ray reject it; the face
   option (porta_set_sc_faces) takes precedence. Drops any captured iteration graph. */
int porta_set_global_sweep(porta_ctx *c, int on);

/* The family of formal solvers compared on the one-ray sigmoid benchmark of
   Sec. 3.4 (Eqs. 15-18, Fig. 5): constant opacity, z = tau, S(z) = sigma(2, -5, z)
   sigma(-2, 5, z), uniform nodes z_i = -12 + shift + i dtau in [-12, 12], the
   exact intensity (Eq. 17) at the first node. Methods of the upwind interval:
   BESSER (Sec. 3.2); PARABOLIC (the parabola through M, O, P: y'_O of Eq. 6 without
   the overshoot tests); LINEAR (psi'_M, psi'_O of Eqs. 9-10); BEZIER_FB (quadratic
   Bezier, y'_O the Fritsch-Butland weighted harmonic mean of the one-sided slopes,
   0 where they differ in sign); CBEZIER (BEZIER_FB with c_M outside [y_M, y_O]
   moved to y_M). */
enum { PORTA_SC_BESSER = 0, PORTA_SC_PARABOLIC = 1, PORTA_SC_LINEAR = 2, PORTA_SC_BEZIER_FB = 3, PORTA_SC_CBEZIER = 4 };

/* E(dtau) of Eq. 18 (maximum over the nodes of |I - I_a| / I_a, I_a of Eq. 17 in
   FP64) for ncase cases, each (method[k], dtau[k], shift[k]) one ray solved on the
   GPU in the given precision; host arrays in and out (E: ncase). Synchronous.
   PORTA_EINVAL for an unknown method, dtau outside [1e-4, 24] or shift outside
   [0, dtau); PORTA_ENOMEM if the device buffers cannot be allocated. */
int porta_sigmoid_error(int precision, int ncase, const int *method, const double *dtau, const double *shift,
                        double *E);

/* Frequency bands: the (ray, frequency) pairs of a formal solution are
   independent and J^K_Q / Lambda-bar* are sums over them (Eq. 1; the band
   parallelization of Sec. 4.3), so a formal solution can be split into bands
   swept on different GPUs and the bands' partial sums added.
   porta_set_freq_range limits the formal solutions of this context to the
   frequencies [j0, j1) (0 <= j0 < j1 <= n_nu; (0, 0) or (0, n_nu) restores the
   whole grid); the profile normalization stays that of the whole grid, so the
   bands' sums add up to J^K_Q and Lambda-bar*. Single-box two-level contexts
   (and batches); PORTA_EINVAL for multilevel contexts and bad bounds.
   porta_partial_size gives the partial sums' element count, (NJ + 1) * nvox
   (and 3 * nvox more, J^1_Q [nvox][3] after Lambda-bar*, on a polarized
   multilevel context), and element size (8 bytes). After porta_formal_solve, porta_get_partial
   copies them to `out` (host or device, `where`): in the FP32 form the exact
   fixed-point sums as int64, [NJ + 1][nvox] (J^K_Q components, then
   Lambda-bar*; the voxels' scales are identical on every context with the same
   unknowns and atmosphere), in the FP64 form doubles, J^K_Q [nvox][NJ] then
   Lambda-bar* [nvox]. Element-wise sums of such buffers over the bands (int64
   in FP32: exact, so independent of the order of the reduction) are again
   partial sums; porta_set_partial loads one into a context that has run a
   formal solution and makes it the J^K_Q / Lambda-bar* that porta_see_update
   uses (PORTA_ESTATE without a formal solution). The paper's distributed
   scheme (domain decomposition, Sec. 4.1-4.2) is not used: every rank holds the
   whole box. */
int porta_set_freq_range(porta_ctx *c, int j0, int j1);
int porta_partial_size(const porta_ctx *c, long long *elements, int *elem_bytes);
int porta_get_partial(porta_ctx *c, void *out, int where);
int porta_set_partial(porta_ctx *c, const void *in, int where);

/* Process-wide cap on the device memory the library allocates (bytes; 0, the
   default, means no cap). Every context allocation (creation, adjoint tapes,
   multigrid levels, scratch of a call) counts against the live total; one that
   would exceed the cap fails with PORTA_ENOMEM before reaching the CUDA
   runtime, and the call that needed it returns PORTA_ENOMEM (porta_create
   returns no context). For callers that share the GPU with other work and must
   bound this library's footprint. porta_device_bytes returns the live total.
   The paper has no counterpart. */
int porta_set_device_limit(long long bytes);
long long porta_device_bytes(void);

/* Create a context: validates sizes, builds the quadratures and the per-ray
   plane geometry, allocates device buffers. Returns PORTA_EINVAL for
   nx, ny < 1, nz < 2, non-increasing z, n_mu, n_chi, n_nu < 1, unknown model
   or precision. *out is NULL on failure. */
int porta_create(const porta_grid *g, const porta_atom *a, const porta_quad *q,
                 const porta_opts *o, porta_ctx **out);

/* Batched problem: nbox independent boxes of uneven size (grids[b]) sharing
   the atomic model and the quadratures. Voxel arrays (atmosphere, rho, J^K_Q,
   Lambda-bar*) are the boxes' arrays concatenated in box order. Every
   formal solution sweeps all (box, ray) pairs in one persistent launch,
   largest boxes first. porta_emergent_stokes and porta_probe_ray take
   single-box contexts only. Errors as porta_create (for every grid). */
int porta_batch_create(int nbox, const porta_grid *grids, const porta_atom *a, const porta_quad *q,
                       const porta_opts *o, porta_ctx **out);

/* Free all device and host memory of the context (NULL is a no-op). */
void porta_destroy(porta_ctx *c);

/* Message of the last failed call on this context (never NULL). */
const char *porta_last_error(const porta_ctx *c);

/* Stream for all subsequent work (a cudaStream_t; NULL = default stream). */
int porta_set_stream(porta_ctx *c, void *stream);

/* Sizes: rays, frequencies, voxels, unknowns per voxel (NL), radiation-field
   components (NJ), Stokes parameters (NS). Any pointer may be NULL. */
int porta_sizes(const porta_ctx *c, int *nray, int *nnu, long long *nvox, int *nl, int *nj, int *ns);

/* Ray directions and weights of the angular quadrature (host arrays of nray). */
int porta_rays(const porta_ctx *c, double *mu, double *chi, double *w);

/* Copy the atmosphere in (Sec. 2). Rejects non-finite values, chi <= 0,
   eps outside (0, 1], and a missing field for the Hanle model. Also
   precomputes the per-voxel, per-ray profile normalization (Sec. 4.2). */
int porta_set_atmosphere(porta_ctx *c, const porta_atmos *a, int where);

/* Set / get the unknowns (nvox*NL doubles, FP64). porta_set_rho rejects
   non-finite values and S^0_0 <= 0. */
int porta_set_rho(porta_ctx *c, const double *rho, int where);
int porta_get_rho(porta_ctx *c, double *rho, int where);

/* Formal solution for all rays and frequencies with the current rho
   (Sec. 3). Requires the atmosphere and rho (PORTA_ESTATE otherwise).
   Enqueues only; results stay on the device until porta_accumulate_jkq. */
int porta_formal_solve(porta_ctx *c);

/* Sum the per-ray partial integrals into J^K_Q (nvox*NJ) and Lambda-bar*
   (nvox), FP64, fixed summation order (Eq. 1). Either output pointer may be
   NULL (result kept on the device for porta_see_update). Requires a
   preceding porta_formal_solve. */
int porta_accumulate_jkq(porta_ctx *c, double *jkq, double *lstar, int where);

/* Jacobi (ALI) update of rho from the accumulated J^K_Q and Lambda-bar*
   (Eq. 2; Sec. 5). max_change (host pointer, may be NULL) receives
   max over voxels of |dS00|/|S00| and, for the Hanle model, of
   |d(S^2_Q/S^0_0)|; passing it synchronizes the stream. */
int porta_see_update(porta_ctx *c, double *max_change);

/* Emergent Stokes vectors at the top plane for ndir outgoing directions
   (host arrays mu in (0, 1], chi in radians). out: ndir*n_nu*ny*nx*NS doubles,
   layout [dir][nu][y][x][stokes]. Uses the current rho. Unless porta_opts
   fixed the launch shape, the first call for a given number of directions
   times the fitting shapes (cluster size x frequencies per pass) and keeps
   the fastest; results do not depend on the shape. */
int porta_emergent_stokes(porta_ctx *c, int ndir, const double *mu, const double *chi,
                          double *out, int where);

/* Diagnostic: Stokes vectors of one ray m for all frequencies at every voxel,
   as computed inside porta_formal_solve (same kernel and launch shape).
   out: n_nu*nvox*NS doubles, layout [nu][voxel][stokes]; lstar: n_nu*nvox
   (may be NULL). Runs a full formal solution. */
int porta_probe_ray(porta_ctx *c, int m, double *out, double *lstar, int where);

/* Autotuner of the sweep launch shape: times every fitting (cluster size,
   frequencies per pass) candidate on one wave of rays of the current problem
   (CUDA events on the context's stream), keeps the fastest for subsequent
   calls and returns it in *cluster / *nu_group (either may be NULL). It then
   times a second, concurrent launch of a smaller cluster shape over the
   cheapest fraction of the (box, ray) work list -- it runs on SMs that the
   main shape's clusters cannot occupy -- and keeps it if it is faster
   (porta_fill_info). With the filler, each launch takes its work items from
   its own device counter; every item is computed by one fixed shape, so the
   results do not depend on scheduling. Requires the atmosphere and rho.
   Overwrites the device-side partial integrals (call porta_formal_solve
   afterwards). */
int porta_autotune(porta_ctx *c, int *cluster, int *nu_group);

/* The concurrent filler launch kept by porta_autotune: CTAs per cluster,
   frequencies per pass and the fraction of the work list it takes
   (cluster size 0: none). */
int porta_fill_info(const porta_ctx *c, int *cluster_size, int *nu_group, double *fraction);

/* Sets (cluster_size >= 1) or removes (cluster_size 0) the concurrent filler
   launch by hand: cluster size, frequencies per pass and the fraction of the
   work list in (0, 1) it takes. PORTA_EINVAL if the shape does not fit. */
int porta_set_fill(porta_ctx *c, int cluster_size, int nu_group, double fraction);

/* Diagnostic: the coefficients of the BESSER-DELO step (Eqs. 9-13; Table 1
   series at small optical path) exactly as the sweep kernels of the given
   precision evaluate them, for n upwind optical paths t (host array, t > 0):
   out[6*i + 0..5] = e^-t, psi'_M, psi'_O, omega_M, omega_O, omega_C (host).
   Synchronous; uses the current device. */
int porta_eval_coefficients(int precision, int n, const double *t, double *out);

/* Allocation-free formal solution. (The paper has no counterpart: this entry
   point exists for callers that cannot allocate device memory, e.g. a host
   program whose device memory is already reserved by another framework's
   pooling allocator, or a latency-sensitive loop that cannot afford the
   implicit synchronization of cudaMalloc/cudaFree.)
   Same computation as porta_formal_solve + porta_accumulate_jkq with FP32
   sweeps, without a context: the caller passes the grid, atom and quadrature
   descriptions (host), the atmosphere arrays and rho (device pointers, FP64,
   layouts as for porta_set_atmosphere / porta_set_rho; values are not
   checked) and receives J^K_Q (nvox*NJ) and Lambda-bar* (nvox) in device
   buffers, enqueued on `stream` (a cudaStream_t, NULL = default stream).
   Every intermediate lives in one file-scope device array of
   PORTA_NOALLOC_SCRATCH_BYTES (32 MiB) that every GPU loading the library
   holds until the process exits; the call allocates nothing, host or device.
   The polarized model needs about nvox * (48 + 20 * nray) bytes, e.g. 10^4
   voxels with 160 rays; larger problems are rejected with PORTA_ESCRATCH
   before anything is enqueued, as are grids of more than PORTA_NOALLOC_MAX_NZ
   levels. n_mu is limited to 32. The heights g->z are read on the host during
   the call (they reach the device inside a kernel's argument block).
   Every call looks up the array's device address on the current device
   (cudaGetSymbolAddress with that device current; the lookup allocates
   nothing, and a device reset between calls is therefore harmless); the first
   call on a device also loads the library's device code there, so make that
   first call before any stream capture. All calls share the array and it keeps
   the last call's contents (each call writes every part it reads); calls that
   overlap on the GPU race on it. */
int porta_formal_solve_noalloc(const porta_grid *g, const porta_atom *a, const porta_quad *q,
                               const porta_atmos *atm, const double *rho, double *jkq, double *lstar,
                               void *stream);

/* Jacobi iterations as a CUDA graph: on first use (and after
   porta_autotune or a stream change) one iteration -- porta_formal_solve,
   porta_accumulate_jkq, porta_see_update with its residual -- is captured on
   the context's stream into a CUDA graph; the graph is then launched
   `iterations` times. Needs a non-default stream (porta_set_stream),
   the atmosphere and rho. max_change (host, may be NULL) receives the
   residual of the last iteration (synchronizes the stream). */
int porta_run_iterations(porta_ctx *c, int iterations, double *max_change);

/* Jacobi (ALI) iterations to a tolerance (Eq. 2 with the Jacobi update of
   Sec. 5; the stop criterion is the maximum relative change R_c of Sec. 5.3):
   replays the captured iteration of porta_run_iterations until the maximum
   change of an iteration is below tol, reading the change after every
   check_every-th iteration (1: after each, so that the count is exact).
   iterations_out and max_change_out (host, may be NULL) receive the number of
   iterations done and the last change read. Returns PORTA_ENOTCONV when
   max_iter iterations leave the change at or above tol (rho is left at the last
   iterate), PORTA_EINVAL for tol <= 0, max_iter < 1 or check_every < 1, and the
   errors of porta_run_iterations. */
int porta_iterate_to(porta_ctx *c, double tol, int max_iter, int check_every, int *iterations_out,
                     double *max_change_out);

/* Launch statistics of the last formal solution: clusters launched, CTAs per
   cluster, frequencies per pass, dynamic shared memory per CTA (bytes). */
int porta_launch_info(const porta_ctx *c, int *clusters, int *cluster_size, int *nu_group, int *smem_bytes);

/* Reverse mode of porta_emergent_stokes (gradients of emergent Stokes
   profiles; the paper has no counterpart, Sec. 3 defines the forward map).
   L = sum(grad_out * out) with out as porta_emergent_stokes writes it, at the
   current atmosphere and rho, as a function of per-voxel
     chi  (line-centre opacity),
     e    = chi S^0_0 (emission scale; the multipoles rho^K_Q scale as e/chi
            with their ratios to S^0_0 held fixed; needs S^0_0 > 0),
     B    (magnetic field vector, through eta_V and eps_V of the weak-field
            Zeeman term).
   Runs the forward emergent sweep keeping the Stokes vectors of every plane
   (a device tape of ndir*n_nu*nvox*NS reals, kept by the context for reuse),
   then the adjoint sweep (planes in reverse order, the forward step
   recomputed and differentiated on the branch the BESSER control point took),
   then a fixed-order sum over directions and frequency groups; the result
   does not depend on scheduling. The sweeps run in the context's precision;
   gradients are accumulated per node in that precision and summed in FP64.
   grad_out: ndir*n_nu*ny*nx*NS doubles, layout of porta_emergent_stokes.
   out: the forward emergent Stokes (may be NULL). g_chi, g_e: nvox doubles;
   g_b: 3*nvox doubles, [component x|y|z][voxel] (NULL allowed for the
   unpolarized model). All caller arrays are host or device per `where`;
   mu, chi are host arrays. Single-box contexts; PORTA_ESTATE without
   atmosphere and rho. Synchronous. */
int porta_emergent_vjp(porta_ctx *c, int ndir, const double *mu, const double *chi, const double *grad_out,
                       double *out, double *g_chi, double *g_e, double *g_b, int where);

/* Launch shape of the adjoint sweep: cluster size (1..16, <= ny) and
   frequencies per pass. With both 0 (the default) the first
   porta_emergent_vjp for a given number of directions times every fitting
   shape once (CUDA events) and keeps the fastest. */
int porta_set_adjoint_launch(porta_ctx *c, int cluster, int nu_group);

/* Device time (ms, CUDA events on the context's stream) of the last
   porta_emergent_vjp: the forward emergent sweep with its tape, and the
   adjoint sweep with the reduction over directions and frequency groups. */
int porta_adjoint_timing(const porta_ctx *c, float *forward_ms, float *adjoint_ms);

/* Launch statistics of the last adjoint sweep (as porta_launch_info). */
int porta_adjoint_info(const porta_ctx *c, int *clusters, int *cluster_size, int *nu_group, int *smem_bytes);

/* Gradients through Jacobi iterations (reverse mode of Eq. 2 composed
   with the formal solution of Sec. 3; the paper has no counterpart).
   porta_iterate_ckpt runs niter Jacobi iterations from the current rho
   (formal solution, J^K_Q and Lambda-bar*, update, as porta_formal_solve,
   porta_accumulate_jkq and porta_see_update) and keeps, on the device,
   rho before every ckpt-th iteration ((niter + ckpt - 1)/ckpt vectors of
   nvox*nl doubles) and rho after the last; rho is left at the last iterate.
   max_change (host, may be NULL): that of the last update. A new call drops
   the previous checkpoints. niter, ckpt >= 1 (PORTA_EINVAL otherwise);
   single-box contexts; PORTA_ESTATE without atmosphere and rho. */
int porta_iterate_ckpt(porta_ctx *c, int niter, int ckpt, double *max_change);

/* L = sum(grad_out * out), out the emergent Stokes profiles (layout of
   porta_emergent_stokes) of the last iterate of porta_iterate_ckpt, as a
   function of per-voxel
     chi  (line-centre opacity; rho follows from the iterations),
     f    (the thermal source term eps B of the update, Eq. 2),
     B    (magnetic field vector: Zeeman term of the sweeps and Hanle term of
           the update).
   The iterates are rebuilt from the checkpoints, each segment of ckpt
   iterations once (its iterates, J^K_Q and Lambda-bar* kept on the device,
   ckpt*nvox*(nl + nj + 1) doubles; where that exceeds the tape limit below
   or the free device memory, each step back rebuilds its iterate from the
   nearest checkpoint instead); each step back
   runs the adjoint of the update, then the adjoint of the formal solution's J^K_Q and Lambda-bar*
   (rays in batches whose forward Stokes vectors fit a device tape of at most
   16 GB, the same gather-form adjoint sweep as porta_emergent_vjp,
   per-cluster FP64 accumulators summed in a fixed order; the limit is
   porta_set_tape_limit's). Gradients at kinks
   of the BESSER control point take the branch the forward took.
   grad_out: ndir*n_nu*ny*nx*NS doubles; out (may be NULL) the forward
   profiles; g_chi, g_f: nvox doubles; g_b: 3*nvox doubles, [x|y|z][voxel]
   (ignored, may be NULL, for the unpolarized model). Caller arrays are host
   or device per `where`; mu, chi are host arrays. PORTA_ESTATE before
   porta_iterate_ckpt. rho is left at the last iterate. Synchronous. */
int porta_iterate_vjp(porta_ctx *c, int ndir, const double *mu, const double *chi, const double *grad_out,
                      double *out, double *g_chi, double *g_f, double *g_b, int where);

/* Device memory for the forward Stokes vectors that porta_iterate_vjp keeps
   per ray batch: at most `bytes` (at least one ray's worth); 0 restores the
   default of 16 GB. Fewer bytes, more batches; the result is the same. */
int porta_set_tape_limit(porta_ctx *c, long long bytes);

/* Device time (ms, CUDA events on the context's stream) of the phases of the
   last porta_iterate_vjp, summed over its steps back: ms[0] rebuilding the
   iterates (checkpoint copy, forward iterations, formal solution, J^K_Q
   sums), ms[1] the update's adjoint, ms[2] the forward sweeps that write the
   tape, ms[3] the J^K_Q / Lambda-bar* adjoint sweeps, ms[4] the sums of the
   per-cluster accumulators. The first call for a batch size also times the
   adjoint launch shapes, outside these figures. */
int porta_iterate_timing(const porta_ctx *c, float *ms);

/* Non-linear multigrid (Sec. 5, full-approximation form). porta_mg_setup
   builds nlevels - 1 coarser grids by keeping every other node on each axis
   (coarse (i, j, k) = fine (2i, 2j, 2k); nz -> (nz + 1)/2 for odd nz, nz/2
   for even nz), each a context of its own with the same atom, quadratures
   and precision and the atmosphere sampled at its nodes. nx and ny must be
   divisible by 2^(nlevels - 1) (PORTA_EINVAL otherwise); requires the
   atmosphere (PORTA_ESTATE); call it again after porta_set_atmosphere. The
   method needs the coarse grids to resolve the transfer problem (about one
   plane per decade of optical depth or more, Sec. 5.3). On a multilevel
   context (porta_ml_create) the coarse levels are multilevel contexts of the
   same atom with the opacity scale, temperature and velocity at the
   coincident nodes. */
int porta_mg_setup(porta_ctx *c, int nlevels);

/* Levels built by porta_mg_setup: *nlevels (0 before setup) and, if shapes is
   not NULL, shapes[3 l + 0..2] = nx, ny, nz of level l, finest first. */
int porta_mg_levels(const porta_ctx *c, int *nlevels, int *shapes);

/* Residual of the statistical-equilibrium equations written as A(x) = f
   (Eq. 30 of the multigrid section, Sec. 5.1) at the current unknowns: a
   formal solution (J^K_Q, Lambda-bar*), then r = f - A(x); *rnorm (host)
   receives max over voxels of max_c |r_c| / max_c |x_c| (the residual relative
   to each voxel's largest unknown). It measures the distance from the discrete
   solution independently of the iteration's step (unlike the maximum change).
   Allocates a temporary of the unknowns' size; leaves no formal solution
   behind (PORTA_ESTATE for porta_accumulate_jkq afterwards). PORTA_ESTATE
   without atmosphere and unknowns, or with a frequency band set. */
int porta_residual(porta_ctx *c, double *rnorm);

/* One V-cycle (Eqs. 30-34) from the finest level: npre Jacobi iterations;
   residual r = f - A(rho), A the statistical-equilibrium operator (J^K_Q from
   a formal solution) and f = eps B delta_K0; restriction of rho and r; coarse
   right-hand side A_c(R rho) + R r; the same cycle on the coarser level
   (ncoarse Jacobi iterations on the coarsest); correction rho += P (rho_c -
   R rho); npost Jacobi iterations (Sec. 5.3 uses npre = 2, npost = 4).
   Prolongation P (porta_mg_set_prolongation): tri-linear, linear in height,
   linear extrapolation above the top coarse plane (even nz); or
   tri-cubic-centered; restriction R: the transpose of the tri-linear P
   normalized to keep constants (adjoint of the tri-linear prolongation, Sec. 5.2).
   max_change (host, may be NULL): the maximum relative change of rho over the
   cycle, defined as for porta_see_update (synchronizes). All work is
   enqueued on the context's stream. Multilevel contexts: the unknowns are the
   populations, A(n)_0 = sum_i n_i and A(n)_i the rate equations with the
   plain radiative rates of the formal solution (i >= 1), f = (1, 0, ..., 0);
   max_change is the largest relative change of a population, and the call
   synchronizes and reports PORTA_EKERNEL for a singular system or a
   non-positive population on any level. */
int porta_mg_vcycle(porta_ctx *c, int npre, int npost, int ncoarse, double *max_change);

/* The prolongation of the multigrid cycles (Sec. 5.2, the two operators the
   paper names): order 1 tri-linear (the default after porta_mg_setup), order 3
   tri-cubic-centered -- a fine node between coarse nodes of an axis takes the
   cubic through the four nearest coarse nodes of that axis (periodic in x and
   y with weights -1/16, 9/16, 9/16, -1/16; in height the Lagrange cubic through
   the four coarse planes around it, the four innermost next to the bottom and
   top, the top four above the coarse grid), a tensor product over the axes,
   injection at coincident nodes. The cubic needs at least 4 coarse nodes per
   axis on every level (PORTA_EINVAL otherwise, and for another order);
   PORTA_ESTATE before porta_mg_setup. */
int porta_mg_set_prolongation(porta_ctx *c, int order);

/* Nested multigrid (Sec. 5.1, the nested method): the unknowns of every
   coarser grid are first set to the finest grid's at the coincident nodes;
   then ncoarse Jacobi iterations solve the coarsest grid's own problem
   (A_c(x) = f_c, the same equations sampled on that grid); then, for each
   finer level up to the finest, its unknowns are set to the prolongation of
   the coarser solution and ncycles V-cycles (as porta_mg_vcycle, with that
   level as the finest) follow. The finest grid's starting unknowns thus
   matter only through their injection (S^0_0 = B, S^2_Q = 0, or LTE
   populations, reproduce those of the coarsest grid). max_change (host, may
   be NULL): as porta_mg_vcycle, over the finest level's last V-cycle.
   PORTA_ESTATE before porta_mg_setup or without atmosphere and unknowns;
   PORTA_EINVAL for ncycles < 1, ncoarse < 1 or negative npre, npost. */
int porta_mg_nested(porta_ctx *c, int ncycles, int npre, int npost, int ncoarse, double *max_change);

/* Multilevel atom without polarization: the non-LTE problem of the first kind
   (Sec. 1; the populations of the levels are the unknowns of Eq. 2, the
   polarized problem with rho^0_0 alone). Levels with total angular momentum
   J (weights 2J + 1) and energies E in eV; lines (upper, lower) with Einstein
   A (s^-1) and collisional destruction probability eps = C/(A + C) in (0, 1).
   Intensities are in units of 2 h nu^3 / c^2 of line 0: the Planck function of
   line k is r^3 / (exp(dE/kT) - 1) with r = dE_k / dE_0 and A/B_ul = r^3; the
   line-centre opacity is chi s_k (n_l - n_u g_l/g_u) with chi the atmosphere's
   opacity scale and s_k = (g_u/g_l) A / dE^2 relative to line 0; the source
   function S = r^3 n_u / (n_l g_u/g_l - n_u) (complete redistribution);
   collisions on the line transitions C_ul = eps A/(1 - eps), C_lu = (g_u/g_l)
   exp(-dE/kT) C_ul. Each line is one unpolarized formal solution (Sec. 3) of
   a batched launch (one box per line on the same grid); the update solves the
   rate equations per voxel in FP64 with the radiative rates preconditioned by
   Lambda-bar* (J_eff = Jbar - Lambda-bar* S_old; P_ul = A (1 - Lambda-bar*) +
   B_ul J_eff + C_ul, P_lu = B_lu J_eff + C_lu), linear in the new populations,
   with the row of level 0 replaced by sum n = 1. 2 <= nlevel <= 8,
   1 <= nline <= 8, 2J integral. */
typedef struct {
    int nlevel, nline;
    const double *J, *E;           /* nlevel */
    const int *upper, *lower;      /* nline level indices, E[upper] > E[lower] */
    const double *A, *eps;         /* nline */
    int polarized;                 /* 0: populations only; 1: all rho^K_Q(J), K <= 2J */
    double zeta;                   /* polarized: weak-field Zeeman splitting per gauss (Doppler widths) */
} porta_ml_atom;

/* The polarized multilevel atom (polarized = 1): the unknowns are the
   multipolar components rho^K_Q(J) of every level (K = 0 .. 2J, Q = -K .. K,
   no interference between levels; sum_J (2J+1)^2 real unknowns per voxel, 69
   for J = 0, 1, 2, 1, 2), stored per voxel in the real order level, K, then
   rho^K_0, Re rho^K_1, Im rho^K_1, ..., Re rho^K_K, Im rho^K_K
   (rho^K_-Q = (-1)^Q conj rho^K_Q). Rate equations (the multilevel atom
   without interference between levels; the paper takes them from LL04 Sect.
   7.2): absorption TA, spontaneous emission TE and stimulated emission TS into
   a level, relaxation RA + RE + RS out of it (Wigner 3j/6j/9j coefficients
   times the line's J^Kr_Qr, Kr = 0, 1, 2), the Hanle term -i 2 pi nu_L g_J (b.J)
   of d rho / dt (counterclockwise precession about the field) with Lande
   factor 1 for every level and nu_L = 1.3996e6 Hz/G, collisions on
   the line transitions moving populations and relaxing every multipole of the
   level they leave. Jacobi: Lambda-bar* preconditioning of the population
   terms as for the unpolarized atom, the trace row sum_J sqrt(2J+1)
   rho^0_0(J) = 1; one warp per voxel solves the FP64 system in shared
   memory. Line transfer: each line is a polarized two-level formal solution
   (Sec. 3) with the line opacity of the populations, the emissivity of the
   upper level's K = 0, 1, 2 multipoles (S^K_Q = S_line w^(K) conj(rho^K_Q /
   rho^0_0), w^(K) = (-1)^(1+Jl+Ju) sqrt(3(2Ju+1)) {1 1 K; Ju Ju Jl}; K = 0, 2
   in eps_I, eps_Q, eps_U, the orientation K = 1 in eps_V through
   T^1_Q(V, Omega) = sqrt(3/2) Omega_Q), the weak-field Zeeman term with
   2 zeta B, and the dichroism of the line's absorption (lower level) and
   stimulated emission (upper level) from their alignment (K = 2; eta_Q,
   eta_U and a rescaled eta_I) and orientation (K = 1; eta_V, the absorption
   term with the sign (-1)^K); J^1_Q = sum_m w_m T^1_Q(V, Omega_m) Vbar_m
   comes from Stokes V. porta_mg_setup / porta_mg_vcycle run the multigrid
   cycle with the multipoles as unknowns (A(x) the plain rate equations with
   the trace row; max_change over the populations). */

/* Create a multilevel context on grid g (PORTA_EINVAL for an invalid atom or
   grid). The generic calls porta_formal_solve, porta_accumulate_jkq,
   porta_see_update, porta_run_iterations, porta_autotune and
   porta_launch_info apply to it (J^K_Q and Lambda-bar* per line, the update
   of the populations); porta_set_rho and porta_iterate_ckpt
   are rejected; porta_mg_setup / porta_mg_vcycle run the multigrid cycle with
   the populations as unknowns. Voxel arrays of the line boxes are
   [line][voxel]. */
int porta_ml_create(const porta_grid *g, const porta_ml_atom *a, const porta_quad *q, const porta_opts *o,
                    porta_ctx **out);

/* Per-voxel atmosphere (nvox doubles each, host or device per `where`):
   chi = opacity scale (> 0), kT = temperature in eV (> 0), vel = vertical
   velocity in Doppler widths (the same for every line); bx, by, bz = magnetic
   field in gauss (required for the polarized atom, ignored (may be NULL)
   otherwise). The polarized atom's first-order Zeeman term must stay a
   propagation matrix: PORTA_EINVAL unless 2 zeta max|B| (x_max + max|vel|) < 1. */
int porta_ml_set_atmosphere(porta_ctx *c, const double *chi, const double *kT, const double *vel, const double *bx,
                            const double *by, const double *bz, int where);

/* Emergent Stokes profiles of line `line` (Sec. 1: the emergent profiles of
   any line and line of sight once the unknowns are known) for ndir
   outgoing directions (mu in (0, 1], azimuth chi; host arrays): the
   emergent-mode formal solution of the line with its opacity, emissivity,
   dichroism and Zeeman term from the current unknowns. out:
   ndir*n_nu*ny*nx*NS doubles (NS = 4 for the polarized atom, 1 otherwise),
   [dir][nu][y][x][stokes], host or device per `where`. Synchronous. */
int porta_ml_emergent_stokes(porta_ctx *c, int line, int ndir, const double *mu, const double *chi, double *out,
                             int where);

/* Solve of the rate equations' K > 0 block (polarized atom, after the population
   block): mode 0 (default) factors it in FP32 with partial pivoting and refines
   the solution with FP64 residuals until the correction is below 1e-13 of it,
   falling back to mode 1 for a voxel whose refinement stalls or whose pivot
   vanishes; mode 1 eliminates the whole system in FP64 with partial pivoting.
   Both give the FP64 solution to its rounding (mode 0 does ~1/8 of the FP64
   arithmetic, which this GPU runs at a small fraction of its FP32 rate).
   PORTA_EINVAL for another mode or a context that is not a polarized
   multilevel one. Drops any captured iteration graph. */
int porta_ml_set_solve(porta_ctx *c, int mode);

/* Number of real unknowns per voxel (nlevel for the unpolarized atom). */
int porta_ml_unknowns(const porta_ctx *c, int *nunk);

/* The full vector of unknowns [voxel][nunk] (populations, or the multipoles of
   the polarized atom in the order given above). set requires the atmosphere
   and rejects non-positive populations or a population inversion. */
int porta_ml_set_unknowns(porta_ctx *c, const double *x, int where);
int porta_ml_get_unknowns(porta_ctx *c, double *x, int where);

/* Populations [voxel][level] (> 0; the update normalizes them to sum 1; for
   the polarized atom: no atomic polarization, rho^0_0 = n / sqrt(2J+1)).
   Writes every line's opacity, source and Planck functions; PORTA_EINVAL if a
   line's opacity is not positive (population inversion). Requires the
   atmosphere. */
int porta_ml_set_pops(porta_ctx *c, const double *pops, int where);
int porta_ml_get_pops(porta_ctx *c, double *pops, int where);

/* Formal solution of every line and the sums Jbar, Lambda-bar* per line
   ([line][voxel] doubles; NULL keeps them on the device). Polarized atom:
   jbar is [line][voxel][9] in the order J00, J10, Re J11, Im J11, J20,
   Re J21, Im J21, Re J22, Im J22 (J^K_-Q = (-1)^Q conj J^K_Q). */
int porta_ml_formal_solve(porta_ctx *c, double *jbar, double *lstar, int where);

/* Update of the populations from the last sums; max_change (host, may be
   NULL) is the maximum relative change of a population (synchronizes and then
   reports PORTA_EKERNEL for a singular system or a non-positive result). */
int porta_ml_see_update(porta_ctx *c, double *max_change);

/* `iterations` eager Jacobi iterations (formal solution of every line, sums,
   update); max_change as for porta_ml_see_update, of the last one. */
int porta_ml_iterate(porta_ctx *c, int iterations, double *max_change);

#ifdef __cplusplus
}
#endif
#endif /* PORTA_H */
