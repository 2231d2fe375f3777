// Host-side state of one solver context (include/porta.h's porta_ctx): the
// problem description, quadratures, device buffers and launch choices.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "ml_kernels.cuh"
#include "mlpol_kernels.cuh"
#include "porta_internal.cuh"

// multilevel atom without polarization: one box of the batch per line
struct MlState {
    porta::MlConst mc{};
    long long nvox1 = 0;               // voxels of the grid (one box)
    double *d_pops = nullptr;          // [nvox1][nlev]
    double *d_chis = nullptr;          // opacity scale, nvox1
    double *d_kT = nullptr;            // kT (eV), nvox1
    unsigned long long *d_bad = nullptr;
    bool have_atm = false, have_pops = false;
    // the atom as given (coarse multigrid levels are created from it)
    std::vector<double> J, E, A, eps;
    std::vector<int> up, lo;
    // polarized atom: multipoles x [nvox1][nunk] and the rate-equation tables
    bool pol = false;
    int nunk = 0;
    double *d_x = nullptr;
    void *d_tab = nullptr;
    porta::MlPolTables tab;
    porta::MlPolDev dev{};
};

// stream, fork/join events and work-list counters of the concurrent launch
struct LaunchFill {
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    int *d_ctr = nullptr;   // [2]: next item of the main and of the filler launch
};

struct porta_ctx {
    int nx = 0, ny = 0, nz = 0;
    double lx = 0, ly = 0;
    std::vector<double> z;
    int model = 0, ns = 1, nl = 1, nj = 1;
    double zeta = 0, gbar = 1, bcrit = 25;
    int n_mu = 0, n_chi = 0, n_nu = 0;
    double x_max = 4;
    int precision = PORTA_FP32;
    bool jk_fits = true;                // a launch shape of the J^K_Q sweep kernel (sweep_j.cu) fits the grid
    int fr0 = 0, fr1 = 0;               // frequency band [fr0, fr1) of the J^K_Q formal solution (fr1 = 0: all)
    bool jkq_loaded = false;            // J^K_Q / Lambda-bar* set by porta_set_partial (not from this context's sweep)
    int opt_cluster = 0, opt_nu_group = 0;
    int user_cluster = 0, user_nu_group = 0;     // as given in porta_opts (0: automatic)
    bool user_shape = false;            // launch shape given in porta_opts (not autotuned)
    std::map<int, porta::LaunchCfg> emg_tuned;   // emergent sweep: shape timed once per direction count
    long long nvox = 0;
    int nray = 0;
    std::vector<double> mu, chi, w, xf, wf, tkq;  // quadratures, T^K_Q per ray (18)
    cudaStream_t stream = nullptr;
    std::string err;
    bool have_atm = false, have_rho = false, have_fs = false, have_jkq = false;

    // device memory
    size_t rsz = 4;                 // sizeof(Real) of the sweep
    void *d_atm = nullptr;          // Real SoA: chi, vel, bx, by, bz, bpl
    double *d_cv64 = nullptr;       // FP64 chi and vel (2*nvox), kept for the multigrid's coarse atmospheres
    double *d_eps = nullptr;        // FP64 per-voxel eps, bpl, B (SEE)
    double *d_bpl = nullptr;
    double *d_b = nullptr;          // 3*nvox
    double *d_rho = nullptr;        // nvox*nl FP64
    void *d_rhoR = nullptr;         // nl*nvox Real
    void *d_invn = nullptr;         // nray*nvox Real
    void *d_geom = nullptr;         // nray*nz PlaneGeom
    void *d_rays = nullptr;         // nray RayDev
    void *d_freq = nullptr;         // xf, wf (Real)
    void *d_part = nullptr;         // nray*nvox*(ns==1 ? 2 : 4) Real (general sweep only; allocated on first use)
    unsigned long long *d_jacc = nullptr;   // J^K_Q sweep: fixed-point sums [nj + 1][nvox] (allocated on first use)
    int *d_jexp = nullptr;                  // J^K_Q sweep: per-voxel fixed-point exponent
    double *d_tw = nullptr;         // nray*19 FP64: w_m, T (18)
    double *d_jkq = nullptr, *d_lstar = nullptr;
    unsigned long long *d_resid = nullptr;
    // batched problems: per-box sizes, grids and offsets
    int nbox = 1;
    std::vector<porta::BoxDev> boxes;
    std::vector<std::vector<double>> bz;
    std::vector<double> blx, bly;
    void *d_boxes = nullptr;       // nbox BoxDev
    int *d_items = nullptr;        // nbox*nray work items ordered by decreasing cost
    int *d_tune_items = nullptr;   // strided sample of the work items for the autotuner
    int n_tune = 0;
    int *d_err = nullptr;
    // CUDA graph of one Jacobi iteration (porta_run_iterations)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    // last launch of the formal solution
    porta::LaunchCfg last{};
    // optional second, concurrent sweep launch of smaller clusters over the
    // cheapest fraction `fill_frac` of the work list: it runs on SMs that the
    // main launch's clusters cannot occupy (fill_cfg.cluster == 0: none)
    porta::LaunchCfg fill_cfg{};
    double fill_frac = 0.0;
    LaunchFill *fill = nullptr;
    // non-linear multigrid (porta_mg_setup): coarse levels, finer first (each a
    // context of its own), and work buffers [voxel][nl] FP64
    std::vector<porta_ctx *> mg;
    double *mg_res = nullptr;       // residual of this level
    double *mg_src = nullptr;       // right-hand side of this level's problem (coarse levels)
    double *mg_rho0 = nullptr;      // restriction of the finer level's unknowns (coarse levels)
    double *mg_prev = nullptr;      // unknowns at the start of a V-cycle (finest level)
    double *mg_zr = nullptr;        // to the next coarser level: per coarse plane 4 x (fine plane, weight)
    double *mg_zp = nullptr;        // from the next coarser level: per fine plane (k0, w0, k1, w1)
    double *mg_zp3 = nullptr;       // the same for the cubic: per fine plane 4 x (coarse plane, weight)
    int mg_order = 1;               // prolongation: 1 tri-linear, 3 tri-cubic-centered (finest level)
    int interp = 1;                 // interpolation at M and P: 1 bilinear, 2 biquadratic (general sweep)
    int sc_faces = 0;               // 1: M and P on the first cell face crossed (faces.cu, J^K_Q formal solution)
    int gsweep = 0;                 // J^K_Q formal solution by the global-memory sweep of faces.cu in the plane
                                    // placement: 1 asked for, 2 where no shared-memory launch shape fits
    bool gsweep_checked = false;    // whether the shared-memory shapes have been checked
    void *d_faces = nullptr;        // its per-ray plane buffers (allocated on first use)
    void *d_fdxy = nullptr;         // its cell sizes, (dx, dy) per box
    size_t faces_bytes = 0;
    double *d_kexpl = nullptr;      // explicit medium: K'/eta_I [6][nvox] and S [4][nvox] (emergent sweep)
    double *d_sexpl = nullptr;
    // reverse mode of the emergent sweep: tape of the forward Stokes vectors,
    // per-item partial gradients, forced launch shape (0 = automatic), last launch
    void *d_tape = nullptr;
    size_t tape_bytes = 0;
    void *d_gpart = nullptr;
    size_t gpart_bytes = 0;
    int adj_cluster = 0, adj_nu_group = 0;
    porta::LaunchCfg last_adj{};
    void *d_gacc = nullptr;         // per-cluster gradient accumulators, Real (gradients in rho)
    void *d_gjR = nullptr;          // dL/dJ^K_Q and dL/dLambda* in the sweep's precision ([nvox][nj], [nvox])
    size_t gjR_bytes = 0;
    double *d_vjp_out = nullptr;    // emergent output of the taped forward sweeps (not read)
    size_t vjp_out_bytes = 0;
    size_t gacc_bytes = 0;
    // differentiation through Jacobi iterations (porta_iterate_ckpt): checkpoints of
    // rho [nvox][nl] every it_ckpt iterations, the iteration count, rho at the end
    std::vector<double *> it_saved;
    double *it_final = nullptr;
    int it_niter = 0, it_ckpt = 0;
    MlState *ml = nullptr;                 // multilevel atom (porta_ml_create), else null
    // polarized lines of a multilevel atom (null: none): Real [11][nvox] the dichroism multipoles
    // D^2_Q (5), D^1_Q (3) and the orientation emission multipoles S^1_Q (3); the per-ray
    // frequency integrals of Stokes V (Real [ray][nvox], allocated on first use), J^1_Q
    // (FP64 [nvox][3]: J10, Re J11, Im J11) and the ray weights times T^1_Q(V, Omega) ([ray][3])
    void *d_dich = nullptr;
    void *d_partv = nullptr;
    double *d_j1 = nullptr, *d_tw1 = nullptr;
    size_t tape_limit = (size_t)16 << 30;  // device tape of the J^K_Q reverse (ray batches)
    std::map<int, porta::LaunchCfg> adj2_tuned;  // J^K_Q adjoint: shape timed once per batch size
    cudaEvent_t it_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // device time (ms) of the last porta_iterate_vjp: recomputation of the iterates,
    // update adjoint, forward tape sweeps, J^K_Q adjoint sweeps, accumulator sums
    float it_ms[5] = {0, 0, 0, 0, 0};
    float adj_fwd_ms = 0.f, adj_rev_ms = 0.f;   // device time of the last porta_emergent_vjp
    int adj_tuned_ndir = 0;                     // automatic shape: timed once per direction count
    porta::LaunchCfg adj_tuned{};
    cudaEvent_t adj_ev[3] = {nullptr, nullptr, nullptr};
};
