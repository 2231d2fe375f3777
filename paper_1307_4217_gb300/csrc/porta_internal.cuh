// Internal declarations of the GB300 formal-solver library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "porta.h"

namespace porta {

// Per-plane geometry of one ray, in sweep order q = 0..nz-1 (q = 0 is the
// boundary plane where the ray enters). The sweep works in a sheared frame
// that follows the characteristics: sheared node (c, r) of plane q is the
// physical node ((c + ax) mod nx, (r + ay) mod ny) of level kz. For q >= 1 the
// horizontal displacement from the upwind point M to O is d = ds * Omega_xy /
// spacing (cells); with ax(q) = ax(q-1) + ceil(d) the upwind corners of sheared
// node (c, r) are sheared (c|c+1, r|r+1) on plane q-1 with weights
// (1-t, t), t = ceil(d) - d, and the downwind corners are (c-1|c, r-1|r) on plane
// q+1 with weights (t', 1-t') taken from plane q+1.
template <typename Real>
struct PlaneGeom {
    int ax, ay, kz, pad;
    Real tx, ty, ds, pad2;   // ds = path length M -> O (q >= 1)
};

// Per-ray constants: direction and the angular tensors T^K_Q(i, Omega) for
// i = I, Q, U (rows of 6: T00, T20, Re T21, Im T21, Re T22, Im T22).
template <typename Real>
struct RayDev {
    Real mu, ox, oy, oz;
    Real t[18];
    Real pad[2];
};

enum SweepMode { MODE_JKQ = 0, MODE_EMERGENT = 1 };

// One box of a (possibly batched) problem: sizes, first voxel in the
// concatenated voxel arrays, first plane record of its ray geometry
// ([ray][nz] PlaneGeom records).
struct BoxDev {
    int nx, ny, nz, pad;
    long long vox0, geom0;
};

template <typename Real>
struct SweepArgs {
    int nnu, nray;
    long long nvox;      // voxels of all boxes
    int nitems;          // work items: (box, ray) pairs (J mode) or directions x groups (emergent)
    const int *items;    // J mode: item -> box * nray + ray, ordered by decreasing cost
    const BoxDev *boxes;
    int ngroups, F;      // frequency groups and frequencies per group
    int ring_plane;      // shared-memory ring plane capacity (16-byte chunks), max over boxes
    int ipts_max;        // Stokes-plane capacity (points), max over boxes
    Real bfac;           // 2 * gbar * zeta (weak-field Zeeman, eta_V / (eta_I x B.Omega))
    const PlaneGeom<Real> *geom;   // per box: [ray][nz]
    const RayDev<Real> *rays;      // [ray]
    const Real *xf, *wf;           // frequency nodes and trapezoid weights
    // atmosphere (SoA, Real) and unknowns
    const Real *chi, *vel, *bx, *by, *bz, *bpl;
    const Real *rho;               // [nl][nvox]
    const Real *invn;              // [ray][nvox] profile normalization (J mode)
    void *part;                    // [ray][nvox] partial integrals (J mode)
    double *out;                   // emergent: [dir][nu][ny][nx][ns]
    int probe_ray;                 // -1 or the ray whose Stokes vectors are written to probe
    Real *probe;                   // [nu][nvox][ns]
    Real *probe_ls;                // [nu][nvox]
    // reverse mode of the emergent sweep (single box)
    Real *store;                   // emergent: null, or the Stokes vectors of every plane [dir][nu][nvox][ns]
    const double *gout;            // adjoint: dL/dI on the top plane [dir][nu][ny][nx][ns]
    Real *gpart;                   // adjoint: per (dir, frequency group) partial gradients [item][3][nvox]
};

struct LaunchCfg {
    int cluster;     // CTAs per cluster
    int F;           // frequencies per pass
    int threads;
    int smem;        // dynamic shared memory bytes
    int clusters;    // clusters launched
};

template <typename Real, int NS>
cudaError_t launch_sweep(const SweepArgs<Real> &a, int mode, LaunchCfg &cfg, cudaStream_t st);

// shared memory of the sweep: ring (3 planes of `ring_plane` chunks),
// Stokes planes (2 x F x ipts_max points), lane-reduction scratch
template <typename Real, int NS>
int sweep_smem_bytes(int ring_plane, int ipts_max, int F, int threads);

template <typename Real, int NS>
cudaError_t max_active_clusters(int cluster, int smem, int threads, int *out);

// adjoint of the emergent sweep (adjoint.cu): shared memory of a launch with
// ring plane `ring_plane` (16-byte chunks), `ipts` points per strip, tape
// tiles of `tile_pts` points and F frequencies per pass; occupancy; launch;
// the fixed-order sum over items
template <typename Real, int NS>
int adjoint_smem_bytes(int ring_plane, int ipts, int tile_pts, int F);
template <typename Real, int NS>
cudaError_t adjoint_max_active_clusters(int cluster, int smem, int threads, int *out);
template <typename Real, int NS>
cudaError_t launch_adjoint(const SweepArgs<Real> &a, const LaunchCfg &cfg, cudaStream_t st);
template <typename Real>
cudaError_t launch_adjoint_reduce(const Real *gpart, int nitems, int ngroups, long long nvox, const RayDev<Real> *rays,
                                  double bfac, double *g_chi, double *g_e, double *g_b, cudaStream_t st);

}  // namespace porta

struct porta_ctx {
    int nx = 0, ny = 0, nz = 0;
    double lx = 0, ly = 0;
    std::vector<double> z;
    int model = 0, ns = 1, nl = 1, nj = 1;
    double zeta = 0, gbar = 1, bcrit = 25;
    int n_mu = 0, n_chi = 0, n_nu = 0;
    double x_max = 4;
    int precision = PORTA_FP32;
    int opt_cluster = 0, opt_nu_group = 0;
    long long nvox = 0;
    int nray = 0;
    std::vector<double> mu, chi, w, xf, wf, tkq;  // quadratures, T^K_Q per ray (18)
    cudaStream_t stream = nullptr;
    std::string err;
    bool have_atm = false, have_rho = false, have_fs = false, have_jkq = false;

    // device memory
    size_t rsz = 4;                 // sizeof(Real) of the sweep
    void *d_atm = nullptr;          // Real SoA: chi, vel, bx, by, bz, bpl
    double *d_eps = nullptr;        // FP64 per-voxel eps, bpl, B (SEE)
    double *d_bpl = nullptr;
    double *d_b = nullptr;          // 3*nvox
    double *d_rho = nullptr;        // nvox*nl FP64
    void *d_rhoR = nullptr;         // nl*nvox Real
    void *d_invn = nullptr;         // nray*nvox Real
    void *d_geom = nullptr;         // nray*nz PlaneGeom
    void *d_rays = nullptr;         // nray RayDev
    void *d_freq = nullptr;         // xf, wf (Real)
    void *d_part = nullptr;         // nray*nvox*(ns==1 ? 2 : 4) Real
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
    // reverse mode of the emergent sweep: tape of the forward Stokes vectors,
    // per-item partial gradients, forced launch shape (0 = automatic), last launch
    void *d_tape = nullptr;
    size_t tape_bytes = 0;
    void *d_gpart = nullptr;
    size_t gpart_bytes = 0;
    int adj_cluster = 0, adj_nu_group = 0;
    porta::LaunchCfg last_adj{};
    float adj_fwd_ms = 0.f, adj_rev_ms = 0.f;   // device time of the last porta_emergent_vjp
    int adj_tuned_ndir = 0;                     // automatic shape: timed once per direction count
    porta::LaunchCfg adj_tuned{};
    cudaEvent_t adj_ev[3] = {nullptr, nullptr, nullptr};
};
