// Internal declarations of the GB300 formal-solver library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

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
    Real w;          // quadrature weight w_m of the ray (0 for a line of sight)
    Real pad;
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
    int cstride, istride;  // J^K_Q sweep: Reals per (slot, frequency) coefficient plane and per (buffer, frequency) Stokes plane
    int interp;            // general sweep: 2 biquadratic interpolation at M and P, else bilinear
    // explicit medium (emergent general sweep, NS = 4): K'/eta_I [6][nvox] and S [4][nvox], FP64
    const double *kexpl, *sexpl;
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
    // polarized lines of the multilevel atom (null: none): [11][nvox] the dichroism
    // multipoles D^2_Q (D20, Re/Im D21, Re/Im D22), D^1_Q (D10, Re/Im D11) and the
    // orientation emission multipoles S^1_Q (S10, Re/Im S11); J mode: partv [ray][nvox]
    // the per-ray frequency integrals of Stokes V (for J^1_Q)
    const Real *dich;
    Real *partv;
    Real *probe;                   // [nu][nvox][ns]
    Real *probe_ls;                // [nu][nvox]
    int *next_item;                // J mode: null (static striding) or the launch's work-list counter
    // reverse mode of the emergent sweep (single box)
    Real *store;                   // emergent: null, or the Stokes vectors of every plane [dir][nu][nvox][ns]
    const double *gout;            // adjoint: dL/dI on the top plane [dir][nu][ny][nx][ns]
    Real *gpart;                   // adjoint: per (dir, frequency group) partial gradients [item][3][nvox]
    // adjoint in the unknowns rho (through iterations): per-cluster accumulators (Real) of
    // dL/dchi (fixed rho), dL/dB (3), dL/drho (6) [cluster][10][nvox]; for the J^K_Q sums
    // of a formal solution also dL/dJ [v][nj], dL/dLambda* [v], ray weights and T ([ray][19])
    void *gacc;
    const Real *gjkq, *glstar;     // (in the sweep's precision)
    const double *tw;
    int ray0;                      // first ray of the batch (rays and geom point at it)
    // J^K_Q formal solution (sweep_j.cu): fixed-point accumulators of the weighted
    // ray sums [NJ + 1][nvox] (J^K_Q components, then Lambda-bar*), the power-of-two
    // exponent of each voxel's fixed-point scale, and the overflow flag
    unsigned long long *jacc;
    const int *jexp;
    int *jerr;
};

struct LaunchCfg {
    int cluster;     // CTAs per cluster
    int F;           // frequencies per pass
    int threads;
    int smem;        // dynamic shared memory bytes
    int clusters;    // clusters launched
    int priority;    // launch priority (0: the stream's; else a value of cudaDeviceGetStreamPriorityRange)
};

template <typename Real, int NS>
cudaError_t launch_sweep(const SweepArgs<Real> &a, int mode, LaunchCfg &cfg, cudaStream_t st);

// shared memory of the sweep: ring (3 planes of `ring_plane` chunks),
// Stokes planes (2 x F x ipts_max points), lane-reduction scratch (na
// accumulated quantities per thread)
template <typename Real, int NS>
int sweep_smem_bytes(int ring_plane, int ipts_max, int F, int threads, int na);

template <typename Real, int NS>
cudaError_t max_active_clusters(int cluster, int smem, int threads, int *out, bool dich = false, bool bq = false,
                                bool gk = false);

// the J^K_Q formal solution (sweep_j.cu): per-frequency node coefficients in
// shared memory; ring capacity `nodes` per slot, Stokes planes of `ipts` points.
// Plane strides are padded to 16 (mod 32) 4-byte words, so that the two
// frequency lanes of a point (adjacent threads) read distinct banks.
__host__ __device__ inline int jsweep_stride(int reals, int real_bytes)
{
    int words = reals * real_bytes / 4;
    words += ((16 - words % 32) + 32) % 32;
    return words * 4 / real_bytes;
}
template <typename Real, int NS>
int jsweep_smem_bytes(int nodes, int ipts, int F, int threads);
template <typename Real, int NS>
cudaError_t jsweep_max_active_clusters(int cluster, int smem, int threads, int *out);
template <typename Real, int NS>
cudaError_t launch_jsweep(const SweepArgs<Real> &a, LaunchCfg &cfg, cudaStream_t st);
// before a J^K_Q formal solution: zero the fixed-point accumulators and set each
// voxel's scale exponent; after it: J^K_Q and Lambda-bar* in FP64 from them
template <typename Real, int NS>
cudaError_t launch_jacc_prepare(const SweepArgs<Real> &a, cudaStream_t st);
template <int NS>
cudaError_t launch_jacc_finalize(long long nvox, const unsigned long long *jacc, const int *jexp, double *jkq,
                                 double *lstar, cudaStream_t st);

// adjoint of the emergent sweep (adjoint.cu): shared memory of a launch with
// ring plane `ring_plane` (16-byte chunks), `ipts` points per strip, tape
// tiles of `tile_pts` points and F frequencies per pass; occupancy; launch;
// the fixed-order sum over items
// form: 0 emergent Stokes, gradients in (chi, e = chi S00, B) per item; 1 emergent Stokes,
// gradients in (chi, B, rho) accumulated per cluster; 2 the J^K_Q / Lambda-bar* of a formal
// solution (rays of a batch), gradients in (chi, B, rho) accumulated per cluster
template <typename Real, int NS>
int adjoint_smem_bytes(int ring_plane, int ipts, int tile_pts, int F);
template <typename Real, int NS>
cudaError_t adjoint_max_active_clusters(int cluster, int smem, int threads, int *out, int form = 0);
template <typename Real, int NS>
cudaError_t launch_adjoint(const SweepArgs<Real> &a, const LaunchCfg &cfg, cudaStream_t st, int form = 0);
template <typename Real>
cudaError_t launch_adjoint_reduce(const Real *gpart, int nitems, int ngroups, long long nvox, const RayDev<Real> *rays,
                                  double bfac, double *g_chi, double *g_e, double *g_b, cudaStream_t st);
// sum of the per-cluster accumulators in cluster order: g_chi and g_b added, g_rho overwritten
template <typename Real>
cudaError_t launch_adjoint_acc_reduce(const Real *gacc, int nclusters, long long nvox, int nl, double *g_chi,
                                      double *g_b, double *g_rho, cudaStream_t st);

}  // namespace porta
