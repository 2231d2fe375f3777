// Host internals of the C ABI (include/porta.h) shared by its translation
// units: api.cu (contexts, formal solution, Jacobi iteration, frequency bands),
// api_adjoint.cu (emergent Stokes profiles and reverse mode), api_mg.cu
// (multigrid, Sec. 5) and api_ml.cu (multilevel atoms). Error reporting, the
// capped device allocator, the per-ray plane geometry and the sweep's launch
// shape selection.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "porta.h"
#include "porta_ctx.h"
#include "porta_internal.cuh"

namespace porta_api {

using namespace porta;

// records msg as the context's last error and returns code
int fail(porta_ctx *c, int code, const std::string &msg);

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(c, PORTA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)

// Device allocations of the library go through pmalloc / pfree, which keep the
// live byte count and honour the process-wide cap of porta_set_device_limit: an
// allocation that would exceed the cap fails with cudaErrorMemoryAllocation
// (reported as PORTA_ENOMEM) without calling the CUDA runtime.
cudaError_t pmalloc_bytes(void **p, size_t bytes);
cudaError_t pfree(void *p);

template <typename T>
cudaError_t pmalloc(T **p, size_t bytes)
{
    void *q = nullptr;
    cudaError_t e = pmalloc_bytes(&q, bytes);
    *p = (T *)q;
    return e;
}

template <typename T>
cudaError_t dalloc(T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) return cudaSuccess;
    return pmalloc(p, n * sizeof(T));
}

// T^K_Q(i, Omega) for i = I, Q, U from the polarization tensors of the ray
// frame: with e_a = dOmega/dtheta and e_b = z x Omega / |z x Omega|, Stokes
// I, Q, U correspond to e_a e_a + e_b e_b, e_a e_a - e_b e_b, e_a e_b + e_b e_a;
// T^0_0 is half the trace and T^2_Q = -sqrt(3)/2 times the spherical
// components of the traceless part (A_0 = sqrt(3/2) A_zz, A_1 = -(A_xz + i A_yz),
// A_2 = (A_xx - A_yy + 2 i A_xy)/2). Output rows of 6 reals per Stokes parameter.
void tkq_tensors(double mu, double chi, double out[18]);

// Gauss-Legendre nodes and weights on (0, 1), n of each, x increasing
void gauss_legendre(int n, double *x, double *w);

// drops the context's captured Jacobi-iteration graph
void drop_graph(porta_ctx *c);
// set c->gsweep = 2 (the global-memory sweep) once, where no shared-memory sweep fits
void check_global_sweep(porta_ctx *c);

inline long long wrapll(long long a, long long n)
{
    long long r = a % n;
    return r < 0 ? r + n : r;
}

// plane geometry of one direction in sweep order (see PlaneGeom) for a grid
// nx x ny x nz with periods lx, ly and heights z
template <typename Real>
void plane_geometry(int nx, int ny, int nz, double lx, double ly, const double *z, double mu, double chi,
                    PlaneGeom<Real> *g)
{
    const bool up = mu > 0;
    const double st = std::sqrt(std::max(0.0, 1.0 - mu * mu));
    const double ox = st * std::cos(chi), oy = st * std::sin(chi);
    const double hx = lx / nx, hy = ly / ny, amu = std::fabs(mu);
    long long ax = 0, ay = 0;
    for (int q = 0; q < nz; ++q) {
        int kz = up ? q : nz - 1 - q;
        PlaneGeom<Real> p{};
        p.kz = kz;
        if (q > 0) {
            int ku = up ? kz - 1 : kz + 1;
            double ds = std::fabs(z[kz] - z[ku]) / amu;
            double dx = ds * ox / hx, dy = ds * oy / hy;
            double cx = std::ceil(dx), cy = std::ceil(dy);
            ax = wrapll(ax + (long long)cx, nx);
            ay = wrapll(ay + (long long)cy, ny);
            p.tx = (Real)(cx - dx);
            p.ty = (Real)(cy - dy);
            p.ds = (Real)ds;
        }
        p.ax = (int)ax;
        p.ay = (int)ay;
        g[q] = p;
    }
}

template <typename Real>
RayDev<Real> ray_dev(double mu, double chi, double w = 0.0)
{
    RayDev<Real> r{};
    r.w = (Real)w;
    double st = std::sqrt(std::max(0.0, 1.0 - mu * mu));
    r.mu = (Real)mu;
    r.ox = (Real)(st * std::cos(chi));
    r.oy = (Real)(st * std::sin(chi));
    r.oz = (Real)mu;
    double t[18];
    tkq_tensors(mu, chi, t);
    for (int i = 0; i < 18; ++i) r.t[i] = (Real)t[i];
    return r;
}

const int kThreads = 512;   // maximum threads per CTA of the sweep kernel
const int kSmemLimit = 220 * 1024;

// Shared-memory capacities of a launch with cluster size C over all boxes:
// ring plane (16-byte chunks) and Stokes-plane points, each the maximum over boxes.
template <typename Real, int NS>
void launch_caps(const porta_ctx *c, int C, int &ring_plane, int &ipts_max, bool jk = false)
{
    const int nch = (NS == 1 ? 4 : 8) * (int)sizeof(Real) / 16;
    const bool dich = NS == 4 && c->d_dich != nullptr;
    ring_plane = 0;
    ipts_max = 0;
    for (const BoxDev &b : c->boxes) {
        const int rmax = (b.ny + C - 1) / C;
        const int chunk = (rmax + 2) * b.nx;
        if (jk) {
            // the J^K_Q sweep (sweep_j.cu): ring capacity in nodes
            ring_plane = std::max(ring_plane, chunk);
            ipts_max = std::max(ipts_max, rmax * b.nx);
            continue;
        }
        // with dichroism the slots of a second ring follow the node ring (eta_U / eta_I and the
        // two orientation terms, 3 words per node); an explicit medium keeps K'/eta_I there
        // (6 words per node); the biquadratic stencils need two halo rows on each side instead of one
        const int gchunk = c->interp == 2 && !c->d_kexpl ? (rmax + 4) * b.nx : chunk;
        const int dwords = dich ? 3 : (c->d_kexpl ? 6 : 0);
        const int dchunks = (dwords * ((chunk * (int)sizeof(Real) + 15) / 16 * 16) + 15) / 16;
        ring_plane = std::max(ring_plane, nch * gchunk + dchunks);
        ipts_max = std::max(ipts_max, rmax * b.nx);
    }
}

// The J^K_Q formal solution runs the kernel of sweep_j.cu (per-frequency
// node coefficients in shared memory) unless the lines carry dichroism, which
// only the general sweep (sweep.cu) implements, or a plane is too wide for its
// shared memory (then the general sweep, which needs less per frequency, runs).
bool use_jk(const porta_ctx *c);

// The J^K_Q sweep sums an FP32 formal solution into fixed-point accumulators;
// an FP64 one keeps per-ray partial integrals summed in ray order in FP64 (a
// fixed-point scale cannot hold 1e-10 relative precision for quantities that
// span many decades within one voxel, as Lambda-bar* does with optical depth).
bool jfixed(const porta_ctx *c);

// frequencies of the J^K_Q formal solution (its band, porta_set_freq_range)
int jnu(const porta_ctx *c);

// largest / smallest plane height ny over the context's boxes
int max_ny(const porta_ctx *c);
int min_ny(const porta_ctx *c);

// Launch shape of the sweep: cluster size C (CTAs sharing one ray's plane)
// and frequencies per pass F. Estimated time of a candidate (in units of one
// point update): the (box, ray) work items spread over the resident clusters,
// each item costing, per plane and frequency pass, the thread slots of its
// point updates, the ring fill (halo rows included), the partial-integral
// writes and a barrier.
template <typename Real, int NS>
int choose_launch(porta_ctx *c, LaunchCfg &best, int force_c, int force_f, int nitems, bool jk = false, int nnu = 0)
{
    const int NU = nnu > 0 ? nnu : c->n_nu;     // frequencies swept
    if (force_f > NU) force_f = NU;
    // accumulated quantities per point (Stokes V too for the polarized lines of a multilevel atom)
    const int NA = NS == 1 ? 2 : (c->d_dich ? 5 : 4);
    double best_cost = 1e300;
    best = LaunchCfg{};
    const int ny_max = max_ny(c);
    for (int C = 1; C <= 16; ++C) {
        if (force_c > 0 && C != force_c) continue;
        if (force_c <= 0 && C > 1 && (C & (C - 1)) != 0 && C != 6 && C != 12) continue;   // heuristic set
        if (C > ny_max) continue;
        // biquadratic stencils reach two rows into the next strip: every CTA needs two rows
        if (c->interp == 2 && !c->d_kexpl && !jk && min_ny(c) / C < 2) continue;
        int ring_plane, ipts_max;
        launch_caps<Real, NS>(c, C, ring_plane, ipts_max, jk);
        int fmax = 0;
        if (jk) {
            // J^K_Q kernel: besides the Stokes planes, each frequency of a pass keeps
            // the nodes' coefficients of three planes (jsweep_smem_bytes)
            for (int f = NU; f >= 1 && fmax == 0; --f)
                if (jsweep_smem_bytes<Real, NS>(ring_plane, ipts_max, f, kThreads) <= kSmemLimit) fmax = f;
            if (fmax == 0) continue;
        } else {
            const long long ring = 3LL * ring_plane * 16;
            const long long per_nu = 2LL * ipts_max * NS * (long long)sizeof(Real);
            const long long scratch = (long long)kThreads * NA * (long long)sizeof(Real);
            if (ring + per_nu + scratch > kSmemLimit) continue;
            fmax = (int)std::min<long long>(NU, (kSmemLimit - ring - scratch) / per_nu);
        }
        if (force_f > 0) {
            if (force_f > fmax) continue;
            fmax = force_f;
        }
        const int G = (NU + fmax - 1) / fmax;
        const int F = (NU + G - 1) / G;
        // threads: the strip's points times the frequency lanes they can use, whole warps, 64..512
        const int threads = std::min(kThreads, std::max(64, (ipts_max * F + 31) / 32 * 32));
        const int smem = jk ? jsweep_smem_bytes<Real, NS>(ring_plane, ipts_max, F, threads)
                            : sweep_smem_bytes<Real, NS>(ring_plane, ipts_max, F, threads, NA);
        if (smem > kSmemLimit + 16) continue;
        int act = 0;
        if ((jk ? jsweep_max_active_clusters<Real, NS>(C, smem, threads, &act)
                : max_active_clusters<Real, NS>(C, smem, threads, &act, c->d_dich != nullptr,
                                                c->interp == 2 && !c->d_kexpl, c->d_kexpl != nullptr)) !=
            cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (act < 1) continue;
        const int ncl = std::min(act, nitems);
        double total = 0.0, item_max = 0.0;
        for (const BoxDev &b : c->boxes) {
            const int rmax = (b.ny + C - 1) / C;
            const double pts = (double)rmax * b.nx;
            const double slots = std::ceil(pts * F / threads) * kThreads;   // per-SM issue slots per pass
            const double item = b.nz * G * (slots + 0.15 * (rmax + 2) * b.nx + 0.05 * pts + 300.0);
            total += item * c->nray;
            item_max = std::max(item_max, item);
        }
        const double cost = c->nbox == 1 ? std::ceil((double)nitems / ncl) * item_max
                                         : std::max(total / ncl, item_max) * 1.05;
        if (cost < best_cost) {
            best_cost = cost;
            best.cluster = C;
            best.F = F;
            best.threads = threads;
            best.smem = smem;
            best.clusters = ncl;
        }
    }
    return best.cluster > 0 ? PORTA_OK : PORTA_EINVAL;
}

// sweep arguments common to every mode: sizes, atmosphere, unknowns, frequencies
template <typename Real>
SweepArgs<Real> base_args(porta_ctx *c)
{
    SweepArgs<Real> a{};
    a.nnu = c->n_nu;
    a.nray = c->nray;
    a.nvox = c->nvox;
    a.boxes = (const BoxDev *)c->d_boxes;
    a.bfac = (Real)(2.0 * c->gbar * c->zeta);
    const Real *atm = (const Real *)c->d_atm;
    a.chi = atm;
    a.vel = atm + c->nvox;
    a.bx = atm + 2 * c->nvox;
    a.by = atm + 3 * c->nvox;
    a.bz = atm + 4 * c->nvox;
    a.bpl = atm + 5 * c->nvox;
    a.rho = (const Real *)c->d_rhoR;
    a.dich = (const Real *)c->d_dich;
    a.xf = (const Real *)c->d_freq;
    a.wf = (const Real *)c->d_freq + c->n_nu;
    a.probe_ray = -1;
    a.interp = c->interp;
    a.kexpl = c->d_kexpl;
    a.sexpl = c->d_sexpl;
    return a;
}

// fill the launch-dependent fields of the arguments
template <typename Real>
void shape_args(porta_ctx *c, SweepArgs<Real> &a, const LaunchCfg &cfg, bool jk = false)
{
    a.F = cfg.F;
    a.ngroups = (a.nnu + cfg.F - 1) / cfg.F;
    if (c->ns == 1)
        launch_caps<Real, 1>(c, cfg.cluster, a.ring_plane, a.ipts_max, jk);
    else
        launch_caps<Real, 4>(c, cfg.cluster, a.ring_plane, a.ipts_max, jk);
    a.cstride = jsweep_stride(a.ring_plane * (c->ns == 1 ? 1 : 2), (int)sizeof(Real));
    a.istride = jsweep_stride(a.ipts_max * c->ns, (int)sizeof(Real));
}

// api.cu
void free_all(porta_ctx *c);
bool finite_host(const double *x, long long n);
// copy n doubles from a caller buffer (host or device) into device memory
int copy_in(porta_ctx *c, double *dst, const double *src, long long n, int where);
// number of entries of a device array outside (lo, hi] (NaN counts)
int count_bad(porta_ctx *c, const double *d, long long n, double lo, double hi, unsigned long long *out);
int create_impl(int nbox, const porta_grid *grids, const porta_atom *at, const porta_quad *q, const porta_opts *o,
                porta_ctx **out);

// api_adjoint.cu: emergent Stokes profiles of ndir directions (device pointers)
template <typename Real>
int emergent_t(porta_ctx *c, int ndir, const double *mu, const double *chi, double *dout, int box = 0);
// releases the checkpoints of porta_iterate_ckpt
void it_free(porta_ctx *c);

// api_mg.cu: releases the coarse levels
void mg_free(porta_ctx *c);
// re-derives the sweep's copy of the unknowns after they changed on the device
cudaError_t mg_rho_changed(porta_ctx *L);

// api_ml.cu: line data of every line from the populations
cudaError_t ml_prepare(porta_ctx *c);
// the error counter of the line data and of the rate equations (synchronizes)
int ml_check(porta_ctx *c, const char *what);

}  // namespace porta_api
