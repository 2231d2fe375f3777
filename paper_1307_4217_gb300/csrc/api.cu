// C ABI of the formal-solver library (include/porta.h): argument checks,
// quadratures and per-ray plane geometry (host, FP64), device buffers, the
// launch sequence formal_solve -> accumulate_jkq -> see_update, the captured
// Jacobi iteration and the frequency bands of a formal solution.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "api_internal.h"
#include "mg_kernels.cuh"
#include "ml_kernels.cuh"
#include "faces_kernels.cuh"
#include "mlpol_kernels.cuh"
#include "see_kernels.cuh"

using namespace porta;

namespace porta_api {

const char *kNullCtx = "null context";

int fail(porta_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}


// Device allocations of the library go through pmalloc / pfree, which keep the
// live byte count and honour the process-wide cap of porta_set_device_limit: an
// allocation that would exceed the cap fails with cudaErrorMemoryAllocation
// (reported as PORTA_ENOMEM) without calling the CUDA runtime.
std::mutex g_alloc_mutex;
std::unordered_map<void *, size_t> g_alloc_sizes;
size_t g_alloc_live = 0, g_alloc_limit = 0;

cudaError_t pmalloc_bytes(void **p, size_t bytes)
{
    *p = nullptr;
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    if (g_alloc_limit > 0 && g_alloc_live + bytes > g_alloc_limit) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return e;
    g_alloc_sizes[*p] = bytes;
    g_alloc_live += bytes;
    return cudaSuccess;
}


cudaError_t pfree(void *p)
{
    if (!p) return cudaSuccess;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mutex);
        auto it = g_alloc_sizes.find(p);
        if (it != g_alloc_sizes.end()) {
            g_alloc_live -= it->second;
            g_alloc_sizes.erase(it);
        }
    }
    return cudaFree(p);
}

// Gauss-Legendre nodes/weights on (0, 1): Newton's method on the Legendre
// polynomial P_n evaluated by its three-term recurrence; x and w receive n values
// in increasing order of x
void gauss_legendre(int n, double *x, double *w)
{
    auto legendre = [n](double t, double &p, double &pm1) {
        pm1 = 1.0;
        p = t;
        for (int k = 1; k < n; ++k) {
            double pn = ((2 * k + 1) * t * p - k * pm1) / (k + 1);
            pm1 = p;
            p = pn;
        }
        if (n == 1) {
            p = t;
            pm1 = 1.0;
        }
    };
    for (int i = 0; i < n; ++i) {
        double t = std::cos(M_PI * (4.0 * i + 3.0) / (4.0 * n + 2.0));
        double p, pm1;
        for (int it = 0; it < 100; ++it) {
            legendre(t, p, pm1);
            double dt = p / (n * (pm1 - t * p) / (1.0 - t * t));
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        legendre(t, p, pm1);   // P'_n at the final node
        const double dp = n * (pm1 - t * p) / (1.0 - t * t);
        x[n - 1 - i] = 0.5 * (t + 1.0);
        w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dp * dp);   // (2/((1-t^2) P'^2)) / 2
    }
}

// T^K_Q(i, Omega) for i = I, Q, U from the polarization tensors of the ray
// frame: with e_a = dOmega/dtheta and e_b = z x Omega / |z x Omega|, Stokes
// I, Q, U correspond to e_a e_a + e_b e_b, e_a e_a - e_b e_b, e_a e_b + e_b e_a;
// T^0_0 is half the trace and T^2_Q = -sqrt(3)/2 times the spherical
// components of the traceless part (A_0 = sqrt(3/2) A_zz, A_1 = -(A_xz + i A_yz),
// A_2 = (A_xx - A_yy + 2 i A_xy)/2). Output rows of 6 reals per Stokes parameter.
void tkq_tensors(double mu, double chi, double out[18])
{
    double st = std::sqrt(std::max(0.0, 1.0 - mu * mu));
    double ea[3] = {mu * std::cos(chi), mu * std::sin(chi), -st};
    double eb[3] = {-std::sin(chi), std::cos(chi), 0.0};
    for (int i = 0; i < 3; ++i) {
        double t[3][3];
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) {
                double aa = ea[r] * ea[s], bb = eb[r] * eb[s], ab = ea[r] * eb[s] + eb[r] * ea[s];
                t[r][s] = i == 0 ? aa + bb : (i == 1 ? aa - bb : ab);
            }
        double tr = t[0][0] + t[1][1] + t[2][2];
        double A[3][3];
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) A[r][s] = t[r][s] - (r == s ? tr / 3.0 : 0.0);
        const double k = -std::sqrt(3.0) / 2.0;
        out[6 * i + 0] = tr / 2.0;
        out[6 * i + 1] = k * std::sqrt(1.5) * A[2][2];
        out[6 * i + 2] = k * (-A[0][2]);
        out[6 * i + 3] = k * (-A[1][2]);
        out[6 * i + 4] = k * 0.5 * (A[0][0] - A[1][1]);
        out[6 * i + 5] = k * A[0][1];
    }
}

void drop_graph(porta_ctx *c)
{
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    c->graph_stream = nullptr;
}

int ns_of(int model) { return model == PORTA_MODEL_TWOLEVEL_UNPOL ? 1 : 4; }
int nl_of(int model) { return model == PORTA_MODEL_TWOLEVEL_UNPOL ? 1 : 6; }

// The J^K_Q formal solution runs the kernel of sweep_j.cu (per-frequency
// node coefficients in shared memory) unless the lines carry dichroism, which
// only the general sweep (sweep.cu) implements, or a plane is too wide for its
// shared memory (then the general sweep, which needs less per frequency, runs).
// (and the biquadratic stencils, which only the general sweep has)
bool use_jk(const porta_ctx *c)
{
    return c->d_dich == nullptr && c->d_kexpl == nullptr && c->jk_fits && c->interp != 2 && !c->sc_faces && !c->gsweep;
}

// The J^K_Q sweep sums an FP32 formal solution into fixed-point accumulators;
// an FP64 one keeps per-ray partial integrals summed in ray order in FP64 (a
// fixed-point scale cannot hold 1e-10 relative precision for quantities that
// span many decades within one voxel, as Lambda-bar* does with optical depth).
bool jfixed(const porta_ctx *c) { return use_jk(c) && c->precision == PORTA_FP32; }

// frequencies of the J^K_Q formal solution (its band, porta_set_freq_range)
int jnu(const porta_ctx *c) { return c->fr1 > c->fr0 ? c->fr1 - c->fr0 : c->n_nu; }

int min_ny(const porta_ctx *c)
{
    int m = 1 << 30;
    for (const BoxDev &b : c->boxes) m = std::min(m, b.ny);
    return m;
}

int max_ny(const porta_ctx *c)
{
    int m = 0;
    for (const BoxDev &b : c->boxes) m = std::max(m, b.ny);
    return m;
}

// all launch shapes that fit, with their resident-cluster counts
template <typename Real, int NS>
std::vector<LaunchCfg> candidates(porta_ctx *c, int nitems)
{
    // every cluster size 1..16 (cluster shapes that are not powers of two can
    // tile the GPU's SM groups better); the three largest frequency passes that fit
    std::vector<LaunchCfg> out;
    const int ny_max = max_ny(c);
    for (int C = 1; C <= 16; ++C) {
        if (C > ny_max) continue;
        int last_f = -1, kept = 0;
        for (int G = 1; G <= jnu(c) && kept < 3; ++G) {
            int F = (jnu(c) + G - 1) / G;
            if (F == last_f) continue;
            last_f = F;
            LaunchCfg cfg{};
            if (choose_launch<Real, NS>(c, cfg, C, F, nitems, use_jk(c), jnu(c)) == PORTA_OK && cfg.F == F) {
                out.push_back(cfg);
                ++kept;
            }
        }
    }
    return out;
}

// one J-mode sweep launch with the kernel use_jk selects
template <typename Real>
cudaError_t launch_j(porta_ctx *c, const SweepArgs<Real> &a, LaunchCfg &cfg, cudaStream_t st)
{
    if (use_jk(c))
        return c->ns == 1 ? launch_jsweep<Real, 1>(a, cfg, st) : launch_jsweep<Real, 4>(a, cfg, st);
    return c->ns == 1 ? launch_sweep<Real, 1>(a, MODE_JKQ, cfg, st) : launch_sweep<Real, 4>(a, MODE_JKQ, cfg, st);
}

template <typename Real>
SweepArgs<Real> jkq_args(porta_ctx *c)
{
    SweepArgs<Real> a = base_args<Real>(c);
    if (c->fr1 > c->fr0) {
        // a frequency band: its nodes and weights (the profile normalization stays
        // the one of the whole frequency grid, so the bands' sums add up to J^K_Q)
        a.xf += c->fr0;
        a.wf += c->fr0;
        a.nnu = c->fr1 - c->fr0;
    }
    a.geom = (const PlaneGeom<Real> *)c->d_geom;
    a.rays = (const RayDev<Real> *)c->d_rays;
    a.invn = (const Real *)c->d_invn;
    a.part = jfixed(c) ? nullptr : c->d_part;
    a.partv = (Real *)c->d_partv;
    a.jacc = jfixed(c) ? c->d_jacc : nullptr;
    a.jexp = c->d_jexp;
    a.jerr = c->d_err;
    a.tw = c->d_tw;
    a.items = c->d_items;
    a.nitems = c->nbox * c->nray;
    return a;
}

// the largest plane of the boxes, and (dx, dy) per box, for the face sweep
long long faces_nxy_max(const porta_ctx *c)
{
    long long n = 0;
    for (const BoxDev &b : c->boxes) n = std::max(n, (long long)b.nx * b.ny);
    return n;
}

std::vector<double> faces_cell_sizes(const porta_ctx *c)
{
    std::vector<double> d(2 * c->boxes.size());
    for (size_t b = 0; b < c->boxes.size(); ++b) {
        d[2 * b] = c->blx[b] / c->boxes[b].nx;
        d[2 * b + 1] = c->bly[b] / c->boxes[b].ny;
    }
    return d;
}

// Device buffers of the J^K_Q formal solution, allocated on first use (before
// any graph capture): the fixed-point sums of the J^K_Q sweep, or the per-ray
// partial integrals of the general sweep.
// whether a shared-memory sweep has some launch shape for this context's planes
static bool smem_sweep_fits(porta_ctx *c)
{
    LaunchCfg cfg{};
    const int n = c->nbox * c->nray;
    int rc;
    if (c->precision == PORTA_FP32)
        rc = c->ns == 1 ? choose_launch<float, 1>(c, cfg, 0, 0, n, use_jk(c), jnu(c))
                        : choose_launch<float, 4>(c, cfg, 0, 0, n, use_jk(c), jnu(c));
    else
        rc = c->ns == 1 ? choose_launch<double, 1>(c, cfg, 0, 0, n, use_jk(c), jnu(c))
                        : choose_launch<double, 4>(c, cfg, 0, 0, n, use_jk(c), jnu(c));
    return rc == 0;
}

// planes too wide for the shared-memory ring: the global-memory sweep (decided on
// the first formal solution's buffers, before any graph capture)
void check_global_sweep(porta_ctx *c)
{
    if (c->gsweep_checked) return;
    c->gsweep_checked = true;
    if (!c->sc_faces && !c->gsweep && c->d_kexpl == nullptr && c->interp != 2 && !smem_sweep_fits(c)) c->gsweep = 2;
}

cudaError_t ensure_sweep_buffers(porta_ctx *c)
{
    check_global_sweep(c);
    if (jfixed(c)) {
        cudaError_t e = cudaSuccess;
        if (!c->d_jacc) e = pmalloc(&c->d_jacc, (size_t)(c->nj + 1) * c->nvox * sizeof(unsigned long long));
        if (e == cudaSuccess && !c->d_jexp) e = pmalloc(&c->d_jexp, (size_t)c->nvox * sizeof(int));
        return e;
    }
    cudaError_t e = cudaSuccess;
    if (!c->d_part) e = pmalloc(&c->d_part, (size_t)c->nray * c->nvox * (c->ns == 1 ? 2 : 4) * c->rsz);
    // polarized lines of a multilevel atom: the per-ray integrals of Stokes V (J^1_Q)
    if (e == cudaSuccess && c->d_dich && !c->d_partv) e = pmalloc(&c->d_partv, (size_t)c->nray * c->nvox * c->rsz);
    // short characteristics on cell faces: the work planes and per-group partials
    if (e == cudaSuccess && (c->sc_faces || c->gsweep || c->d_kexpl)) {
        const long long nxy = faces_nxy_max(c);
        const size_t need =
            c->precision == PORTA_FP32
                ? (c->ns == 1 ? faces_scratch_bytes<float, 1>(c->nbox, c->nray, jnu(c), nxy, c->nvox, c->d_dich ? 1 : (c->d_kexpl ? 2 : 0))
                              : faces_scratch_bytes<float, 4>(c->nbox, c->nray, jnu(c), nxy, c->nvox, c->d_dich ? 1 : (c->d_kexpl ? 2 : 0)))
                : (c->ns == 1 ? faces_scratch_bytes<double, 1>(c->nbox, c->nray, jnu(c), nxy, c->nvox, c->d_dich ? 1 : (c->d_kexpl ? 2 : 0))
                              : faces_scratch_bytes<double, 4>(c->nbox, c->nray, jnu(c), nxy, c->nvox, c->d_dich ? 1 : (c->d_kexpl ? 2 : 0)));
        if (!c->d_fdxy) {
            const std::vector<double> dxy = faces_cell_sizes(c);
            e = pmalloc(&c->d_fdxy, dxy.size() * sizeof(double));
            if (e == cudaSuccess) e = cudaMemcpy(c->d_fdxy, dxy.data(), dxy.size() * sizeof(double), cudaMemcpyHostToDevice);
        }
        if (c->faces_bytes < need) {
            if (c->d_faces) pfree(c->d_faces);
            c->d_faces = nullptr;
            c->faces_bytes = 0;
            e = pmalloc(&c->d_faces, need);
            if (e == cudaSuccess) c->faces_bytes = need;
        }
    }
    return e;
}

// zero the fixed-point sums and set the voxels' scales before a J^K_Q sweep
template <typename Real>
cudaError_t jacc_prepare(porta_ctx *c, const SweepArgs<Real> &a)
{
    if (!jfixed(c)) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    return c->ns == 1 ? launch_jacc_prepare<Real, 1>(a, c->stream) : launch_jacc_prepare<Real, 4>(a, c->stream);
}

// J^K_Q and Lambda-bar* (FP64) from the sums of the last formal solution; for the
// polarized lines of a multilevel atom also J^1_Q (d_j1)
cudaError_t finalize_jkq(porta_ctx *c)
{
    if (c->d_j1) {
        cudaError_t e = c->precision == PORTA_FP32
                            ? run_j1_finalize<float>(c->nvox, c->nray, c->d_partv, c->d_tw1, c->d_j1, c->stream)
                            : run_j1_finalize<double>(c->nvox, c->nray, c->d_partv, c->d_tw1, c->d_j1, c->stream);
        if (e != cudaSuccess) return e;
    }
    if (jfixed(c))
        return c->ns == 1 ? launch_jacc_finalize<1>(c->nvox, c->d_jacc, c->d_jexp, c->d_jkq, c->d_lstar, c->stream)
                          : launch_jacc_finalize<4>(c->nvox, c->d_jacc, c->d_jexp, c->d_jkq, c->d_lstar, c->stream);
    if (c->precision == PORTA_FP32)
        return c->ns == 1 ? run_jkq_finalize<float, 1>(c->nvox, c->nray, c->d_part, c->d_tw, c->d_jkq, c->d_lstar, c->stream)
                          : run_jkq_finalize<float, 4>(c->nvox, c->nray, c->d_part, c->d_tw, c->d_jkq, c->d_lstar, c->stream);
    return c->ns == 1 ? run_jkq_finalize<double, 1>(c->nvox, c->nray, c->d_part, c->d_tw, c->d_jkq, c->d_lstar, c->stream)
                      : run_jkq_finalize<double, 4>(c->nvox, c->nray, c->d_part, c->d_tw, c->d_jkq, c->d_lstar, c->stream);
}

// the fixed-point sums' overflow flag (reads device memory: synchronizes the stream)
int check_jacc(porta_ctx *c)
{
    if (!jfixed(c) && !c->sc_faces && !c->gsweep && !c->d_kexpl) return PORTA_OK;
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (flag & 2) return fail(c, PORTA_ENOTCONV, "formal solution: a plane of face points did not converge");
    if (flag) return fail(c, PORTA_EKERNEL, "formal solution: a J^K_Q term exceeded the fixed-point range (2^16 times "
                                            "max(|S^0_0|, |B|) of its voxel), or was not finite");
    return PORTA_OK;
}

cudaError_t ensure_fill(porta_ctx *c)
{
    if (c->fill) return cudaSuccess;
    LaunchFill *f = new (std::nothrow) LaunchFill;
    if (!f) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = pmalloc((void **)&f->d_ctr, 2 * sizeof(int));
    c->fill = f;   // released by free_all also on failure
    return e;
}

// J-mode sweep over the work items [items, items + nitems): one launch of the
// main shape, or, with a filler configured, the main launch over the first
// (costliest) items and a concurrent launch of the filler shape over the last
// fraction, each taking its items dynamically from its own counter (every item
// is computed by one fixed shape, so results do not depend on scheduling)
template <typename Real>
cudaError_t sweep_jkq(porta_ctx *c, SweepArgs<Real> a, LaunchCfg cfg, const int *items, int nitems, bool allow_fill)
{
    a.items = items;
    a.nitems = nitems;
    const int nB = (int)std::lround(c->fill_frac * nitems);
    if (!allow_fill || c->fill_cfg.cluster <= 0 || nB < 1 || nB >= nitems) return launch_j<Real>(c, a, cfg, c->stream);
    cudaError_t e = ensure_fill(c);
    if (e != cudaSuccess) return e;
    const int nA = nitems - nB;
    SweepArgs<Real> b = a;
    LaunchCfg fc = c->fill_cfg;
    shape_args<Real>(c, b, fc, use_jk(c));
    b.items = items + nA;
    b.nitems = nB;
    b.next_item = c->fill->d_ctr + 1;
    fc.clusters = std::min(fc.clusters, nB);
    a.nitems = nA;
    a.next_item = c->fill->d_ctr;
    cfg.clusters = std::min(cfg.clusters, nA);
    // the main launch's clusters are placed first; the filler takes what is left
    int least = 0, greatest = 0;
    e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e != cudaSuccess) return e;
    cfg.priority = greatest;
    fc.priority = least;
    e = cudaMemsetAsync(c->fill->d_ctr, 0, 2 * sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->fill->fork, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->fill->stream, c->fill->fork, 0);
    if (e == cudaSuccess) e = launch_j<Real>(c, a, cfg, c->stream);
    if (e == cudaSuccess) e = launch_j<Real>(c, b, fc, c->fill->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->fill->join, c->fill->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->fill->join, 0);
    return e;
}

// the formal solution with short characteristics on the first cell face crossed,
// or (planes) the plane placement by the same global-memory sweep
template <typename Real>
int faces_solve_t(porta_ctx *c, bool planes)
{
    cudaError_t e = ensure_sweep_buffers(c);   // (with the face work planes)
    const long long nxy = faces_nxy_max(c);
    if (e != cudaSuccess) return fail(c, PORTA_ENOMEM, std::string("formal solution buffers: ") + cudaGetErrorString(e));
    SweepArgs<Real> a = jkq_args<Real>(c);
    a.part = c->d_part;
    e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    const double *dxy = (const double *)c->d_fdxy;
    if (e == cudaSuccess)
        e = c->ns == 1 ? launch_faces<Real, 1>(a, (Real *)c->d_faces, c->nbox, nxy, dxy, 100000, c->d_err, c->stream,
                                               false, planes)
                       : launch_faces<Real, 4>(a, (Real *)c->d_faces, c->nbox, nxy, dxy, 100000, c->d_err, c->stream,
                                               false, planes);
    if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("face sweep: ") + cudaGetErrorString(e));
    return PORTA_OK;
}

template <typename Real>
int formal_solve_t(porta_ctx *c, int probe_ray, Real *probe, Real *probe_ls)
{
    if (c->d_kexpl) {
        // an explicit medium: the seven-element step of the global-memory sweep
        if (probe_ray >= 0) return fail(c, PORTA_EINVAL, "probe ray: not with an explicit medium");
        return faces_solve_t<Real>(c, true);
    }
    if (c->sc_faces || c->gsweep) {
        if (probe_ray >= 0) return fail(c, PORTA_EINVAL, "probe ray: not with the global-memory sweep");
        return faces_solve_t<Real>(c, !c->sc_faces);
    }
    SweepArgs<Real> a = jkq_args<Real>(c);
    a.probe_ray = probe_ray;
    a.probe = probe;
    a.probe_ls = probe_ls;
    LaunchCfg cfg{};
    int rc = c->ns == 1 ? choose_launch<Real, 1>(c, cfg, c->opt_cluster, c->opt_nu_group, a.nitems, use_jk(c), jnu(c))
                        : choose_launch<Real, 4>(c, cfg, c->opt_cluster, c->opt_nu_group, a.nitems, use_jk(c), jnu(c));
    if (rc) {
        // planes too wide for the shared-memory ring: the global-memory sweep (a
        // forced shape that does not fit is an error)
        if (probe_ray >= 0 || smem_sweep_fits(c))
            return fail(c, rc, "no sweep launch shape fits this grid (shared memory / cluster limits)");
        c->gsweep = 2;
        c->gsweep_checked = true;
        return faces_solve_t<Real>(c, true);
    }
    shape_args<Real>(c, a, cfg, use_jk(c));
    cudaError_t e = ensure_sweep_buffers(c);
    if (e != cudaSuccess) return fail(c, PORTA_ENOMEM, std::string("formal solution buffers: ") + cudaGetErrorString(e));
    a.part = jfixed(c) ? nullptr : c->d_part;
    a.partv = (Real *)c->d_partv;
    a.jacc = jfixed(c) ? c->d_jacc : nullptr;
    a.jexp = c->d_jexp;
    e = jacc_prepare<Real>(c, a);
    if (e == cudaSuccess) e = sweep_jkq<Real>(c, a, cfg, a.items, a.nitems, probe_ray < 0);
    if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("sweep launch: ") + cudaGetErrorString(e));
    c->last = cfg;
    return PORTA_OK;
}

template <typename Real>
int autotune_t(porta_ctx *c)
{
    const int nitems = c->nbox * c->nray;
    std::vector<LaunchCfg> cand = c->ns == 1 ? candidates<Real, 1>(c, nitems) : candidates<Real, 4>(c, nitems);
    if (cand.empty()) return fail(c, PORTA_EINVAL, "autotune: no launch shape fits");
    {
        // the timing launches write the formal solution's buffers (their sums are
        // discarded: every formal solution starts from zero)
        cudaError_t eb = ensure_sweep_buffers(c);
        if (eb == cudaSuccess) eb = jacc_prepare<Real>(c, jkq_args<Real>(c));
        if (eb != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("autotune: ") + cudaGetErrorString(eb));
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = 1e300;
    LaunchCfg pick = cand[0];
    int rc = PORTA_OK;
    std::vector<double> est_of(cand.size(), 1e300);
    for (size_t ci = 0; ci < cand.size(); ++ci) {
        const LaunchCfg &cfg0 = cand[ci];
        LaunchCfg cfg = cfg0;
        SweepArgs<Real> a = jkq_args<Real>(c);
        shape_args<Real>(c, a, cfg, use_jk(c));
        // one box: time one wave (every resident cluster sweeps one ray);
        // batches: time a strided sample of the (box, ray) items
        if (c->nbox == 1) {
            a.nitems = cfg.clusters;
        } else {
            a.items = c->d_tune_items;
            a.nitems = c->n_tune;
        }
        float ms = 1e30f;
        for (int rep = 0; rep < 2 && rc == PORTA_OK; ++rep) {
            cudaError_t e = cudaEventRecord(e0, c->stream);
            if (e == cudaSuccess) e = launch_j<Real>(c, a, cfg, c->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
            ms = std::min(ms, t);
        }
        if (rc != PORTA_OK) break;
        double waves = c->nbox == 1 ? std::ceil((double)c->nray / cfg.clusters)
                                    : (double)c->nbox * c->nray / c->n_tune;
        double est = ms * waves;
        est_of[ci] = est;
        if (est < best) {
            best = est;
            pick = cfg;
        }
    }
    c->fill_cfg = LaunchCfg{};
    c->fill_frac = 0.0;
    if (rc == PORTA_OK) {
        c->opt_cluster = pick.cluster;
        c->opt_nu_group = pick.F;
        // Concurrent filler: smaller clusters over the cheapest fraction of the
        // work list, on the SMs the main shape's clusters leave idle. Timed on the
        // whole work list (one box) or the strided sample (batches) for every
        // smaller cluster size up to 8 (its best F) x split fractions.
        const int *titems = c->nbox == 1 ? c->d_items : c->d_tune_items;
        const int tn = c->nbox == 1 ? nitems : c->n_tune;
        auto time_split = [&](float &ms) {
            SweepArgs<Real> a = jkq_args<Real>(c);
            LaunchCfg cfg = pick;
            shape_args<Real>(c, a, cfg, use_jk(c));
            ms = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {
                cudaError_t e = cudaEventRecord(e0, c->stream);
                if (e == cudaSuccess) e = sweep_jkq<Real>(c, a, cfg, titems, tn, true);
                if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float t = 0;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
                if (e != cudaSuccess) return e;
                ms = std::min(ms, t);
            }
            return cudaSuccess;
        };
        std::vector<std::pair<double, LaunchCfg>> small;
        for (int C = 1; C < std::min(pick.cluster, 9); ++C) {
            double b = 1e300;
            LaunchCfg k{};
            for (size_t ci = 0; ci < cand.size(); ++ci)
                if (cand[ci].cluster == C && est_of[ci] < b) {
                    b = est_of[ci];
                    k = cand[ci];
                }
            if (k.cluster > 0) small.push_back({b, k});
        }

        float base = 0;
        cudaError_t e = tn >= 8 && !small.empty() ? ensure_fill(c) : cudaSuccess;
        if (e == cudaSuccess && tn >= 8 && !small.empty()) e = time_split(base);
        float best_split = base;
        LaunchCfg best_fill{};
        double best_frac = 0.0;
        // split points: one box -> the main launch keeps a whole number of rounds
        // of its resident clusters (rays cost the same); batches -> fractions
        std::vector<double> fracs;
        if (c->nbox == 1) {
            const int rounds = (tn + pick.clusters - 1) / pick.clusters;
            for (int r = rounds - 1; r >= std::max(1, rounds - 6); --r) {
                const int nB = tn - r * pick.clusters;
                if (nB > 0 && nB < tn) fracs.push_back((double)nB / tn);
            }
        } else {
            fracs = {0.05, 0.1, 0.15, 0.2, 0.25, 0.3};
        }
        for (const auto &sk : small) {
            if (e != cudaSuccess || tn < 8) break;
            for (double frac : fracs) {
                c->fill_cfg = sk.second;
                c->fill_frac = frac;
                float t = 0;
                e = time_split(t);
                if (e != cudaSuccess) break;
                if (t < best_split) {
                    best_split = t;
                    best_fill = sk.second;
                    best_frac = frac;
                }
            }
        }
        if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, std::string("autotune (filler): ") + cudaGetErrorString(e));
        // keep a filler only if it beats the single launch by more than the timing noise
        const bool keep = rc == PORTA_OK && best_fill.cluster > 0 && best_split < 0.98f * base;
        c->fill_cfg = keep ? best_fill : LaunchCfg{};
        c->fill_frac = keep ? best_frac : 0.0;
        c->have_fs = c->have_jkq = false;
        drop_graph(c);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

void free_all(porta_ctx *c)
{
    drop_graph(c);
    mg_free(c);
    it_free(c);
    if (c->d_dich) pfree(c->d_dich);
    if (c->ml) {
        pfree(c->ml->d_x);
        pfree(c->ml->d_tab);
        pfree(c->ml->d_pops);
        pfree(c->ml->d_chis);
        pfree(c->ml->d_kT);
        pfree(c->ml->d_bad);
        delete c->ml;
        c->ml = nullptr;
    }
    if (c->d_gacc) pfree(c->d_gacc);
    for (cudaEvent_t &ev : c->it_ev)
        if (ev) cudaEventDestroy(ev);
    if (c->d_cv64) pfree(c->d_cv64);
    if (c->fill) {
        if (c->fill->stream) cudaStreamDestroy(c->fill->stream);
        if (c->fill->fork) cudaEventDestroy(c->fill->fork);
        if (c->fill->join) cudaEventDestroy(c->fill->join);
        if (c->fill->d_ctr) pfree(c->fill->d_ctr);
        delete c->fill;
        c->fill = nullptr;
    }
    for (cudaEvent_t &ev : c->adj_ev)
        if (ev) cudaEventDestroy(ev);
    void *ptrs[] = {c->d_atm, c->d_eps, c->d_bpl, c->d_b, c->d_rho, c->d_rhoR, c->d_invn, c->d_geom, c->d_rays,
                    c->d_freq, c->d_part, c->d_tw, c->d_jkq, c->d_lstar, c->d_resid, c->d_err, c->d_boxes,
                    c->d_items, c->d_tune_items, c->d_tape, c->d_gpart, c->d_jacc, c->d_jexp, c->d_kexpl, c->d_sexpl,
                    c->d_partv, c->d_j1, c->d_tw1, c->d_gjR, c->d_vjp_out, c->d_faces, c->d_fdxy};
    for (void *p : ptrs)
        if (p) pfree(p);
}

bool finite_host(const double *x, long long n)
{
    for (long long i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

// copy n doubles from a caller buffer (host or device) into device memory
int copy_in(porta_ctx *c, double *dst, const double *src, long long n, int where)
{
    cudaError_t e = cudaMemcpyAsync(dst, src, n * sizeof(double),
                                    where == PORTA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("copy in: ") + cudaGetErrorString(e));
    return PORTA_OK;
}

// number of entries of a device array outside (lo, hi] (NaN counts)
int count_bad(porta_ctx *c, const double *d, long long n, double lo, double hi, unsigned long long *out)
{
    CK(cudaMemsetAsync(c->d_resid, 0, sizeof(unsigned long long), c->stream));
    CK(run_count_bad(n, d, lo, hi, c->d_resid, c->stream));
    CK(cudaMemcpyAsync(out, c->d_resid, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PORTA_OK;
}

// the update step of a Jacobi iteration, enqueued on the context's stream
// (capturable): residual reset, then the two-level SEE update, or for the
// multilevel atom the rate equations and the next iteration's line data
cudaError_t enqueue_update(porta_ctx *c)
{
    cudaError_t e = cudaMemsetAsync(c->d_resid, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
    if (!c->ml)
        return c->precision == PORTA_FP32
                   ? run_see<float>(c->nvox, c->nl, c->model, c->bcrit, c->d_eps, c->d_bpl, c->d_b, c->d_jkq,
                                    c->d_lstar, c->d_rho, c->d_rhoR, c->d_resid, c->stream)
                   : run_see<double>(c->nvox, c->nl, c->model, c->bcrit, c->d_eps, c->d_bpl, c->d_b, c->d_jkq,
                                     c->d_lstar, c->d_rho, c->d_rhoR, c->d_resid, c->stream);
    MlState *m = c->ml;
    if (m->pol)
        e = run_mlpol_see(m->mc, m->dev, m->nvox1, m->d_kT, c->d_jkq, c->d_j1, c->d_lstar, c->d_b, m->d_x, c->d_resid,
                          m->d_bad, c->stream);
    else
        e = run_ml_see(m->mc, m->nvox1, m->d_kT, c->d_jkq, c->d_lstar, m->d_pops, c->d_resid, m->d_bad, c->stream);
    if (e != cudaSuccess) return e;
    return ml_prepare(c);
}


int create_impl(int nbox, const porta_grid *grids, const porta_atom *at, const porta_quad *q,
                const porta_opts *o, porta_ctx **out)
{
    if (!out) return PORTA_EINVAL;
    *out = nullptr;
    if (nbox < 1 || !grids || !at || !q) return PORTA_EINVAL;
    long long nvox = 0, nplane = 0;
    for (int b = 0; b < nbox; ++b) {
        const porta_grid *gb = &grids[b];
        if (!gb->z || gb->nx < 1 || gb->ny < 1 || gb->nz < 2 || !(gb->lx > 0) || !(gb->ly > 0)) return PORTA_EINVAL;
        for (int k = 0; k < gb->nz; ++k)
            if (!std::isfinite(gb->z[k]) || (k > 0 && !(gb->z[k] > gb->z[k - 1]))) return PORTA_EINVAL;
        nvox += (long long)gb->nx * gb->ny * gb->nz;
        nplane += gb->nz;
    }
    const porta_grid *g = &grids[0];
    if (q->n_mu < 1 || q->n_chi < 1 || q->n_nu < 1 || !(q->x_max > 0) || !std::isfinite(q->x_max)) return PORTA_EINVAL;
    if (at->model != PORTA_MODEL_TWOLEVEL_UNPOL && at->model != PORTA_MODEL_TWOLEVEL_HANLE) return PORTA_EINVAL;
    if (at->model == PORTA_MODEL_TWOLEVEL_HANLE && !(at->bcrit > 0)) return PORTA_EINVAL;
    int prec = o ? o->precision : PORTA_FP32;
    if (prec != PORTA_FP32 && prec != PORTA_FP64) return PORTA_EINVAL;
    if (nvox > (1LL << 31)) return PORTA_EINVAL;

    porta_ctx *c = new (std::nothrow) porta_ctx();
    if (!c) return PORTA_ENOMEM;
    c->nx = g->nx; c->ny = g->ny; c->nz = g->nz;
    c->lx = g->lx; c->ly = g->ly;
    c->z.assign(g->z, g->z + g->nz);
    c->model = at->model;
    c->ns = ns_of(at->model);
    c->nl = nl_of(at->model);
    c->nj = c->nl;
    c->zeta = at->zeta; c->gbar = at->gbar; c->bcrit = at->bcrit;
    c->n_mu = q->n_mu; c->n_chi = q->n_chi; c->n_nu = q->n_nu; c->x_max = q->x_max;
    c->precision = prec;
    c->user_shape = o && (o->cluster > 0 || o->nu_group > 0);
    c->opt_cluster = c->user_cluster = o ? o->cluster : 0;
    c->opt_nu_group = c->user_nu_group = o ? o->nu_group : 0;
    c->nvox = nvox;
    c->nray = 2 * q->n_mu * q->n_chi;
    c->nbox = nbox;
    {
        long long v0 = 0, g0 = 0;
        for (int b = 0; b < nbox; ++b) {
            const porta_grid *gb = &grids[b];
            BoxDev d{};
            d.nx = gb->nx; d.ny = gb->ny; d.nz = gb->nz;
            d.vox0 = v0;
            d.geom0 = g0;
            v0 += (long long)gb->nx * gb->ny * gb->nz;
            g0 += (long long)c->nray * gb->nz;
            c->boxes.push_back(d);
            c->bz.emplace_back(gb->z, gb->z + gb->nz);
            c->blx.push_back(gb->lx);
            c->bly.push_back(gb->ly);
        }
    }
    c->rsz = prec == PORTA_FP32 ? sizeof(float) : sizeof(double);

    // angular quadrature: Gauss inclinations per hemisphere x equally weighted azimuths at midpoints
    std::vector<double> xg(q->n_mu), wg(q->n_mu);
    gauss_legendre(q->n_mu, xg.data(), wg.data());
    c->mu.resize(c->nray); c->chi.resize(c->nray); c->w.resize(c->nray);
    for (int h = 0; h < 2; ++h)
        for (int i = 0; i < q->n_mu; ++i)
            for (int a = 0; a < q->n_chi; ++a) {
                int m = (h * q->n_mu + i) * q->n_chi + a;
                c->mu[m] = h == 0 ? xg[i] : -xg[i];
                c->chi[m] = (a + 0.5) * 2.0 * M_PI / q->n_chi;
                c->w[m] = 0.5 * wg[i] / q->n_chi;
            }
    // frequency quadrature: uniform nodes, trapezoid weights
    c->xf.resize(q->n_nu); c->wf.resize(q->n_nu);
    if (q->n_nu == 1) { c->xf[0] = 0.0; c->wf[0] = 1.0; }
    else {
        double dx = 2.0 * q->x_max / (q->n_nu - 1);
        for (int j = 0; j < q->n_nu; ++j) {
            c->xf[j] = -q->x_max + j * dx;
            c->wf[j] = (j == 0 || j == q->n_nu - 1) ? 0.5 * dx : dx;
        }
    }
    c->tkq.resize((size_t)c->nray * 18);
    for (int m = 0; m < c->nray; ++m) tkq_tensors(c->mu[m], c->chi[m], &c->tkq[(size_t)m * 18]);

    int rc = PORTA_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == PORTA_OK) {
            rc = e == cudaErrorMemoryAllocation ? PORTA_ENOMEM : PORTA_ECUDA;
            c->err = cudaGetErrorString(e);
        }
    };
    const size_t R = c->rsz;
    ok(pmalloc(&c->d_atm, 6 * nvox * R));
    ok(dalloc(&c->d_eps, nvox));
    ok(dalloc(&c->d_bpl, nvox));
    ok(dalloc(&c->d_b, 3 * nvox));
    ok(dalloc(&c->d_rho, nvox * c->nl));
    ok(pmalloc(&c->d_rhoR, nvox * c->nl * R));
    ok(pmalloc(&c->d_invn, (size_t)c->nray * nvox * R));
    ok(pmalloc(&c->d_geom, (size_t)c->nray * nplane * (prec == PORTA_FP32 ? sizeof(PlaneGeom<float>) : sizeof(PlaneGeom<double>))));
    ok(pmalloc(&c->d_boxes, (size_t)nbox * sizeof(BoxDev)));
    ok(dalloc(&c->d_items, (size_t)nbox * c->nray));
    c->n_tune = (int)std::min<long long>((long long)nbox * c->nray, 256);
    ok(dalloc(&c->d_tune_items, (size_t)c->n_tune));
    ok(pmalloc(&c->d_rays, (size_t)c->nray * (prec == PORTA_FP32 ? sizeof(RayDev<float>) : sizeof(RayDev<double>))));
    ok(pmalloc(&c->d_freq, 2 * (size_t)c->n_nu * R));
    ok(dalloc(&c->d_tw, (size_t)c->nray * 19));
    ok(dalloc(&c->d_jkq, nvox * c->nj));
    ok(dalloc(&c->d_lstar, nvox));
    ok(dalloc(&c->d_resid, 1));
    ok(dalloc(&c->d_err, 1));
    if (rc == PORTA_OK) {
        ok(cudaMemset(c->d_atm, 0, 6 * nvox * R));
        // geometry, rays, frequencies, angular weights
        std::vector<double> tw((size_t)c->nray * 19);
        for (int m = 0; m < c->nray; ++m) {
            tw[m * 19] = c->w[m];
            for (int i = 0; i < 18; ++i) tw[m * 19 + 1 + i] = c->tkq[(size_t)m * 18 + i];
        }
        ok(cudaMemcpy(c->d_tw, tw.data(), tw.size() * sizeof(double), cudaMemcpyHostToDevice));
        // boxes and work items: (box, ray) pairs by decreasing box size (longest first)
        ok(cudaMemcpy(c->d_boxes, c->boxes.data(), nbox * sizeof(BoxDev), cudaMemcpyHostToDevice));
        std::vector<int> items((size_t)nbox * c->nray);
        std::vector<int> order(nbox);
        for (int b = 0; b < nbox; ++b) order[b] = b;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            const BoxDev &p = c->boxes[x], &r = c->boxes[y];
            return (long long)p.nx * p.ny * p.nz > (long long)r.nx * r.ny * r.nz;
        });
        for (int i = 0; i < nbox; ++i)
            for (int m = 0; m < c->nray; ++m) items[(size_t)i * c->nray + m] = order[i] * c->nray + m;
        ok(cudaMemcpy(c->d_items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice));
        // autotuner sample: every k-th item, keeping the mix of box sizes
        std::vector<int> tune(c->n_tune);
        for (int i = 0; i < c->n_tune; ++i) tune[i] = items[(size_t)i * items.size() / c->n_tune];
        ok(cudaMemcpy(c->d_tune_items, tune.data(), tune.size() * sizeof(int), cudaMemcpyHostToDevice));
        if (prec == PORTA_FP32) {
            std::vector<PlaneGeom<float>> geom((size_t)c->nray * nplane);
            std::vector<RayDev<float>> rays(c->nray);
            std::vector<float> fr(2 * c->n_nu);
            for (int b = 0; b < nbox; ++b)
                for (int m = 0; m < c->nray; ++m)
                    plane_geometry<float>(c->boxes[b].nx, c->boxes[b].ny, c->boxes[b].nz, c->blx[b], c->bly[b],
                                          c->bz[b].data(), c->mu[m], c->chi[m],
                                          geom.data() + c->boxes[b].geom0 + (size_t)m * c->boxes[b].nz);
            for (int m = 0; m < c->nray; ++m) rays[m] = ray_dev<float>(c->mu[m], c->chi[m], c->w[m]);
            for (int j = 0; j < c->n_nu; ++j) { fr[j] = (float)c->xf[j]; fr[c->n_nu + j] = (float)c->wf[j]; }
            ok(cudaMemcpy(c->d_geom, geom.data(), geom.size() * sizeof(geom[0]), cudaMemcpyHostToDevice));
            ok(cudaMemcpy(c->d_rays, rays.data(), rays.size() * sizeof(rays[0]), cudaMemcpyHostToDevice));
            ok(cudaMemcpy(c->d_freq, fr.data(), fr.size() * sizeof(float), cudaMemcpyHostToDevice));
        } else {
            std::vector<PlaneGeom<double>> geom((size_t)c->nray * nplane);
            std::vector<RayDev<double>> rays(c->nray);
            std::vector<double> fr(2 * c->n_nu);
            for (int b = 0; b < nbox; ++b)
                for (int m = 0; m < c->nray; ++m)
                    plane_geometry<double>(c->boxes[b].nx, c->boxes[b].ny, c->boxes[b].nz, c->blx[b], c->bly[b],
                                           c->bz[b].data(), c->mu[m], c->chi[m],
                                           geom.data() + c->boxes[b].geom0 + (size_t)m * c->boxes[b].nz);
            for (int m = 0; m < c->nray; ++m) rays[m] = ray_dev<double>(c->mu[m], c->chi[m], c->w[m]);
            for (int j = 0; j < c->n_nu; ++j) { fr[j] = c->xf[j]; fr[c->n_nu + j] = c->wf[j]; }
            ok(cudaMemcpy(c->d_geom, geom.data(), geom.size() * sizeof(geom[0]), cudaMemcpyHostToDevice));
            ok(cudaMemcpy(c->d_rays, rays.data(), rays.size() * sizeof(rays[0]), cudaMemcpyHostToDevice));
            ok(cudaMemcpy(c->d_freq, fr.data(), fr.size() * sizeof(double), cudaMemcpyHostToDevice));
        }
        // a launch shape must exist for this grid
        LaunchCfg cfg{};
        int r2 = PORTA_OK;
        for (int jk = 1; jk >= 0; --jk) {
            r2 = prec == PORTA_FP32
                     ? (c->ns == 1 ? choose_launch<float, 1>(c, cfg, c->opt_cluster, c->opt_nu_group, c->nray, jk)
                                   : choose_launch<float, 4>(c, cfg, c->opt_cluster, c->opt_nu_group, c->nray, jk))
                     : (c->ns == 1 ? choose_launch<double, 1>(c, cfg, c->opt_cluster, c->opt_nu_group, c->nray, jk)
                                   : choose_launch<double, 4>(c, cfg, c->opt_cluster, c->opt_nu_group, c->nray, jk));
            if (jk) c->jk_fits = r2 == PORTA_OK;
        }
        if (rc == PORTA_OK && r2 != PORTA_OK) {
            if (c->opt_cluster > 0 || c->opt_nu_group > 0) {
                rc = PORTA_EINVAL;
                c->err = "the forced sweep launch shape does not fit this grid (shared memory / cluster limits)";
            } else {
                // planes too wide for every shared-memory ring: the global-memory sweep
                c->gsweep = 2;
                c->gsweep_checked = true;
            }
        }
    }
    if (rc != PORTA_OK) {
        free_all(c);
        delete c;
        return rc;
    }
    *out = c;
    return PORTA_OK;
}

}  // namespace porta_api

using namespace porta_api;

extern "C" {

int porta_create(const porta_grid *g, const porta_atom *at, const porta_quad *q, const porta_opts *o, porta_ctx **out)
{
    if (!g) {
        if (out) *out = nullptr;
        return PORTA_EINVAL;
    }
    return create_impl(1, g, at, q, o, out);
}

int porta_batch_create(int nbox, const porta_grid *grids, const porta_atom *at, const porta_quad *q,
                       const porta_opts *o, porta_ctx **out)
{
    return create_impl(nbox, grids, at, q, o, out);
}

void porta_destroy(porta_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    free_all(c);
    delete c;
}

const char *porta_last_error(const porta_ctx *c) { return c ? c->err.c_str() : kNullCtx; }

int porta_set_stream(porta_ctx *c, void *stream)
{
    if (!c) return PORTA_EINVAL;
    c->stream = (cudaStream_t)stream;
    return PORTA_OK;
}

int porta_sizes(const porta_ctx *c, int *nray, int *nnu, long long *nvox, int *nl, int *nj, int *ns)
{
    if (!c) return PORTA_EINVAL;
    if (nray) *nray = c->nray;
    if (nnu) *nnu = c->n_nu;
    if (nvox) *nvox = c->nvox;
    if (nl) *nl = c->nl;
    if (nj) *nj = c->nj;
    if (ns) *ns = c->ns;
    return PORTA_OK;
}

int porta_rays(const porta_ctx *c, double *mu, double *chi, double *w)
{
    if (!c) return PORTA_EINVAL;
    for (int m = 0; m < c->nray; ++m) {
        if (mu) mu[m] = c->mu[m];
        if (chi) chi[m] = c->chi[m];
        if (w) w[m] = c->w[m];
    }
    return PORTA_OK;
}

int porta_set_atmosphere(porta_ctx *c, const porta_atmos *a, int where)
{
    if (!c) return PORTA_EINVAL;
    if (!a || !a->chi || !a->eps || !a->bpl || !a->vel) return fail(c, PORTA_EINVAL, "atmosphere: missing array");
    const bool pol = c->model == PORTA_MODEL_TWOLEVEL_HANLE;
    if (pol && (!a->bx || !a->by || !a->bz)) return fail(c, PORTA_EINVAL, "atmosphere: magnetic field required");
    if (where != PORTA_HOST && where != PORTA_DEVICE) return fail(c, PORTA_EINVAL, "atmosphere: bad `where`");
    const long long n = c->nvox;
    // stage FP64 copies on the device: eps, bpl, field, chi and vel (all kept)
    if (!c->d_cv64) CK(dalloc(&c->d_cv64, 2 * n));
    double *tmp = c->d_cv64;
    int rc = PORTA_OK;
    do {
        if ((rc = copy_in(c, tmp, a->chi, n, where))) break;
        if ((rc = copy_in(c, tmp + n, a->vel, n, where))) break;
        if ((rc = copy_in(c, c->d_eps, a->eps, n, where))) break;
        if ((rc = copy_in(c, c->d_bpl, a->bpl, n, where))) break;
        if (pol) {
            if ((rc = copy_in(c, c->d_b, a->bx, n, where))) break;
            if ((rc = copy_in(c, c->d_b + n, a->by, n, where))) break;
            if ((rc = copy_in(c, c->d_b + 2 * n, a->bz, n, where))) break;
        } else {
            cudaMemsetAsync(c->d_b, 0, 3 * n * sizeof(double), c->stream);
        }
        unsigned long long bad = 0;
        if ((rc = count_bad(c, tmp, n, 0.0, 1e300, &bad))) break;
        if (bad) { rc = fail(c, PORTA_EINVAL, "atmosphere: chi must be finite and > 0"); break; }
        if ((rc = count_bad(c, c->d_eps, n, 0.0, 1.0, &bad))) break;
        if (bad) { rc = fail(c, PORTA_EINVAL, "atmosphere: eps must lie in (0, 1]"); break; }
        if ((rc = count_bad(c, c->d_bpl, n, -1e300, 1e300, &bad))) break;
        if (bad) { rc = fail(c, PORTA_EINVAL, "atmosphere: Planck function must be finite"); break; }
        if ((rc = count_bad(c, tmp + n, n, -1e300, 1e300, &bad))) break;
        if (bad) { rc = fail(c, PORTA_EINVAL, "atmosphere: velocity must be finite"); break; }
        if (pol) {
            if ((rc = count_bad(c, c->d_b, 3 * n, -1e300, 1e300, &bad))) break;
            if (bad) { rc = fail(c, PORTA_EINVAL, "atmosphere: magnetic field must be finite"); break; }
        }
        // sweep copies (Real): chi, vel, bx, by, bz, bpl
        cudaError_t e;
        const size_t R = c->rsz;
        char *atm = (char *)c->d_atm;
        if (c->precision == PORTA_FP32) {
            e = run_to_real<float>(n, tmp, atm, c->stream);
            if (e == cudaSuccess) e = run_to_real<float>(n, tmp + n, atm + n * R, c->stream);
            if (e == cudaSuccess) e = run_to_real<float>(3 * n, c->d_b, atm + 2 * n * R, c->stream);
            if (e == cudaSuccess) e = run_to_real<float>(n, c->d_bpl, atm + 5 * n * R, c->stream);
        } else {
            e = run_to_real<double>(n, tmp, atm, c->stream);
            if (e == cudaSuccess) e = run_to_real<double>(n, tmp + n, atm + n * R, c->stream);
            if (e == cudaSuccess) e = run_to_real<double>(3 * n, c->d_b, atm + 2 * n * R, c->stream);
            if (e == cudaSuccess) e = run_to_real<double>(n, c->d_bpl, atm + 5 * n * R, c->stream);
        }
        if (e != cudaSuccess) { rc = fail(c, PORTA_ECUDA, cudaGetErrorString(e)); break; }
        // profile normalization per voxel and ray
        double *dq = nullptr;
        e = dalloc(&dq, (size_t)c->nray + 2 * c->n_nu);
        if (e != cudaSuccess) { rc = fail(c, PORTA_ENOMEM, "atmosphere: allocation"); break; }
        std::vector<double> hq(c->mu);
        hq.insert(hq.end(), c->xf.begin(), c->xf.end());
        hq.insert(hq.end(), c->wf.begin(), c->wf.end());
        e = cudaMemcpyAsync(dq, hq.data(), hq.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = c->precision == PORTA_FP32
                    ? run_profile_norm<float>(n, c->nray, c->n_nu, dq, dq + c->nray, dq + c->nray + c->n_nu, tmp + n, c->d_invn, c->stream)
                    : run_profile_norm<double>(n, c->nray, c->n_nu, dq, dq + c->nray, dq + c->nray + c->n_nu, tmp + n, c->d_invn, c->stream);
        cudaError_t e2 = cudaStreamSynchronize(c->stream);
        pfree(dq);
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess) { rc = fail(c, PORTA_ECUDA, cudaGetErrorString(e)); break; }
    } while (0);
    cudaStreamSynchronize(c->stream);
    if (rc == PORTA_OK) {
        c->have_atm = true;
        c->have_fs = c->have_jkq = false;
    }
    return rc;
}

int porta_set_rho(porta_ctx *c, const double *rho, int where)
{
    if (!c) return PORTA_EINVAL;
    if (c->ml) return fail(c, PORTA_EINVAL, "set_rho: not for a multilevel context (porta_ml_*)");
    if (!rho || (where != PORTA_HOST && where != PORTA_DEVICE)) return fail(c, PORTA_EINVAL, "set_rho: bad argument");
    const long long n = c->nvox * c->nl;
    if (where == PORTA_HOST) {
        if (!finite_host(rho, n)) return fail(c, PORTA_EINVAL, "set_rho: non-finite value");
        for (long long v = 0; v < c->nvox; ++v)
            if (!(rho[v * c->nl] > 0)) return fail(c, PORTA_EINVAL, "set_rho: S^0_0 must be > 0");
    }
    int rc = copy_in(c, c->d_rho, rho, n, where);
    if (rc) return rc;
    if (where == PORTA_DEVICE) {
        unsigned long long bad = 0;
        if ((rc = count_bad(c, c->d_rho, n, -1e300, 1e300, &bad))) return rc;
        if (bad) return fail(c, PORTA_EINVAL, "set_rho: non-finite value");
    }
    cudaError_t e = c->precision == PORTA_FP32 ? run_rho_convert<float>(c->nvox, c->nl, c->d_rho, c->d_rhoR, c->stream)
                                               : run_rho_convert<double>(c->nvox, c->nl, c->d_rho, c->d_rhoR, c->stream);
    if (e != cudaSuccess) return fail(c, PORTA_ECUDA, cudaGetErrorString(e));
    if (where == PORTA_HOST) CK(cudaStreamSynchronize(c->stream));
    c->have_rho = true;
    c->have_fs = c->have_jkq = false;
    return PORTA_OK;
}

int porta_get_rho(porta_ctx *c, double *rho, int where)
{
    if (!c) return PORTA_EINVAL;
    if (!rho || (where != PORTA_HOST && where != PORTA_DEVICE)) return fail(c, PORTA_EINVAL, "get_rho: bad argument");
    if (!c->have_rho) return fail(c, PORTA_ESTATE, "get_rho: rho has not been set");
    CK(cudaMemcpyAsync(rho, c->d_rho, c->nvox * c->nl * sizeof(double),
                       where == PORTA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (where == PORTA_HOST) CK(cudaStreamSynchronize(c->stream));
    return PORTA_OK;
}

int porta_formal_solve(porta_ctx *c)
{
    if (!c) return PORTA_EINVAL;
    if (!c->have_atm) return fail(c, PORTA_ESTATE, "formal_solve: atmosphere not set");
    if (!c->have_rho) return fail(c, PORTA_ESTATE, "formal_solve: rho not set");
    int rc = c->precision == PORTA_FP32 ? formal_solve_t<float>(c, -1, nullptr, nullptr)
                                        : formal_solve_t<double>(c, -1, nullptr, nullptr);
    if (rc == PORTA_OK) {
        c->have_fs = true;
        c->jkq_loaded = false;
        c->have_jkq = false;
    }
    return rc;
}

int porta_accumulate_jkq(porta_ctx *c, double *jkq, double *lstar, int where)
{
    if (!c) return PORTA_EINVAL;
    if (!c->have_fs) return fail(c, PORTA_ESTATE, "accumulate_jkq: no formal solution");
    if (where != PORTA_HOST && where != PORTA_DEVICE) return fail(c, PORTA_EINVAL, "accumulate_jkq: bad `where`");
    // (J^K_Q loaded by porta_set_partial is already final)
    cudaError_t e = c->jkq_loaded ? cudaSuccess : finalize_jkq(c);
    if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("accumulate_jkq: ") + cudaGetErrorString(e));
    cudaMemcpyKind k = where == PORTA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (jkq) CK(cudaMemcpyAsync(jkq, c->d_jkq, c->nvox * c->nj * sizeof(double), k, c->stream));
    if (lstar) CK(cudaMemcpyAsync(lstar, c->d_lstar, c->nvox * sizeof(double), k, c->stream));
    if (where == PORTA_HOST && (jkq || lstar)) {
        int rc = check_jacc(c);
        if (rc != PORTA_OK) return rc;
    }
    c->have_jkq = true;
    return PORTA_OK;
}

int porta_see_update(porta_ctx *c, double *max_change)
{
    if (!c) return PORTA_EINVAL;
    if (!c->have_jkq) return fail(c, PORTA_ESTATE, "see_update: J^K_Q not accumulated");
    cudaError_t e = enqueue_update(c);
    if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("see_update: ") + cudaGetErrorString(e));
    c->have_fs = c->have_jkq = false;
    if (max_change) {
        unsigned long long bits = 0;
        CK(cudaMemcpyAsync(&bits, c->d_resid, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        double v;
        std::memcpy(&v, &bits, sizeof(v));
        *max_change = v;
    }
    return PORTA_OK;
}

int porta_probe_ray(porta_ctx *c, int m, double *out, double *lstar, int where)
{
    if (!c) return PORTA_EINVAL;
    if (m < 0 || m >= c->nray || !out || (where != PORTA_HOST && where != PORTA_DEVICE))
        return fail(c, PORTA_EINVAL, "probe_ray: bad argument");
    if (c->nbox != 1) return fail(c, PORTA_EINVAL, "probe_ray: single-box contexts only");
    if (c->fr1 > c->fr0) return fail(c, PORTA_ESTATE, "probe_ray: needs the whole frequency grid (porta_set_freq_range)");
    if (!c->have_atm || !c->have_rho) return fail(c, PORTA_ESTATE, "probe_ray: atmosphere or rho not set");
    const long long n = (long long)c->n_nu * c->nvox;
    void *pr = nullptr, *pl = nullptr;
    CK(pmalloc(&pr, n * c->ns * c->rsz));
    cudaError_t e = pmalloc(&pl, n * c->rsz);
    if (e != cudaSuccess) { pfree(pr); return fail(c, PORTA_ENOMEM, "probe_ray: allocation"); }
    int rc = c->precision == PORTA_FP32 ? formal_solve_t<float>(c, m, (float *)pr, (float *)pl)
                                        : formal_solve_t<double>(c, m, (double *)pr, (double *)pl);
    double *d1 = nullptr, *d2 = nullptr;
    if (rc == PORTA_OK) {
        e = dalloc(&d1, n * c->ns);
        if (e == cudaSuccess) e = dalloc(&d2, n);
        if (e == cudaSuccess) {
            if (c->precision == PORTA_FP32) {
                // widen float -> double on the host side of the copy
                std::vector<float> h1(n * c->ns), h2(n);
                e = cudaMemcpyAsync(h1.data(), pr, h1.size() * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
                if (e == cudaSuccess) e = cudaMemcpyAsync(h2.data(), pl, h2.size() * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
                std::vector<double> g1(h1.begin(), h1.end()), g2(h2.begin(), h2.end());
                if (e == cudaSuccess) e = cudaMemcpy(d1, g1.data(), g1.size() * sizeof(double), cudaMemcpyHostToDevice);
                if (e == cudaSuccess) e = cudaMemcpy(d2, g2.data(), g2.size() * sizeof(double), cudaMemcpyHostToDevice);
            } else {
                e = cudaMemcpyAsync(d1, pr, n * c->ns * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
                if (e == cudaSuccess) e = cudaMemcpyAsync(d2, pl, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
            }
        }
        cudaMemcpyKind k = where == PORTA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, d1, n * c->ns * sizeof(double), k, c->stream);
        if (e == cudaSuccess && lstar) e = cudaMemcpyAsync(lstar, d2, n * sizeof(double), k, c->stream);
        cudaError_t e2 = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, std::string("probe_ray: ") + cudaGetErrorString(e));
    }
    cudaStreamSynchronize(c->stream);
    pfree(pr);
    pfree(pl);
    if (d1) pfree(d1);
    if (d2) pfree(d2);
    if (rc == PORTA_OK) {
        c->have_fs = true;
        c->jkq_loaded = false;
        c->have_jkq = false;
    }
    return rc;
}

int porta_eval_coefficients(int precision, int n, const double *t, double *out)
{
    if (n < 1 || !t || !out || (precision != PORTA_FP32 && precision != PORTA_FP64)) return PORTA_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!(t[i] > 0) || !std::isfinite(t[i])) return PORTA_EINVAL;
    double *d = nullptr;
    if (pmalloc(&d, sizeof(double) * 7 * (size_t)n) != cudaSuccess) return PORTA_ENOMEM;
    cudaError_t e = cudaMemcpy(d, t, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = precision == PORTA_FP32 ? run_coefficients<float>(n, d, d + n, nullptr) : run_coefficients<double>(n, d, d + n, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d + n, sizeof(double) * 6 * (size_t)n, cudaMemcpyDeviceToHost);
    pfree(d);
    return e == cudaSuccess ? PORTA_OK : PORTA_ECUDA;
}

int porta_eval_step(int precision, int n, const double *in, double *out)
{
    if (n < 1 || !in || !out || (precision != PORTA_FP32 && precision != PORTA_FP64)) return PORTA_EINVAL;
    for (int i = 0; i < n; ++i) {
        const double *p = in + (size_t)i * 34;
        for (int k = 0; k < 34; ++k)
            if (!std::isfinite(p[k])) return PORTA_EINVAL;
        if (!(p[4] > 0) || !(p[15] > 0) || !(p[31] > 0) || (p[33] != 0.0 && (!(p[26] > 0) || !(p[32] > 0))))
            return PORTA_EINVAL;
    }
    double *d = nullptr;
    if (pmalloc(&d, sizeof(double) * 39 * (size_t)n) != cudaSuccess) return PORTA_ENOMEM;
    cudaError_t e = cudaMemcpy(d, in, sizeof(double) * 34 * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = run_step_eval(precision, n, d, d + 34 * (size_t)n, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d + 34 * (size_t)n, sizeof(double) * 5 * (size_t)n, cudaMemcpyDeviceToHost);
    pfree(d);
    return e == cudaSuccess ? PORTA_OK : PORTA_ECUDA;
}

int porta_autotune(porta_ctx *c, int *cluster, int *nu_group)
{
    if (!c) return PORTA_EINVAL;
    if (!c->have_atm || !c->have_rho) return fail(c, PORTA_ESTATE, "autotune: atmosphere or rho not set");
    int rc = c->precision == PORTA_FP32 ? autotune_t<float>(c) : autotune_t<double>(c);
    if (rc == PORTA_OK) {
        if (cluster) *cluster = c->opt_cluster;
        if (nu_group) *nu_group = c->opt_nu_group;
    }
    return rc;
}

int porta_run_iterations(porta_ctx *c, int iterations, double *max_change)
{
    if (!c) return PORTA_EINVAL;
    if (iterations < 0) return fail(c, PORTA_EINVAL, "run_iterations: negative count");
    if (!c->have_atm || !c->have_rho) return fail(c, PORTA_ESTATE, "run_iterations: atmosphere or rho not set");
    if (!c->stream) return fail(c, PORTA_ESTATE, "run_iterations: needs a non-default stream (porta_set_stream)");
    if (c->graph_exec && c->graph_stream != c->stream) drop_graph(c);
    if (!c->graph_exec) {
        cudaError_t eb = ensure_sweep_buffers(c);   // no allocation inside the capture
        if (eb != cudaSuccess) return fail(c, PORTA_ENOMEM, std::string("run_iterations: ") + cudaGetErrorString(eb));
        // capture one iteration: formal solution, J^K_Q sums, SEE update and residual
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        int rc = c->precision == PORTA_FP32 ? formal_solve_t<float>(c, -1, nullptr, nullptr)
                                            : formal_solve_t<double>(c, -1, nullptr, nullptr);
        cudaError_t e = cudaSuccess;
        if (rc == PORTA_OK) {
            e = finalize_jkq(c);
            if (e == cudaSuccess) e = enqueue_update(c);
        }
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
        if (rc != PORTA_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph_exec, g, cudaGraphInstantiateFlagUseNodePriority);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            c->graph_exec = nullptr;
            return fail(c, PORTA_ECUDA, std::string("run_iterations: graph capture: ") + cudaGetErrorString(e));
        }
        c->graph = g;
        c->graph_stream = c->stream;
    }
    for (int it = 0; it < iterations; ++it) CK(cudaGraphLaunch(c->graph_exec, c->stream));
    c->have_fs = c->have_jkq = false;
    if (max_change) {
        unsigned long long bits = 0;
        CK(cudaMemcpyAsync(&bits, c->d_resid, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        double v;
        std::memcpy(&v, &bits, sizeof(v));
        *max_change = v;
        int rc = check_jacc(c);
        if (rc != PORTA_OK) return rc;
    }
    return PORTA_OK;
}

int porta_set_device_limit(long long bytes)
{
    if (bytes < 0) return PORTA_EINVAL;
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    g_alloc_limit = (size_t)bytes;
    return PORTA_OK;
}

long long porta_device_bytes(void)
{
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    return (long long)g_alloc_live;
}

int porta_iterate_to(porta_ctx *c, double tol, int max_iter, int check_every, int *iterations_out,
                     double *max_change_out)
{
    if (!c) return PORTA_EINVAL;
    if (!(tol > 0) || max_iter < 1 || check_every < 1)
        return fail(c, PORTA_EINVAL, "iterate_to: tol > 0, max_iter >= 1 and check_every >= 1 required");
    int done = 0;
    double change = 0.0;
    while (done < max_iter) {
        const int n = std::min(check_every, max_iter - done);
        int rc = porta_run_iterations(c, n, &change);
        if (rc != PORTA_OK) return rc;
        done += n;
        if (iterations_out) *iterations_out = done;
        if (max_change_out) *max_change_out = change;
        if (change < tol) return PORTA_OK;
    }
    return fail(c, PORTA_ENOTCONV, "iterate_to: maximum change " + std::to_string(change) + " >= tolerance after " +
                                       std::to_string(done) + " iterations");
}

int porta_set_freq_range(porta_ctx *c, int j0, int j1)
{
    if (!c) return PORTA_EINVAL;
    if (c->ml) return fail(c, PORTA_EINVAL, "set_freq_range: two-level contexts only");
    if (j0 == 0 && (j1 == 0 || j1 == c->n_nu)) {
        c->fr0 = c->fr1 = 0;
    } else {
        if (j0 < 0 || j1 <= j0 || j1 > c->n_nu) return fail(c, PORTA_EINVAL, "set_freq_range: need 0 <= j0 < j1 <= n_nu");
        c->fr0 = j0;
        c->fr1 = j1;
    }
    c->have_fs = c->have_jkq = false;
    drop_graph(c);
    return PORTA_OK;
}

int porta_partial_size(const porta_ctx *c, long long *elements, int *elem_bytes)
{
    if (!c) return PORTA_EINVAL;
    // (polarized lines of a multilevel atom: J^1_Q, 3 per voxel, follow)
    if (elements) *elements = (long long)(c->nj + 1 + (c->d_j1 ? 3 : 0)) * c->nvox;
    if (elem_bytes) *elem_bytes = 8;
    return PORTA_OK;
}

int porta_get_partial(porta_ctx *c, void *out, int where)
{
    if (!c || !out) return PORTA_EINVAL;
    if (!c->have_fs) return fail(c, PORTA_ESTATE, "get_partial: no formal solution");
    if (where != PORTA_HOST && where != PORTA_DEVICE) return fail(c, PORTA_EINVAL, "get_partial: bad `where`");
    const cudaMemcpyKind k = where == PORTA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (jfixed(c)) {
        CK(cudaMemcpyAsync(out, c->d_jacc, (size_t)(c->nj + 1) * c->nvox * sizeof(unsigned long long), k, c->stream));
    } else {
        cudaError_t e = finalize_jkq(c);
        if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("get_partial: ") + cudaGetErrorString(e));
        double *o = (double *)out;
        CK(cudaMemcpyAsync(o, c->d_jkq, (size_t)c->nj * c->nvox * sizeof(double), k, c->stream));
        CK(cudaMemcpyAsync(o + (size_t)c->nj * c->nvox, c->d_lstar, (size_t)c->nvox * sizeof(double), k, c->stream));
        if (c->d_j1)
            CK(cudaMemcpyAsync(o + (size_t)(c->nj + 1) * c->nvox, c->d_j1, (size_t)3 * c->nvox * sizeof(double), k, c->stream));
    }
    if (where == PORTA_HOST) CK(cudaStreamSynchronize(c->stream));
    return PORTA_OK;
}

int porta_set_partial(porta_ctx *c, const void *in, int where)
{
    if (!c || !in) return PORTA_EINVAL;
    if (!c->have_fs) return fail(c, PORTA_ESTATE, "set_partial: no formal solution on this context");
    if (where != PORTA_HOST && where != PORTA_DEVICE) return fail(c, PORTA_EINVAL, "set_partial: bad `where`");
    const cudaMemcpyKind k = where == PORTA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (jfixed(c)) {
        CK(cudaMemcpyAsync(c->d_jacc, in, (size_t)(c->nj + 1) * c->nvox * sizeof(unsigned long long), k, c->stream));
        cudaError_t e = finalize_jkq(c);
        if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("set_partial: ") + cudaGetErrorString(e));
    } else {
        const double *i = (const double *)in;
        CK(cudaMemcpyAsync(c->d_jkq, i, (size_t)c->nj * c->nvox * sizeof(double), k, c->stream));
        CK(cudaMemcpyAsync(c->d_lstar, i + (size_t)c->nj * c->nvox, (size_t)c->nvox * sizeof(double), k, c->stream));
        if (c->d_j1)
            CK(cudaMemcpyAsync(c->d_j1, i + (size_t)(c->nj + 1) * c->nvox, (size_t)3 * c->nvox * sizeof(double), k, c->stream));
    }
    if (where == PORTA_HOST) CK(cudaStreamSynchronize(c->stream));
    c->have_jkq = true;
    c->jkq_loaded = true;
    return PORTA_OK;
}

int porta_set_fill(porta_ctx *c, int cluster, int nu_group, double fraction)
{
    if (!c) return PORTA_EINVAL;
    if (cluster == 0) {
        c->fill_cfg = LaunchCfg{};
        c->fill_frac = 0.0;
        drop_graph(c);
        return PORTA_OK;
    }
    if (cluster < 1 || cluster > 16 || nu_group < 1 || nu_group > c->n_nu || !(fraction > 0.0 && fraction < 1.0))
        return fail(c, PORTA_EINVAL, "set_fill: cluster in 1..16, nu_group in 1..n_nu, fraction in (0, 1)");
    LaunchCfg k{};
    const int nitems = c->nbox * c->nray;
    const bool jk = use_jk(c);
    const int nu = jnu(c);
    int rc = c->precision == PORTA_FP32
                 ? (c->ns == 1 ? choose_launch<float, 1>(c, k, cluster, nu_group, nitems, jk, nu) : choose_launch<float, 4>(c, k, cluster, nu_group, nitems, jk, nu))
                 : (c->ns == 1 ? choose_launch<double, 1>(c, k, cluster, nu_group, nitems, jk, nu) : choose_launch<double, 4>(c, k, cluster, nu_group, nitems, jk, nu));
    if (rc || k.F != nu_group) return fail(c, PORTA_EINVAL, "set_fill: this launch shape does not fit");
    // stream, events and counters exist before any graph capture uses them
    cudaError_t e = ensure_fill(c);
    if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("set_fill: ") + cudaGetErrorString(e));
    c->fill_cfg = k;
    c->fill_frac = fraction;
    c->have_fs = c->have_jkq = false;
    drop_graph(c);
    return PORTA_OK;
}

int porta_fill_info(const porta_ctx *c, int *cluster_size, int *nu_group, double *fraction)
{
    if (!c) return PORTA_EINVAL;
    if (cluster_size) *cluster_size = c->fill_cfg.cluster;
    if (nu_group) *nu_group = c->fill_cfg.F;
    if (fraction) *fraction = c->fill_frac;
    return PORTA_OK;
}

int porta_launch_info(const porta_ctx *c, int *clusters, int *cluster_size, int *nu_group, int *smem_bytes)
{
    if (!c) return PORTA_EINVAL;
    if (clusters) *clusters = c->last.clusters;
    if (cluster_size) *cluster_size = c->last.cluster;
    if (nu_group) *nu_group = c->last.F;
    if (smem_bytes) *smem_bytes = c->last.smem;
    return PORTA_OK;
}
int porta_set_explicit_medium(porta_ctx *c, const double *kexpl, const double *sexpl, int where)
{
    if (!c) return PORTA_EINVAL;
    if (!kexpl || !sexpl) {
        if (c->d_kexpl) pfree(c->d_kexpl);
        if (c->d_sexpl) pfree(c->d_sexpl);
        c->d_kexpl = c->d_sexpl = nullptr;
        c->emg_tuned.clear();
        return PORTA_OK;
    }
    if (c->ns != 4 || c->ml || c->d_dich || c->nbox != 1)
        return fail(c, PORTA_EINVAL, "set_explicit_medium: polarized two-level single-box contexts only");
    if (c->interp == 2) return fail(c, PORTA_EINVAL, "set_explicit_medium: bilinear interpolation only");
    if (where != PORTA_HOST && where != PORTA_DEVICE) return fail(c, PORTA_EINVAL, "set_explicit_medium: where");
    if (where == PORTA_HOST && (!finite_host(kexpl, 6 * c->nvox) || !finite_host(sexpl, 4 * c->nvox)))
        return fail(c, PORTA_EINVAL, "set_explicit_medium: non-finite values");
    if (!c->d_kexpl) CK(dalloc(&c->d_kexpl, 6 * (size_t)c->nvox));
    if (!c->d_sexpl) CK(dalloc(&c->d_sexpl, 4 * (size_t)c->nvox));
    int rc = copy_in(c, c->d_kexpl, kexpl, 6 * c->nvox, where);
    if (rc == PORTA_OK) rc = copy_in(c, c->d_sexpl, sexpl, 4 * c->nvox, where);
    if (rc == PORTA_OK) CK(cudaStreamSynchronize(c->stream));
    c->emg_tuned.clear();
    return rc;
}

int porta_set_global_sweep(porta_ctx *c, int on)
{
    if (!c) return PORTA_EINVAL;
    if (on != 0 && on != 1) return fail(c, PORTA_EINVAL, "set_global_sweep: 0 or 1");
    if (on && (c->d_kexpl || c->interp == 2))
        return fail(c, PORTA_EINVAL, "set_global_sweep: bilinear stencils only, and not with an explicit medium");
    c->gsweep = on;
    c->gsweep_checked = on != 0;           // off: the shared-memory shapes are checked again
    c->have_fs = c->have_jkq = false;
    drop_graph(c);
    return PORTA_OK;
}

int porta_set_sc_faces(porta_ctx *c, int on)
{
    if (!c) return PORTA_EINVAL;
    if (on != 0 && on != 1) return fail(c, PORTA_EINVAL, "set_sc_faces: 0 or 1");
    if (on && (c->d_kexpl || c->interp == 2))
        return fail(c, PORTA_EINVAL, "set_sc_faces: bilinear stencils only, and not with an explicit medium");
    if (on == c->sc_faces) return PORTA_OK;
    c->sc_faces = on;
    c->have_fs = c->have_jkq = false;
    drop_graph(c);
    return PORTA_OK;
}

int porta_set_interpolation(porta_ctx *c, int order)
{
    if (!c) return PORTA_EINVAL;
    if (order != 1 && order != 2) return fail(c, PORTA_EINVAL, "set_interpolation: order 1 (bilinear) or 2 (biquadratic)");
    if (order == 2 && (c->ml || c->d_dich))
        return fail(c, PORTA_EINVAL, "set_interpolation: the biquadratic stencils have no dichroism (multilevel lines)");
    if (order == 2 && min_ny(c) < 2) return fail(c, PORTA_EINVAL, "set_interpolation: biquadratic needs ny >= 2");
    if (order == 2 && c->d_kexpl) return fail(c, PORTA_EINVAL, "set_interpolation: explicit media are bilinear");
    if (order == 2 && (c->sc_faces || c->gsweep))
        return fail(c, PORTA_EINVAL, "set_interpolation: the global-memory sweep (face intersections) is bilinear");
    if (order == c->interp) return PORTA_OK;
    c->interp = order;
    // an autotuned shape of the other stencil need not fit: back to porta_opts' choice
    c->opt_cluster = c->user_cluster;
    c->opt_nu_group = c->user_nu_group;
    c->fill_cfg = LaunchCfg{};
    c->fill_frac = 0.0;
    c->emg_tuned.clear();
    c->have_fs = c->have_jkq = false;
    drop_graph(c);
    return PORTA_OK;
}

}  // extern "C"
