// C ABI of the formal-solver library (include/porta.h): argument checks,
// quadratures and per-ray plane geometry (host, FP64), device buffers, and the
// launch sequence formal_solve -> accumulate_jkq -> see_update.
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

#include "porta.h"
#include "porta_ctx.h"
#include "porta_internal.cuh"
#include "mg_kernels.cuh"
#include "ml_kernels.cuh"
#include "mlpol_kernels.cuh"
#include "see_kernels.cuh"

using namespace porta;

namespace {

const char *kNullCtx = "null context";

int fail(porta_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

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

template <typename T>
cudaError_t pmalloc(T **p, size_t bytes)
{
    void *q = nullptr;
    cudaError_t e = pmalloc_bytes(&q, bytes);
    *p = (T *)q;
    return e;
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

template <typename T>
cudaError_t dalloc(T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) return cudaSuccess;
    return pmalloc(p, n * sizeof(T));
}

// Gauss-Legendre nodes/weights on (0, 1): Newton's method on the Legendre
// polynomial P_n evaluated by its three-term recurrence.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double t = std::cos(M_PI * (4.0 * i + 3.0) / (4.0 * n + 2.0));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double pm1 = 1.0, p = t;
            for (int k = 1; k < n; ++k) {
                double pn = ((2 * k + 1) * t * p - k * pm1) / (k + 1);
                pm1 = p;
                p = pn;
            }
            if (n == 1) { p = t; pm1 = 1.0; }
            dp = n * (pm1 - t * p) / (1.0 - t * t);
            double dt = p / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-16) {
                // one more derivative evaluation at the final node
                pm1 = 1.0; p = t;
                for (int k = 1; k < n; ++k) {
                    double pn = ((2 * k + 1) * t * p - k * pm1) / (k + 1);
                    pm1 = p;
                    p = pn;
                }
                if (n == 1) { p = t; pm1 = 1.0; }
                dp = n * (pm1 - t * p) / (1.0 - t * t);
                break;
            }
        }
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

long long wrapll(long long a, long long n)
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

int ns_of(int model) { return model == PORTA_MODEL_TWOLEVEL_UNPOL ? 1 : 4; }
int nl_of(int model) { return model == PORTA_MODEL_TWOLEVEL_UNPOL ? 1 : 6; }

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
        // with dichroism the slots of a second ring (eta_U / eta_I per node) follow the node ring
        const int dchunks = dich ? (chunk * (int)sizeof(Real) + 15) / 16 : 0;
        ring_plane = std::max(ring_plane, nch * chunk + dchunks);
        ipts_max = std::max(ipts_max, rmax * b.nx);
    }
}

// The J^K_Q formal solution runs the kernel of sweep_j.cu (per-frequency
// node coefficients in shared memory) unless the lines carry dichroism, which
// only the general sweep (sweep.cu) implements, or a plane is too wide for its
// shared memory (then the general sweep, which needs less per frequency, runs).
bool use_jk(const porta_ctx *c) { return c->d_dich == nullptr && c->jk_fits; }

// The J^K_Q sweep sums an FP32 formal solution into fixed-point accumulators;
// an FP64 one keeps per-ray partial integrals summed in ray order in FP64 (a
// fixed-point scale cannot hold 1e-10 relative precision for quantities that
// span many decades within one voxel, as Lambda-bar* does with optical depth).
bool jfixed(const porta_ctx *c) { return use_jk(c) && c->precision == PORTA_FP32; }

// frequencies of the J^K_Q formal solution (its band, porta_set_freq_range)
int jnu(const porta_ctx *c) { return c->fr1 > c->fr0 ? c->fr1 - c->fr0 : c->n_nu; }

int max_ny(const porta_ctx *c)
{
    int m = 0;
    for (const BoxDev &b : c->boxes) m = std::max(m, b.ny);
    return m;
}

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
    const int NA = NS == 1 ? 2 : 4;
    double best_cost = 1e300;
    best = LaunchCfg{};
    const int ny_max = max_ny(c);
    for (int C = 1; C <= 16; ++C) {
        if (force_c > 0 && C != force_c) continue;
        if (force_c <= 0 && C > 1 && (C & (C - 1)) != 0 && C != 6 && C != 12) continue;   // heuristic set
        if (C > ny_max) continue;
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
                            : sweep_smem_bytes<Real, NS>(ring_plane, ipts_max, F, threads);
        if (smem > kSmemLimit + 16) continue;
        int act = 0;
        if ((jk ? jsweep_max_active_clusters<Real, NS>(C, smem, threads, &act)
                : max_active_clusters<Real, NS>(C, smem, threads, &act, c->d_dich != nullptr)) != cudaSuccess) {
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
    a.jacc = jfixed(c) ? c->d_jacc : nullptr;
    a.jexp = c->d_jexp;
    a.jerr = c->d_err;
    a.tw = c->d_tw;
    a.items = c->d_items;
    a.nitems = c->nbox * c->nray;
    return a;
}

// Device buffers of the J^K_Q formal solution, allocated on first use (before
// any graph capture): the fixed-point sums of the J^K_Q sweep, or the per-ray
// partial integrals of the general sweep.
cudaError_t ensure_sweep_buffers(porta_ctx *c)
{
    if (jfixed(c)) {
        cudaError_t e = cudaSuccess;
        if (!c->d_jacc) e = pmalloc(&c->d_jacc, (size_t)(c->nj + 1) * c->nvox * sizeof(unsigned long long));
        if (e == cudaSuccess && !c->d_jexp) e = pmalloc(&c->d_jexp, (size_t)c->nvox * sizeof(int));
        return e;
    }
    if (c->d_part) return cudaSuccess;
    return pmalloc(&c->d_part, (size_t)c->nray * c->nvox * (c->ns == 1 ? 2 : 4) * c->rsz);
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

// J^K_Q and Lambda-bar* (FP64) from the sums of the last formal solution
cudaError_t finalize_jkq(porta_ctx *c)
{
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
    if (!jfixed(c)) return PORTA_OK;
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
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

template <typename Real>
int formal_solve_t(porta_ctx *c, int probe_ray, Real *probe, Real *probe_ls)
{
    SweepArgs<Real> a = jkq_args<Real>(c);
    a.probe_ray = probe_ray;
    a.probe = probe;
    a.probe_ls = probe_ls;
    LaunchCfg cfg{};
    int rc = c->ns == 1 ? choose_launch<Real, 1>(c, cfg, c->opt_cluster, c->opt_nu_group, a.nitems, use_jk(c), jnu(c))
                        : choose_launch<Real, 4>(c, cfg, c->opt_cluster, c->opt_nu_group, a.nitems, use_jk(c), jnu(c));
    if (rc) return fail(c, rc, "no sweep launch shape fits this grid (shared memory / cluster limits)");
    shape_args<Real>(c, a, cfg, use_jk(c));
    cudaError_t e = ensure_sweep_buffers(c);
    if (e != cudaSuccess) return fail(c, PORTA_ENOMEM, std::string("formal solution buffers: ") + cudaGetErrorString(e));
    a.part = jfixed(c) ? nullptr : c->d_part;
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

// Launch shape of the emergent sweep for ndir directions: the one given in
// porta_opts, else timed once per direction count over the fitting shapes
// (cluster sizes x frequencies per pass; each trial rewrites the same outputs).
// Leaves the arguments shaped for the chosen launch.
template <typename Real, int NS>
int emergent_shape(porta_ctx *c, SweepArgs<Real> &a, int ndir, LaunchCfg &cfg)
{
    auto shape = [&](LaunchCfg &k) {
        shape_args<Real>(c, a, k);
        a.nitems = ndir * a.ngroups;
        k.clusters = std::min(k.clusters, a.nitems);
    };
    if (c->user_shape || c->emg_tuned.count(ndir)) {
        if (c->user_shape) {
            int rc = choose_launch<Real, NS>(c, cfg, c->opt_cluster, c->opt_nu_group, ndir);
            if (rc) return fail(c, rc, "no sweep launch shape fits this grid");
        } else {
            cfg = c->emg_tuned[ndir];
        }
        shape(cfg);
        return PORTA_OK;
    }
    std::vector<LaunchCfg> cand;
    const int sizes[] = {1, 2, 3, 4, 6, 8, 12, 16};
    for (int C : sizes) {
        if (C > c->ny) continue;
        int last_f = -1;
        for (int G = 1; G <= c->n_nu; ++G) {
            const int F = (c->n_nu + G - 1) / G;
            if (F == last_f) continue;
            last_f = F;
            LaunchCfg k{};
            if (choose_launch<Real, NS>(c, k, C, F, ndir * G) == PORTA_OK && k.F == F) cand.push_back(k);
        }
    }
    if (cand.empty()) return fail(c, PORTA_EINVAL, "no sweep launch shape fits this grid");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    cudaError_t e = cudaSuccess;
    for (LaunchCfg k : cand) {
        shape(k);
        float ms = 0;
        e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess) e = launch_sweep<Real, NS>(a, MODE_EMERGENT, k, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        if (ms < best) {
            best = ms;
            cfg = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("emergent shape timing: ") + cudaGetErrorString(e));
    c->emg_tuned[ndir] = cfg;
    shape(cfg);
    return PORTA_OK;
}

template <typename Real>
int emergent_t(porta_ctx *c, int ndir, const double *mu, const double *chi, double *dout, int box = 0)
{
    std::vector<PlaneGeom<Real>> geom((size_t)ndir * c->nz);
    std::vector<RayDev<Real>> rays(ndir);
    for (int d = 0; d < ndir; ++d) {
        plane_geometry<Real>(c->nx, c->ny, c->nz, c->lx, c->ly, c->z.data(), mu[d], chi[d], geom.data() + (size_t)d * c->nz);
        rays[d] = ray_dev<Real>(mu[d], chi[d]);
    }
    PlaneGeom<Real> *dg = nullptr;
    RayDev<Real> *dr = nullptr;
    BoxDev *dbox = nullptr;
    CK(dalloc(&dg, geom.size()));
    cudaError_t e2 = dalloc(&dr, rays.size());
    if (e2 == cudaSuccess) e2 = pmalloc(&dbox, sizeof(BoxDev));
    if (e2 != cudaSuccess) {
        pfree(dg);
        if (dr) pfree(dr);
        return fail(c, PORTA_ENOMEM, "emergent: device allocation");
    }
    int rc = PORTA_OK;
    do {
        // the box of this call (a line of a multilevel context shares the grid): its
        // voxels, with the per-direction geometry of this call (geometry offset 0)
        BoxDev hb = c->boxes[box];
        hb.geom0 = 0;
        cudaError_t e = cudaMemcpyAsync(dg, geom.data(), geom.size() * sizeof(geom[0]), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dr, rays.data(), rays.size() * sizeof(rays[0]), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dbox, &hb, sizeof(hb), cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) { rc = fail(c, PORTA_ECUDA, cudaGetErrorString(e)); break; }
        SweepArgs<Real> a = base_args<Real>(c);
        a.boxes = dbox;
        a.geom = dg;
        a.rays = dr;
        a.out = dout;
        LaunchCfg cfg{};
        rc = c->ns == 1 ? emergent_shape<Real, 1>(c, a, ndir, cfg) : emergent_shape<Real, 4>(c, a, ndir, cfg);
        if (rc) break;
        e = c->ns == 1 ? launch_sweep<Real, 1>(a, MODE_EMERGENT, cfg, c->stream)
                       : launch_sweep<Real, 4>(a, MODE_EMERGENT, cfg, c->stream);
        if (e != cudaSuccess) { rc = fail(c, PORTA_ECUDA, std::string("emergent launch: ") + cudaGetErrorString(e)); break; }
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, std::string("emergent: ") + cudaGetErrorString(e));
    } while (0);
    cudaStreamSynchronize(c->stream);
    pfree(dg);
    pfree(dr);
    pfree(dbox);
    return rc;
}

// grow-only device buffer held by the context
cudaError_t ensure_buf(void **p, size_t &cap, size_t need)
{
    if (need <= cap && *p) return cudaSuccess;
    if (*p) pfree(*p);
    *p = nullptr;
    cap = 0;
    cudaError_t e = pmalloc(p, need);
    if (e == cudaSuccess) cap = need;
    return e;
}

const int kAdjThreads = 256;   // maximum threads per CTA of the adjoint kernel

// Launch shape of the adjoint sweep: cluster size C and frequencies per pass
// F. Estimated time: the (direction, frequency group) items spread over the
// resident clusters, each costing per plane its point passes (F frequencies
// per pass) plus the two cluster barriers, the ring fill and the node
// finalization.
template <typename Real, int NS>
int choose_adjoint(porta_ctx *c, LaunchCfg &best, int force_c, int force_f, int ndir,
                   std::vector<LaunchCfg> *all = nullptr)
{
    best = LaunchCfg{};
    double best_cost = 1e300;
    for (int C = 1; C <= 16; ++C) {
        if (force_c > 0 && C != force_c) continue;
        if (force_c <= 0 && C > 1 && (C & (C - 1)) != 0 && C != 6 && C != 12) continue;
        if (C > c->ny) continue;
        int ring_plane, ipts;
        launch_caps<Real, NS>(c, C, ring_plane, ipts);
        const int threads = std::min(kAdjThreads, std::max(64, (ipts + 31) / 32 * 32));
        int last_f = -1;
        for (int G = 1; G <= c->n_nu; ++G) {
            const int F = force_f > 0 ? force_f : (c->n_nu + G - 1) / G;
            if (F == last_f) continue;
            last_f = F;
            const int smem = adjoint_smem_bytes<Real, NS>(ring_plane, ipts, ipts + c->nx, F);
            if (smem > kSmemLimit) continue;
            int act = 0;
            if (adjoint_max_active_clusters<Real, NS>(C, smem, threads, &act) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (act < 1) continue;
            const int Gr = (c->n_nu + F - 1) / F;
            const int items = ndir * Gr;
            const int ncl = std::min(act, items);
            const double passes = std::ceil((double)ipts / threads);
            const double item = c->nz * (passes * F * 3.0 + 0.5 * F + 4.0);
            const double cost = std::ceil((double)items / ncl) * item;
            if (all) {
                LaunchCfg k{};
                k.cluster = C;
                k.F = F;
                k.threads = threads;
                k.smem = smem;
                k.clusters = ncl;
                all->push_back(k);
            }
            if (cost < best_cost) {
                best_cost = cost;
                best.cluster = C;
                best.F = F;
                best.threads = threads;
                best.smem = smem;
                best.clusters = ncl;
            }
        }
    }
    return best.cluster > 0 ? PORTA_OK : PORTA_EINVAL;
}

// forward emergent sweep with the tape, adjoint sweep, fixed-order reduction;
// all pointers are device memory; dout may be null
template <typename Real>
int emergent_vjp_t(porta_ctx *c, int ndir, const double *mu, const double *chi, const double *dgrad, double *dout,
                   double *dg_chi, double *dg_e, double *dg_b, double *dg_rho = nullptr)
{
    std::vector<PlaneGeom<Real>> geom((size_t)ndir * c->nz);
    std::vector<RayDev<Real>> rays(ndir);
    for (int d = 0; d < ndir; ++d) {
        plane_geometry<Real>(c->nx, c->ny, c->nz, c->lx, c->ly, c->z.data(), mu[d], chi[d], geom.data() + (size_t)d * c->nz);
        rays[d] = ray_dev<Real>(mu[d], chi[d]);
    }
    const long long nxy = (long long)c->nx * c->ny;
    PlaneGeom<Real> *dg = nullptr;
    RayDev<Real> *dr = nullptr;
    double *scratch_out = nullptr;
    CK(dalloc(&dg, geom.size()));
    cudaError_t e2 = dalloc(&dr, rays.size());
    if (e2 == cudaSuccess && !dout) e2 = dalloc(&scratch_out, (size_t)ndir * c->n_nu * nxy * c->ns);
    int rc = PORTA_OK;
    do {
        if (e2 != cudaSuccess) { rc = fail(c, PORTA_ENOMEM, "emergent_vjp: device allocation"); break; }
        cudaError_t e = cudaMemcpyAsync(dg, geom.data(), geom.size() * sizeof(geom[0]), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dr, rays.data(), rays.size() * sizeof(rays[0]), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = ensure_buf(&c->d_tape, c->tape_bytes, (size_t)ndir * c->n_nu * c->nvox * c->ns * sizeof(Real));
        if (e != cudaSuccess) { rc = fail(c, PORTA_ENOMEM, std::string("emergent_vjp: ") + cudaGetErrorString(e)); break; }
        // forward: emergent Stokes and the Stokes vectors of every plane
        for (int k = 0; k < 3 && e == cudaSuccess; ++k)
            if (!c->adj_ev[k]) e = cudaEventCreate(&c->adj_ev[k]);
        if (e != cudaSuccess) { rc = fail(c, PORTA_ECUDA, std::string("emergent_vjp: ") + cudaGetErrorString(e)); break; }
        SweepArgs<Real> a = base_args<Real>(c);
        a.geom = dg;
        a.rays = dr;
        a.out = dout ? dout : scratch_out;
        a.store = (Real *)c->d_tape;
        LaunchCfg cfg{};
        rc = c->ns == 1 ? emergent_shape<Real, 1>(c, a, ndir, cfg) : emergent_shape<Real, 4>(c, a, ndir, cfg);
        if (rc) break;
        e = cudaEventRecord(c->adj_ev[0], c->stream);
        if (e == cudaSuccess)
            e = c->ns == 1 ? launch_sweep<Real, 1>(a, MODE_EMERGENT, cfg, c->stream)
                           : launch_sweep<Real, 4>(a, MODE_EMERGENT, cfg, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(c->adj_ev[1], c->stream);
        if (e != cudaSuccess) { rc = fail(c, PORTA_ECUDA, std::string("emergent_vjp forward: ") + cudaGetErrorString(e)); break; }
        // adjoint: launch shape forced, or timed once per direction count over
        // every fitting shape (each trial overwrites the same outputs)
        LaunchCfg acfg{};
        std::vector<LaunchCfg> cand;
        const bool forced = c->adj_cluster > 0 || c->adj_nu_group > 0;
        const bool tune = !forced && c->adj_tuned_ndir != ndir;
        rc = c->ns == 1 ? choose_adjoint<Real, 1>(c, acfg, c->adj_cluster, c->adj_nu_group, ndir, tune ? &cand : nullptr)
                        : choose_adjoint<Real, 4>(c, acfg, c->adj_cluster, c->adj_nu_group, ndir, tune ? &cand : nullptr);
        if (rc) { rc = fail(c, rc, "no adjoint launch shape fits this grid"); break; }
        if (!forced && !tune) acfg = c->adj_tuned;
        e = ensure_buf(&c->d_gpart, c->gpart_bytes, (size_t)ndir * c->n_nu * 3 * c->nvox * sizeof(Real));
        if (e != cudaSuccess) { rc = fail(c, PORTA_ENOMEM, "emergent_vjp: partial-gradient allocation"); break; }
        auto args_for = [&](LaunchCfg &k) {
            SweepArgs<Real> b = base_args<Real>(c);
            b.geom = dg;
            b.rays = dr;
            b.store = (Real *)c->d_tape;
            b.gout = dgrad;
            b.gpart = (Real *)c->d_gpart;
            b.F = k.F;
            b.ngroups = (c->n_nu + k.F - 1) / k.F;
            if (c->ns == 1)
                launch_caps<Real, 1>(c, k.cluster, b.ring_plane, b.ipts_max);
            else
                launch_caps<Real, 4>(c, k.cluster, b.ring_plane, b.ipts_max);
            b.nitems = ndir * b.ngroups;
            k.clusters = std::min(k.clusters, b.nitems);
            return b;
        };
        if (tune) {
            // the forward's time is read before the trials reuse the events
            e = cudaEventSynchronize(c->adj_ev[1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&c->adj_fwd_ms, c->adj_ev[0], c->adj_ev[1]);
            float best_ms = 1e30f;
            for (LaunchCfg k : cand) {
                SweepArgs<Real> b = args_for(k);
                float ms = 0;
                e = cudaEventRecord(c->adj_ev[1], c->stream);
                if (e == cudaSuccess)
                    e = c->ns == 1 ? launch_adjoint<Real, 1>(b, k, c->stream) : launch_adjoint<Real, 4>(b, k, c->stream);
                if (e == cudaSuccess) e = cudaEventRecord(c->adj_ev[2], c->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(c->adj_ev[2]);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->adj_ev[1], c->adj_ev[2]);
                if (e != cudaSuccess) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    acfg = k;
                }
            }
            if (e != cudaSuccess) { rc = fail(c, PORTA_ECUDA, std::string("emergent_vjp tuning: ") + cudaGetErrorString(e)); break; }
            c->adj_tuned = acfg;
            c->adj_tuned_ndir = ndir;
            e = cudaEventRecord(c->adj_ev[1], c->stream);
        }
        SweepArgs<Real> b = args_for(acfg);
        if (!dg_rho) {
            if (e == cudaSuccess)
                e = c->ns == 1 ? launch_adjoint<Real, 1>(b, acfg, c->stream) : launch_adjoint<Real, 4>(b, acfg, c->stream);
            if (e == cudaSuccess)
                e = launch_adjoint_reduce<Real>((const Real *)c->d_gpart, b.nitems, b.ngroups, c->nvox, dr,
                                                2.0 * c->gbar * c->zeta, dg_chi, dg_e, c->ns == 1 ? nullptr : dg_b, c->stream);
        } else {
            // gradients in the unknowns: per-cluster accumulators, then their sum
            if (e == cudaSuccess)
                e = ensure_buf((void **)&c->d_gacc, c->gacc_bytes, (size_t)acfg.clusters * 10 * c->nvox * sizeof(double));
            if (e == cudaSuccess) e = cudaMemsetAsync(c->d_gacc, 0, (size_t)acfg.clusters * 10 * c->nvox * sizeof(double), c->stream);
            b.gacc = c->d_gacc;
            if (e == cudaSuccess)
                e = c->ns == 1 ? launch_adjoint<Real, 1>(b, acfg, c->stream, 1) : launch_adjoint<Real, 4>(b, acfg, c->stream, 1);
            if (e == cudaSuccess)
                e = launch_adjoint_acc_reduce(c->d_gacc, acfg.clusters, c->nvox, c->nl, dg_chi, c->ns == 1 ? nullptr : dg_b,
                                              dg_rho, c->stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(c->adj_ev[2], c->stream);
        if (e != cudaSuccess) { rc = fail(c, PORTA_ECUDA, std::string("emergent_vjp adjoint: ") + cudaGetErrorString(e)); break; }
        c->last_adj = acfg;
        e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess && !tune) e = cudaEventElapsedTime(&c->adj_fwd_ms, c->adj_ev[0], c->adj_ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&c->adj_rev_ms, c->adj_ev[1], c->adj_ev[2]);
        if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, std::string("emergent_vjp: ") + cudaGetErrorString(e));
    } while (0);
    cudaStreamSynchronize(c->stream);
    pfree(dg);
    pfree(dr);
    if (scratch_out) pfree(scratch_out);
    return rc;
}

void mg_free(porta_ctx *c);
void it_free(porta_ctx *c);

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
                    c->d_items, c->d_tune_items, c->d_tape, c->d_gpart, c->d_jacc, c->d_jexp};
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


// ---------------------------------------------------------------- differentiation through iterations

// Gradients of sum g_J J^K_Q + sum g_L Lambda-bar* (the sums of a formal solution at
// the current rho) with respect to chi at fixed rho (added), B (added) and rho
// (overwritten). Rays in batches: the emergent-mode sweep over a batch's rays writes
// the tape, the adjoint (form 2) accumulates per cluster; one sum at the end.
template <typename Real>
int jkq_vjp_t(porta_ctx *c, const double *dgj, const double *dgl, double *dg_chi, double *dg_b, double *dg_rho)
{
    const long long nxy = (long long)c->nx * c->ny;
    const size_t per_ray = (size_t)c->n_nu * c->nvox * c->ns * sizeof(Real);
    // batches of equal size (the last one may be smaller) within the tape limit
    const int nbmax = (int)std::max<size_t>(1, std::min<size_t>(c->nray, c->tape_limit / per_ray));
    const int nbatch = (c->nray + nbmax - 1) / nbmax;
    const int nb = (c->nray + nbatch - 1) / nbatch;
    cudaError_t e = ensure_buf(&c->d_tape, c->tape_bytes, (size_t)nb * per_ray);
    double *scratch = nullptr;
    if (e == cudaSuccess) e = dalloc(&scratch, (size_t)nb * c->n_nu * nxy * c->ns);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        if (!c->it_ev[k]) e = cudaEventCreate(&c->it_ev[k]);
    if (e != cudaSuccess) {
        if (scratch) pfree(scratch);
        return fail(c, PORTA_ENOMEM, "iterate_vjp: tape allocation");
    }
    // adjoint launch shape: forced, else timed once per batch size on the first batch
    LaunchCfg acfg{};
    std::vector<LaunchCfg> cand;
    const bool forced = c->adj_cluster > 0 || c->adj_nu_group > 0;
    const bool tune = !forced && !c->adj2_tuned.count(nb);
    int rc = c->ns == 1 ? choose_adjoint<Real, 1>(c, acfg, c->adj_cluster, c->adj_nu_group, nb, tune ? &cand : nullptr)
                        : choose_adjoint<Real, 4>(c, acfg, c->adj_cluster, c->adj_nu_group, nb, tune ? &cand : nullptr);
    if (rc) {
        pfree(scratch);
        return fail(c, rc, "iterate_vjp: no adjoint launch shape fits");
    }
    if (!forced && !tune) acfg = c->adj2_tuned[nb];
    int maxcl = acfg.clusters;
    for (const LaunchCfg &k : cand) maxcl = std::max(maxcl, k.clusters);
    e = ensure_buf((void **)&c->d_gacc, c->gacc_bytes, (size_t)maxcl * 10 * c->nvox * sizeof(double));
    if (e != cudaSuccess) {
        pfree(scratch);
        return fail(c, PORTA_ENOMEM, "iterate_vjp: accumulator allocation");
    }
    // forward: Stokes vectors of every node for rays r0 .. r0 + n - 1
    auto forward = [&](int r0, int n) -> int {
        SweepArgs<Real> a = base_args<Real>(c);
        a.geom = (const PlaneGeom<Real> *)c->d_geom + (size_t)r0 * c->nz;
        a.rays = (const RayDev<Real> *)c->d_rays + r0;
        a.out = scratch;
        a.store = (Real *)c->d_tape;
        LaunchCfg cfg{};
        int r = c->ns == 1 ? emergent_shape<Real, 1>(c, a, n, cfg) : emergent_shape<Real, 4>(c, a, n, cfg);
        if (r) return r;
        e = c->ns == 1 ? launch_sweep<Real, 1>(a, MODE_EMERGENT, cfg, c->stream)
                       : launch_sweep<Real, 4>(a, MODE_EMERGENT, cfg, c->stream);
        return e == cudaSuccess ? PORTA_OK : fail(c, PORTA_ECUDA, std::string("iterate_vjp: ") + cudaGetErrorString(e));
    };
    // reverse: the J^K_Q and Lambda-bar* terms of the same rays
    auto reverse = [&](int r0, int n, LaunchCfg k) -> int {
        SweepArgs<Real> b = base_args<Real>(c);
        b.geom = (const PlaneGeom<Real> *)c->d_geom + (size_t)r0 * c->nz;
        b.rays = (const RayDev<Real> *)c->d_rays + r0;
        b.store = (Real *)c->d_tape;
        b.invn = (const Real *)c->d_invn;
        b.gjkq = dgj;
        b.glstar = dgl;
        b.tw = c->d_tw;
        b.ray0 = r0;
        b.gacc = c->d_gacc;
        b.F = k.F;
        b.ngroups = (c->n_nu + k.F - 1) / k.F;
        if (c->ns == 1)
            launch_caps<Real, 1>(c, k.cluster, b.ring_plane, b.ipts_max);
        else
            launch_caps<Real, 4>(c, k.cluster, b.ring_plane, b.ipts_max);
        b.nitems = n * b.ngroups;
        k.clusters = std::min(k.clusters, b.nitems);
        e = c->ns == 1 ? launch_adjoint<Real, 1>(b, k, c->stream, 2) : launch_adjoint<Real, 4>(b, k, c->stream, 2);
        return e == cudaSuccess ? PORTA_OK : fail(c, PORTA_ECUDA, std::string("iterate_vjp adjoint: ") + cudaGetErrorString(e));
    };
    cudaEvent_t *ev = c->it_ev;
    if (tune) {
        rc = forward(0, nb);
        float best = 1e30f;
        for (const LaunchCfg &k : cand) {
            if (rc) break;
            float ms = 0;
            e = cudaEventRecord(ev[0], c->stream);
            if (e == cudaSuccess) rc = reverse(0, nb, k);
            if (rc) break;
            e = cudaEventRecord(ev[1], c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (e != cudaSuccess) {
                rc = fail(c, PORTA_ECUDA, std::string("iterate_vjp tuning: ") + cudaGetErrorString(e));
                break;
            }
            if (ms < best) {
                best = ms;
                acfg = k;
            }
        }
        if (rc == PORTA_OK) c->adj2_tuned[nb] = acfg;
    }
    if (rc == PORTA_OK) {
        e = cudaMemsetAsync(c->d_gacc, 0, (size_t)acfg.clusters * 10 * c->nvox * sizeof(double), c->stream);
        if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, cudaGetErrorString(e));
    }
    for (int r0 = 0; r0 < c->nray && rc == PORTA_OK; r0 += nb) {
        const int n = std::min(nb, c->nray - r0);
        float t0 = 0, t1 = 0;
        e = cudaEventRecord(ev[0], c->stream);
        if (e == cudaSuccess) rc = forward(r0, n);
        if (rc) break;
        e = cudaEventRecord(ev[1], c->stream);
        if (e == cudaSuccess) rc = reverse(r0, n, acfg);
        if (rc) break;
        e = cudaEventRecord(ev[2], c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t0, ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, ev[1], ev[2]);
        if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, std::string("iterate_vjp: ") + cudaGetErrorString(e));
        c->it_ms[2] += t0;
        c->it_ms[3] += t1;
    }
    if (rc == PORTA_OK) {
        float t = 0;
        e = cudaEventRecord(ev[0], c->stream);
        if (e == cudaSuccess)
            e = launch_adjoint_acc_reduce(c->d_gacc, acfg.clusters, c->nvox, c->nl, dg_chi, c->ns == 1 ? nullptr : dg_b,
                                          dg_rho, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
        if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, std::string("iterate_vjp: ") + cudaGetErrorString(e));
        c->it_ms[4] += t;
        c->last_adj = acfg;
    }
    cudaStreamSynchronize(c->stream);
    pfree(scratch);
    return rc;
}

cudaError_t mg_rho_changed(porta_ctx *L);

void it_free(porta_ctx *c)
{
    for (double *b : c->it_saved) pfree(b);
    c->it_saved.clear();
    if (c->it_final) pfree(c->it_final);
    c->it_final = nullptr;
    c->it_niter = c->it_ckpt = 0;
}

int it_load(porta_ctx *c, const double *src)
{
    cudaError_t e = cudaMemcpyAsync(c->d_rho, src, sizeof(double) * c->nvox * c->nl, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = mg_rho_changed(c);
    if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("iterate: ") + cudaGetErrorString(e));
    c->have_rho = true;
    c->have_fs = c->have_jkq = false;
    return PORTA_OK;
}

template <typename Real>
int iterate_vjp_t(porta_ctx *c, int ndir, const double *mu, const double *chi, const double *dgrad, double *dout,
                  double *dg_chi, double *dg_f, double *dg_b)
{
    const size_t nr = (size_t)c->nvox * c->nl;
    double *blk = nullptr;
    // gbar (dL/drho of the current iterate), explicit part, dL/dJ, dL/dLambda*
    CK(dalloc(&blk, 3 * nr + c->nvox));
    double *gbar = blk, *gexp = blk + nr, *gj = blk + 2 * nr, *gl = blk + 3 * nr;
    int rc = PORTA_OK;
    cudaError_t e = cudaMemsetAsync(dg_chi, 0, sizeof(double) * c->nvox, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dg_f, 0, sizeof(double) * c->nvox, c->stream);
    if (e == cudaSuccess && dg_b) e = cudaMemsetAsync(dg_b, 0, sizeof(double) * 3 * c->nvox, c->stream);
    if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, cudaGetErrorString(e));
    // the loss: emergent Stokes of the final unknowns
    if (rc == PORTA_OK) rc = it_load(c, c->it_final);
    if (rc == PORTA_OK) rc = emergent_vjp_t<Real>(c, ndir, mu, chi, dgrad, dout, dg_chi, nullptr, dg_b, gbar);
    for (float &t : c->it_ms) t = 0.f;
    for (int k = 0; k < 4 && rc == PORTA_OK; ++k)
        if (!c->it_ev[k] && cudaEventCreate(&c->it_ev[k]) != cudaSuccess) rc = fail(c, PORTA_ECUDA, "iterate_vjp: events");
    cudaEvent_t *ev = c->it_ev;
    // The iterates of one checkpoint segment with their J^K_Q and Lambda-bar*:
    // each segment is rebuilt once from its checkpoint (ckpt formal solutions in
    // all, as many as the forward iterations) and its steps back read them from
    // here. Where that store exceeds the tape limit or the free device memory,
    // every step back rebuilds its iterate from the checkpoint instead
    // (ckpt (ckpt + 1) / 2 formal solutions per segment).
    const int nslot = std::min(c->it_ckpt, c->it_niter);
    const size_t nj = (size_t)c->nvox * c->nj, per_slot = nr + nj + c->nvox;
    double *seg = nullptr;
    const size_t seg_bytes = sizeof(double) * per_slot * nslot;
    if (rc == PORTA_OK && seg_bytes <= c->tape_limit && pmalloc(&seg, seg_bytes) != cudaSuccess) {
        cudaGetLastError();
        seg = nullptr;
    }
    auto slot = [&](int i) { return seg + per_slot * i; };
    auto save = [&](int i) {
        cudaError_t r = cudaMemcpyAsync(slot(i), c->d_rho, sizeof(double) * nr, cudaMemcpyDeviceToDevice, c->stream);
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(slot(i) + nr, c->d_jkq, sizeof(double) * nj, cudaMemcpyDeviceToDevice, c->stream);
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(slot(i) + nr + nj, c->d_lstar, sizeof(double) * c->nvox, cudaMemcpyDeviceToDevice,
                                c->stream);
        return r == cudaSuccess ? PORTA_OK : fail(c, PORTA_ECUDA, std::string("iterate_vjp: ") + cudaGetErrorString(r));
    };
    auto restore = [&](int i) {
        int r = it_load(c, slot(i));
        cudaError_t x = cudaSuccess;
        if (r == PORTA_OK)
            x = cudaMemcpyAsync(c->d_jkq, slot(i) + nr, sizeof(double) * nj, cudaMemcpyDeviceToDevice, c->stream);
        if (r == PORTA_OK && x == cudaSuccess)
            x = cudaMemcpyAsync(c->d_lstar, slot(i) + nr + nj, sizeof(double) * c->nvox, cudaMemcpyDeviceToDevice,
                                c->stream);
        if (r == PORTA_OK && x != cudaSuccess) r = fail(c, PORTA_ECUDA, std::string("iterate_vjp: ") + cudaGetErrorString(x));
        return r;
    };
    int seg_base = -1;
    for (int k = c->it_niter - 1; k >= 0 && rc == PORTA_OK; --k) {
        // the iterate rho_k with J^K_Q and Lambda-bar* at rho_k
        const int base = k / c->it_ckpt, b0 = base * c->it_ckpt;
        e = cudaEventRecord(ev[0], c->stream);
        if (seg && base == seg_base) {
            rc = restore(k - b0);
        } else {
            rc = it_load(c, c->it_saved[base]);
            for (int s = b0; s <= k && rc == PORTA_OK; ++s) {
                rc = porta_formal_solve(c);
                if (rc == PORTA_OK) rc = porta_accumulate_jkq(c, nullptr, nullptr, PORTA_DEVICE);
                if (rc == PORTA_OK && seg) rc = save(s - b0);
                if (rc == PORTA_OK && s < k) rc = porta_see_update(c, nullptr);
            }
            seg_base = seg ? base : -1;
        }
        if (rc) break;
        e = cudaEventRecord(ev[1], c->stream);
        // reverse mode of the update rho_{k+1} = U(rho_k, J, Lambda*, f, B)
        if (e == cudaSuccess)
            e = run_see_vjp(c->nvox, c->nl, c->model, c->bcrit, c->d_eps, c->d_bpl, c->d_b, c->d_jkq, c->d_lstar, nullptr,
                            c->d_rho, gbar, gexp, gj, gl, dg_f, dg_b, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2], c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
        float t0 = 0, t1 = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t0, ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, ev[1], ev[2]);
        if (e != cudaSuccess) { rc = fail(c, PORTA_ECUDA, std::string("iterate_vjp: ") + cudaGetErrorString(e)); break; }
        c->it_ms[0] += t0;
        c->it_ms[1] += t1;
        // ... and of J^K_Q, Lambda-bar* (gbar <- their gradient in rho_k), plus the explicit term
        rc = jkq_vjp_t<Real>(c, gj, gl, dg_chi, dg_b, gbar);
        if (rc) break;
        e = run_axpy((long long)nr, 1.0, gexp, gbar, c->stream);
        if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, std::string("iterate_vjp: ") + cudaGetErrorString(e));
    }
    // leave the context at the final unknowns
    int rc2 = it_load(c, c->it_final);
    cudaStreamSynchronize(c->stream);
    pfree(blk);
    if (seg) pfree(seg);
    return rc ? rc : rc2;
}

// ---------------------------------------------------------------- multigrid (Sec. 5)

int coarse_nz(int nz) { return nz % 2 ? (nz + 1) / 2 : nz / 2; }

void mg_free(porta_ctx *c)
{
    for (porta_ctx *L : c->mg) porta_destroy(L);
    c->mg.clear();
    double *bufs[] = {c->mg_res, c->mg_src, c->mg_rho0, c->mg_prev, c->mg_zr, c->mg_zp};
    for (double *b : bufs)
        if (b) pfree(b);
    c->mg_res = c->mg_src = c->mg_rho0 = c->mg_prev = c->mg_zr = c->mg_zp = nullptr;
}

// z tables between a level with heights zf and the next coarser one (coarse
// plane i = fine plane 2i): per fine plane (k0, w0, k1, w1) of the linear
// interpolation in height (extrapolation from the top two coarse planes above
// the coarse grid), and per coarse plane up to 4 (fine plane, weight) pairs of
// the transposed interpolation
void mg_ztables(const std::vector<double> &zf, std::vector<double> &zr, std::vector<double> &zp)
{
    const int nf = (int)zf.size(), nc = coarse_nz(nf);
    zp.assign(4 * (size_t)nf, 0.0);
    for (int k = 0; k < nf; ++k) {
        if (k % 2 == 0) {
            zp[4 * k] = zp[4 * k + 2] = k / 2;
            zp[4 * k + 1] = 1.0;
            continue;
        }
        int k0 = (k - 1) / 2;
        if (k0 + 1 >= nc) k0 = nc - 2;
        const int k1 = k0 + 1;
        const double t = (zf[k] - zf[2 * k0]) / (zf[2 * k1] - zf[2 * k0]);
        zp[4 * k] = k0;
        zp[4 * k + 1] = 1.0 - t;
        zp[4 * k + 2] = k1;
        zp[4 * k + 3] = t;
    }
    zr.assign(8 * (size_t)nc, 0.0);
    std::vector<int> used(nc, 0);
    for (int k = 0; k < nf; ++k)
        for (int e = 0; e < 2; ++e) {
            const double w = zp[4 * k + 2 * e + 1];
            if (w == 0.0) continue;
            const int K = (int)zp[4 * k + 2 * e];
            zr[8 * K + 2 * used[K]] = k;
            zr[8 * K + 2 * used[K] + 1] = w;
            ++used[K];
        }
}

// formal solution and J^K_Q / Lambda-bar* of one level, kept on the device
int mg_fs(porta_ctx *L)
{
    int rc = porta_formal_solve(L);
    if (rc == PORTA_OK) rc = porta_accumulate_jkq(L, nullptr, nullptr, PORTA_DEVICE);
    return rc;
}

cudaError_t ml_prepare(porta_ctx *c);

// the unknowns of a level: rho [v][nl] of the two-level atom, or the
// populations [v][nlevel] of the multilevel atom
double *mg_unk(porta_ctx *L) { return L->ml ? (L->ml->pol ? L->ml->d_x : L->ml->d_pops) : L->d_rho; }
long long mg_nunk(const porta_ctx *L) { return L->ml ? L->ml->nvox1 : L->nvox; }
int mg_ncomp(const porta_ctx *L) { return L->ml ? L->ml->nunk : L->nl; }

cudaError_t mg_rho_changed(porta_ctx *L)
{
    if (L->ml) return ml_prepare(L);
    return L->precision == PORTA_FP32 ? run_rho_convert<float>(L->nvox, L->nl, L->d_rho, L->d_rhoR, L->stream)
                                      : run_rho_convert<double>(L->nvox, L->nl, L->d_rho, L->d_rhoR, L->stream);
}

// out = alpha A(unknowns) + add + with_f f_fine, with J^K_Q of the last formal solution
cudaError_t mg_apply(porta_ctx *L, double alpha, const double *add, int with_f, double *out)
{
    if (L->ml && L->ml->pol)
        return run_mlpol_apply(L->ml->mc, L->ml->dev, L->ml->nvox1, L->ml->d_kT, L->d_jkq, L->d_b, L->ml->d_x, alpha, add,
                               with_f, out, L->stream);
    if (L->ml)
        return run_ml_apply(L->ml->mc, L->ml->nvox1, L->ml->d_kT, L->d_jkq, L->ml->d_pops, alpha, add, with_f, out,
                            L->stream);
    return run_see_apply(L->nvox, L->nl, L->model, L->bcrit, L->d_eps, L->d_bpl, L->d_b, L->d_jkq, L->d_rho, alpha,
                         add, with_f, out, L->stream);
}

// n Jacobi iterations of A(x) = src on one level (src null: the fine right-hand side)
int mg_jacobi(porta_ctx *L, const double *src, int n)
{
    for (int it = 0; it < n; ++it) {
        int rc = mg_fs(L);
        if (rc) return rc;
        cudaError_t e;
        if (L->ml) {
            e = L->ml->pol ? run_mlpol_see(L->ml->mc, L->ml->dev, L->ml->nvox1, L->ml->d_kT, L->d_jkq, L->d_lstar, L->d_b,
                                           L->ml->d_x, L->d_resid, L->ml->d_bad, L->stream, src)
                           : run_ml_see(L->ml->mc, L->ml->nvox1, L->ml->d_kT, L->d_jkq, L->d_lstar, L->ml->d_pops, L->d_resid,
                                        L->ml->d_bad, L->stream, src);
            if (e == cudaSuccess) e = ml_prepare(L);
        } else {
            e = L->precision == PORTA_FP32
                    ? run_see<float>(L->nvox, L->nl, L->model, L->bcrit, L->d_eps, L->d_bpl, L->d_b, L->d_jkq,
                                     L->d_lstar, L->d_rho, L->d_rhoR, L->d_resid, L->stream, src)
                    : run_see<double>(L->nvox, L->nl, L->model, L->bcrit, L->d_eps, L->d_bpl, L->d_b, L->d_jkq,
                                      L->d_lstar, L->d_rho, L->d_rhoR, L->d_resid, L->stream, src);
        }
        if (e != cudaSuccess) return fail(L, PORTA_ECUDA, std::string("mg jacobi: ") + cudaGetErrorString(e));
        L->have_fs = L->have_jkq = false;
    }
    return PORTA_OK;
}

// One V-cycle (Eqs. 30-34) from level l of levels[0..n) down to the coarsest.
int mg_vcycle(porta_ctx *const *levels, int n, int l, int npre, int npost, int ncoarse)
{
    porta_ctx *L = levels[l];
    const double *src = l == 0 ? nullptr : L->mg_src;
    if (l == n - 1) return mg_jacobi(L, src, ncoarse);
    int rc = mg_jacobi(L, src, npre);
    if (rc) return rc;
    // residual r = f - A(x)
    if ((rc = mg_fs(L))) return rc;
    cudaError_t e = mg_apply(L, -1.0, src, src ? 0 : 1, L->mg_res);
    porta_ctx *C = levels[l + 1];
    const int nc = mg_ncomp(L);
    // coarse unknowns R x, coarse right-hand side A_c(R x) + R r
    if (e == cudaSuccess)
        e = run_restrict(C->nx, C->ny, C->nz, L->nx, L->ny, nc, L->mg_zr, mg_unk(L), C->mg_rho0, L->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(mg_unk(C), C->mg_rho0, sizeof(double) * mg_nunk(C) * nc, cudaMemcpyDeviceToDevice, L->stream);
    if (e == cudaSuccess) e = mg_rho_changed(C);
    if (e == cudaSuccess)
        e = run_restrict(C->nx, C->ny, C->nz, L->nx, L->ny, nc, L->mg_zr, L->mg_res, C->mg_src, L->stream);
    if (e != cudaSuccess) return fail(L, PORTA_ECUDA, std::string("mg restrict: ") + cudaGetErrorString(e));
    C->have_rho = true;
    if (C->ml) C->ml->have_pops = true;
    if ((rc = mg_fs(C))) return fail(L, rc, std::string("mg coarse level: ") + C->err);
    e = mg_apply(C, 1.0, C->mg_src, 0, C->mg_src);
    if (e != cudaSuccess) return fail(L, PORTA_ECUDA, std::string("mg coarse rhs: ") + cudaGetErrorString(e));
    if ((rc = mg_vcycle(levels, n, l + 1, npre, npost, ncoarse))) return fail(L, rc, C->err);
    // coarse-grid correction x += P (x_c - R x)
    e = run_prolong_add(L->nx, L->ny, L->nz, C->nx, C->ny, nc, L->mg_zp, mg_unk(C), C->mg_rho0, mg_unk(L), L->stream);
    if (e == cudaSuccess) e = mg_rho_changed(L);
    if (e != cudaSuccess) return fail(L, PORTA_ECUDA, std::string("mg prolong: ") + cudaGetErrorString(e));
    return mg_jacobi(L, src, npost);
}

// line data of every line from the populations (sweep arrays of the line boxes)
cudaError_t ml_prepare(porta_ctx *c)
{
    MlState *m = c->ml;
    const size_t R = c->rsz;
    char *atm = (char *)c->d_atm;
    const long long n = c->nvox;
    if (m->pol) {
        if (c->precision == PORTA_FP32)
            return run_mlpol_prepare<float>(m->mc, m->dev, m->nvox1, m->d_x, m->d_chis, m->d_kT, (float *)atm,
                                            (float *)(atm + 5 * n * R), (float *)c->d_rhoR, c->d_rho,
                                            (float *)c->d_dich, m->d_bad, c->stream);
        return run_mlpol_prepare<double>(m->mc, m->dev, m->nvox1, m->d_x, m->d_chis, m->d_kT, (double *)atm,
                                         (double *)(atm + 5 * n * R), (double *)c->d_rhoR, c->d_rho,
                                         (double *)c->d_dich, m->d_bad, c->stream);
    }
    if (c->precision == PORTA_FP32)
        return run_ml_prepare<float>(m->mc, m->nvox1, m->d_pops, m->d_chis, m->d_kT, (float *)atm,
                                     (float *)(atm + 5 * n * R), (float *)c->d_rhoR, c->d_rho, m->d_bad, c->stream);
    return run_ml_prepare<double>(m->mc, m->nvox1, m->d_pops, m->d_chis, m->d_kT, (double *)atm,
                                  (double *)(atm + 5 * n * R), (double *)c->d_rhoR, c->d_rho, m->d_bad, c->stream);
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
        e = run_mlpol_see(m->mc, m->dev, m->nvox1, m->d_kT, c->d_jkq, c->d_lstar, c->d_b, m->d_x, c->d_resid, m->d_bad,
                          c->stream);
    else
        e = run_ml_see(m->mc, m->nvox1, m->d_kT, c->d_jkq, c->d_lstar, m->d_pops, c->d_resid, m->d_bad, c->stream);
    if (e != cudaSuccess) return e;
    return ml_prepare(c);
}

}  // namespace

extern "C" {

static int create_impl(int nbox, const porta_grid *grids, const porta_atom *at, const porta_quad *q,
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
    c->opt_cluster = o ? o->cluster : 0;
    c->opt_nu_group = o ? o->nu_group : 0;
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
    std::vector<double> xg, wg;
    gauss_legendre(q->n_mu, xg, wg);
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
            rc = PORTA_EINVAL;
            c->err = "no sweep launch shape fits this grid (nx too large for shared memory)";
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

int porta_emergent_stokes(porta_ctx *c, int ndir, const double *mu, const double *chi, double *out, int where)
{
    if (!c) return PORTA_EINVAL;
    if (ndir < 1 || !mu || !chi || !out || (where != PORTA_HOST && where != PORTA_DEVICE))
        return fail(c, PORTA_EINVAL, "emergent_stokes: bad argument");
    for (int d = 0; d < ndir; ++d)
        if (!(mu[d] > 0.0 && mu[d] <= 1.0) || !std::isfinite(chi[d]))
            return fail(c, PORTA_EINVAL, "emergent_stokes: mu must lie in (0, 1], chi finite");
    if (c->nbox != 1) return fail(c, PORTA_EINVAL, "emergent_stokes: single-box contexts only");
    if (!c->have_atm || !c->have_rho) return fail(c, PORTA_ESTATE, "emergent_stokes: atmosphere or rho not set");
    const long long n = (long long)ndir * c->n_nu * c->nx * c->ny * c->ns;
    double *dout = out;
    if (where == PORTA_HOST) CK(dalloc(&dout, n));
    int rc = c->precision == PORTA_FP32 ? emergent_t<float>(c, ndir, mu, chi, dout) : emergent_t<double>(c, ndir, mu, chi, dout);
    if (where == PORTA_HOST) {
        if (rc == PORTA_OK) {
            cudaError_t e = cudaMemcpy(out, dout, n * sizeof(double), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, cudaGetErrorString(e));
        }
        pfree(dout);
    }
    return rc;
}

int porta_emergent_vjp(porta_ctx *c, int ndir, const double *mu, const double *chi, const double *grad_out,
                       double *out, double *g_chi, double *g_e, double *g_b, int where)
{
    if (!c) return PORTA_EINVAL;
    if (ndir < 1 || !mu || !chi || !grad_out || !g_chi || !g_e || (c->ns > 1 && !g_b) ||
        (where != PORTA_HOST && where != PORTA_DEVICE))
        return fail(c, PORTA_EINVAL, "emergent_vjp: bad argument");
    for (int d = 0; d < ndir; ++d)
        if (!(mu[d] > 0.0 && mu[d] <= 1.0) || !std::isfinite(chi[d]))
            return fail(c, PORTA_EINVAL, "emergent_vjp: mu must lie in (0, 1], chi finite");
    if (c->nbox != 1) return fail(c, PORTA_EINVAL, "emergent_vjp: single-box contexts only");
    if (!c->have_atm || !c->have_rho) return fail(c, PORTA_ESTATE, "emergent_vjp: atmosphere or rho not set");
    const long long nout = (long long)ndir * c->n_nu * c->nx * c->ny * c->ns;
    const long long nv = c->nvox;
    if (where == PORTA_DEVICE)
        return c->precision == PORTA_FP32 ? emergent_vjp_t<float>(c, ndir, mu, chi, grad_out, out, g_chi, g_e, g_b)
                                          : emergent_vjp_t<double>(c, ndir, mu, chi, grad_out, out, g_chi, g_e, g_b);
    // host buffers: one device block for grad_out, out, g_chi, g_e, g_b
    const long long nb = c->ns > 1 ? 3 * nv : 0;
    double *blk = nullptr;
    CK(dalloc(&blk, (size_t)(nout + (out ? nout : 0) + 2 * nv + nb)));
    double *dgrad = blk, *dout = out ? blk + nout : nullptr;
    double *dchi = blk + nout + (out ? nout : 0), *de = dchi + nv, *db = nb ? de + nv : nullptr;
    int rc = PORTA_OK;
    cudaError_t e = cudaMemcpy(dgrad, grad_out, nout * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, cudaGetErrorString(e));
    if (rc == PORTA_OK)
        rc = c->precision == PORTA_FP32 ? emergent_vjp_t<float>(c, ndir, mu, chi, dgrad, dout, dchi, de, db)
                                        : emergent_vjp_t<double>(c, ndir, mu, chi, dgrad, dout, dchi, de, db);
    if (rc == PORTA_OK) {
        e = cudaMemcpy(g_chi, dchi, nv * sizeof(double), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(g_e, de, nv * sizeof(double), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && db) e = cudaMemcpy(g_b, db, 3 * nv * sizeof(double), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && out) e = cudaMemcpy(out, dout, nout * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, cudaGetErrorString(e));
    }
    pfree(blk);
    return rc;
}

int porta_iterate_ckpt(porta_ctx *c, int niter, int ckpt, double *max_change)
{
    if (!c) return PORTA_EINVAL;
    if (c->ml) return fail(c, PORTA_EINVAL, "iterate_ckpt: not for a multilevel context (porta_ml_*)");
    if (niter < 1 || ckpt < 1) return fail(c, PORTA_EINVAL, "iterate_ckpt: niter >= 1, ckpt >= 1");
    if (c->nbox != 1) return fail(c, PORTA_EINVAL, "iterate_ckpt: single-box contexts only");
    if (!c->have_atm || !c->have_rho) return fail(c, PORTA_ESTATE, "iterate_ckpt: atmosphere or rho not set");
    it_free(c);
    const size_t nr = (size_t)c->nvox * c->nl;
    const int nsave = (niter + ckpt - 1) / ckpt;
    for (int i = 0; i <= nsave; ++i) {
        double *b = nullptr;
        cudaError_t e = dalloc(&b, nr);
        if (e != cudaSuccess) {
            it_free(c);
            return fail(c, PORTA_ENOMEM, "iterate_ckpt: checkpoint allocation");
        }
        if (i < nsave)
            c->it_saved.push_back(b);
        else
            c->it_final = b;
    }
    int rc = PORTA_OK;
    for (int k = 0; k < niter && rc == PORTA_OK; ++k) {
        if (k % ckpt == 0) {
            cudaError_t e = cudaMemcpyAsync(c->it_saved[k / ckpt], c->d_rho, sizeof(double) * nr, cudaMemcpyDeviceToDevice,
                                            c->stream);
            if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, std::string("iterate_ckpt: ") + cudaGetErrorString(e));
        }
        if (rc == PORTA_OK) rc = porta_formal_solve(c);
        if (rc == PORTA_OK) rc = porta_accumulate_jkq(c, nullptr, nullptr, PORTA_DEVICE);
        if (rc == PORTA_OK) rc = porta_see_update(c, k == niter - 1 ? max_change : nullptr);
    }
    if (rc == PORTA_OK) {
        cudaError_t e = cudaMemcpyAsync(c->it_final, c->d_rho, sizeof(double) * nr, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, std::string("iterate_ckpt: ") + cudaGetErrorString(e));
    }
    if (rc) {
        it_free(c);
        return rc;
    }
    c->it_niter = niter;
    c->it_ckpt = ckpt;
    return PORTA_OK;
}

int porta_iterate_timing(const porta_ctx *c, float *ms)
{
    if (!c || !ms) return PORTA_EINVAL;
    for (int k = 0; k < 5; ++k) ms[k] = c->it_ms[k];
    return PORTA_OK;
}

int porta_set_tape_limit(porta_ctx *c, long long bytes)
{
    if (!c) return PORTA_EINVAL;
    if (bytes < 0) return fail(c, PORTA_EINVAL, "set_tape_limit: bytes >= 0");
    c->tape_limit = bytes ? (size_t)bytes : (size_t)16 << 30;
    return PORTA_OK;
}

int porta_iterate_vjp(porta_ctx *c, int ndir, const double *mu, const double *chi, const double *grad_out, double *out,
                      double *g_chi, double *g_f, double *g_b, int where)
{
    if (!c) return PORTA_EINVAL;
    if (ndir < 1 || !mu || !chi || !grad_out || !g_chi || !g_f || (c->ns > 1 && !g_b) ||
        (where != PORTA_HOST && where != PORTA_DEVICE))
        return fail(c, PORTA_EINVAL, "iterate_vjp: bad argument");
    for (int d = 0; d < ndir; ++d)
        if (!(mu[d] > 0.0 && mu[d] <= 1.0) || !std::isfinite(chi[d]))
            return fail(c, PORTA_EINVAL, "iterate_vjp: mu must lie in (0, 1], chi finite");
    if (c->it_niter < 1) return fail(c, PORTA_ESTATE, "iterate_vjp: call porta_iterate_ckpt first");
    if (c->ns == 1) g_b = nullptr;
    const long long nout = (long long)ndir * c->n_nu * c->nx * c->ny * c->ns;
    const long long nv = c->nvox;
    auto run = [&](const double *dgrad, double *dout, double *dchi, double *df, double *db) {
        return c->precision == PORTA_FP32 ? iterate_vjp_t<float>(c, ndir, mu, chi, dgrad, dout, dchi, df, db)
                                          : iterate_vjp_t<double>(c, ndir, mu, chi, dgrad, dout, dchi, df, db);
    };
    if (where == PORTA_DEVICE) return run(grad_out, out, g_chi, g_f, g_b);
    const long long nb = g_b ? 3 * nv : 0;
    double *blk = nullptr;
    CK(dalloc(&blk, (size_t)(nout + (out ? nout : 0) + 2 * nv + nb)));
    double *dgrad = blk, *dout = out ? blk + nout : nullptr;
    double *dchi = blk + nout + (out ? nout : 0), *df = dchi + nv, *db = nb ? df + nv : nullptr;
    int rc = PORTA_OK;
    cudaError_t e = cudaMemcpy(dgrad, grad_out, nout * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, cudaGetErrorString(e));
    if (rc == PORTA_OK) rc = run(dgrad, dout, dchi, df, db);
    if (rc == PORTA_OK) {
        e = cudaMemcpy(g_chi, dchi, nv * sizeof(double), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(g_f, df, nv * sizeof(double), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && db) e = cudaMemcpy(g_b, db, 3 * nv * sizeof(double), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && out) e = cudaMemcpy(out, dout, nout * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, cudaGetErrorString(e));
    }
    pfree(blk);
    return rc;
}

int porta_set_adjoint_launch(porta_ctx *c, int cluster, int nu_group)
{
    if (!c) return PORTA_EINVAL;
    if (cluster < 0 || cluster > 16 || nu_group < 0 || nu_group > c->n_nu)
        return fail(c, PORTA_EINVAL, "set_adjoint_launch: cluster in 0..16, nu_group in 0..n_nu");
    if (cluster > c->ny) return fail(c, PORTA_EINVAL, "set_adjoint_launch: cluster larger than ny");
    c->adj_cluster = cluster;
    c->adj_nu_group = nu_group;
    c->adj_tuned_ndir = 0;
    c->adj2_tuned.clear();
    return PORTA_OK;
}

int porta_adjoint_timing(const porta_ctx *c, float *forward_ms, float *adjoint_ms)
{
    if (!c) return PORTA_EINVAL;
    if (forward_ms) *forward_ms = c->adj_fwd_ms;
    if (adjoint_ms) *adjoint_ms = c->adj_rev_ms;
    return PORTA_OK;
}

int porta_adjoint_info(const porta_ctx *c, int *clusters, int *cluster_size, int *nu_group, int *smem_bytes)
{
    if (!c) return PORTA_EINVAL;
    if (clusters) *clusters = c->last_adj.clusters;
    if (cluster_size) *cluster_size = c->last_adj.cluster;
    if (nu_group) *nu_group = c->last_adj.F;
    if (smem_bytes) *smem_bytes = c->last_adj.smem;
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
    if (elements) *elements = (long long)(c->nj + 1) * c->nvox;
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


static int ml_check(porta_ctx *c, const char *what);

int porta_mg_setup(porta_ctx *c, int nlevels)
{
    if (!c) return PORTA_EINVAL;
    if (c->nbox != 1 && !c->ml) return fail(c, PORTA_EINVAL, "mg_setup: single-box contexts only");
    if (c->ml && !c->ml->have_atm) return fail(c, PORTA_ESTATE, "mg_setup: atmosphere not set");
    if (nlevels < 2 || nlevels > 8) return fail(c, PORTA_EINVAL, "mg_setup: nlevels in 2..8");
    if (!c->have_atm) return fail(c, PORTA_ESTATE, "mg_setup: atmosphere not set");
    {
        int nx = c->nx, ny = c->ny, nz = c->nz;
        for (int l = 1; l < nlevels; ++l) {
            if (nx % 2 || ny % 2)
                return fail(c, PORTA_EINVAL, "mg_setup: nx and ny must be divisible by 2^(nlevels-1)");
            nx /= 2;
            ny /= 2;
            nz = coarse_nz(nz);
            if (nz < 2) return fail(c, PORTA_EINVAL, "mg_setup: too many levels for nz");
        }
    }
    mg_free(c);
    porta_ctx *F = c;
    int rc = PORTA_OK;
    for (int l = 1; l < nlevels && rc == PORTA_OK; ++l) {
        const int nzc = coarse_nz(F->nz);
        std::vector<double> zc(nzc);
        for (int k = 0; k < nzc; ++k) zc[k] = F->z[2 * k];
        porta_grid g{};
        g.nx = F->nx / 2;
        g.ny = F->ny / 2;
        g.nz = nzc;
        g.lx = c->lx;
        g.ly = c->ly;
        g.z = zc.data();
        porta_atom a{};
        a.model = c->model;
        a.zeta = c->zeta;
        a.gbar = c->gbar;
        a.bcrit = c->bcrit;
        porta_quad q{};
        q.n_mu = c->n_mu;
        q.n_chi = c->n_chi;
        q.n_nu = c->n_nu;
        q.x_max = c->x_max;
        porta_opts o{};
        o.precision = c->precision;
        porta_ctx *L = nullptr;
        if (c->ml) {
            // multilevel: a coarse multilevel context of the same atom; its opacity
            // scale, temperature and velocity at the coincident nodes
            const MlState *m = c->ml;
            porta_ml_atom ma{m->mc.nlev, m->mc.nline, m->J.data(), m->E.data(), m->up.data(), m->lo.data(),
                             m->A.data(), m->eps.data(), m->pol ? 1 : 0, c->zeta};
            if ((rc = porta_ml_create(&g, &ma, &q, &o, &L))) {
                rc = fail(c, rc, "mg_setup: coarse level creation");
                break;
            }
            c->mg.push_back(L);
            porta_set_stream(L, c->stream);
            const MlState *mf = F->ml;
            const long long ncv = L->ml->nvox1;
            double *tmp = nullptr;
            cudaError_t e = dalloc(&tmp, 6 * (size_t)ncv);
            // F->d_cv64 + F->nvox: FP64 velocity of the line boxes (box 0 first); F->d_b the field
            const double *srcs[6] = {mf->d_chis, mf->d_kT, F->d_cv64 + F->nvox, F->d_b, F->d_b + F->nvox,
                                     F->d_b + 2 * F->nvox};
            for (int f = 0; f < (m->pol ? 6 : 3) && e == cudaSuccess; ++f)
                e = run_inject(L->nx, L->ny, L->nz, F->nx, F->ny, srcs[f], tmp + f * ncv, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) {
                pfree(tmp);
                rc = fail(c, PORTA_ECUDA, std::string("mg_setup: ") + cudaGetErrorString(e));
                break;
            }
            rc = porta_ml_set_atmosphere(L, tmp, tmp + ncv, tmp + 2 * ncv, m->pol ? tmp + 3 * ncv : nullptr,
                                         m->pol ? tmp + 4 * ncv : nullptr, m->pol ? tmp + 5 * ncv : nullptr, PORTA_DEVICE);
            pfree(tmp);
            if (rc) {
                rc = fail(c, rc, std::string("mg_setup: coarse atmosphere: ") + L->err);
                break;
            }
            std::vector<double> zr, zp;
            mg_ztables(F->z, zr, zp);
            const int nl = mg_ncomp(c);
            e = dalloc(&L->mg_src, (size_t)ncv * nl);
            if (e == cudaSuccess) e = dalloc(&L->mg_rho0, (size_t)ncv * nl);
            if (e == cudaSuccess) e = dalloc(&L->mg_res, (size_t)ncv * nl);
            if (e == cudaSuccess) e = dalloc(&F->mg_zr, zr.size());
            if (e == cudaSuccess) e = dalloc(&F->mg_zp, zp.size());
            if (e == cudaSuccess) e = cudaMemcpy(F->mg_zr, zr.data(), zr.size() * sizeof(double), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(F->mg_zp, zp.data(), zp.size() * sizeof(double), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                rc = fail(c, PORTA_ENOMEM, "mg_setup: allocation");
                break;
            }
            F = L;
            continue;
        }
        if ((rc = porta_create(&g, &a, &q, &o, &L))) {
            rc = fail(c, rc, "mg_setup: coarse level creation");
            break;
        }
        c->mg.push_back(L);
        porta_set_stream(L, c->stream);
        // coarse atmosphere: the finer level's values at the coincident nodes
        const long long nf = F->nvox, ncv = L->nvox;
        double *tmp = nullptr;
        cudaError_t e = dalloc(&tmp, 7 * (size_t)ncv);
        const double *src[7] = {F->d_cv64, F->d_eps, F->d_bpl, F->d_cv64 + nf, F->d_b, F->d_b + nf, F->d_b + 2 * nf};
        for (int f = 0; f < 7 && e == cudaSuccess; ++f)
            e = run_inject(L->nx, L->ny, L->nz, F->nx, F->ny, src[f], tmp + f * ncv, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            pfree(tmp);
            rc = fail(c, PORTA_ECUDA, std::string("mg_setup: ") + cudaGetErrorString(e));
            break;
        }
        porta_atmos at{};
        at.chi = tmp;
        at.eps = tmp + ncv;
        at.bpl = tmp + 2 * ncv;
        at.vel = tmp + 3 * ncv;
        at.bx = tmp + 4 * ncv;
        at.by = tmp + 5 * ncv;
        at.bz = tmp + 6 * ncv;
        rc = porta_set_atmosphere(L, &at, PORTA_DEVICE);
        pfree(tmp);
        if (rc) {
            rc = fail(c, rc, std::string("mg_setup: coarse atmosphere: ") + L->err);
            break;
        }
        std::vector<double> zr, zp;
        mg_ztables(F->z, zr, zp);
        e = dalloc(&L->mg_src, (size_t)ncv * c->nl);
        if (e == cudaSuccess) e = dalloc(&L->mg_rho0, (size_t)ncv * c->nl);
        if (e == cudaSuccess) e = dalloc(&L->mg_res, (size_t)ncv * c->nl);
        if (e == cudaSuccess) e = dalloc(&F->mg_zr, zr.size());
        if (e == cudaSuccess) e = dalloc(&F->mg_zp, zp.size());
        if (e == cudaSuccess) e = cudaMemcpy(F->mg_zr, zr.data(), zr.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(F->mg_zp, zp.data(), zp.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            rc = fail(c, PORTA_ENOMEM, "mg_setup: allocation");
            break;
        }
        F = L;
    }
    if (rc == PORTA_OK) {
        cudaError_t e = dalloc(&c->mg_res, (size_t)mg_nunk(c) * mg_ncomp(c));
        if (e == cudaSuccess) e = dalloc(&c->mg_prev, (size_t)mg_nunk(c) * mg_ncomp(c));
        if (e != cudaSuccess) rc = fail(c, PORTA_ENOMEM, "mg_setup: allocation");
    }
    if (rc) mg_free(c);
    return rc;
}

int porta_mg_levels(const porta_ctx *c, int *nlevels, int *shapes)
{
    if (!c) return PORTA_EINVAL;
    if (nlevels) *nlevels = c->mg.empty() ? 0 : 1 + (int)c->mg.size();
    if (shapes && !c->mg.empty()) {
        shapes[0] = c->nx;
        shapes[1] = c->ny;
        shapes[2] = c->nz;
        for (size_t l = 0; l < c->mg.size(); ++l) {
            shapes[3 * (l + 1)] = c->mg[l]->nx;
            shapes[3 * (l + 1) + 1] = c->mg[l]->ny;
            shapes[3 * (l + 1) + 2] = c->mg[l]->nz;
        }
    }
    return PORTA_OK;
}

int porta_residual(porta_ctx *c, double *rnorm)
{
    if (!c || !rnorm) return PORTA_EINVAL;
    if (!c->have_atm || !c->have_rho) return fail(c, PORTA_ESTATE, "residual: atmosphere or unknowns not set");
    if (c->ml && !c->ml->have_pops) return fail(c, PORTA_ESTATE, "residual: populations not set");
    if (c->fr1 > c->fr0) return fail(c, PORTA_ESTATE, "residual: needs the whole frequency grid");
    const long long nu = mg_nunk(c);
    const int nc = mg_ncomp(c);
    double *r = nullptr;
    cudaError_t e = pmalloc(&r, sizeof(double) * nu * nc);
    if (e != cudaSuccess) return fail(c, PORTA_ENOMEM, "residual: allocation");
    int rc = mg_fs(c);
    if (rc == PORTA_OK) {
        e = mg_apply(c, -1.0, nullptr, 1, r);                    // r = f - A(x)
        if (e == cudaSuccess) e = cudaMemsetAsync(c->d_resid, 0, sizeof(unsigned long long), c->stream);
        if (e == cudaSuccess) e = run_rel_residual(nu, nc, r, mg_unk(c), c->d_resid, c->stream);
        unsigned long long bits = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, c->d_resid, sizeof(bits), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess) std::memcpy(rnorm, &bits, sizeof(double));
        else rc = fail(c, PORTA_ECUDA, std::string("residual: ") + cudaGetErrorString(e));
    }
    pfree(r);
    c->have_fs = c->have_jkq = false;
    return rc;
}

int porta_mg_vcycle(porta_ctx *c, int npre, int npost, int ncoarse, double *max_change)
{
    if (!c) return PORTA_EINVAL;
    if (c->mg.empty()) return fail(c, PORTA_ESTATE, "mg_vcycle: call porta_mg_setup first");
    if (!c->have_atm || !c->have_rho) return fail(c, PORTA_ESTATE, "mg_vcycle: atmosphere or rho not set");
    if (npre < 0 || npost < 0 || ncoarse < 1) return fail(c, PORTA_EINVAL, "mg_vcycle: npre, npost >= 0, ncoarse >= 1");
    std::vector<porta_ctx *> levels{c};
    for (porta_ctx *L : c->mg) {
        L->stream = c->stream;
        levels.push_back(L);
    }
    if (c->ml && !c->ml->have_pops) return fail(c, PORTA_ESTATE, "mg_vcycle: populations not set");
    const long long nu = mg_nunk(c);
    const int nc = mg_ncomp(c);
    CK(cudaMemcpyAsync(c->mg_prev, mg_unk(c), sizeof(double) * nu * nc, cudaMemcpyDeviceToDevice, c->stream));
    int rc = mg_vcycle(levels.data(), (int)levels.size(), 0, npre, npost, ncoarse);
    if (rc) return rc;
    c->have_fs = c->have_jkq = false;
    CK(cudaMemsetAsync(c->d_resid, 0, sizeof(unsigned long long), c->stream));
    cudaError_t e = c->ml && c->ml->pol
                        ? run_mlpol_change(c->ml->mc, c->ml->dev, nu, c->mg_prev, mg_unk(c), c->d_resid, c->stream)
                        : run_change(nu, nc, c->mg_prev, mg_unk(c), c->d_resid, c->stream, c->ml ? 1 : 0);
    if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("mg_vcycle: ") + cudaGetErrorString(e));
    if (max_change) {
        unsigned long long bits = 0;
        CK(cudaMemcpyAsync(&bits, c->d_resid, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        std::memcpy(max_change, &bits, sizeof(double));
    }
    if (c->ml) {
        for (porta_ctx *L : levels)
            if ((rc = ml_check(L, "mg_vcycle"))) return L == c ? rc : fail(c, rc, L->err);
    }
    return PORTA_OK;
}

// ---------------------------------------------------------------- multilevel atom (Sec. 1)

int porta_ml_create(const porta_grid *g, const porta_ml_atom *a, const porta_quad *q, const porta_opts *o,
                    porta_ctx **out)
{
    if (!out) return PORTA_EINVAL;
    *out = nullptr;
    if (!g || !a || !q || !a->J || !a->E || !a->upper || !a->lower || !a->A || !a->eps) return PORTA_EINVAL;
    if (a->nlevel < 2 || a->nlevel > kMlMaxLevel || a->nline < 1 || a->nline > kMlMaxLine) return PORTA_EINVAL;
    MlConst mc{};
    mc.nlev = a->nlevel;
    mc.nline = a->nline;
    for (int i = 0; i < a->nlevel; ++i) {
        const double j2 = 2.0 * a->J[i];
        if (!(a->J[i] >= 0.0) || j2 != std::floor(j2) || j2 > 64 || !std::isfinite(a->E[i])) return PORTA_EINVAL;
        mc.g[i] = j2 + 1.0;
    }
    for (int k = 0; k < a->nline; ++k) {
        const int u = a->upper[k], l = a->lower[k];
        if (u < 0 || u >= a->nlevel || l < 0 || l >= a->nlevel || !(a->E[u] > a->E[l])) return PORTA_EINVAL;
        if (!(a->A[k] > 0.0) || !std::isfinite(a->A[k]) || !(a->eps[k] > 0.0 && a->eps[k] < 1.0)) return PORTA_EINVAL;
        mc.up[k] = u;
        mc.lo[k] = l;
        mc.A[k] = a->A[k];
        mc.dE[k] = a->E[u] - a->E[l];
        mc.Cul[k] = a->eps[k] / (1.0 - a->eps[k]) * a->A[k];
    }
    // intensities in units of 2 h nu^3 / c^2 of line 0; opacity strengths relative to line 0
    for (int k = 0; k < a->nline; ++k) {
        const double r = mc.dE[k] / mc.dE[0];
        mc.r3[k] = r * r * r;
        mc.Bul[k] = mc.A[k] / mc.r3[k];
        mc.Blu[k] = mc.g[mc.up[k]] / mc.g[mc.lo[k]] * mc.Bul[k];
        mc.s[k] = mc.g[mc.up[k]] / mc.g[mc.lo[k]] * mc.A[k] / (mc.dE[k] * mc.dE[k]);
    }
    for (int k = a->nline - 1; k >= 0; --k) mc.s[k] /= mc.s[0];
    if (a->polarized != 0 && a->polarized != 1) return PORTA_EINVAL;
    if (a->polarized && !(a->zeta >= 0.0 && std::isfinite(a->zeta))) return PORTA_EINVAL;
    MlPolTables tab;
    if (a->polarized) {
        std::vector<double> J(a->J, a->J + a->nlevel), E(a->E, a->E + a->nlevel), A(a->A, a->A + a->nline),
            eps(a->eps, a->eps + a->nline);
        std::vector<int> up(a->upper, a->upper + a->nline), lo(a->lower, a->lower + a->nline);
        if (mlpol_tables(J, E, up, lo, A, eps, tab)) return PORTA_EINVAL;
    }
    std::vector<porta_grid> grids(a->nline, *g);
    porta_atom at{a->polarized ? PORTA_MODEL_TWOLEVEL_HANLE : PORTA_MODEL_TWOLEVEL_UNPOL,
                  a->polarized ? a->zeta : 0.0, 1.0, 25.0};
    porta_ctx *c = nullptr;
    int rc = create_impl(a->nline, grids.data(), &at, q, o, &c);
    if (rc) return rc;
    MlState *m = new (std::nothrow) MlState();
    if (!m) {
        porta_destroy(c);
        return PORTA_ENOMEM;
    }
    c->ml = m;
    m->mc = mc;
    m->J.assign(a->J, a->J + a->nlevel);
    m->E.assign(a->E, a->E + a->nlevel);
    m->A.assign(a->A, a->A + a->nline);
    m->eps.assign(a->eps, a->eps + a->nline);
    m->up.assign(a->upper, a->upper + a->nline);
    m->lo.assign(a->lower, a->lower + a->nline);
    m->nvox1 = (long long)g->nx * g->ny * g->nz;
    cudaError_t e = dalloc(&m->d_pops, (size_t)m->nvox1 * mc.nlev);
    if (e == cudaSuccess) e = dalloc(&m->d_chis, (size_t)m->nvox1);
    if (e == cudaSuccess) e = dalloc(&m->d_kT, (size_t)m->nvox1);
    if (e == cudaSuccess) e = pmalloc(&m->d_bad, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(m->d_bad, 0, sizeof(unsigned long long));
    m->nunk = mc.nlev;
    if (e == cudaSuccess && a->polarized) {
        // the tables in one device allocation: ints first, then doubles (8-byte aligned)
        m->pol = true;
        m->tab = tab;
        m->nunk = tab.nunk;
        const size_t ni = tab.pop_idx.size() + tab.up2.size() + tab.cell_rc.size() + tab.cell_start.size() +
                          tab.ent_src.size() + tab.act.size() + tab.inact.size() + tab.apop.size() + tab.lo2.size();
        const size_t nd = tab.w2.size() + tab.trace.size() + tab.ent_coef.size() + tab.w2lo.size();
        const size_t ibytes = (ni * sizeof(int) + 7) / 8 * 8;
        std::vector<char> h(ibytes + nd * sizeof(double));
        int *ip = (int *)h.data();
        double *dp = (double *)(h.data() + ibytes);
        size_t io[9], doff[4], k = 0, kd = 0;
        const std::vector<int> *iv[9] = {&tab.pop_idx, &tab.up2, &tab.cell_rc, &tab.cell_start, &tab.ent_src,
                                         &tab.act, &tab.inact, &tab.apop, &tab.lo2};
        for (int q2 = 0; q2 < 9; ++q2) {
            io[q2] = k;
            for (int x : *iv[q2]) ip[k++] = x;
        }
        const std::vector<double> *dv[4] = {&tab.w2, &tab.trace, &tab.ent_coef, &tab.w2lo};
        for (int q2 = 0; q2 < 4; ++q2) {
            doff[q2] = kd;
            for (double x : *dv[q2]) dp[kd++] = x;
        }
        e = pmalloc(&m->d_tab, h.size());
        if (e == cudaSuccess) e = cudaMemcpy(m->d_tab, h.data(), h.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = dalloc(&m->d_x, (size_t)m->nvox1 * tab.nunk);
        if (e == cudaSuccess) e = pmalloc(&c->d_dich, (size_t)5 * c->nvox * c->rsz);
        if (e == cudaSuccess) e = cudaMemset(c->d_dich, 0, (size_t)5 * c->nvox * c->rsz);
        const int *di = (const int *)m->d_tab;
        const double *dd = (const double *)((const char *)m->d_tab + ibytes);
        MlPolDev &d = m->dev;
        d.nunk = tab.nunk;
        d.nsrc = tab.nsrc;
        d.ncell = (int)tab.cell_start.size() - 1;
        d.row0 = tab.row0;
        d.src_j = tab.src_j; d.src_b = tab.src_b; d.src_clu = tab.src_clu; d.src_pop = tab.src_pop; d.src_spop = tab.src_spop;
        d.pop_idx = di + io[0]; d.up2 = di + io[1]; d.cell_rc = di + io[2]; d.cell_start = di + io[3]; d.ent_src = di + io[4];
        d.act = di + io[5]; d.inact = di + io[6]; d.apop = di + io[7]; d.lo2 = di + io[8];
        d.w2lo = dd + doff[3];
        d.nact = tab.nact;
        d.ninact = (int)tab.inact.size();
        d.w2 = dd + doff[0]; d.trace = dd + doff[1]; d.ent_coef = dd + doff[2];
    }
    if (e != cudaSuccess) {
        porta_destroy(c);
        return PORTA_ENOMEM;
    }
    *out = c;
    return PORTA_OK;
}

int porta_ml_set_atmosphere(porta_ctx *c, const double *chi, const double *kT, const double *vel, const double *bx,
                            const double *by, const double *bz, int where)
{
    if (!c) return PORTA_EINVAL;
    MlState *m = c->ml;
    if (!m) return fail(c, PORTA_EINVAL, "ml_set_atmosphere: not a multilevel context");
    if (!chi || !kT || !vel || (where != PORTA_HOST && where != PORTA_DEVICE))
        return fail(c, PORTA_EINVAL, "ml_set_atmosphere: bad argument");
    if (m->pol && (!bx || !by || !bz)) return fail(c, PORTA_EINVAL, "ml_set_atmosphere: magnetic field required");
    const long long n1 = m->nvox1, n = c->nvox;
    std::vector<double> hv(n1);
    cudaMemcpyKind k = where == PORTA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(m->d_chis, chi, n1 * sizeof(double), k, c->stream));
    CK(cudaMemcpyAsync(m->d_kT, kT, n1 * sizeof(double), k, c->stream));
    unsigned long long bad = 0;
    int rc = count_bad(c, m->d_chis, n1, 0.0, 1e300, &bad);
    if (rc) return rc;
    if (bad) return fail(c, PORTA_EINVAL, "ml_set_atmosphere: chi must be finite and > 0");
    if ((rc = count_bad(c, m->d_kT, n1, 0.0, 1e300, &bad))) return rc;
    if (bad) return fail(c, PORTA_EINVAL, "ml_set_atmosphere: kT must be finite and > 0");
    if (where == PORTA_DEVICE)
        CK(cudaMemcpy(hv.data(), vel, n1 * sizeof(double), cudaMemcpyDeviceToHost));
    else
        std::memcpy(hv.data(), vel, n1 * sizeof(double));
    // the line boxes share the grid and the velocity; their opacity, Planck
    // function and source function are written from the populations
    std::vector<double> vrep(n), ones(n, 1.0), half(n, 0.5);
    for (int b = 0; b < m->mc.nline; ++b) std::memcpy(vrep.data() + b * n1, hv.data(), n1 * sizeof(double));
    std::vector<double> brep[3];
    if (m->pol) {
        const double *src[3] = {bx, by, bz};
        for (int d = 0; d < 3; ++d) {
            brep[d].resize(n);
            if (where == PORTA_DEVICE)
                CK(cudaMemcpy(brep[d].data(), src[d], n1 * sizeof(double), cudaMemcpyDeviceToHost));
            else
                std::memcpy(brep[d].data(), src[d], n1 * sizeof(double));
            for (int b = 1; b < m->mc.nline; ++b) std::memcpy(brep[d].data() + b * n1, brep[d].data(), n1 * sizeof(double));
        }
        // the first-order (weak-field) Zeeman term eta_V = 2 zeta (B.Omega)(x - s) eta_I is a
        // propagation matrix only while |eta_V| < eta_I over the frequency grid
        double bmax = 0.0, vmax = 0.0;
        for (long long v = 0; v < n1; ++v) {
            bmax = std::max(bmax, std::sqrt(brep[0][v] * brep[0][v] + brep[1][v] * brep[1][v] + brep[2][v] * brep[2][v]));
            vmax = std::max(vmax, std::fabs(hv[v]));
        }
        if (!(2.0 * c->zeta * bmax * (c->x_max + vmax) < 1.0))
            return fail(c, PORTA_EINVAL, "ml_set_atmosphere: the weak-field Zeeman term 2 zeta |B| (x_max + |v|) reaches 1 "
                                         "(|eta_V| > eta_I); lower zeta or the field");
    }
    porta_atmos at{ones.data(), half.data(), ones.data(), vrep.data(), m->pol ? brep[0].data() : nullptr,
                   m->pol ? brep[1].data() : nullptr, m->pol ? brep[2].data() : nullptr};
    rc = porta_set_atmosphere(c, &at, PORTA_HOST);
    if (rc) return rc;
    m->have_atm = true;
    if (m->have_pops) {
        cudaError_t e = ml_prepare(c);
        if (e != cudaSuccess) return fail(c, PORTA_ECUDA, cudaGetErrorString(e));
    }
    return PORTA_OK;
}

int porta_ml_set_pops(porta_ctx *c, const double *pops, int where)
{
    if (!c) return PORTA_EINVAL;
    MlState *m = c->ml;
    if (!m) return fail(c, PORTA_EINVAL, "ml_set_pops: not a multilevel context");
    if (!pops || (where != PORTA_HOST && where != PORTA_DEVICE)) return fail(c, PORTA_EINVAL, "ml_set_pops: bad argument");
    if (!m->have_atm) return fail(c, PORTA_ESTATE, "ml_set_pops: atmosphere not set");
    const long long n = m->nvox1 * m->mc.nlev;
    int rc = copy_in(c, m->d_pops, pops, n, where);
    if (rc) return rc;
    unsigned long long bad = 0;
    if ((rc = count_bad(c, m->d_pops, n, 0.0, 1e300, &bad))) return rc;
    if (bad) return fail(c, PORTA_EINVAL, "ml_set_pops: populations must be finite and > 0");
    if (m->pol) {
        // no atomic polarization: rho^0_0 = n / sqrt(2J+1)
        std::vector<double> hp(n), hx((size_t)m->nvox1 * m->nunk, 0.0);
        CK(cudaStreamSynchronize(c->stream));
        CK(cudaMemcpy(hp.data(), m->d_pops, n * sizeof(double), cudaMemcpyDeviceToHost));
        for (long long v = 0; v < m->nvox1; ++v)
            for (int i = 0; i < m->mc.nlev; ++i)
                hx[v * m->nunk + m->tab.pop_idx[i]] = hp[v * m->mc.nlev + i] / std::sqrt(m->mc.g[i]);
        CK(cudaMemcpy(m->d_x, hx.data(), hx.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    CK(cudaMemsetAsync(m->d_bad, 0, sizeof(unsigned long long), c->stream));
    CK(ml_prepare(c));
    unsigned long long hb = 0;
    CK(cudaMemcpyAsync(&hb, m->d_bad, sizeof(hb), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (hb) return fail(c, PORTA_EINVAL, "ml_set_pops: a line has a non-positive opacity (population inversion)");
    m->have_pops = true;
    c->have_rho = true;
    c->have_fs = c->have_jkq = false;
    return PORTA_OK;
}

int porta_ml_get_pops(porta_ctx *c, double *pops, int where)
{
    if (!c) return PORTA_EINVAL;
    MlState *m = c->ml;
    if (!m) return fail(c, PORTA_EINVAL, "ml_get_pops: not a multilevel context");
    if (!pops || (where != PORTA_HOST && where != PORTA_DEVICE)) return fail(c, PORTA_EINVAL, "ml_get_pops: bad argument");
    if (!m->have_pops) return fail(c, PORTA_ESTATE, "ml_get_pops: populations not set");
    if (m->pol) {
        std::vector<double> hx((size_t)m->nvox1 * m->nunk), hp((size_t)m->nvox1 * m->mc.nlev);
        CK(cudaMemcpyAsync(hx.data(), m->d_x, hx.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (long long v = 0; v < m->nvox1; ++v)
            for (int i = 0; i < m->mc.nlev; ++i)
                hp[v * m->mc.nlev + i] = std::sqrt(m->mc.g[i]) * hx[v * m->nunk + m->tab.pop_idx[i]];
        CK(cudaMemcpy(pops, hp.data(), hp.size() * sizeof(double),
                      where == PORTA_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
        return PORTA_OK;
    }
    CK(cudaMemcpyAsync(pops, m->d_pops, m->nvox1 * m->mc.nlev * sizeof(double),
                       where == PORTA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (where == PORTA_HOST) CK(cudaStreamSynchronize(c->stream));
    return PORTA_OK;
}

int porta_ml_emergent_stokes(porta_ctx *c, int line, int ndir, const double *mu, const double *chi, double *out,
                             int where)
{
    if (!c) return PORTA_EINVAL;
    MlState *m = c->ml;
    if (!m) return fail(c, PORTA_EINVAL, "ml_emergent_stokes: not a multilevel context");
    if (line < 0 || line >= m->mc.nline || ndir < 1 || !mu || !chi || !out ||
        (where != PORTA_HOST && where != PORTA_DEVICE))
        return fail(c, PORTA_EINVAL, "ml_emergent_stokes: bad argument");
    for (int d = 0; d < ndir; ++d)
        if (!(mu[d] > 0.0 && mu[d] <= 1.0) || !std::isfinite(chi[d]))
            return fail(c, PORTA_EINVAL, "ml_emergent_stokes: mu must lie in (0, 1], chi finite");
    if (!m->have_atm || !m->have_pops) return fail(c, PORTA_ESTATE, "ml_emergent_stokes: atmosphere or populations not set");
    const long long n = (long long)ndir * c->n_nu * c->nx * c->ny * c->ns;
    double *dout = out;
    if (where == PORTA_HOST) CK(dalloc(&dout, n));
    int rc = c->precision == PORTA_FP32 ? emergent_t<float>(c, ndir, mu, chi, dout, line)
                                        : emergent_t<double>(c, ndir, mu, chi, dout, line);
    if (where == PORTA_HOST) {
        if (rc == PORTA_OK) {
            cudaError_t e = cudaMemcpy(out, dout, n * sizeof(double), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, cudaGetErrorString(e));
        }
        pfree(dout);
    }
    return rc;
}

int porta_ml_unknowns(const porta_ctx *c, int *nunk)
{
    if (!c || !nunk) return PORTA_EINVAL;
    if (!c->ml) return PORTA_EINVAL;
    *nunk = c->ml->nunk;
    return PORTA_OK;
}

int porta_ml_set_unknowns(porta_ctx *c, const double *x, int where)
{
    if (!c) return PORTA_EINVAL;
    MlState *m = c->ml;
    if (!m) return fail(c, PORTA_EINVAL, "ml_set_unknowns: not a multilevel context");
    if (!m->pol) return porta_ml_set_pops(c, x, where);
    if (!x || (where != PORTA_HOST && where != PORTA_DEVICE)) return fail(c, PORTA_EINVAL, "ml_set_unknowns: bad argument");
    if (!m->have_atm) return fail(c, PORTA_ESTATE, "ml_set_unknowns: atmosphere not set");
    const long long n = m->nvox1 * m->nunk;
    int rc = copy_in(c, m->d_x, x, n, where);
    if (rc) return rc;
    unsigned long long bad = 0;
    if ((rc = count_bad(c, m->d_x, n, -1e300, 1e300, &bad))) return rc;
    if (bad) return fail(c, PORTA_EINVAL, "ml_set_unknowns: non-finite value");
    CK(cudaMemsetAsync(m->d_bad, 0, sizeof(unsigned long long), c->stream));
    CK(ml_prepare(c));
    unsigned long long hb = 0;
    CK(cudaMemcpyAsync(&hb, m->d_bad, sizeof(hb), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (hb) return fail(c, PORTA_EINVAL, "ml_set_unknowns: non-positive population or line opacity");
    m->have_pops = true;
    c->have_rho = true;
    c->have_fs = c->have_jkq = false;
    return PORTA_OK;
}

int porta_ml_get_unknowns(porta_ctx *c, double *x, int where)
{
    if (!c) return PORTA_EINVAL;
    MlState *m = c->ml;
    if (!m) return fail(c, PORTA_EINVAL, "ml_get_unknowns: not a multilevel context");
    if (!m->pol) return porta_ml_get_pops(c, x, where);
    if (!x || (where != PORTA_HOST && where != PORTA_DEVICE)) return fail(c, PORTA_EINVAL, "ml_get_unknowns: bad argument");
    if (!m->have_pops) return fail(c, PORTA_ESTATE, "ml_get_unknowns: unknowns not set");
    CK(cudaMemcpyAsync(x, m->d_x, m->nvox1 * m->nunk * sizeof(double),
                       where == PORTA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (where == PORTA_HOST) CK(cudaStreamSynchronize(c->stream));
    return PORTA_OK;
}

// the error counter of the line data and of the rate equations (synchronizes)
static int ml_check(porta_ctx *c, const char *what)
{
    unsigned long long hb = 0;
    CK(cudaMemcpyAsync(&hb, c->ml->d_bad, sizeof(hb), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (hb) {
        cudaMemsetAsync(c->ml->d_bad, 0, sizeof(hb), c->stream);
        return fail(c, PORTA_EKERNEL, std::string(what) + ": singular rate equations, non-positive population or "
                                                          "line opacity (population inversion)");
    }
    return PORTA_OK;
}

int porta_ml_formal_solve(porta_ctx *c, double *jbar, double *lstar, int where)
{
    if (!c) return PORTA_EINVAL;
    MlState *m = c->ml;
    if (!m) return fail(c, PORTA_EINVAL, "ml_formal_solve: not a multilevel context");
    if (!m->have_atm || !m->have_pops) return fail(c, PORTA_ESTATE, "ml_formal_solve: atmosphere or populations not set");
    int rc = porta_formal_solve(c);
    if (rc == PORTA_OK) rc = porta_accumulate_jkq(c, jbar, lstar, where);
    return rc;
}

int porta_ml_see_update(porta_ctx *c, double *max_change)
{
    if (!c) return PORTA_EINVAL;
    if (!c->ml) return fail(c, PORTA_EINVAL, "ml_see_update: not a multilevel context");
    int rc = porta_see_update(c, max_change);
    if (rc == PORTA_OK && max_change) rc = ml_check(c, "ml_see_update");
    return rc;
}

int porta_ml_iterate(porta_ctx *c, int iterations, double *max_change)
{
    if (!c) return PORTA_EINVAL;
    MlState *m = c->ml;
    if (!m) return fail(c, PORTA_EINVAL, "ml_iterate: not a multilevel context");
    if (!m->have_atm || !m->have_pops) return fail(c, PORTA_ESTATE, "ml_iterate: atmosphere or populations not set");
    if (iterations < 0) return fail(c, PORTA_EINVAL, "ml_iterate: negative count");
    int rc = PORTA_OK;
    for (int it = 0; it < iterations && rc == PORTA_OK; ++it) {
        rc = porta_ml_formal_solve(c, nullptr, nullptr, PORTA_DEVICE);
        if (rc == PORTA_OK) rc = porta_see_update(c, it == iterations - 1 ? max_change : nullptr);
    }
    if (rc == PORTA_OK) rc = ml_check(c, "ml_iterate");
    return rc;
}

}  // extern "C"
