// Allocation-free formal solution: porta_formal_solve_noalloc (include/porta.h).
//
// Some callers cannot call cudaMalloc: a host program whose device memory is
// fully reserved up front by another framework's pooling allocator (where a
// further cudaMalloc fails or fragments the pool), or a latency-sensitive loop
// that cannot afford the implicit device synchronization and unpredictable
// latency of cudaMalloc / cudaFree. For them this entry point runs the FP32
// formal solution and the J^K_Q / Lambda-bar* sums on caller-provided device
// inputs and outputs, and keeps every intermediate (atmosphere and unknowns in
// the sweep's precision, profile normalization, per-ray geometry and tensor
// tables, per-ray partial integrals) in one file-scope device array of fixed
// size. It calls no allocating routine, host or device.
//
// The array is reserved on every GPU that loads the library, for the life of
// the process. All calls share it and it keeps the contents of the last call;
// every region is fully written by a call before it is read, so nothing needs
// clearing between calls. Calls that overlap on the GPU (concurrent streams,
// threads, or several problems in flight) race on the array.
#include <cuda_runtime.h>

#include <cmath>

#include "api_internal.h"
#include "porta.h"
#include "porta_internal.cuh"
#include "see_kernels.cuh"

using namespace porta;

namespace {

constexpr size_t kScratchBytes = (size_t)PORTA_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxMu = 32;
constexpr int kMaxNz = PORTA_NOALLOC_MAX_NZ;   // heights travel in the kernel's argument block

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[PORTA_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of the scratch array on the current device. The host-side
// symbol itself is not a device address. The address is looked up on every
// call with the caller's device current: the lookup allocates nothing, and a
// cached address would go stale if the caller reset the device (a new context
// loads the module again, possibly elsewhere). The first call on a device also
// loads the library's device code there.
cudaError_t scratch_address(void **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

struct GaussNodes {
    double x[kMaxMu], w[kMaxMu];
};

// Gauss-Legendre nodes and weights on (0, 1) into a fixed-size argument block
void gauss_nodes(int n, GaussNodes &g) { porta_api::gauss_legendre(n, g.x, g.w); }

struct TableArgs {
    int n_mu, n_chi, n_nu, nx, ny, nz;
    double lx, ly, x_max;
    GaussNodes gl;
    double z[kMaxNz];
    BoxDev *box;
    RayDev<float> *rays;
    PlaneGeom<float> *geom;
    double *mu, *tw, *xd, *wd;
    float *xf, *wf;
};

// Per-ray tables: direction, weight, T^K_Q(i, Omega) for i = I, Q, U (from the
// polarization tensors of the ray frame), the sheared plane geometry, and the
// frequency grid.
__global__ void noalloc_tables_kernel(TableArgs a)
{
    const int nray = 2 * a.n_mu * a.n_chi;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m == 0) {
        BoxDev b{};
        b.nx = a.nx; b.ny = a.ny; b.nz = a.nz;
        *a.box = b;
        for (int j = 0; j < a.n_nu; ++j) {
            double x = 0.0, w = 1.0;
            if (a.n_nu > 1) {
                double dx = 2.0 * a.x_max / (a.n_nu - 1);
                x = -a.x_max + j * dx;
                w = (j == 0 || j == a.n_nu - 1) ? 0.5 * dx : dx;
            }
            a.xd[j] = x; a.wd[j] = w;
            a.xf[j] = (float)x; a.wf[j] = (float)w;
        }
    }
    if (m >= nray) return;
    const int h = m / (a.n_mu * a.n_chi), rem = m - h * a.n_mu * a.n_chi;
    const int i = rem / a.n_chi, az = rem - i * a.n_chi;
    const double mu = h == 0 ? a.gl.x[i] : -a.gl.x[i];
    const double chi = (az + 0.5) * 2.0 * M_PI / a.n_chi;
    const double w = 0.5 * a.gl.w[i] / a.n_chi;
    const double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    const double ox = st * cos(chi), oy = st * sin(chi);
    double ea[3] = {mu * cos(chi), mu * sin(chi), -st};
    double eb[3] = {-sin(chi), cos(chi), 0.0};
    RayDev<float> r{};
    r.mu = (float)mu; r.ox = (float)ox; r.oy = (float)oy; r.oz = (float)mu;
    a.mu[m] = mu;
    a.tw[m * 19] = w;
    const double k = -0.8660254037844386;   // -sqrt(3)/2
    for (int s = 0; s < 3; ++s) {
        double t[3][3];
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) {
                double aa = ea[p] * ea[q], bb = eb[p] * eb[q], ab = ea[p] * eb[q] + eb[p] * ea[q];
                t[p][q] = s == 0 ? aa + bb : (s == 1 ? aa - bb : ab);
            }
        double tr = t[0][0] + t[1][1] + t[2][2];
        double v[6] = {tr / 2.0, k * 1.2247448713915890 * (t[2][2] - tr / 3.0), k * (-t[0][2]), k * (-t[1][2]),
                       k * 0.5 * (t[0][0] - t[1][1]), k * t[0][1]};
        for (int c = 0; c < 6; ++c) {
            r.t[6 * s + c] = (float)v[c];
            a.tw[m * 19 + 1 + 6 * s + c] = v[c];
        }
    }
    a.rays[m] = r;
    const bool up = mu > 0;
    const double hx = a.lx / a.nx, hy = a.ly / a.ny, amu = fabs(mu);
    long long ax = 0, ay = 0;
    for (int q = 0; q < a.nz; ++q) {
        const int kz = up ? q : a.nz - 1 - q;
        PlaneGeom<float> g{};
        g.kz = kz;
        if (q > 0) {
            const int ku = up ? kz - 1 : kz + 1;
            const double ds = fabs(a.z[kz] - a.z[ku]) / amu;
            const double dx = ds * ox / hx, dy = ds * oy / hy;
            const double cx = ceil(dx), cy = ceil(dy);
            ax = ((ax + (long long)cx) % a.nx + a.nx) % a.nx;
            ay = ((ay + (long long)cy) % a.ny + a.ny) % a.ny;
            g.tx = (float)(cx - dx);
            g.ty = (float)(cy - dy);
            g.ds = (float)ds;
        }
        g.ax = (int)ax;
        g.ay = (int)ay;
        a.geom[(size_t)m * a.nz + q] = g;
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t atm, rho, invn, part, geom, rays, xf, xd, mu, tw, box, total;
};

Layout layout(long long nvox, int nray, int nz, int nnu, int nl, int ns)
{
    Layout L{};
    size_t o = 0;
    L.atm = o;  o = align256(o + 6 * (size_t)nvox * sizeof(float));
    L.rho = o;  o = align256(o + (size_t)nl * nvox * sizeof(float));
    L.invn = o; o = align256(o + (size_t)nray * nvox * sizeof(float));
    L.part = o; o = align256(o + (size_t)nray * nvox * (ns == 1 ? 2 : 4) * sizeof(float));
    L.geom = o; o = align256(o + (size_t)nray * nz * sizeof(PlaneGeom<float>));
    L.rays = o; o = align256(o + (size_t)nray * sizeof(RayDev<float>));
    L.xf = o;   o = align256(o + 2 * (size_t)nnu * sizeof(float));
    L.xd = o;   o = align256(o + 2 * (size_t)nnu * sizeof(double));
    L.mu = o;   o = align256(o + (size_t)nray * sizeof(double));
    L.tw = o;   o = align256(o + (size_t)nray * 19 * sizeof(double));
    L.box = o;  o = align256(o + sizeof(BoxDev));
    L.total = o;
    return L;
}

template <int NS>
int run(const porta_grid *g, const porta_atom *at, const porta_quad *q, const porta_atmos *atm, const double *rho,
        double *jkq, double *lstar, cudaStream_t st)
{
    const long long nvox = (long long)g->nx * g->ny * g->nz;
    const int nray = 2 * q->n_mu * q->n_chi;
    const int nl = NS == 1 ? 1 : 6;
    const Layout L = layout(nvox, nray, g->nz, q->n_nu, nl, NS);
    if (L.total > kScratchBytes) return PORTA_ESCRATCH;

    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return PORTA_ECUDA;
    unsigned char *B = (unsigned char *)base;
    float *d_atm = (float *)(B + L.atm);

    // launch shape by the same cost estimate as porta_formal_solve's default
    // (waves of rays x per-ray plane work), without timing runs
    LaunchCfg best{};
    double best_cost = 1e300;
    for (int C = 1; C <= 16; ++C) {
        if (C > g->ny) break;
        const int rmax = (g->ny + C - 1) / C;
        const int ring_plane = (NS == 1 ? 1 : 2) * (rmax + 2) * g->nx;
        const int ipts = rmax * g->nx;
        const long long ring = 3LL * ring_plane * 16;
        const long long per_nu = 2LL * ipts * NS * 4;
        const long long scratch = 512LL * (NS == 1 ? 2 : 4) * 4;
        const long long limit = 220 * 1024;
        if (ring + per_nu + scratch > limit) continue;
        const int fmax = (int)std::min<long long>(q->n_nu, (limit - ring - scratch) / per_nu);
        const int G = (q->n_nu + fmax - 1) / fmax, F = (q->n_nu + G - 1) / G;
        const int threads = std::min(512, std::max(64, (ipts * F + 31) / 32 * 32));
        const int smem = sweep_smem_bytes<float, NS>(ring_plane, ipts, F, threads, NS == 1 ? 2 : 4);
        int act = 0;
        if (max_active_clusters<float, NS>(C, smem, threads, &act) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (act < 1) continue;
        const int ncl = std::min(act, nray);
        const double slots = std::ceil((double)ipts * F / threads) * 512.0;
        const double cost = std::ceil((double)nray / ncl) * G *
                            (slots + 0.15 * (rmax + 2) * g->nx + 0.05 * ipts + 300.0);
        if (cost < best_cost) {
            best_cost = cost;
            best.cluster = C; best.F = F; best.threads = threads; best.smem = smem; best.clusters = ncl;
        }
    }
    if (best.cluster == 0) return PORTA_EINVAL;

    cudaError_t e = cudaSuccess;
    TableArgs ta{};
    ta.n_mu = q->n_mu; ta.n_chi = q->n_chi; ta.n_nu = q->n_nu;
    ta.nx = g->nx; ta.ny = g->ny; ta.nz = g->nz;
    ta.lx = g->lx; ta.ly = g->ly; ta.x_max = q->x_max;
    gauss_nodes(q->n_mu, ta.gl);
    for (int k = 0; k < g->nz; ++k) ta.z[k] = g->z[k];
    ta.box = (BoxDev *)(B + L.box);
    ta.rays = (RayDev<float> *)(B + L.rays);
    ta.geom = (PlaneGeom<float> *)(B + L.geom);
    ta.mu = (double *)(B + L.mu);
    ta.tw = (double *)(B + L.tw);
    ta.xd = (double *)(B + L.xd);
    ta.wd = ta.xd + q->n_nu;
    ta.xf = (float *)(B + L.xf);
    ta.wf = ta.xf + q->n_nu;
    if (e == cudaSuccess) {
        noalloc_tables_kernel<<<(nray + 63) / 64, 64, 0, st>>>(ta);
        e = cudaGetLastError();
    }
    // atmosphere and unknowns in the sweep's precision (SoA: chi, vel, bx, by, bz, bpl)
    if (e == cudaSuccess) e = run_to_real<float>(nvox, atm->chi, d_atm, st);
    if (e == cudaSuccess) e = run_to_real<float>(nvox, atm->vel, d_atm + nvox, st);
    if (NS == 4) {
        if (e == cudaSuccess) e = run_to_real<float>(nvox, atm->bx, d_atm + 2 * nvox, st);
        if (e == cudaSuccess) e = run_to_real<float>(nvox, atm->by, d_atm + 3 * nvox, st);
        if (e == cudaSuccess) e = run_to_real<float>(nvox, atm->bz, d_atm + 4 * nvox, st);
    }
    if (e == cudaSuccess) e = run_to_real<float>(nvox, atm->bpl, d_atm + 5 * nvox, st);
    if (e == cudaSuccess) e = run_rho_convert<float>(nvox, nl, rho, B + L.rho, st);
    if (e == cudaSuccess) e = run_profile_norm<float>(nvox, nray, q->n_nu, ta.mu, ta.xd, ta.wd, atm->vel, B + L.invn, st);
    if (e != cudaSuccess) return PORTA_ECUDA;

    SweepArgs<float> a{};
    a.nnu = q->n_nu; a.nray = nray; a.nvox = nvox;
    a.boxes = ta.box;
    a.items = nullptr;
    a.bfac = (float)(2.0 * at->gbar * at->zeta);
    a.chi = d_atm; a.vel = d_atm + nvox; a.bx = d_atm + 2 * nvox; a.by = d_atm + 3 * nvox; a.bz = d_atm + 4 * nvox;
    a.bpl = d_atm + 5 * nvox;
    a.rho = (const float *)(B + L.rho);
    a.invn = (const float *)(B + L.invn);
    a.part = B + L.part;
    a.xf = ta.xf; a.wf = ta.wf;
    a.geom = ta.geom; a.rays = ta.rays;
    a.probe_ray = -1;
    a.nitems = nray;
    a.F = best.F;
    a.ngroups = (q->n_nu + best.F - 1) / best.F;
    {
        const int rmax = (g->ny + best.cluster - 1) / best.cluster;
        a.ring_plane = (NS == 1 ? 1 : 2) * (rmax + 2) * g->nx;
        a.ipts_max = rmax * g->nx;
    }
    e = launch_sweep<float, NS>(a, MODE_JKQ, best, st);
    if (e == cudaSuccess) e = run_jkq_finalize<float, NS>(nvox, nray, B + L.part, ta.tw, jkq, lstar, st);
    return e == cudaSuccess ? PORTA_OK : PORTA_ECUDA;
}

}  // namespace

extern "C" int porta_formal_solve_noalloc(const porta_grid *g, const porta_atom *at, const porta_quad *q,
                                          const porta_atmos *atm, const double *rho, double *jkq, double *lstar,
                                          void *stream)
{
    if (!g || !at || !q || !atm || !g->z || !rho || !jkq || !lstar) return PORTA_EINVAL;
    if (g->nx < 1 || g->ny < 1 || g->nz < 2 || !(g->lx > 0) || !(g->ly > 0)) return PORTA_EINVAL;
    if (g->nz > kMaxNz) return PORTA_ESCRATCH;
    if (q->n_mu < 1 || q->n_mu > kMaxMu || q->n_chi < 1 || q->n_nu < 1 || !(q->x_max > 0)) return PORTA_EINVAL;
    for (int k = 1; k < g->nz; ++k)
        if (!(g->z[k] > g->z[k - 1])) return PORTA_EINVAL;
    if (!atm->chi || !atm->vel || !atm->bpl) return PORTA_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (at->model == PORTA_MODEL_TWOLEVEL_UNPOL) return run<1>(g, at, q, atm, rho, jkq, lstar, st);
    if (at->model == PORTA_MODEL_TWOLEVEL_HANLE) {
        if (!atm->bx || !atm->by || !atm->bz) return PORTA_EINVAL;
        return run<4>(g, at, q, atm, rho, jkq, lstar, st);
    }
    return PORTA_EINVAL;
}
