// C ABI, emergent Stokes profiles and reverse mode: the emergent sweep for
// given directions, the vector-Jacobian products of the emergent profiles, of
// one formal solution's J^K_Q and Lambda-bar*, and of a run of Jacobi
// iterations (checkpointed forward, reverse sweeps).
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
int emergent_t(porta_ctx *c, int ndir, const double *mu, const double *chi, double *dout, int box)
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
        check_global_sweep(c);
        if (c->sc_faces || c->gsweep) {
            // short characteristics on cell faces, or the plane placement of the
            // global-memory sweep (faces.cu), its own work buffer
            a.nray = ndir;
            const BoxDev &hb0 = c->boxes[box];
            const long long nxy = (long long)hb0.nx * hb0.ny;
            const double dxy[2] = {c->blx[box] / hb0.nx, c->bly[box] / hb0.ny};
            Real *ws = nullptr;
            double *ddxy = nullptr;
            e = pmalloc((void **)&ws, c->ns == 1 ? faces_scratch_bytes<Real, 1>(1, ndir, c->n_nu, nxy, c->nvox, c->d_dich ? 1 : (c->d_kexpl ? 2 : 0))
                                                 : faces_scratch_bytes<Real, 4>(1, ndir, c->n_nu, nxy, c->nvox, c->d_dich ? 1 : (c->d_kexpl ? 2 : 0)));
            if (e == cudaSuccess) e = pmalloc((void **)&ddxy, sizeof(dxy));
            if (e == cudaSuccess) e = cudaMemcpyAsync(ddxy, dxy, sizeof(dxy), cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
            if (e == cudaSuccess)
                e = c->ns == 1 ? launch_faces<Real, 1>(a, ws, 1, nxy, ddxy, 100000, c->d_err, c->stream, true, !c->sc_faces)
                               : launch_faces<Real, 4>(a, ws, 1, nxy, ddxy, 100000, c->d_err, c->stream, true, !c->sc_faces);
            int flag = 0;
            if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (ws) pfree(ws);
            if (ddxy) pfree(ddxy);
            if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, std::string("emergent (faces): ") + cudaGetErrorString(e));
            else if (flag & 2) rc = fail(c, PORTA_ENOTCONV, "emergent (faces): a plane of face points did not converge");
            break;
        }
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
                e = ensure_buf((void **)&c->d_gacc, c->gacc_bytes, (size_t)acfg.clusters * 10 * c->nvox * sizeof(Real));
            if (e == cudaSuccess) e = cudaMemsetAsync(c->d_gacc, 0, (size_t)acfg.clusters * 10 * c->nvox * sizeof(Real), c->stream);
            b.gacc = c->d_gacc;
            if (e == cudaSuccess)
                e = c->ns == 1 ? launch_adjoint<Real, 1>(b, acfg, c->stream, 1) : launch_adjoint<Real, 4>(b, acfg, c->stream, 1);
            if (e == cudaSuccess)
                e = launch_adjoint_acc_reduce<Real>((const Real *)c->d_gacc, acfg.clusters, c->nvox, c->nl, dg_chi, c->ns == 1 ? nullptr : dg_b,
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

template int emergent_t<float>(porta_ctx *, int, const double *, const double *, double *, int);
template int emergent_t<double>(porta_ctx *, int, const double *, const double *, double *, int);

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
    if (e == cudaSuccess)
        e = ensure_buf((void **)&c->d_vjp_out, c->vjp_out_bytes, (size_t)nb * c->n_nu * nxy * c->ns * sizeof(double));
    // dL/dJ^K_Q and dL/dLambda* in the sweep's precision (read per point and item)
    if (e == cudaSuccess) e = ensure_buf(&c->d_gjR, c->gjR_bytes, (size_t)c->nvox * (c->nj + 1) * sizeof(Real));
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        if (!c->it_ev[k]) e = cudaEventCreate(&c->it_ev[k]);
    if (e != cudaSuccess) return fail(c, PORTA_ENOMEM, "iterate_vjp: tape allocation");
    double *scratch = c->d_vjp_out;
    Real *gjR = (Real *)c->d_gjR;
    e = run_to_real<Real>((long long)c->nvox * c->nj, dgj, gjR, c->stream);
    if (e == cudaSuccess) e = run_to_real<Real>((long long)c->nvox, dgl, gjR + (size_t)c->nvox * c->nj, c->stream);
    if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("iterate_vjp: ") + cudaGetErrorString(e));
    // adjoint launch shape: forced, else timed once per batch size on the first batch
    LaunchCfg acfg{};
    std::vector<LaunchCfg> cand;
    const bool forced = c->adj_cluster > 0 || c->adj_nu_group > 0;
    const bool tune = !forced && !c->adj2_tuned.count(nb);
    int rc = c->ns == 1 ? choose_adjoint<Real, 1>(c, acfg, c->adj_cluster, c->adj_nu_group, nb, tune ? &cand : nullptr)
                        : choose_adjoint<Real, 4>(c, acfg, c->adj_cluster, c->adj_nu_group, nb, tune ? &cand : nullptr);
    if (rc) return fail(c, rc, "iterate_vjp: no adjoint launch shape fits");
    if (!forced && !tune) acfg = c->adj2_tuned[nb];
    int maxcl = acfg.clusters;
    for (const LaunchCfg &k : cand) maxcl = std::max(maxcl, k.clusters);
    e = ensure_buf((void **)&c->d_gacc, c->gacc_bytes, (size_t)maxcl * 10 * c->nvox * sizeof(Real));
    if (e != cudaSuccess) return fail(c, PORTA_ENOMEM, "iterate_vjp: accumulator allocation");
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
        b.gjkq = gjR;
        b.glstar = gjR + (size_t)c->nvox * c->nj;
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
        e = cudaMemsetAsync(c->d_gacc, 0, (size_t)acfg.clusters * 10 * c->nvox * sizeof(Real), c->stream);
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
            e = launch_adjoint_acc_reduce<Real>((const Real *)c->d_gacc, acfg.clusters, c->nvox, c->nl, dg_chi, c->ns == 1 ? nullptr : dg_b,
                                          dg_rho, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
        if (e != cudaSuccess) rc = fail(c, PORTA_ECUDA, std::string("iterate_vjp: ") + cudaGetErrorString(e));
        c->it_ms[4] += t;
        c->last_adj = acfg;
    }
    cudaStreamSynchronize(c->stream);
    return rc;
}

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

}  // namespace porta_api

using namespace porta_api;

extern "C" {

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
    if (c && (c->interp == 2 || c->d_kexpl || c->sc_faces || c->gsweep))
        return fail(c, PORTA_EINVAL, "reverse mode: bilinear interpolation on the horizontal planes, two-level media only");
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
    if (c && (c->interp == 2 || c->d_kexpl || c->sc_faces || c->gsweep))
        return fail(c, PORTA_EINVAL, "reverse mode: bilinear interpolation on the horizontal planes, two-level media only");
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
}  // extern "C"
