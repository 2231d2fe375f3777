// C ABI, multigrid (Sec. 5): coarse levels as solver contexts of their own,
// restriction / prolongation, the full-approximation-scheme V-cycle
// (Eqs. 30-34) and the residual of the fine-grid equations.
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
#include "mlpol_kernels.cuh"
#include "see_kernels.cuh"

using namespace porta;

namespace porta_api {

// ---------------------------------------------------------------- multigrid (Sec. 5)

int coarse_nz(int nz) { return nz % 2 ? (nz + 1) / 2 : nz / 2; }

void mg_free(porta_ctx *c)
{
    for (porta_ctx *L : c->mg) porta_destroy(L);
    c->mg.clear();
    double *bufs[] = {c->mg_res, c->mg_src, c->mg_rho0, c->mg_prev, c->mg_zr, c->mg_zp, c->mg_zp3};
    for (double *b : bufs)
        if (b) pfree(b);
    c->mg_res = c->mg_src = c->mg_rho0 = c->mg_prev = c->mg_zr = c->mg_zp = c->mg_zp3 = nullptr;
    c->mg_order = 1;
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

// the cubic prolongation in height between a level with heights zf and the next
// coarser one: per fine plane 4 (coarse plane, weight) pairs -- the coarse plane
// itself (weight 1) for a coincident plane, else the Lagrange cubic through the
// four coarse planes around it (the four innermost next to the bottom and top, the
// top four for a fine plane above the coarse grid). Needs at least 4 coarse planes.
void mg_ztable_cubic(const std::vector<double> &zf, std::vector<double> &zp3)
{
    const int nf = (int)zf.size(), nc = coarse_nz(nf);
    zp3.assign(8 * (size_t)nf, 0.0);
    for (int k = 0; k < nf; ++k) {
        if (k % 2 == 0) {
            for (int a = 0; a < 4; ++a) zp3[8 * k + 2 * a] = k / 2;
            zp3[8 * k + 1] = 1.0;
            continue;
        }
        const int s = std::min(std::max((k - 1) / 2 - 1, 0), nc - 4);
        for (int a = 0; a < 4; ++a) {
            double w = 1.0;
            for (int b = 0; b < 4; ++b)
                if (b != a) w *= (zf[k] - zf[2 * (s + b)]) / (zf[2 * (s + a)] - zf[2 * (s + b)]);
            zp3[8 * k + 2 * a] = s + a;
            zp3[8 * k + 2 * a + 1] = w;
        }
    }
}

// the cubic table of the prolongation from coarse level L to F (null where L has
// fewer than 4 nodes on an axis: the cubic is then not available)
cudaError_t mg_cubic_table(porta_ctx *F, const porta_ctx *L)
{
    if (L->nx < 4 || L->ny < 4 || L->nz < 4) return cudaSuccess;
    std::vector<double> zp3;
    mg_ztable_cubic(F->z, zp3);
    cudaError_t e = dalloc(&F->mg_zp3, zp3.size());
    if (e == cudaSuccess) e = cudaMemcpy(F->mg_zp3, zp3.data(), zp3.size() * sizeof(double), cudaMemcpyHostToDevice);
    return e;
}

// formal solution and J^K_Q / Lambda-bar* of one level, kept on the device
int mg_fs(porta_ctx *L)
{
    int rc = porta_formal_solve(L);
    if (rc == PORTA_OK) rc = porta_accumulate_jkq(L, nullptr, nullptr, PORTA_DEVICE);
    return rc;
}

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
        return run_mlpol_apply(L->ml->mc, L->ml->dev, L->ml->nvox1, L->ml->d_kT, L->d_jkq, L->d_j1, L->d_b, L->ml->d_x,
                               alpha, add, with_f, out, L->stream);
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
            e = L->ml->pol ? run_mlpol_see(L->ml->mc, L->ml->dev, L->ml->nvox1, L->ml->d_kT, L->d_jkq, L->d_j1, L->d_lstar, L->d_b,
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

// One V-cycle (Eqs. 30-34) from level l of levels[0..n) down to the coarsest;
// level `top` solves its own problem (right-hand side f), the coarser ones the
// FAS equations; order: the prolongation (1 tri-linear, 3 tri-cubic-centered).
int mg_vcycle(porta_ctx *const *levels, int n, int l, int top, int order, int npre, int npost, int ncoarse)
{
    porta_ctx *L = levels[l];
    const double *src = l == top ? nullptr : L->mg_src;
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
    if ((rc = mg_vcycle(levels, n, l + 1, top, order, npre, npost, ncoarse))) return fail(L, rc, C->err);
    // coarse-grid correction x += P (x_c - R x)
    e = run_prolong(L->nx, L->ny, L->nz, C->nx, C->ny, nc, order, order == 3 ? L->mg_zp3 : L->mg_zp, mg_unk(C),
                    C->mg_rho0, mg_unk(L), 0, L->stream);
    if (e == cudaSuccess) e = mg_rho_changed(L);
    if (e != cudaSuccess) return fail(L, PORTA_ECUDA, std::string("mg prolong: ") + cudaGetErrorString(e));
    return mg_jacobi(L, src, npost);
}


}  // namespace porta_api

using namespace porta_api;

extern "C" {

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
            if (e == cudaSuccess) e = mg_cubic_table(F, L);
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
        if (e == cudaSuccess) e = mg_cubic_table(F, L);
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
    int rc = mg_vcycle(levels.data(), (int)levels.size(), 0, 0, c->mg_order, npre, npost, ncoarse);
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

int porta_mg_set_prolongation(porta_ctx *c, int order)
{
    if (!c) return PORTA_EINVAL;
    if (c->mg.empty()) return fail(c, PORTA_ESTATE, "mg_set_prolongation: call porta_mg_setup first");
    if (order != 1 && order != 3) return fail(c, PORTA_EINVAL, "mg_set_prolongation: order 1 or 3");
    if (order == 3) {
        porta_ctx *F = c;
        for (porta_ctx *L : c->mg) {
            if (!F->mg_zp3)
                return fail(c, PORTA_EINVAL, "mg_set_prolongation: the cubic needs 4 coarse nodes per axis on every level");
            F = L;
        }
    }
    c->mg_order = order;
    return PORTA_OK;
}

int porta_mg_nested(porta_ctx *c, int ncycles, int npre, int npost, int ncoarse, double *max_change)
{
    if (!c) return PORTA_EINVAL;
    if (c->mg.empty()) return fail(c, PORTA_ESTATE, "mg_nested: call porta_mg_setup first");
    if (!c->have_atm || !c->have_rho) return fail(c, PORTA_ESTATE, "mg_nested: atmosphere or rho not set");
    if (c->ml && !c->ml->have_pops) return fail(c, PORTA_ESTATE, "mg_nested: populations not set");
    if (ncycles < 1 || npre < 0 || npost < 0 || ncoarse < 1)
        return fail(c, PORTA_EINVAL, "mg_nested: ncycles >= 1, npre, npost >= 0, ncoarse >= 1");
    std::vector<porta_ctx *> levels{c};
    for (porta_ctx *L : c->mg) {
        L->stream = c->stream;
        levels.push_back(L);
    }
    const int n = (int)levels.size(), nc = mg_ncomp(c), order = c->mg_order;
    // the starting unknowns of the coarsest grid: the finest grid's at the coincident nodes
    cudaError_t e = cudaSuccess;
    for (int l = 1; l < n && e == cudaSuccess; ++l) {
        porta_ctx *F = levels[l - 1], *L = levels[l];
        e = run_inject_vec(L->nx, L->ny, L->nz, F->nx, F->ny, nc, mg_unk(F), mg_unk(L), c->stream);
    }
    if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("mg_nested: ") + cudaGetErrorString(e));
    porta_ctx *K = levels[n - 1];
    if ((e = mg_rho_changed(K)) != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("mg_nested: ") + cudaGetErrorString(e));
    K->have_rho = true;
    if (K->ml) K->ml->have_pops = true;
    // the coarsest grid's own problem, then each finer level from the prolonged solution
    int rc = mg_jacobi(K, nullptr, ncoarse);
    if (rc) return fail(c, rc, std::string("mg_nested: coarsest level: ") + K->err);
    const long long nu = mg_nunk(c);
    for (int l = n - 2; l >= 0 && rc == PORTA_OK; --l) {
        porta_ctx *L = levels[l], *C = levels[l + 1];
        e = run_prolong(L->nx, L->ny, L->nz, C->nx, C->ny, nc, order, order == 3 ? L->mg_zp3 : L->mg_zp, mg_unk(C),
                        nullptr, mg_unk(L), 1, c->stream);
        if (e == cudaSuccess) e = mg_rho_changed(L);
        if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("mg_nested: ") + cudaGetErrorString(e));
        L->have_rho = true;
        if (L->ml) L->ml->have_pops = true;
        for (int k = 0; k < ncycles && rc == PORTA_OK; ++k) {
            if (l == 0 && k == ncycles - 1)
                CK(cudaMemcpyAsync(c->mg_prev, mg_unk(c), sizeof(double) * nu * nc, cudaMemcpyDeviceToDevice, c->stream));
            rc = mg_vcycle(levels.data(), n, l, l, order, npre, npost, ncoarse);
        }
        if (rc && L != c) rc = fail(c, rc, L->err);
    }
    if (rc) return rc;
    c->have_fs = c->have_jkq = false;
    // the change over the finest level's last V-cycle
    CK(cudaMemsetAsync(c->d_resid, 0, sizeof(unsigned long long), c->stream));
    e = c->ml && c->ml->pol ? run_mlpol_change(c->ml->mc, c->ml->dev, nu, c->mg_prev, mg_unk(c), c->d_resid, c->stream)
                            : run_change(nu, nc, c->mg_prev, mg_unk(c), c->d_resid, c->stream, c->ml ? 1 : 0);
    if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("mg_nested: ") + cudaGetErrorString(e));
    if (max_change) {
        unsigned long long bits = 0;
        CK(cudaMemcpyAsync(&bits, c->d_resid, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        std::memcpy(max_change, &bits, sizeof(double));
    }
    if (c->ml) {
        for (porta_ctx *L : levels)
            if ((rc = ml_check(L, "mg_nested"))) return L == c ? rc : fail(c, rc, L->err);
    }
    return PORTA_OK;
}

}  // extern "C"
