// C ABI, multilevel atoms: creation from the atomic model, the populations
// (or multipole components) as unknowns, their line data for the sweeps, the
// rate equations and the emergent profiles of each line.
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

// the error counter of the line data and of the rate equations (synchronizes)
int ml_check(porta_ctx *c, const char *what)
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

}  // namespace porta_api

using namespace porta_api;

extern "C" {

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
        const std::vector<int> *iv[6] = {&tab.pop_idx, &tab.upk, &tab.lok, &tab.cell_rc, &tab.cell_start, &tab.ent_src};
        const std::vector<double> *dv[4] = {&tab.wu, &tab.wl, &tab.trace, &tab.ent_coef};
        size_t ni = 0, nd = 0;
        for (auto *p : iv) ni += p->size();
        for (auto *p : dv) nd += p->size();
        const size_t ibytes = (ni * sizeof(int) + 7) / 8 * 8;
        std::vector<char> h(ibytes + nd * sizeof(double));
        int *ip = (int *)h.data();
        double *dp = (double *)(h.data() + ibytes);
        size_t io[6], doff[4], k = 0, kd = 0;
        for (int q2 = 0; q2 < 6; ++q2) {
            io[q2] = k;
            for (int x : *iv[q2]) ip[k++] = x;
        }
        for (int q2 = 0; q2 < 4; ++q2) {
            doff[q2] = kd;
            for (double x : *dv[q2]) dp[kd++] = x;
        }
        e = pmalloc(&m->d_tab, h.size());
        if (e == cudaSuccess) e = cudaMemcpy(m->d_tab, h.data(), h.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = dalloc(&m->d_x, (size_t)m->nvox1 * tab.nunk);
        // line polarization terms of the sweep ([11][line voxel]), J^1_Q and w_m T^1_Q(V, Omega_m)
        // = w_m sqrt(3/2) Omega_Q per ray (T10 = sqrt(3/2) Omega_z, T11 = -sqrt(3/4) (Omega_x + i Omega_y))
        if (e == cudaSuccess) e = pmalloc(&c->d_dich, (size_t)11 * c->nvox * c->rsz);
        if (e == cudaSuccess) e = cudaMemset(c->d_dich, 0, (size_t)11 * c->nvox * c->rsz);
        if (e == cudaSuccess) e = dalloc(&c->d_j1, (size_t)3 * c->nvox);
        if (e == cudaSuccess) e = cudaMemset(c->d_j1, 0, (size_t)3 * c->nvox * sizeof(double));
        if (e == cudaSuccess) e = dalloc(&c->d_tw1, (size_t)3 * c->nray);
        if (e == cudaSuccess) {
            std::vector<double> tw1((size_t)3 * c->nray);
            for (int r = 0; r < c->nray; ++r) {
                const double st = std::sqrt(1.0 - c->mu[r] * c->mu[r]);
                tw1[3 * r] = c->w[r] * std::sqrt(1.5) * c->mu[r];
                tw1[3 * r + 1] = -c->w[r] * std::sqrt(0.75) * st * std::cos(c->chi[r]);
                tw1[3 * r + 2] = -c->w[r] * std::sqrt(0.75) * st * std::sin(c->chi[r]);
            }
            e = cudaMemcpy(c->d_tw1, tw1.data(), tw1.size() * sizeof(double), cudaMemcpyHostToDevice);
        }
        const int *di = (const int *)m->d_tab;
        const double *dd = (const double *)((const char *)m->d_tab + ibytes);
        MlPolDev &d = m->dev;
        d.nunk = tab.nunk;
        d.solve = 0;
        d.nsrc = tab.nsrc;
        d.ncell = (int)tab.cell_start.size() - 1;
        d.row0 = tab.row0;
        d.src_j = tab.src_j; d.src_b = tab.src_b; d.src_clu = tab.src_clu; d.src_pop = tab.src_pop; d.src_spop = tab.src_spop;
        d.pop_idx = di + io[0]; d.upk = di + io[1]; d.lok = di + io[2];
        d.cell_rc = di + io[3]; d.cell_start = di + io[4]; d.ent_src = di + io[5];
        d.wu = dd + doff[0]; d.wl = dd + doff[1]; d.trace = dd + doff[2]; d.ent_coef = dd + doff[3];
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

int porta_ml_set_solve(porta_ctx *c, int mode)
{
    if (!c) return PORTA_EINVAL;
    if (!c->ml || !c->ml->pol) return fail(c, PORTA_EINVAL, "ml_set_solve: not a polarized multilevel context");
    if (mode != 0 && mode != 1) return fail(c, PORTA_EINVAL, "ml_set_solve: mode 0 or 1");
    c->ml->dev.solve = mode;
    drop_graph(c);
    return PORTA_OK;
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

int porta_ml_formal_solve(porta_ctx *c, double *jbar, double *lstar, int where)
{
    if (!c) return PORTA_EINVAL;
    MlState *m = c->ml;
    if (!m) return fail(c, PORTA_EINVAL, "ml_formal_solve: not a multilevel context");
    if (!m->have_atm || !m->have_pops) return fail(c, PORTA_ESTATE, "ml_formal_solve: atmosphere or populations not set");
    int rc = porta_formal_solve(c);
    if (rc != PORTA_OK) return rc;
    if (!m->pol) return porta_accumulate_jkq(c, jbar, lstar, where);
    // polarized lines: jbar [line voxel][9] in the Kr = 0, 1, 2 layout
    rc = porta_accumulate_jkq(c, nullptr, lstar, where);
    if (rc != PORTA_OK || !jbar) return rc;
    double *d9 = jbar;
    if (where == PORTA_HOST) CK(dalloc(&d9, (size_t)9 * c->nvox));
    cudaError_t e = run_mlpol_jbar9(c->nvox, c->d_jkq, c->d_j1, d9, c->stream);
    if (e == cudaSuccess && where == PORTA_HOST) {
        e = cudaMemcpyAsync(jbar, d9, (size_t)9 * c->nvox * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (where == PORTA_HOST) pfree(d9);
    if (e != cudaSuccess) return fail(c, PORTA_ECUDA, std::string("ml_formal_solve: ") + cudaGetErrorString(e));
    return PORTA_OK;
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
