// Launchers of the per-voxel kernels (see.cu); internal to the library.
#pragma once
#include <cuda_runtime.h>

#include "porta.h"

namespace porta {

template <typename Real>
cudaError_t run_profile_norm(long long nvox, int nray, int nnu, const double *mu, const double *xf, const double *wf,
                             const double *vel, void *invn, cudaStream_t st);
template <typename Real>
cudaError_t run_rho_convert(long long nvox, int nl, const double *rho, void *out, cudaStream_t st);
template <typename Real, int NS>
cudaError_t run_jkq_finalize(long long nvox, int nray, const void *part, const double *tw, double *jkq, double *lstar,
                             cudaStream_t st);
// J^1_Q [v][3] (J10, Re J11, Im J11) = sum_m tw1[m][c] partv[m][v]: tw1 = w_m T^1_Q(V, Omega_m),
// partv (Real [ray][nvox]) the per-ray frequency integrals of Stokes V
template <typename Real>
cudaError_t run_j1_finalize(long long nvox, int nray, const void *partv, const double *tw1, double *j1, cudaStream_t st);
// src: null (right-hand side eps B delta_K0) or a per-voxel right-hand side [v][nl]
template <typename Real>
cudaError_t run_see(long long nvox, int nl, int model, double bcrit, const double *eps, const double *bpl,
                    const double *bvec, const double *jkq, const double *lstar, double *rho, void *rhoR,
                    unsigned long long *resid, cudaStream_t st, const double *src = nullptr);
// reverse mode of the Jacobi update: dL/drho (explicit, overwritten), dL/dJ and dL/dLambda*
// (overwritten), dL/d(thermal term) and dL/dB (added)
cudaError_t run_see_vjp(long long nvox, int nl, int model, double bcrit, const double *eps, const double *bpl,
                        const double *bvec, const double *jkq, const double *lstar, const double *src,
                        const double *rho, const double *g, double *g_rho, double *g_jkq, double *g_lstar,
                        double *g_f, double *g_b, cudaStream_t st);
// out = alpha A(rho) + add (+ eps B delta_K0 if with_eb); out may alias add
cudaError_t run_see_apply(long long nvox, int nl, int model, double bcrit, const double *eps, const double *bpl,
                          const double *bvec, const double *jkq, const double *rho, double alpha, const double *add,
                          int with_eb, double *out, cudaStream_t st);
cudaError_t run_count_bad(long long n, const double *x, double lo_excl, double hi_incl, unsigned long long *bad,
                          cudaStream_t st);
template <typename Real>
cudaError_t run_coefficients(int n, const double *t, double *out, cudaStream_t st);
cudaError_t run_step_eval(int precision, int n, const double *in, double *out, cudaStream_t st);
template <typename Real>
cudaError_t run_to_real(long long n, const double *x, void *y, cudaStream_t st);

}  // namespace porta
