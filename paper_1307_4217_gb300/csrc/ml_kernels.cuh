// Multilevel atom without polarization (populations only): constants of the
// model atom and the launchers of ml.cu; internal to the library.
#pragma once
#include <cuda_runtime.h>

namespace porta {

constexpr int kMlMaxLevel = 8;
constexpr int kMlMaxLine = 8;

// per-line constants derived on the host from the atom (energies in eV,
// intensities in units of 2 h nu^3 / c^2 of line 0)
struct MlConst {
    int nlev, nline;
    double g[kMlMaxLevel];          // 2J + 1
    int up[kMlMaxLine], lo[kMlMaxLine];
    double A[kMlMaxLine];           // Einstein A (s^-1)
    double Bul[kMlMaxLine];         // A / r^3 (r = dE / dE_ref)
    double Blu[kMlMaxLine];         // (g_u / g_l) Bul
    double Cul[kMlMaxLine];         // eps A / (1 - eps)
    double dE[kMlMaxLine];          // E_u - E_l (eV)
    double r3[kMlMaxLine];          // r^3
    double s[kMlMaxLine];           // opacity strength relative to line 0
};

// per line k and voxel v: line-centre opacity, source function and Planck
// function into the sweep arrays of box k (chi, bpl: the Real atmosphere
// planes; S: the Real and FP64 unknowns); counts voxels whose line opacity is
// not positive or whose source function is not finite into *bad
template <typename Real>
cudaError_t run_ml_prepare(const MlConst &mc, long long nvox1, const double *pops, const double *chis, const double *kT,
                           Real *chi_out, Real *bpl_out, Real *S_out, double *S64_out, unsigned long long *bad,
                           cudaStream_t st);

// preconditioned rate equations per voxel (Jbar, Lambda-bar* per line in
// [line][voxel] order), populations updated in place; the maximum relative
// change goes to *resid as the IEEE bits of a non-negative double (atomic
// max), non-finite or non-positive results count into *bad
// src (per voxel, nlev; null: (1, 0, ..., 0)) is the right-hand side of the
// rate equations with their conservation row (coarse-grid equations)
cudaError_t run_ml_see(const MlConst &mc, long long nvox1, const double *kT, const double *jbar, const double *lstar,
                       double *pops, unsigned long long *resid, unsigned long long *bad, cudaStream_t st,
                       const double *src = nullptr);

// out = alpha A(n) + add + with_f (1, 0, ..., 0) with A(n)_0 = sum_i n_i and
// A(n)_i = (M n)_i for the plain radiative rates of Jbar (i >= 1); add may be null
cudaError_t run_ml_apply(const MlConst &mc, long long nvox1, const double *kT, const double *jbar, const double *pops,
                         double alpha, const double *add, int with_f, double *out, cudaStream_t st);

}  // namespace porta
