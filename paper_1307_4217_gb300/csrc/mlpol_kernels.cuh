// Polarized multilevel atom: rate-equation tables (host) and the launchers of
// mlpol.cu; internal to the library.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "ml_kernels.cuh"

namespace porta {

constexpr int kMlPolMaxUnk = 128;           // real unknowns per voxel (sum of (2J+1)^2)
constexpr double kLarmorPerGauss = 1.3996e6;   // Larmor frequency per gauss (Hz)

// the rate equations as sparse (row, column) cells over the real unknowns,
// each cell a sum of coefficient x source; sources per voxel: 1, the line
// radiation tensors (J00, J10, Re J11, Im J11, J20, Re J21, Im J21, Re J22,
// Im J22 per line), the field (3), the collisional excitation rate per line,
// -Lambda* S_old and -Lambda* per line
struct MlPolTables {
    // J^1_Q (from Stokes V) couples the odd-K multipoles to the even ones: the
    // system is assembled and solved over all nunk unknowns
    int nline = 0, nunk = 0, nsrc = 0, row0 = -1;
    int src_j = 0, src_b = 0, src_clu = 0, src_pop = 0, src_spop = 0;
    std::vector<double> trace;       // trace row (sqrt(2J+1) on each rho^0_0)
    std::vector<int> pop_idx;        // per level: index of rho^0_0
    // per line: indices of rho^0_0, rho^1_0, Re/Im rho^1_1, rho^2_0, Re/Im rho^2_1,
    // Re/Im rho^2_2 of the upper level (upk) and of the lower level (lok); -1: none
    std::vector<int> upk, lok;
    std::vector<double> wu, wl;      // per line: (w^(1), w^(2)) of the upper level {Ju Jl} and of the lower {Jl Ju}
    std::vector<int> cell_rc, cell_start, ent_src;
    std::vector<double> ent_coef;
};

// device copy (pointers into one allocation)
struct MlPolDev {
    int nunk, nsrc, ncell, row0;
    int solve;                       // K > 0 block: 0 FP32 factors + FP64 refinement, 1 FP64 elimination
    int src_j, src_b, src_clu, src_pop, src_spop;
    const int *pop_idx, *upk, *lok, *cell_rc, *cell_start, *ent_src;
    const double *wu, *wl, *trace, *ent_coef;
};

// build the tables of an atom (levels J, energies E in eV; lines up/lo with A, eps); 0 on success
int mlpol_tables(const std::vector<double> &J, const std::vector<double> &E, const std::vector<int> &up,
                 const std::vector<int> &lo, const std::vector<double> &A, const std::vector<double> &eps,
                 MlPolTables &t);

// per line and voxel: opacity, Planck function and the emission multipoles
// S^K_Q (K = 0, 2; two-level real layout, AoS FP64 and SoA Real) from the unknowns
// x [v][nunk]; pol_out (Real SoA [11][line voxel]): the dichroism multipoles D^2_Q
// (5), D^1_Q (3) and the orientation emission multipoles S^1_Q (3) of each line
template <typename Real>
cudaError_t run_mlpol_prepare(const MlConst &mc, const MlPolDev &T, long long nvox1, const double *x, const double *chis,
                              const double *kT, Real *chi_out, Real *bpl_out, Real *S_out, double *S64_out,
                              Real *pol_out, unsigned long long *bad, cudaStream_t st);

// the rate equations per voxel (jkq [line voxel][6] = J00, J20, Re/Im J21, Re/Im J22,
// j1 [line voxel][3] = J10, Re/Im J11, lstar [line voxel], bvec [3][line voxel]);
// x updated in place, max relative population change into *resid
// src (per voxel, nunk; null: e_row0) is the right-hand side (coarse-grid equations)
cudaError_t run_mlpol_see(const MlConst &mc, const MlPolDev &T, long long nvox1, const double *kT, const double *jkq,
                          const double *j1, const double *lstar, const double *bvec, double *x, unsigned long long *resid,
                          unsigned long long *bad, cudaStream_t st, const double *src = nullptr);

// out = alpha A(x) + add + with_f e_row0 with A the plain rate operator (trace row for
// level 0's population); add may be null; full layout [v][nunk]
cudaError_t run_mlpol_apply(const MlConst &mc, const MlPolDev &T, long long nvox1, const double *kT, const double *jkq,
                            const double *j1, const double *bvec, const double *x, double alpha, const double *add, int with_f,
                            double *out, cudaStream_t st);

// dynamic shared memory of the rate-equation kernels for `voxels` voxels per CTA
size_t mlpol_see_smem(const MlPolDev &T, int voxels);

// jbar [line voxel][9] (J00, J10, Re/Im J11, J20, Re/Im J21, Re/Im J22) from jkq and j1
cudaError_t run_mlpol_jbar9(long long n, const double *jkq, const double *j1, double *jbar, cudaStream_t st);

// max relative change of the populations between two vectors of unknowns (atomic max on the bits in *resid)
cudaError_t run_mlpol_change(const MlConst &mc, const MlPolDev &T, long long nvox1, const double *old, const double *cur,
                             unsigned long long *resid, cudaStream_t st);

}  // namespace porta
