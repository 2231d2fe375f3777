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
// radiation tensors (J00, J20, Re J21, Im J21, Re J22, Im J22 per line), the
// field (3), the collisional excitation rate per line, -Lambda* S_old and
// -Lambda* per line
struct MlPolTables {
    // With J^1_Q = 0 the odd-K multipoles decouple from the even ones and their
    // equations are homogeneous (zero solution): the system is assembled and
    // solved over the nact even-K unknowns act[] only; cells, trace, row0 and apop
    // are in that compact numbering, pop_idx and up2 in the full one.
    int nline = 0, nunk = 0, nsrc = 0, row0 = -1, nact = 0;
    std::vector<int> act, inact, apop;
    int src_j = 0, src_b = 0, src_clu = 0, src_pop = 0, src_spop = 0;
    std::vector<double> trace;       // trace row (sqrt(2J+1) on each rho^0_0)
    std::vector<int> pop_idx;        // per level: index of rho^0_0
    std::vector<int> up2;            // per line: rho^0_0, rho^2_0, Re/Im rho^2_1, Re/Im rho^2_2 of the upper level (-1: none)
    std::vector<double> w2;          // per line: w^(2)_{Ju Jl}
    std::vector<int> lo2;            // per line: the same six indices for the lower level (-1: none)
    std::vector<double> w2lo;        // per line: w^(2)_{Jl Ju}
    std::vector<int> cell_rc, cell_start, ent_src;
    std::vector<double> ent_coef;
};

// device copy (pointers into one allocation)
struct MlPolDev {
    int nunk, nsrc, ncell, row0, nact, ninact;
    int src_j, src_b, src_clu, src_pop, src_spop;
    const int *pop_idx, *up2, *cell_rc, *cell_start, *ent_src, *act, *inact, *apop, *lo2;
    const double *w2, *trace, *ent_coef, *w2lo;
};

// build the tables of an atom (levels J, energies E in eV; lines up/lo with A, eps); 0 on success
int mlpol_tables(const std::vector<double> &J, const std::vector<double> &E, const std::vector<int> &up,
                 const std::vector<int> &lo, const std::vector<double> &A, const std::vector<double> &eps,
                 MlPolTables &t);

// per line and voxel: opacity, Planck function and the emission multipoles
// S^K_Q (two-level real layout, AoS FP64 and SoA Real) from the unknowns x [v][nunk]
// and the dichroism multipoles D^2_Q of each line (Real SoA [5][line voxel])
template <typename Real>
cudaError_t run_mlpol_prepare(const MlConst &mc, const MlPolDev &T, long long nvox1, const double *x, const double *chis,
                              const double *kT, Real *chi_out, Real *bpl_out, Real *S_out, double *S64_out,
                              Real *dich_out, unsigned long long *bad, cudaStream_t st);

// the rate equations per voxel (jkq [line voxel][6], lstar [line voxel], bvec [3][line voxel]);
// x updated in place, max relative population change into *resid
// src (per voxel, nunk; null: e_row0) is the right-hand side (coarse-grid equations)
cudaError_t run_mlpol_see(const MlConst &mc, const MlPolDev &T, long long nvox1, const double *kT, const double *jkq,
                          const double *lstar, const double *bvec, double *x, unsigned long long *resid,
                          unsigned long long *bad, cudaStream_t st, const double *src = nullptr);

// out = alpha A(x) + add + with_f e_row0 with A the plain rate operator (trace row for
// level 0's population); add may be null; full layout [v][nunk]
cudaError_t run_mlpol_apply(const MlConst &mc, const MlPolDev &T, long long nvox1, const double *kT, const double *jkq,
                            const double *bvec, const double *x, double alpha, const double *add, int with_f,
                            double *out, cudaStream_t st);

size_t mlpol_see_smem(const MlPolDev &T, int warps);

// max relative change of the populations between two vectors of unknowns (atomic max on the bits in *resid)
cudaError_t run_mlpol_change(const MlConst &mc, const MlPolDev &T, long long nvox1, const double *old, const double *cur,
                             unsigned long long *resid, cudaStream_t st);

}  // namespace porta
