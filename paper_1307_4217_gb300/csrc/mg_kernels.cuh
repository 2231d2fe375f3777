// Launchers of the multigrid grid-transfer kernels (mg.cu); internal to the library.
#pragma once
#include <cuda_runtime.h>

namespace porta {

constexpr int kMgMaxComp = 8;   // unknowns per voxel the transfer kernels accumulate at a time

// coarse = fine at the coincident nodes, one per-voxel array
cudaError_t run_inject(int nxc, int nyc, int nzc, int nxf, int nyf, const double *fine, double *coarse, cudaStream_t st);
// restriction [v][nl] fine -> coarse; zr: per coarse plane 4 x (fine plane, weight)
cudaError_t run_restrict(int nxc, int nyc, int nzc, int nxf, int nyf, int nl, const double *zr, const double *fine,
                         double *coarse, cudaStream_t st);
// fine += P (cnew - cold), or with assign fine = P (cnew - cold); cold may be null (zero);
// order 1 (tri-linear; zp: per fine plane 2 (coarse plane, weight) pairs) or 3
// (tri-cubic-centered; zp: 4 pairs per fine plane)
cudaError_t run_prolong(int nxf, int nyf, int nzf, int nxc, int nyc, int nl, int order, const double *zp,
                        const double *cnew, const double *cold, double *fine, int assign, cudaStream_t st);
// coarse = fine at the coincident nodes, nl components per voxel
cudaError_t run_inject_vec(int nxc, int nyc, int nzc, int nxf, int nyf, int nl, const double *fine, double *coarse,
                           cudaStream_t st);
// max relative change between two vectors of unknowns (atomic max on the IEEE bits in *resid):
// of S00 and of S2/S00, or with rel_all of every component
cudaError_t run_change(long long nvox, int nl, const double *old, const double *cur, unsigned long long *resid,
                       cudaStream_t st, int rel_all = 0);
// max over voxels of max_c |r| / max_c |x| (atomic max on the IEEE bits in *out)
cudaError_t run_rel_residual(long long nvox, int nl, const double *r, const double *x, unsigned long long *out,
                             cudaStream_t st);
// y += alpha x
cudaError_t run_axpy(long long n, double alpha, const double *x, double *y, cudaStream_t st);

}  // namespace porta
