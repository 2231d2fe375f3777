// Short characteristics ending on the first cell face they cross (faces.cu);
// internal to the library.
#pragma once
#include <cuda_runtime.h>

#include "porta_internal.cuh"

namespace porta {

// The J^K_Q formal solution of nbox boxes (at most nxy_max points per plane;
// dxy[2 b], dxy[2 b + 1]: the cell sizes of box b, on the device) with the face
// placement: per-ray partials into a.part; scratch holds the per-CTA work planes
// and, with more than one frequency group, the per-(ray, group) partial sums
// (faces_scratch_bytes; medium 1: the dichroism variant, used when a.dich is set,
// with the Stokes-V integrals into a.partv; medium 2: an explicit medium, used when
// a.kexpl is set, with the seven-element step); a plane still changing after maxpass passes sets bit 2
// of *err. emergent: one box, a.rays are lines of sight (mu > 0) and the top
// plane's Stokes vectors go to a.out ([dir][nu][y][x][ns], FP64) instead of the sums.
// planes: M and P on the neighbouring horizontal planes at any offset (the plane
// placement of the shared-memory sweeps, here with the work planes in global memory:
// the sweep for planes too wide for the shared-memory ring)
template <typename Real, int NS>
cudaError_t launch_faces(const SweepArgs<Real> &a, Real *scratch, int nbox, long long nxy_max, const double *dxy,
                         int maxpass, int *err, cudaStream_t st, bool emergent = false, bool planes = false);
template <typename Real, int NS>
size_t faces_scratch_bytes(int nbox, int nray, int nnu, long long nxy_max, long long nvox, int medium = 0);

}  // namespace porta
