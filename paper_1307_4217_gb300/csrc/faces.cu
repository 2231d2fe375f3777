// Short characteristics that end on the first cell face they cross (Sec. 3.1:
// the upwind and downwind points M and P may lie on a vertical plane of the
// grid), for the J^K_Q formal solution of one box.
//
// Where the horizontal offset of a ray over a layer, (f_x, f_y) cells, exceeds
// one cell, the characteristic through a node leaves its cell through the
// vertical face x = x_(i + sgn f_x) (|f_x| >= |f_y|) or y = y_(j + sgn f_y), at
// the fraction s = 1 / max(|f_x|, |f_y|) of the layer; the face point's
// quantities are bilinear in the face's horizontal coordinate and in height
// between the two planes. The upwind face's upper nodes belong to the point's
// own plane, so the plane's intensities depend on each other; with periodic
// horizontal boundaries their chains close on themselves (Sec. 4.2). Each such
// plane is swept line by line in the upwind order (the points of a line depend
// only on the line before it), in place, and the pass repeated until no
// intensity changes by more than a tolerance of the plane's largest: the fixed
// point of the plane's SC relations (a pass carries the chain once around the
// periodic domain, so the wrap converges geometrically, by ~(1 - s)^n per pass
// over n lines). Where the offset stays within a cell, M (or P) lies on the
// neighbouring plane and one parallel pass is exact.
//
// One CTA of four warps per (ray, frequency group) item (a grid-stride loop over
// the items, about eight CTAs per SM), the group's frequencies in order, the
// planes in sweep order; the CTA's Stokes planes (upwind and current), its
// Lambda* plane and the per-frequency transfer coefficients of the planes ku, k
// and kd (computed once per plane and frequency) live in global scratch memory
// (L2-resident at these sizes); each item's partial sums (stored on its first
// frequency, added on the later ones) are added over the groups in group order
// into the general sweep's per-ray partials, which the J^K_Q finalize sums over
// rays in ray order. A plane that does not converge
// within maxpass passes sets bit 2 of the error flag and keeps its last pass.
#include <algorithm>

#include "device_math.cuh"
#include "faces_kernels.cuh"
#include "sweep_common.cuh"

namespace porta {

namespace {

// bilinear stencil (4 nodes, periodic) of the point at offset (fx, fy) cells from
// node (i, j) on a neighbouring plane
__device__ __forceinline__ void plane_stencil(int nx, int ny, int i, int j, double fx, double fy, int *ii, int *jj,
                                              double *w)
{
    const double xc = i + fx, yc = j + fy;
    const double x0 = floor(xc), y0 = floor(yc);
    const double gx = xc - x0, gy = yc - y0;
    const long long i0 = (long long)x0, j0 = (long long)y0;
    const int ia = (int)(((i0 % nx) + nx) % nx), ja = (int)(((j0 % ny) + ny) % ny);
    const int ib = ia + 1 == nx ? 0 : ia + 1, jb = ja + 1 == ny ? 0 : ja + 1;
    ii[0] = ia; jj[0] = ja; w[0] = (1 - gx) * (1 - gy);
    ii[1] = ib; jj[1] = ja; w[1] = gx * (1 - gy);
    ii[2] = ia; jj[2] = jb; w[2] = (1 - gx) * gy;
    ii[3] = ib; jj[3] = jb; w[3] = gx * gy;
}

// face stencil: nodes 0, 1 on the point's own plane (weight 1 - s), 2, 3 on the
// neighbouring plane (weight s); returns s
__device__ __forceinline__ double face_stencil(int nx, int ny, int i, int j, double fx, double fy, int *ii, int *jj,
                                               double *w)
{
    const double ax = fabs(fx), ay = fabs(fy);
    const double s = 1.0 / (ax >= ay ? ax : ay);
    const int sx = fx > 0 ? 1 : (fx < 0 ? -1 : 0), sy = fy > 0 ? 1 : (fy < 0 ? -1 : 0);
    int i0, j0, i1, j1;
    double g;
    if (ax >= ay) {
        i0 = i1 = i + sx;
        j0 = j;
        j1 = j + (sy != 0 ? sy : 1);
        g = ay * s;
    } else {
        j0 = j1 = j + sy;
        i0 = i;
        i1 = i + (sx != 0 ? sx : 1);
        g = ax * s;
    }
    i0 = ((i0 % nx) + nx) % nx; i1 = ((i1 % nx) + nx) % nx;
    j0 = ((j0 % ny) + ny) % ny; j1 = ((j1 % ny) + ny) % ny;
    ii[0] = i0; jj[0] = j0; w[0] = (1 - g) * (1 - s);
    ii[1] = i1; jj[1] = j1; w[1] = g * (1 - s);
    ii[2] = i0; jj[2] = j0; w[2] = (1 - g) * s;
    ii[3] = i1; jj[3] = j1; w[3] = g * s;
    return s;
}

template <typename Real>
__device__ __forceinline__ Real block_max(Real v, Real *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    Real t = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    return t;
}

// transfer coefficients of node v at frequency x: eta_I, eta_V (weak-field Zeeman) and
// eps (I, Q, U, V) as the general sweep forms them (Sec. 2)
template <typename Real, int NS>
__device__ __forceinline__ void node_coef(const Node<Real, NS> &n, Real x, Real &etaI, Real &etaV, Real *eps)
{
    const Real xs = x - n.s;
    etaI = n.chi * profile_shape(xs);
    if constexpr (NS == 1) {
        etaV = Real(0);
        eps[0] = etaI * n.S;
    } else {
        etaV = etaI * n.b * xs;
        eps[0] = etaI * n.SI;
        eps[1] = etaI * n.SQ;
        eps[2] = etaI * n.SU;
        eps[3] = etaV * n.S00;
    }
}

// the transfer coefficients of every node of plane k at frequency x: eta_I, eta_V,
// eps (NS) at cw[(c * nxy) + p], c = 0 .. NS + 1
template <typename Real, int NS>
__device__ __forceinline__ void plane_coefs(const SweepArgs<Real> &a, const RayDev<Real> &ray, int m, long long base,
                                            long long nxy, Real x, Real *cw)
{
    for (long long p = threadIdx.x; p < nxy; p += blockDim.x) {
        const Node<Real, NS> n = make_node<Real, NS>(a, ray, base + p, m, false);
        Real eI, eV, e4[NS];
        node_coef<Real, NS>(n, x, eI, eV, e4);
        cw[p] = eI;
        cw[nxy + p] = eV;
#pragma unroll
        for (int s = 0; s < NS; ++s) cw[(2 + s) * nxy + p] = e4[s];
    }
}

// One CTA per (ray, frequency group). Per frequency and plane: the coefficients of the planes k (the
// points and the upper nodes of their faces), ku (upwind) and kd (downwind) in the
// ray's scratch, then the plane's points. Where M lies on the upwind plane (offset
// within a cell) one parallel pass is exact; where it lies on vertical faces the
// plane is swept line by line in the upwind order (columns for x faces, rows for y
// faces: a line's points depend only on the line before), in place, and the pass is
// repeated until no intensity changes by more than tol of the plane's largest (the
// first line of a pass reads the last line of the previous one: the periodic chain).
template <typename Real, int NS>
__global__ void __launch_bounds__(128) faces_kernel(const SweepArgs<Real> a, Real *scratch, Real *gpart, int ngroups,
                                                   double dx, double dy, int maxpass, Real tol, int *err, int emergent)
{
    constexpr int NC = NS + 2;                    // coefficient words per node
    __shared__ Real red[4];
    const BoxDev B = a.boxes[0];
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const long long nxy = (long long)nx * ny;
    const int fper = (a.nnu + ngroups - 1) / ngroups;
    // work items: (ray, frequency group), each CTA with its own scratch slot
    for (int item = blockIdx.x; item < a.nray * ngroups; item += gridDim.x) {
        const int m = item / ngroups, grp = item - m * ngroups;
        const RayDev<Real> ray = a.rays[m];
        const PlaneGeom<Real> *G = a.geom + B.geom0 + (long long)m * nz;
        const bool upward = ray.mu > Real(0);
        // scratch of the CTA: I of the upwind plane and of the current one, Lambda*,
        // the coefficients of planes ku, k, kd
        Real *Iu = scratch + (long long)blockIdx.x * (2 * NS + 1 + 3 * NC) * nxy;
        Real *Ik = Iu + NS * nxy;
        Real *lsb = Ik + NS * nxy;
        Real *cu = lsb + nxy, *ck = cu + NC * nxy, *cd = ck + NC * nxy;
        // this item's partial sums over its frequencies: [ray][group][nvox]
        Real *part = gpart + ((long long)m * ngroups + grp) * a.nvox * (NS == 1 ? 2 : 4);
        const int jb = grp * fper, je = min(a.nnu, jb + fper);
        for (int j = jb; j < je; ++j) {
            const Real x = a.xf[j], wf = a.wf[j];
            for (int q = 0; q < nz; ++q) {
                const int k = G[q].kz;
                const long long base = B.vox0 + (long long)k * nxy;
                if (q == 0) {
                    for (long long p = threadIdx.x; p < nxy; p += blockDim.x) {
                        const long long v = base + p;
                        Real I0[NS];
#pragma unroll
                        for (int s = 0; s < NS; ++s) I0[s] = Real(0);
                        if (upward) I0[0] = a.bpl[v];
#pragma unroll
                        for (int s = 0; s < NS; ++s) Ik[s * nxy + p] = I0[s];
                        lsb[p] = Real(0);
                    }
                } else {
                    const int ku = G[q - 1].kz;
                    const bool has_p = q + 1 < nz;
                    const int kd = has_p ? G[q + 1].kz : k;
                    const double dsM = (double)G[q].ds, dsP = has_p ? (double)G[q + 1].ds : 0.0;
                    const double fxM = -dsM * (double)ray.ox / dx, fyM = -dsM * (double)ray.oy / dy;
                    const double fxP = dsP * (double)ray.ox / dx, fyP = dsP * (double)ray.oy / dy;
                    const bool vertM = fabs(fxM) > 1.0 || fabs(fyM) > 1.0;
                    const bool vertP = has_p && (fabs(fxP) > 1.0 || fabs(fyP) > 1.0);
                    // the finished plane becomes the upwind one; coefficients of ku, k, kd
                    for (long long e = threadIdx.x; e < NS * nxy; e += blockDim.x) {
                        Iu[e] = Ik[e];
                        Ik[e] = Real(0);
                    }
                    plane_coefs<Real, NS>(a, ray, m, B.vox0 + (long long)ku * nxy, nxy, x, cu);
                    plane_coefs<Real, NS>(a, ray, m, base, nxy, x, ck);
                    if (has_p) plane_coefs<Real, NS>(a, ray, m, B.vox0 + (long long)kd * nxy, nxy, x, cd);
                    __syncthreads();
                    // one point's update (in place into Ik); returns the change of its Stokes vector
                    auto update = [&](int ix, int jy, Real &chg, Real &mag) {
                        const long long p = (long long)jy * nx + ix;
                        int ii[4], jj[4];
                        double w[4];
                        Real etaM = 0, etaVM = 0, epsM[NS], IM[NS];
#pragma unroll
                        for (int s = 0; s < NS; ++s) epsM[s] = IM[s] = Real(0);
                        double sM = 1.0;
                        if (vertM) sM = face_stencil(nx, ny, ix, jy, fxM, fyM, ii, jj, w);
                        else plane_stencil(nx, ny, ix, jy, fxM, fyM, ii, jj, w);
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const bool own = vertM && c < 2;
                            const Real *cc = own ? ck : cu;
                            const Real *Ib = own ? Ik : Iu;
                            const long long pc = (long long)jj[c] * nx + ii[c];
                            const Real wc = (Real)w[c];
                            etaM += wc * cc[pc];
                            etaVM += wc * cc[nxy + pc];
#pragma unroll
                            for (int s = 0; s < NS; ++s) {
                                epsM[s] += wc * cc[(2 + s) * nxy + pc];
                                IM[s] += wc * Ib[s * nxy + pc];
                            }
                        }
                        const Real etaO = ck[p], etaVO = ck[nxy + p];
                        Real epsO[NS];
#pragma unroll
                        for (int s = 0; s < NS; ++s) epsO[s] = ck[(2 + s) * nxy + p];
                        Real etaP = 0, epsP[NS];
#pragma unroll
                        for (int s = 0; s < NS; ++s) epsP[s] = Real(0);
                        double sP = 1.0;
                        if (has_p) {
                            if (vertP) sP = face_stencil(nx, ny, ix, jy, fxP, fyP, ii, jj, w);
                            else plane_stencil(nx, ny, ix, jy, fxP, fyP, ii, jj, w);
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const Real *cc = vertP && c < 2 ? ck : cd;
                                const long long pc = (long long)jj[c] * nx + ii[c];
                                const Real wc = (Real)w[c];
                                etaP += wc * cc[pc];
#pragma unroll
                                for (int s = 0; s < NS; ++s) epsP[s] += wc * cc[(2 + s) * nxy + pc];
                            }
                        }
                        const Real dM = (Real)(sM * dsM), dP = (Real)(sP * dsP);
                        Real IO[NS], ls;
                        if constexpr (NS == 1) {
                            const Real SM = epsM[0] / etaM, SO = epsO[0] / etaO;
                            const Real tMO = Real(0.5) * (etaM + etaO) * dM;
                            const Coef<Real> co = coefficients(tMO);
                            Real cM;
                            if (has_p) {
                                const Real SP = epsP[0] / etaP, tOP = Real(0.5) * (etaO + etaP) * dP;
                                cM = control_point(SM, SO, SP, besser_geom(tMO, tOP));
                            } else {
                                cM = Real(0.5) * (SM + SO);
                            }
                            IO[0] = co.e * IM[0] + co.wm * SM + co.wo * SO + co.wc * cM;
                            ls = co.wo + (has_p ? co.wc : Real(0.5) * co.wc);
                        } else {
                            const Real etaM7[7] = {etaM, 0, 0, etaVM, 0, 0, 0}, etaO7[7] = {etaO, 0, 0, etaVO, 0, 0, 0};
                            delo_step_general<Real>(IM, etaM7, epsM, etaO7, epsO, etaP, epsP, dM, dP, has_p, IO, ls);
                        }
#pragma unroll
                        for (int s = 0; s < NS; ++s) {
                            chg = fmax(chg, fabs(IO[s] - Ik[s * nxy + p]));
                            mag = fmax(mag, fabs(IO[s]));
                            Ik[s * nxy + p] = IO[s];
                        }
                        lsb[p] = ls;
                    };
                    if (!vertM) {
                        Real chg = 0, mag = 0;
                        for (long long p = threadIdx.x; p < nxy; p += blockDim.x) {
                            const int jy = (int)(p / nx), ix = (int)(p - (long long)jy * nx);
                            update(ix, jy, chg, mag);
                        }
                    } else {
                        // lines in the upwind order: a point depends on the line at +sgn(f)
                        const bool xface = fabs(fxM) >= fabs(fyM);
                        const int n_lines = xface ? nx : ny, n_pts = xface ? ny : nx;
                        const int step = xface ? (fxM > 0 ? -1 : 1) : (fyM > 0 ? -1 : 1);
                        for (int pass = 0;; ++pass) {
                            Real chg = 0, mag = 0;
                            for (int t = 0; t < n_lines; ++t) {
                                const int line = (((step * t) % n_lines) + n_lines) % n_lines;
                                for (int i = threadIdx.x; i < n_pts; i += blockDim.x) {
                                    if (xface) update(line, i, chg, mag);
                                    else update(i, line, chg, mag);
                                }
                                __syncthreads();
                            }
                            chg = block_max(chg, red);
                            mag = block_max(mag, red);
                            if (!(chg > tol * mag)) break;
                            if (pass + 1 >= maxpass) {
                                if (threadIdx.x == 0) atomicOr(err, 2);
                                break;
                            }
                        }
                    }
                }
                __syncthreads();
                if (emergent) {
                    // lines of sight: the Stokes vectors of the top plane, [dir][nu][y][x][ns]
                    if (q == nz - 1)
                        for (long long p = threadIdx.x; p < nxy; p += blockDim.x)
#pragma unroll
                            for (int s = 0; s < NS; ++s)
                                a.out[(((long long)m * a.nnu + j) * nxy + p) * NS + s] = (double)Ik[s * nxy + p];
                    __syncthreads();
                    continue;
                }
                // the plane's sums: w_j phi_O / N (I, Q, U, Lambda*) added to the ray's partials
                for (long long p = threadIdx.x; p < nxy; p += blockDim.x) {
                    const long long vO = base + p;
                    const Node<Real, NS> nO = make_node<Real, NS>(a, ray, vO, m, true);
                    const Real wt = wf * profile_shape(x - nO.s) * nO.invn;
                    if constexpr (NS == 1) {
                        R2<Real> *pp = reinterpret_cast<R2<Real> *>(part) + vO;
                        R2<Real> o = {wt * Ik[p], wt * lsb[p]};
                        if (j > jb) { const R2<Real> old = *pp; o.x += old.x; o.y += old.y; }
                        *pp = o;
                    } else {
                        R4<Real> *pp = reinterpret_cast<R4<Real> *>(part) + vO;
                        R4<Real> o = {wt * Ik[p], wt * Ik[nxy + p], wt * Ik[2 * nxy + p], wt * lsb[p]};
                        if (j > jb) { const R4<Real> old = *pp; o.x += old.x; o.y += old.y; o.z += old.z; o.w += old.w; }
                        *pp = o;
                    }
                }
                __syncthreads();
            }
        }
    }
}

// per ray and voxel: the frequency groups' partial sums added in group order
template <typename Real, int NA>
__global__ void faces_group_sum_kernel(const Real *gpart, int ngroups, long long nvox, int nray, Real *part)
{
    const long long n = (long long)nray * nvox;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long m = e / nvox, v = e - m * nvox;
        Real s[NA] = {};
        for (int g = 0; g < ngroups; ++g) {
            const Real *p = gpart + ((m * ngroups + g) * nvox + v) * NA;
#pragma unroll
            for (int c = 0; c < NA; ++c) s[c] += p[c];
        }
#pragma unroll
        for (int c = 0; c < NA; ++c) part[e * NA + c] = s[c];
    }
}

}  // namespace

// frequency groups per ray: enough (ray, group) items for ~8 CTAs per SM
int faces_groups(int nray, int nnu)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, std::min(nnu, (8 * std::max(1, nsm) + nray - 1) / std::max(1, nray)));
}

template <typename Real, int NS>
size_t faces_scratch_bytes(int nray, int nnu, long long nxy, long long nvox)
{
    const int ng = faces_groups(nray, nnu);
    const long long items = (long long)nray * ng;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long ctas = std::min<long long>(items, 8LL * std::max(1, nsm));
    return sizeof(Real) * ((size_t)ctas * (2 * NS + 1 + 3 * (NS + 2)) * nxy + (size_t)items * nvox * (NS == 1 ? 2 : 4));
}

template <typename Real, int NS>
cudaError_t launch_faces(const SweepArgs<Real> &a, Real *scratch, long long nxy, double dx, double dy, int maxpass,
                         int *err, cudaStream_t st, bool emergent)
{
    const Real tol = sizeof(Real) == 8 ? Real(1e-15) : Real(2e-7);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int ng = faces_groups(a.nray, a.nnu);
    const long long items = (long long)a.nray * ng;
    const int ctas = (int)std::min<long long>(items, 8LL * std::max(1, nsm));
    Real *gpart = scratch + (size_t)ctas * (2 * NS + 1 + 3 * (NS + 2)) * nxy;
    faces_kernel<Real, NS><<<ctas, 128, 0, st>>>(a, scratch, gpart, ng, dx, dy, maxpass, tol, err, emergent ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || emergent) return e;
    const long long n = (long long)a.nray * a.nvox;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 16LL * std::max(1, nsm));
    faces_group_sum_kernel<Real, NS == 1 ? 2 : 4><<<blocks, 256, 0, st>>>(gpart, ng, a.nvox, a.nray, (Real *)a.part);
    return cudaGetLastError();
}

#define PORTA_FACES_INST(R, N)                                                                              \
    template cudaError_t launch_faces<R, N>(const SweepArgs<R> &, R *, long long, double, double, int, int *,   \
                                            cudaStream_t, bool);                                               \
    template size_t faces_scratch_bytes<R, N>(int, int, long long, long long);
PORTA_FACES_INST(float, 1)
PORTA_FACES_INST(float, 4)
PORTA_FACES_INST(double, 1)
PORTA_FACES_INST(double, 4)
#undef PORTA_FACES_INST

}  // namespace porta
