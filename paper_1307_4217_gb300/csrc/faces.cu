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
// plane is solved here by Jacobi passes over all its points (every pass from
// the previous pass's values of the plane and the finished upwind plane)
// repeated until no intensity changes by more than a tolerance of the plane's
// largest: the fixed point of the plane's SC relations. Where the offset stays
// within a cell, M (or P) lies on the neighbouring plane and one pass is exact.
//
// One CTA per ray (a grid-stride loop over rays), the frequencies in order, the
// planes in sweep order; the ray's three plane buffers (the upwind plane and
// two iterates of the current one) and its Lambda* plane live in global scratch
// memory; the per-ray partial sums are those of the general sweep (stored on
// the first frequency, added on the later ones, then summed over rays in ray
// order by the J^K_Q finalize). A plane that does not converge within maxpass
// passes sets bit 2 of the error flag and keeps its last pass.
#include <algorithm>

#include "device_math.cuh"
#include "porta_internal.cuh"
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

template <typename Real, int NS>
__global__ void __launch_bounds__(256) faces_kernel(const SweepArgs<Real> a, Real *scratch, double dx, double dy,
                                                   int maxpass, Real tol, int *err)
{
    __shared__ Real red[8];
    const BoxDev B = a.boxes[0];
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const long long nxy = (long long)nx * ny;
    for (int m = blockIdx.x; m < a.nray; m += gridDim.x) {
        const RayDev<Real> ray = a.rays[m];
        const PlaneGeom<Real> *G = a.geom + B.geom0 + (long long)m * nz;
        const bool upward = ray.mu > Real(0);
        Real *buf[3] = {scratch + ((long long)m * (3 * NS + 1)) * nxy, nullptr, nullptr};
        buf[1] = buf[0] + NS * nxy;
        buf[2] = buf[1] + NS * nxy;
        Real *lsb = buf[2] + NS * nxy;
        for (int j = 0; j < a.nnu; ++j) {
            const Real x = a.xf[j], wf = a.wf[j];
            int up = 0;                                   // buffer of the finished upwind plane
            for (int q = 0; q < nz; ++q) {
                const int k = G[q].kz;
                if (q == 0) {
                    for (long long p = threadIdx.x; p < nxy; p += blockDim.x) {
                        const long long v = B.vox0 + (long long)k * nxy + p;
                        Real I0[NS];
#pragma unroll
                        for (int s = 0; s < NS; ++s) I0[s] = Real(0);
                        if (upward) I0[0] = a.bpl[v];
#pragma unroll
                        for (int s = 0; s < NS; ++s) buf[0][s * nxy + p] = I0[s];
                        const Node<Real, NS> nO = make_node<Real, NS>(a, ray, v, m, true);
                        const Real wt = wf * profile_shape(x - nO.s) * nO.invn;
                        Real acc[NS == 1 ? 2 : 4] = {};
                        acc[0] = wt * I0[0];
                        if constexpr (NS == 1) {
                            R2<Real> *pp = reinterpret_cast<R2<Real> *>(a.part) + (long long)m * a.nvox + v;
                            R2<Real> o = {acc[0], acc[1]};
                            if (j > 0) { const R2<Real> old = *pp; o.x += old.x; o.y += old.y; }
                            *pp = o;
                        } else {
                            R4<Real> *pp = reinterpret_cast<R4<Real> *>(a.part) + (long long)m * a.nvox + v;
                            R4<Real> o = {acc[0], acc[1], acc[2], acc[3]};
                            if (j > 0) { const R4<Real> old = *pp; o.x += old.x; o.y += old.y; o.z += old.z; o.w += old.w; }
                            *pp = o;
                        }
                    }
                    __syncthreads();
                    continue;
                }
                const int ku = G[q - 1].kz;
                const bool has_p = q + 1 < nz;
                const int kd = has_p ? G[q + 1].kz : k;
                const double dsM = (double)G[q].ds, dsP = has_p ? (double)G[q + 1].ds : 0.0;
                const double fxM = -dsM * (double)ray.ox / dx, fyM = -dsM * (double)ray.oy / dy;
                const double fxP = dsP * (double)ray.ox / dx, fyP = dsP * (double)ray.oy / dy;
                const bool vertM = fabs(fxM) > 1.0 || fabs(fyM) > 1.0;
                const bool vertP = has_p && (fabs(fxP) > 1.0 || fabs(fyP) > 1.0);
                int cur = (up + 1) % 3, nxt = (up + 2) % 3;
                // start the plane's iterate from zero
                for (long long p = threadIdx.x; p < NS * nxy; p += blockDim.x) buf[cur][p] = Real(0);
                __syncthreads();
                int pass = 0;
                for (;; ++pass) {
                    Real change = 0, big = 0;
                    for (long long p = threadIdx.x; p < nxy; p += blockDim.x) {
                        const int jy = (int)(p / nx), ix = (int)(p - (long long)jy * nx);
                        const long long vO = B.vox0 + (long long)k * nxy + p;
                        int ii[4], jj[4];
                        double w[4];
                        // upwind point M
                        Real etaM = 0, etaVM = 0, epsM[NS], IM[NS];
#pragma unroll
                        for (int s = 0; s < NS; ++s) epsM[s] = IM[s] = Real(0);
                        double sM = 1.0;
                        if (vertM) sM = face_stencil(nx, ny, ix, jy, fxM, fyM, ii, jj, w);
                        else plane_stencil(nx, ny, ix, jy, fxM, fyM, ii, jj, w);
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int kk = vertM && c < 2 ? k : ku;
                            const Real *Ib = vertM && c < 2 ? buf[cur] : buf[up];
                            const long long pc = (long long)jj[c] * nx + ii[c];
                            const long long u = B.vox0 + (long long)kk * nxy + pc;
                            const Node<Real, NS> n = make_node<Real, NS>(a, ray, u, m, false);
                            Real eI, eV, e4[NS];
                            node_coef<Real, NS>(n, x, eI, eV, e4);
                            const Real wc = (Real)w[c];
                            etaM += wc * eI;
                            etaVM += wc * eV;
#pragma unroll
                            for (int s = 0; s < NS; ++s) {
                                epsM[s] += wc * e4[s];
                                IM[s] += wc * Ib[s * nxy + pc];
                            }
                        }
                        // the point O
                        const Node<Real, NS> nO = make_node<Real, NS>(a, ray, vO, m, true);
                        Real etaO, etaVO, epsO[NS];
                        node_coef<Real, NS>(nO, x, etaO, etaVO, epsO);
                        // downwind point P
                        Real etaP = 0, epsP[NS];
#pragma unroll
                        for (int s = 0; s < NS; ++s) epsP[s] = Real(0);
                        double sP = 1.0;
                        if (has_p) {
                            if (vertP) sP = face_stencil(nx, ny, ix, jy, fxP, fyP, ii, jj, w);
                            else plane_stencil(nx, ny, ix, jy, fxP, fyP, ii, jj, w);
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const int kk = vertP && c < 2 ? k : kd;
                                const long long u = B.vox0 + (long long)kk * nxy + (long long)jj[c] * nx + ii[c];
                                const Node<Real, NS> n = make_node<Real, NS>(a, ray, u, m, false);
                                Real eI, eV, e4[NS];
                                node_coef<Real, NS>(n, x, eI, eV, e4);
                                const Real wc = (Real)w[c];
                                etaP += wc * eI;
#pragma unroll
                                for (int s = 0; s < NS; ++s) epsP[s] += wc * e4[s];
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
                            const Real old = buf[cur][s * nxy + p];
                            change = fmax(change, fabs(IO[s] - old));
                            big = fmax(big, fabs(IO[s]));
                            buf[nxt][s * nxy + p] = IO[s];
                        }
                        lsb[p] = ls;
                    }
                    change = block_max(change, red);
                    big = block_max(big, red);
                    {
                        const int t = cur; cur = nxt; nxt = t;
                    }
                    __syncthreads();
                    if (!vertM || !(change > tol * big)) break;
                    if (pass + 1 >= maxpass) {
                        if (threadIdx.x == 0) atomicOr(err, 2);
                        break;
                    }
                }
                // the plane's sums: w_j phi_O / N (I, Q, U, Lambda*) added to the ray's partials
                for (long long p = threadIdx.x; p < nxy; p += blockDim.x) {
                    const long long vO = B.vox0 + (long long)k * nxy + p;
                    const Node<Real, NS> nO = make_node<Real, NS>(a, ray, vO, m, true);
                    const Real wt = wf * profile_shape(x - nO.s) * nO.invn;
                    if constexpr (NS == 1) {
                        R2<Real> *pp = reinterpret_cast<R2<Real> *>(a.part) + (long long)m * a.nvox + vO;
                        R2<Real> o = {wt * buf[cur][p], wt * lsb[p]};
                        if (j > 0) { const R2<Real> old = *pp; o.x += old.x; o.y += old.y; }
                        *pp = o;
                    } else {
                        R4<Real> *pp = reinterpret_cast<R4<Real> *>(a.part) + (long long)m * a.nvox + vO;
                        R4<Real> o = {wt * buf[cur][p], wt * buf[cur][nxy + p], wt * buf[cur][2 * nxy + p], wt * lsb[p]};
                        if (j > 0) { const R4<Real> old = *pp; o.x += old.x; o.y += old.y; o.z += old.z; o.w += old.w; }
                        *pp = o;
                    }
                }
                __syncthreads();
                up = cur;
            }
        }
    }
}

}  // namespace

template <typename Real, int NS>
cudaError_t launch_faces(const SweepArgs<Real> &a, Real *scratch, double dx, double dy, int maxpass, int *err,
                         cudaStream_t st)
{
    const Real tol = sizeof(Real) == 8 ? Real(1e-15) : Real(2e-7);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = std::max(1, std::min(a.nray, 4 * nsm));
    faces_kernel<Real, NS><<<blocks, 256, 0, st>>>(a, scratch, dx, dy, maxpass, tol, err);
    return cudaGetLastError();
}

#define PORTA_FACES_INST(R, N)                                                                              \
    template cudaError_t launch_faces<R, N>(const SweepArgs<R> &, R *, double, double, int, int *, cudaStream_t);
PORTA_FACES_INST(float, 1)
PORTA_FACES_INST(float, 4)
PORTA_FACES_INST(double, 1)
PORTA_FACES_INST(double, 4)
#undef PORTA_FACES_INST

}  // namespace porta
