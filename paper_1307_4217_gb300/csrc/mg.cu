// Grid transfer of the non-linear multigrid method (Sec. 5): the coarse grid
// keeps every other node on each axis (coarse (i, j, k) = fine (2i, 2j, 2k),
// Sec. 5.1). Prolongation (Sec. 5.2), tri-linear or tri-cubic-centered: a fine
// node on a coarse node takes its value, others interpolate along each axis
// where they fall between coarse nodes -- linearly between the two neighbours,
// or with the cubic through the four nearest coarse nodes (periodic in x and y
// with unit spacing: -1/16, 9/16, 9/16, -1/16; in the height z with the
// weights of a table; above the top coarse plane -- an even number of fine
// planes -- extrapolation from the top two or four). Restriction is the
// transpose of the tri-linear prolongation normalized so that constants are
// kept: its adjoint over the 3 x 3 x (up to 4) fine nodes around a coarse node.
// The z weights come as tables built on the host: per fine plane 2 (linear) or
// 4 (cubic) (coarse plane, weight) pairs for the prolongation, per coarse plane
// up to 4 (fine plane, weight) pairs for the restriction. Vectors of unknowns
// are [voxel][nl], FP64.
#include "mg_kernels.cuh"

namespace porta {

namespace {

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

// coarse[v_c] = fine[v_f] at the coincident node, one per-voxel array
__global__ void inject_kernel(int nxc, int nyc, long long nvc, int nxf, int nyf, const double *fine, double *coarse)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nvc) return;
    const int i = (int)(v % nxc);
    const int j = (int)((v / nxc) % nyc);
    const long long k = v / ((long long)nxc * nyc);
    coarse[v] = fine[((2 * k) * nyf + 2 * j) * (long long)nxf + 2 * i];
}

__global__ void restrict_kernel(int nxc, int nyc, long long nvc, int nxf, int nyf, int nl, const double *zr,
                                const double *fine, double *coarse)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nvc) return;
    const int I = (int)(v % nxc);
    const int J = (int)((v / nxc) % nyc);
    const int K = (int)(v / ((long long)nxc * nyc));
    double den = 0.0;
    for (int e = 0; e < 4; ++e) den += zr[8 * K + 2 * e + 1];
    // the horizontal weights sum to 2 per axis
    const double inv = 1.0 / (4.0 * den);
    // components in chunks of kMgMaxComp
    for (int c0 = 0; c0 < nl; c0 += kMgMaxComp) {
        const int nc = min(kMgMaxComp, nl - c0);
        double acc[kMgMaxComp] = {};
        for (int e = 0; e < 4; ++e) {
            const double w = zr[8 * K + 2 * e + 1];
            if (w == 0.0) continue;
            const long long kf = (long long)zr[8 * K + 2 * e];
            for (int dy = -1; dy <= 1; ++dy) {
                const double wy = dy == 0 ? 1.0 : 0.5;
                const int jf = (2 * J + dy + nyf) % nyf;
                for (int dx = -1; dx <= 1; ++dx) {
                    const double wx = dx == 0 ? 1.0 : 0.5;
                    const int xf = (2 * I + dx + nxf) % nxf;
                    const double *p = fine + ((kf * nyf + jf) * nxf + xf) * nl + c0;
                    const double wt = w * wy * wx;
                    for (int c = 0; c < nc; ++c) acc[c] += wt * p[c];
                }
            }
        }
        for (int c = 0; c < nc; ++c) coarse[v * nl + c0 + c] = acc[c] * inv;
    }
}

// one axis of the horizontal prolongation: the NP coarse nodes of fine node i and their weights
template <int NP>
__device__ __forceinline__ void prolong_axis(int i, int nc, int idx[NP], double w[NP])
{
    for (int a = 0; a < NP; ++a) {
        idx[a] = i / 2;
        w[a] = 0.0;
    }
    if (i % 2 == 0) {
        w[0] = 1.0;
    } else if (NP == 2) {
        idx[0] = (i - 1) / 2;
        idx[1] = ((i + 1) / 2) % nc;
        w[0] = w[1] = 0.5;
    } else {
        // the cubic through coarse nodes left-1 .. left+2 at the midpoint of [left, left+1]
        const double cw[4] = {-1.0 / 16.0, 9.0 / 16.0, 9.0 / 16.0, -1.0 / 16.0};
        const int left = (i - 1) / 2;
        for (int a = 0; a < NP && a < 4; ++a) {
            idx[a] = ((left - 1 + a) % nc + nc) % nc;
            w[a] = cw[a];
        }
    }
}

// fine (+)= P (cnew - cold); cold may be null (zero); NP = 2 tri-linear, 4 tri-cubic;
// zp: per fine plane NP (coarse plane, weight) pairs
template <int NP>
__global__ void prolong_kernel(int nxf, int nyf, long long nvf, int nxc, int nyc, int nl, const double *zp,
                               const double *cnew, const double *cold, double *fine, int assign)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nvf) return;
    const int i = (int)(v % nxf);
    const int j = (int)((v / nxf) % nyf);
    const int k = (int)(v / ((long long)nxf * nyf));
    int xi[NP], yj[NP];
    double wx[NP], wy[NP];
    prolong_axis<NP>(i, nxc, xi, wx);
    prolong_axis<NP>(j, nyc, yj, wy);
    long long kz[NP];
    double wz[NP];
    for (int a = 0; a < NP; ++a) {
        kz[a] = (long long)zp[2 * NP * k + 2 * a];
        wz[a] = zp[2 * NP * k + 2 * a + 1];
    }
    for (int c0 = 0; c0 < nl; c0 += kMgMaxComp) {
        const int nc = min(kMgMaxComp, nl - c0);
        double d[kMgMaxComp] = {};
        for (int a = 0; a < NP; ++a) {
            if (wz[a] == 0.0) continue;
            for (int b = 0; b < NP; ++b) {
                if (wy[b] == 0.0) continue;
                for (int cx = 0; cx < NP; ++cx) {
                    if (wx[cx] == 0.0) continue;
                    const long long vc = (kz[a] * nyc + yj[b]) * nxc + xi[cx];
                    const double w = wz[a] * wy[b] * wx[cx];
                    for (int c = 0; c < nc; ++c)
                        d[c] += w * (cnew[vc * nl + c0 + c] - (cold ? cold[vc * nl + c0 + c] : 0.0));
                }
            }
        }
        for (int c = 0; c < nc; ++c) {
            double *o = fine + v * nl + c0 + c;
            *o = assign ? d[c] : *o + d[c];
        }
    }
}

// coarse[v_c][c] = fine[v_f][c] at the coincident node, nl components per voxel
__global__ void inject_vec_kernel(int nxc, int nyc, long long nvc, int nxf, int nyf, int nl, const double *fine,
                                  double *coarse)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nvc) return;
    const int i = (int)(v % nxc);
    const int j = (int)((v / nxc) % nyc);
    const long long k = v / ((long long)nxc * nyc);
    const double *src = fine + (((2 * k) * nyf + 2 * j) * (long long)nxf + 2 * i) * nl;
    for (int c = 0; c < nl; ++c) coarse[v * nl + c] = src[c];
}

// max over voxels of |dS00| / |S00_old| and |S2/S00 (new) - S2/S00 (old)|
// (the residual of the Jacobi update), or with rel_all the relative change of
// every component (populations), as the IEEE bits of a non-negative double
__global__ void change_kernel(long long nvox, int nl, const double *old, const double *cur, int rel_all,
                              unsigned long long *resid)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double ch = 0.0;
    if (v < nvox) {
        const double *o = old + v * nl, *n = cur + v * nl;
        ch = fabs(n[0] - o[0]) / fabs(o[0]);
        for (int c = 1; c < nl; ++c)
            ch = fmax(ch, rel_all ? fabs(n[c] - o[c]) / fabs(o[c]) : fabs(n[c] / n[0] - o[c] / o[0]));
    }
    if (!(ch <= 1e300)) ch = 1e300;
    for (int s = 16; s > 0; s >>= 1) ch = fmax(ch, __shfl_xor_sync(0xffffffffu, ch, s));
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = ch;
    __syncthreads();
    if (wid == 0) {
        ch = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int s = 16; s > 0; s >>= 1) ch = fmax(ch, __shfl_xor_sync(0xffffffffu, ch, s));
        if (lane == 0) atomicMax(resid, (unsigned long long)__double_as_longlong(ch));
    }
}

// max over voxels of max_c |r[v][c]| / max_c |x[v][c]|: a residual relative to each
// voxel's largest unknown, as the IEEE bits of a non-negative double
__global__ void rel_residual_kernel(long long nvox, int nl, const double *r, const double *x,
                                    unsigned long long *out)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double q = 0.0;
    if (v < nvox) {
        double rm = 0.0, xm = 0.0;
        for (int c = 0; c < nl; ++c) {
            rm = fmax(rm, fabs(r[v * nl + c]));
            xm = fmax(xm, fabs(x[v * nl + c]));
        }
        q = rm / xm;
    }
    if (!(q <= 1e300)) q = 1e300;
    for (int s = 16; s > 0; s >>= 1) q = fmax(q, __shfl_xor_sync(0xffffffffu, q, s));
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = q;
    __syncthreads();
    if (wid == 0) {
        q = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int s = 16; s > 0; s >>= 1) q = fmax(q, __shfl_xor_sync(0xffffffffu, q, s));
        if (lane == 0) atomicMax(out, (unsigned long long)__double_as_longlong(q));
    }
}

__global__ void axpy_kernel(long long n, double alpha, const double *x, double *y)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] += alpha * x[i];
}

}  // namespace

cudaError_t run_axpy(long long n, double alpha, const double *x, double *y, cudaStream_t st)
{
    axpy_kernel<<<nblk(n, 256), 256, 0, st>>>(n, alpha, x, y);
    return cudaGetLastError();
}

cudaError_t run_inject(int nxc, int nyc, int nzc, int nxf, int nyf, const double *fine, double *coarse, cudaStream_t st)
{
    const long long n = (long long)nxc * nyc * nzc;
    inject_kernel<<<nblk(n, 256), 256, 0, st>>>(nxc, nyc, n, nxf, nyf, fine, coarse);
    return cudaGetLastError();
}

cudaError_t run_restrict(int nxc, int nyc, int nzc, int nxf, int nyf, int nl, const double *zr, const double *fine,
                         double *coarse, cudaStream_t st)
{
    const long long n = (long long)nxc * nyc * nzc;
    restrict_kernel<<<nblk(n, 256), 256, 0, st>>>(nxc, nyc, n, nxf, nyf, nl, zr, fine, coarse);
    return cudaGetLastError();
}

cudaError_t run_prolong(int nxf, int nyf, int nzf, int nxc, int nyc, int nl, int order, const double *zp,
                        const double *cnew, const double *cold, double *fine, int assign, cudaStream_t st)
{
    const long long n = (long long)nxf * nyf * nzf;
    if (order == 3)
        prolong_kernel<4><<<nblk(n, 256), 256, 0, st>>>(nxf, nyf, n, nxc, nyc, nl, zp, cnew, cold, fine, assign);
    else
        prolong_kernel<2><<<nblk(n, 256), 256, 0, st>>>(nxf, nyf, n, nxc, nyc, nl, zp, cnew, cold, fine, assign);
    return cudaGetLastError();
}

cudaError_t run_inject_vec(int nxc, int nyc, int nzc, int nxf, int nyf, int nl, const double *fine, double *coarse,
                           cudaStream_t st)
{
    const long long n = (long long)nxc * nyc * nzc;
    inject_vec_kernel<<<nblk(n, 256), 256, 0, st>>>(nxc, nyc, n, nxf, nyf, nl, fine, coarse);
    return cudaGetLastError();
}

cudaError_t run_rel_residual(long long nvox, int nl, const double *r, const double *x, unsigned long long *out,
                             cudaStream_t st)
{
    rel_residual_kernel<<<nblk(nvox, 256), 256, 0, st>>>(nvox, nl, r, x, out);
    return cudaGetLastError();
}

cudaError_t run_change(long long nvox, int nl, const double *old, const double *cur, unsigned long long *resid,
                       cudaStream_t st, int rel_all)
{
    change_kernel<<<nblk(nvox, 256), 256, 0, st>>>(nvox, nl, old, cur, rel_all, resid);
    return cudaGetLastError();
}

}  // namespace porta
