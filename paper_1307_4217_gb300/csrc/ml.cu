// Multilevel atom without polarization (Sec. 1: the non-LTE problem of the
// first kind, populations n_i of the levels as the unknowns of Eq. 2).
//
// Per Jacobi iteration: ml_prepare turns the populations into each line's
// line-centre opacity chi_ul = chi s_ul (n_l - n_u g_l / g_u), source function
// S_ul = r^3 n_u / (n_l g_u / g_l - n_u) and Planck function B_ul(T) (the
// bottom boundary), written into the sweep arrays of the line's box, so that
// every line is one unpolarized formal solution of a batched launch; ml_see
// then solves the rate equations per voxel in FP64 with the radiative rates
// preconditioned by Lambda-bar* (J_eff = Jbar - Lambda-bar* S_old, P_ul = A (1 -
// Lambda-bar*) + B_ul J_eff + C_ul, P_lu = B_lu J_eff + C_lu), which makes them
// linear in the new populations; the equation of level 0 is replaced by
// sum_i n_i = 1. Collisions: C_lu = (g_u / g_l) exp(-dE / kT) C_ul.
#include <cmath>

#include "ml_kernels.cuh"

namespace porta {

namespace {

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

template <typename Real>
__global__ void ml_prepare_kernel(const MlConst mc, long long nvox1, const double *pops, const double *chis,
                                  const double *kT, Real *chi_out, Real *bpl_out, Real *S_out, double *S64_out,
                                  unsigned long long *bad)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nvox1) return;
    const double *n = pops + v * mc.nlev;
    const double chi = chis[v], t = kT[v];
    int nbad = 0;
    for (int k = 0; k < mc.nline; ++k) {
        const int u = mc.up[k], l = mc.lo[k];
        const double op = chi * mc.s[k] * (n[l] - n[u] * mc.g[l] / mc.g[u]);
        const double S = mc.r3[k] * n[u] / (n[l] * mc.g[u] / mc.g[l] - n[u]);
        const double B = mc.r3[k] / expm1(mc.dE[k] / t);
        const long long o = (long long)k * nvox1 + v;
        nbad += !(op > 0.0 && op < 1e300) || !(fabs(S) < 1e300);
        chi_out[o] = (Real)op;
        bpl_out[o] = (Real)B;
        S_out[o] = (Real)S;
        S64_out[o] = S;
    }
    if (nbad) atomicAdd(bad, (unsigned long long)nbad);
}

// rate coefficients of line k at voxel v: P_ul, P_lu with radiation jrad and
// escape factor (1 - ls) on the spontaneous rate
__device__ __forceinline__ void ml_rates(const MlConst &mc, int k, double t, double jrad, double ls, double &pul,
                                         double &plu)
{
    const int u = mc.up[k], l = mc.lo[k];
    const double clu = mc.g[u] / mc.g[l] * exp(-mc.dE[k] / t) * mc.Cul[k];
    pul = mc.A[k] * (1.0 - ls) + mc.Bul[k] * jrad + mc.Cul[k];
    plu = mc.Blu[k] * jrad + clu;
}

// out = alpha A(n) + add + with_f (1, 0, ..., 0): A(n)_0 = sum_i n_i, A(n)_i =
// (M n)_i with the plain rates of Jbar (i >= 1)
__global__ void ml_apply_kernel(const MlConst mc, long long nvox1, const double *kT, const double *jbar,
                                const double *pops, double alpha, const double *add, int with_f, double *out)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nvox1) return;
    const int L = mc.nlev;
    double n[kMlMaxLevel], y[kMlMaxLevel];
    for (int i = 0; i < L; ++i) {
        n[i] = pops[v * L + i];
        y[i] = 0.0;
    }
    const double t = kT[v];
    for (int k = 0; k < mc.nline; ++k) {
        const int u = mc.up[k], l = mc.lo[k];
        double pul, plu;
        ml_rates(mc, k, t, jbar[(long long)k * nvox1 + v], 0.0, pul, plu);
        const double down = pul * n[u], up = plu * n[l];
        y[l] += down - up;
        y[u] += up - down;
    }
    double sum = 0.0;
    for (int i = 0; i < L; ++i) sum += n[i];
    y[0] = sum;
    for (int i = 0; i < L; ++i)
        out[v * L + i] = alpha * y[i] + (add ? add[v * L + i] : 0.0) + (with_f && i == 0 ? 1.0 : 0.0);
}

__global__ void ml_see_kernel(const MlConst mc, long long nvox1, const double *kT, const double *jbar,
                              const double *lstar, const double *src, double *pops, unsigned long long *resid,
                              unsigned long long *bad)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double ch = 0.0;
    if (v < nvox1) {
        const int L = mc.nlev;
        double n[kMlMaxLevel], M[kMlMaxLevel][kMlMaxLevel], x[kMlMaxLevel];
        for (int i = 0; i < L; ++i) {
            n[i] = pops[v * L + i];
            for (int j = 0; j < L; ++j) M[i][j] = 0.0;
        }
        const double t = kT[v];
        for (int k = 0; k < mc.nline; ++k) {
            const int u = mc.up[k], l = mc.lo[k];
            const long long o = (long long)k * nvox1 + v;
            const double Sold = mc.r3[k] * n[u] / (n[l] * mc.g[u] / mc.g[l] - n[u]);
            const double ls = lstar[o];
            double pul, plu;
            ml_rates(mc, k, t, jbar[o] - ls * Sold, ls, pul, plu);
            M[l][u] += pul;
            M[u][u] -= pul;
            M[u][l] += plu;
            M[l][l] -= plu;
        }
        // conservation row; Gaussian elimination with partial pivoting
        for (int j = 0; j < L; ++j) M[0][j] = 1.0;
        for (int i = 0; i < L; ++i) x[i] = src ? src[v * L + i] : (i == 0 ? 1.0 : 0.0);
        bool ok = true;
        for (int c = 0; c < L; ++c) {
            int p = c;
            for (int r = c + 1; r < L; ++r)
                if (fabs(M[r][c]) > fabs(M[p][c])) p = r;
            if (!(fabs(M[p][c]) > 0.0)) { ok = false; break; }
            if (p != c) {
                for (int j = 0; j < L; ++j) {
                    const double tmp = M[c][j]; M[c][j] = M[p][j]; M[p][j] = tmp;
                }
                const double tmp = x[c]; x[c] = x[p]; x[p] = tmp;
            }
            const double inv = 1.0 / M[c][c];
            for (int r = c + 1; r < L; ++r) {
                const double f = M[r][c] * inv;
                if (f == 0.0) continue;
                for (int j = c; j < L; ++j) M[r][j] -= f * M[c][j];
                x[r] -= f * x[c];
            }
        }
        if (ok) {
            for (int i = L - 1; i >= 0; --i) {
                double acc = x[i];
                for (int j = i + 1; j < L; ++j) acc -= M[i][j] * x[j];
                x[i] = acc / M[i][i];
            }
        }
        int nbad = ok ? 0 : 1;
        for (int i = 0; i < L && ok; ++i) {
            nbad += !(x[i] > 0.0 && x[i] < 1e300);
            ch = fmax(ch, fabs(x[i] - n[i]) / fabs(n[i]));
        }
        if (nbad) {
            atomicAdd(bad, (unsigned long long)nbad);
            ch = 1e300;
        } else {
            for (int i = 0; i < L; ++i) pops[v * L + i] = x[i];
        }
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

}  // namespace

template <typename Real>
cudaError_t run_ml_prepare(const MlConst &mc, long long nvox1, const double *pops, const double *chis, const double *kT,
                           Real *chi_out, Real *bpl_out, Real *S_out, double *S64_out, unsigned long long *bad,
                           cudaStream_t st)
{
    ml_prepare_kernel<Real><<<nblk(nvox1, 256), 256, 0, st>>>(mc, nvox1, pops, chis, kT, chi_out, bpl_out, S_out,
                                                              S64_out, bad);
    return cudaGetLastError();
}
template cudaError_t run_ml_prepare<float>(const MlConst &, long long, const double *, const double *, const double *,
                                           float *, float *, float *, double *, unsigned long long *, cudaStream_t);
template cudaError_t run_ml_prepare<double>(const MlConst &, long long, const double *, const double *, const double *,
                                            double *, double *, double *, double *, unsigned long long *, cudaStream_t);

cudaError_t run_ml_see(const MlConst &mc, long long nvox1, const double *kT, const double *jbar, const double *lstar,
                       double *pops, unsigned long long *resid, unsigned long long *bad, cudaStream_t st,
                       const double *src)
{
    ml_see_kernel<<<nblk(nvox1, 128), 128, 0, st>>>(mc, nvox1, kT, jbar, lstar, src, pops, resid, bad);
    return cudaGetLastError();
}

cudaError_t run_ml_apply(const MlConst &mc, long long nvox1, const double *kT, const double *jbar, const double *pops,
                         double alpha, const double *add, int with_f, double *out, cudaStream_t st)
{
    ml_apply_kernel<<<nblk(nvox1, 128), 128, 0, st>>>(mc, nvox1, kT, jbar, pops, alpha, add, with_f, out);
    return cudaGetLastError();
}

}  // namespace porta
