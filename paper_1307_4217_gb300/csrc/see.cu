// Per-voxel kernels around the formal solution: profile normalization
// (Sec. 4.2), conversion of the unknowns for the sweep, the FP64 sum of the
// per-ray partial integrals into J^K_Q and Lambda-bar* (Eq. 1), and the
// Jacobi (ALI) statistical-equilibrium update with its convergence residual
// (Eq. 2, Sec. 5).
#include "device_math.cuh"
#include "adjoint_math.cuh"
#include "see_kernels.cuh"

namespace porta {

// Sign of the Hanle (magnetic) term of the update: the unknowns S^K_Q follow the
// convention of J^K_Q (the complex conjugates of the atomic rho^K_Q), in which the
// counterclockwise Larmor precession of the atom about B (Lande factor > 0) reads
//   S^K_Q - i (1-eps) Gamma_u sum_Q' K_QQ'(B) S^K_Q' = (1-eps) J^K_Q + eps B delta_K0
constexpr double kHanleSense = -1.0;

// invn[m][v] = 1 / sum_j w_j exp(-(x_j - vel_v mu_m)^2): the profile is
// renormalized on the frequency quadrature for each voxel and direction.
template <typename Real>
__global__ void profile_norm_kernel(long long nvox, int nray, int nnu, const double *mu, const double *xf,
                                    const double *wf, const double *vel, Real *invn)
{
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= nvox * nray) return;
    int m = (int)(idx / nvox);
    long long v = idx - (long long)m * nvox;
    if constexpr (sizeof(Real) == 4) {
        // FP32 sweeps: the sum of the profile they evaluate (FP32 shift and profile),
        // compensated, so that their integration weights w_j phi_j / N sum to 1 in
        // their own arithmetic (and without the low-rate FP64 exponential)
        const float s = (float)vel[v] * (float)mu[m];
        float sum = 0.0f, comp = 0.0f;
        for (int j = 0; j < nnu; ++j) {
            const float y = (float)wf[j] * profile_shape((float)xf[j] - s) - comp;
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
        invn[idx] = (Real)(1.0f / sum);
    } else {
        double s = vel[v] * mu[m], sum = 0.0;
        for (int j = 0; j < nnu; ++j) {
            double xs = xf[j] - s;
            sum += wf[j] * exp(-xs * xs);
        }
        invn[idx] = (Real)(1.0 / sum);
    }
}

// rho (FP64, [v][nl]) -> sweep copy (Real, [c][v])
template <typename Real>
__global__ void rho_convert_kernel(long long nvox, int nl, const double *rho, Real *out)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    for (int c = 0; c < nl; ++c) out[c * nvox + v] = (Real)rho[v * nl + c];
}

// J^K_Q(v) = sum_m w_m sum_p T^K_Q(p, m) P_p(m, v) and Lambda-bar*(v) = sum_m w_m P_L(m, v),
// summed over rays in ascending order (deterministic). FP64 partials are summed
// in FP64; FP32 partials (FP32 sweep) in FP32 with compensated (Kahan) sums,
// whose error for nray terms is ~2 ulp independent of nray, instead of FP64
// arithmetic on the GPU's low-rate FP64 pipe.
template <typename Real>
struct KahanSum {
    Real s = 0, c = 0;
    __device__ __forceinline__ void add(Real x)
    {
        if constexpr (sizeof(Real) == 8) {
            s += x;                       // FP64: plain sum
        } else {
            Real y = x - c;
            Real t = s + y;
            c = (t - s) - y;
            s = t;
        }
    }
};

template <typename Real, int NS>
__global__ void jkq_finalize_kernel(long long nvox, int nray, const void *part, const double *tw,
                                    double *jkq, double *lstar)
{
    // the ray weights and tensors in the sums' precision, converted once per block
    extern __shared__ __align__(16) unsigned char fin_smem[];
    Real *stw = reinterpret_cast<Real *>(fin_smem);
    for (int i = threadIdx.x; i < nray * 19; i += blockDim.x) stw[i] = (Real)tw[i];
    __syncthreads();
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const Real *p = reinterpret_cast<const Real *>(part);
    if constexpr (NS == 1) {
        KahanSum<Real> J, L;
#pragma unroll 4
        for (int m = 0; m < nray; ++m) {
            const Real *q = p + 2 * ((long long)m * nvox + v);
            const Real w = stw[m * 19];
            J.add(w * q[0]);
            L.add(w * q[1]);
        }
        jkq[v] = (double)J.s;
        lstar[v] = (double)L.s;
    } else {
        KahanSum<Real> J[6], L;
#pragma unroll 2
        for (int m = 0; m < nray; ++m) {
            const Real *q = p + 4 * ((long long)m * nvox + v);
            const Real *t = stw + m * 19;
            const Real w = t[0];
            const Real pI = w * q[0], pQ = w * q[1], pU = w * q[2];
#pragma unroll
            for (int c = 0; c < 6; ++c) J[c].add(t[1 + c] * pI + t[7 + c] * pQ + t[13 + c] * pU);
            L.add(w * q[3]);
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) jkq[v * 6 + c] = (double)J[c].s;
        lstar[v] = (double)L.s;
    }
}

// J^1_Q of polarized lines from the per-ray frequency integrals of Stokes V:
// J^1_Q = sum_m w_m T^1_Q(V, Omega_m) Vbar_m, tw1 [ray][3] = w_m T^1_Q (J10, Re J11, Im J11)
template <typename Real>
__global__ void j1_finalize_kernel(long long nvox, int nray, const Real *partv, const double *tw1, double *j1)
{
    extern __shared__ __align__(16) unsigned char fin_smem[];
    Real *stw = reinterpret_cast<Real *>(fin_smem);
    for (int i = threadIdx.x; i < nray * 3; i += blockDim.x) stw[i] = (Real)tw1[i];
    __syncthreads();
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    KahanSum<Real> J[3];
#pragma unroll 4
    for (int m = 0; m < nray; ++m) {
        const Real pv = partv[(long long)m * nvox + v];
#pragma unroll
        for (int c = 0; c < 3; ++c) J[c].add(stw[3 * m + c] * pv);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) j1[v * 3 + c] = (double)J[c].s;
}

// atomic max of non-negative doubles through their IEEE bit patterns (the
// ordering of the bit patterns is that of the values for non-negative doubles)
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *addr, double v)
{
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// Jacobi update (FP64). Unpolarized: S <- S + [(1-eps)J + eps B - S] / [1 - (1-eps) L*].
// Hanle: S^0_0 as above with J^0_0; K = 2 from (1 + i (1-eps) Gamma_u K(B)) S^2 = (1-eps) J^2.
template <typename Real>
__global__ void see_kernel(long long nvox, int nl, int model, double bcrit, const double *eps, const double *bpl,
                           const double *bvec, const double *jkq, const double *lstar, double *rho, Real *rhoR,
                           unsigned long long *resid, const double *src)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double change = 0.0;
    if (v < nvox) {
        const double e = eps[v], B = bpl[v];
        // right-hand side of A(S) = f: eps B delta_K0, or a given source (coarse-grid problems)
        const double f0 = src ? src[v * nl] : e * B;
        if (model == PORTA_MODEL_TWOLEVEL_UNPOL) {
            const double S = rho[v];
            const double dS = ((1.0 - e) * jkq[v] + f0 - S) / (1.0 - (1.0 - e) * lstar[v]);
            const double Sn = S + dS;
            change = fabs(dS) / fabs(S);
            rho[v] = Sn;
            rhoR[v] = (Real)Sn;
        } else {
            double *s = rho + 6 * v;
            const double *J = jkq + 6 * v;
            const double S00 = s[0];
            const double dS = ((1.0 - e) * J[0] + f0 - S00) / (1.0 - (1.0 - e) * lstar[v]);
            const double S00n = S00 + dS;
            const double bx = bvec[v], by = bvec[nvox + v], bz = bvec[2 * nvox + v];
            const double gam = kHanleSense * (1.0 - e) / bcrit;   // Gamma = (1-eps) |B| / bcrit; times B/|B| below
            double r[5], x[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) r[c] = (1.0 - e) * J[1 + c] + (src ? src[v * nl + 1 + c] : 0.0);
            hanle_solve5(gam * bx, gam * by, gam * bz, r, x);
            change = fabs(dS) / fabs(S00);
#pragma unroll
            for (int c = 0; c < 5; ++c) change = fmax(change, fabs(x[c] / S00n - s[1 + c] / S00));
            s[0] = S00n;
            rhoR[v] = (Real)S00n;
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                s[1 + c] = x[c];
                rhoR[(1 + c) * nvox + v] = (Real)x[c];
            }
        }
    }
    // a non-finite change (NaN input or breakdown) is reported as 1e300
    if (!(change <= 1e300)) change = 1e300;
    // block max, then one atomic per block
    __shared__ double red[32];
    double m = change;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = m;
    __syncthreads();
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        double mm = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) mm = fmax(mm, __shfl_xor_sync(0xffffffffu, mm, o));
        if (lane == 0) atomic_max_nonneg(resid, mm);
    }
}

// finite-value checks of inputs (count of offending entries)
__global__ void count_bad_kernel(long long n, const double *x, double lo_excl, double hi_incl, unsigned long long *bad)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = x[i];
    if (!(v > lo_excl && v <= hi_incl)) atomicAdd(bad, 1ULL);
}

template <typename Real>
__global__ void to_real_kernel(long long n, const double *x, Real *y)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = (Real)x[i];
}

// diagnostic: the general BESSER-DELO step (delo_step_general) on a batch of
// inputs [n][34]: IM 4, eta_M 7, eps_M 4, eta_O 7, eps_O 4, eta_P,I 1, eps_P 4,
// ds_M, ds_P, has_p; outputs [n][5]: I_O 4, Lambda*
template <typename Real>
__global__ void step_eval_kernel(int n, const double *in, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *p = in + (long long)i * 34;
    Real IM[4], eM[7], sM[4], eO[7], sO[4], sP[4];
    for (int k = 0; k < 4; ++k) { IM[k] = (Real)p[k]; sM[k] = (Real)p[11 + k]; sO[k] = (Real)p[22 + k]; sP[k] = (Real)p[27 + k]; }
    for (int k = 0; k < 7; ++k) { eM[k] = (Real)p[4 + k]; eO[k] = (Real)p[15 + k]; }
    Real IO[4], ls;
    delo_step_general<Real>(IM, eM, sM, eO, sO, (Real)p[26], sP, (Real)p[31], (Real)p[32], p[33] != 0.0, IO, ls);
    for (int k = 0; k < 4; ++k) out[(long long)i * 5 + k] = (double)IO[k];
    out[(long long)i * 5 + 4] = (double)ls;
}

cudaError_t run_step_eval(int precision, int n, const double *in, double *out, cudaStream_t st)
{
    const int bs = 128;
    if (precision == PORTA_FP32) step_eval_kernel<float><<<(n + bs - 1) / bs, bs, 0, st>>>(n, in, out);
    else step_eval_kernel<double><<<(n + bs - 1) / bs, bs, 0, st>>>(n, in, out);
    return cudaGetLastError();
}

// diagnostic: the sweep's coefficient function (Eqs. 9-13 / Table 1) on the GPU
template <typename Real>
__global__ void coefficients_kernel(int n, const double *t, double *out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Coef<Real> c = coefficients((Real)t[i]);
    out[6 * i + 0] = (double)c.e;
    out[6 * i + 1] = (double)c.pm;
    out[6 * i + 2] = (double)c.po;
    out[6 * i + 3] = (double)c.wm;
    out[6 * i + 4] = (double)c.wo;
    out[6 * i + 5] = (double)c.wc;
}

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename Real>
cudaError_t run_profile_norm(long long nvox, int nray, int nnu, const double *mu, const double *xf, const double *wf,
                             const double *vel, void *invn, cudaStream_t st)
{
    profile_norm_kernel<Real><<<nblk(nvox * nray, 256), 256, 0, st>>>(nvox, nray, nnu, mu, xf, wf, vel, (Real *)invn);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t run_rho_convert(long long nvox, int nl, const double *rho, void *out, cudaStream_t st)
{
    rho_convert_kernel<Real><<<nblk(nvox, 256), 256, 0, st>>>(nvox, nl, rho, (Real *)out);
    return cudaGetLastError();
}

template <typename Real, int NS>
cudaError_t run_jkq_finalize(long long nvox, int nray, const void *part, const double *tw, double *jkq, double *lstar,
                             cudaStream_t st)
{
    const size_t smem = (size_t)nray * 19 * sizeof(Real);
    cudaError_t e = cudaFuncSetAttribute(jkq_finalize_kernel<Real, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    jkq_finalize_kernel<Real, NS><<<nblk(nvox, 256), 256, smem, st>>>(nvox, nray, part, tw, jkq, lstar);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t run_j1_finalize(long long nvox, int nray, const void *partv, const double *tw1, double *j1, cudaStream_t st)
{
    const size_t smem = (size_t)nray * 3 * sizeof(Real);
    cudaError_t e = cudaFuncSetAttribute(j1_finalize_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    j1_finalize_kernel<Real><<<nblk(nvox, 256), 256, smem, st>>>(nvox, nray, (const Real *)partv, tw1, j1);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t run_see(long long nvox, int nl, int model, double bcrit, const double *eps, const double *bpl,
                    const double *bvec, const double *jkq, const double *lstar, double *rho, void *rhoR,
                    unsigned long long *resid, cudaStream_t st, const double *src)
{
    see_kernel<Real><<<nblk(nvox, 256), 256, 0, st>>>(nvox, nl, model, bcrit, eps, bpl, bvec, jkq, lstar, rho,
                                                      (Real *)rhoR, resid, src);
    return cudaGetLastError();
}

// out = alpha A(S) + add (+ eps B delta_K0 if with_eb), A the statistical-
// equilibrium operator of A(S) = f: A(S)^0_0 = S^0_0 - (1-eps) J^0_0,
// A(S)^2 = M S^2 - (1-eps) J^2 with M = 1 + i (1-eps) Gamma_u K (Eq. 2).
// out may alias add (each element is read before it is written).
__global__ void see_apply_kernel(long long nvox, int nl, int model, double bcrit, const double *eps, const double *bpl,
                                 const double *bvec, const double *jkq, const double *rho, double alpha,
                                 const double *add, int with_eb, double *out)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const double e = eps[v];
    const double *s = rho + v * nl, *J = jkq + v * nl;
    double a[6];
    a[0] = s[0] - (1.0 - e) * J[0];
    if (model != PORTA_MODEL_TWOLEVEL_UNPOL) {
        const double gam = kHanleSense * (1.0 - e) / bcrit;
        double y[5];
        hanle_apply5(gam * bvec[v], gam * bvec[nvox + v], gam * bvec[2 * nvox + v], s + 1, y);
#pragma unroll
        for (int c = 0; c < 5; ++c) a[1 + c] = y[c] - (1.0 - e) * J[1 + c];
    }
    for (int c = 0; c < nl; ++c) {
        double o = alpha * a[c];
        if (add) o += add[v * nl + c];
        if (with_eb && c == 0) o += e * bpl[v];
        out[v * nl + c] = o;
    }
}

// Reverse mode of the Jacobi update (src as in see_kernel): from g = dL/d(rho
// after the update) to dL/drho through the explicit S^0_0 term (overwritten),
// dL/dJ^K_Q and dL/dLambda-bar* (overwritten), dL/d(thermal term) and, through
// the Hanle matrix M = 1 + sum_c g_c E_c (affine in g = kHanleSense (1-eps) B / bcrit),
// dL/dB (both added):
//   S00' = S00 + ((1-eps) J00 + f - S00) / D,  D = 1 - (1-eps) Lambda*,
//   S2'  = M^-1 ((1-eps) J2 + f2),  dL/dJ2 = (1-eps) M^-T g2,
//   dL/dB_c = -kHanleSense (1-eps)/bcrit (M^-T g2) . E_c S2'.
__global__ void see_vjp_kernel(long long nvox, int nl, int model, double bcrit, const double *eps, const double *bpl,
                               const double *bvec, const double *jkq, const double *lstar, const double *src,
                               const double *rho, const double *g, double *g_rho, double *g_jkq, double *g_lstar,
                               double *g_f, double *g_b)
{
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const double e = eps[v];
    const double f0 = src ? src[v * nl] : e * bpl[v];
    const double *s = rho + v * nl, *J = jkq + v * nl, *gv = g + v * nl;
    const double D = 1.0 - (1.0 - e) * lstar[v];
    const double num = (1.0 - e) * J[0] + f0 - s[0];
    g_rho[v * nl] = gv[0] * (1.0 - 1.0 / D);
    g_jkq[v * nl] = gv[0] * (1.0 - e) / D;
    g_lstar[v] = gv[0] * num * (1.0 - e) / (D * D);
    g_f[v] += gv[0] / D;
    if (model == PORTA_MODEL_TWOLEVEL_UNPOL) return;
    const double gam = kHanleSense * (1.0 - e) / bcrit;
    const double gx = gam * bvec[v], gy = gam * bvec[nvox + v], gz = gam * bvec[2 * nvox + v];
    double r[5], s2[5], z[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) r[c] = (1.0 - e) * J[1 + c] + (src ? src[v * nl + 1 + c] : 0.0);
    hanle_solve5(gx, gy, gz, r, s2);
    hanle_solve5_t(gx, gy, gz, gv + 1, z);
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        g_rho[v * nl + 1 + c] = 0.0;
        g_jkq[v * nl + 1 + c] = (1.0 - e) * z[c];
    }
    // E_c S2' = (M(unit g along c) - 1) S2'
    const double unit[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double y[5];
        hanle_apply5(unit[c][0], unit[c][1], unit[c][2], s2, y);
        double acc = 0.0;
#pragma unroll
        for (int a = 0; a < 5; ++a) acc += z[a] * (y[a] - s2[a]);
        g_b[c * nvox + v] += -gam * acc;
    }
}

cudaError_t run_see_vjp(long long nvox, int nl, int model, double bcrit, const double *eps, const double *bpl,
                        const double *bvec, const double *jkq, const double *lstar, const double *src,
                        const double *rho, const double *g, double *g_rho, double *g_jkq, double *g_lstar,
                        double *g_f, double *g_b, cudaStream_t st)
{
    see_vjp_kernel<<<nblk(nvox, 256), 256, 0, st>>>(nvox, nl, model, bcrit, eps, bpl, bvec, jkq, lstar, src, rho, g,
                                                    g_rho, g_jkq, g_lstar, g_f, g_b);
    return cudaGetLastError();
}

cudaError_t run_see_apply(long long nvox, int nl, int model, double bcrit, const double *eps, const double *bpl,
                          const double *bvec, const double *jkq, const double *rho, double alpha, const double *add,
                          int with_eb, double *out, cudaStream_t st)
{
    see_apply_kernel<<<nblk(nvox, 256), 256, 0, st>>>(nvox, nl, model, bcrit, eps, bpl, bvec, jkq, rho, alpha, add,
                                                      with_eb, out);
    return cudaGetLastError();
}

cudaError_t run_count_bad(long long n, const double *x, double lo_excl, double hi_incl, unsigned long long *bad,
                          cudaStream_t st)
{
    count_bad_kernel<<<nblk(n, 256), 256, 0, st>>>(n, x, lo_excl, hi_incl, bad);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t run_to_real(long long n, const double *x, void *y, cudaStream_t st)
{
    to_real_kernel<Real><<<nblk(n, 256), 256, 0, st>>>(n, x, (Real *)y);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t run_coefficients(int n, const double *t, double *out, cudaStream_t st)
{
    coefficients_kernel<Real><<<nblk(n, 128), 128, 0, st>>>(n, t, out);
    return cudaGetLastError();
}
template cudaError_t run_coefficients<float>(int, const double *, double *, cudaStream_t);
template cudaError_t run_coefficients<double>(int, const double *, double *, cudaStream_t);

#define INST(R)                                                                                                \
    template cudaError_t run_profile_norm<R>(long long, int, int, const double *, const double *, const double *,\
                                             const double *, void *, cudaStream_t);                           \
    template cudaError_t run_rho_convert<R>(long long, int, const double *, void *, cudaStream_t);              \
    template cudaError_t run_jkq_finalize<R, 1>(long long, int, const void *, const double *, double *, double *, \
                                                cudaStream_t);                                                 \
    template cudaError_t run_jkq_finalize<R, 4>(long long, int, const void *, const double *, double *, double *, \
                                                cudaStream_t);                                                 \
    template cudaError_t run_j1_finalize<R>(long long, int, const void *, const double *, double *, cudaStream_t); \
    template cudaError_t run_see<R>(long long, int, int, double, const double *, const double *, const double *, \
                                    const double *, const double *, double *, void *, unsigned long long *,     \
                                    cudaStream_t, const double *);                                             \
    template cudaError_t run_to_real<R>(long long, const double *, void *, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace porta
