// The family of short-characteristics formal solvers that Sec. 3.4 compares on
// a one-ray benchmark (Eqs. 15-18, Fig. 5): constant opacity, z = tau, the
// source function S(z) = sigma(2, -5, z) sigma(-2, 5, z) of Eq. 15 (Eq. 16
// sigmoids) on the uniform nodes z = -12 + shift + i dtau within [-12, 12],
// starting from the exact intensity of Eq. 17 at the first node. Each case
// (method, dtau, shift) is one thread that steps along its ray and keeps the
// maximum relative true error E (Eq. 18) against Eq. 17 evaluated in FP64.
//
// Methods of the upwind interval MO, all written as I_O = e I_M + w_M S_M +
// w_O S_O + w_C c_M (Eq. 7 for Stokes I) except the linear one:
//   BESSER     c_M of Sec. 3.2 (steps 1-9), as in the sweeps;
//   PARABOLIC  c_M = y_O - h_M y'_O / 2 with y'_O of Eq. 6 unclipped (the parabola
//              through M, O, P: standard parabolic short characteristics);
//   LINEAR     I_O = e I_M + psi'_M S_M + psi'_O S_O (Eqs. 9-10);
//   BEZIER_FB  c_M from the Fritsch-Butland derivative at O (weighted harmonic
//              mean of the one-sided slopes, 0 where they differ in sign);
//   CBEZIER    BEZIER_FB with c_M outside [y_M, y_O] moved to y_M.
// The last interval has no downwind point: c_M = (y_M + y_O)/2 (linear).
#include <cuda_runtime.h>

#include <cmath>

#include "api_internal.h"
#include "device_math.cuh"

namespace porta {

namespace {

// Eq. 16
template <typename Real>
__device__ __forceinline__ Real sigma(Real a, Real d, Real z)
{
    return Real(1) / (Real(1) + exp(-a * (z - d)));
}

// Eq. 15
template <typename Real>
__device__ __forceinline__ Real sig_source(Real z)
{
    return sigma(Real(2), Real(-5), z) * sigma(Real(-2), Real(5), z);
}

// Eq. 17 (FP64): the intensity towards +z with I(-inf) = 0
__device__ __forceinline__ double sig_exact(double z)
{
    return exp(15.0 - z) / (exp(20.0) - 1.0) * (exp(10.0) * atan(exp(z - 5.0)) - atan(exp(z + 5.0)));
}

template <typename Real>
__device__ __forceinline__ Real upwind_control(int method, Real yM, Real yO, Real yP, Real hM, Real hP)
{
    if (method == PORTA_SC_BESSER) return control_point(yM, yO, yP, besser_geom(hM, hP));
    const Real dM = (yO - yM) / hM, dP = (yP - yO) / hP;
    if (method == PORTA_SC_PARABOLIC) return yO - Real(0.5) * hM * ((hM * dP + hP * dM) / (hM + hP));
    // BEZIER_FB, CBEZIER: 1/y'_O = alpha/d_M + (1 - alpha)/d_P, alpha = (1 + h_P/(h_M + h_P))/3
    if (dM * dP <= Real(0)) return yO;
    const Real alpha = (Real(1) + hP / (hM + hP)) / Real(3);
    const Real yp = dM * dP / (alpha * dP + (Real(1) - alpha) * dM);
    const Real c = yO - Real(0.5) * hM * yp;
    if (method == PORTA_SC_CBEZIER && (c < fmin(yM, yO) || c > fmax(yM, yO))) return yM;
    return c;
}

template <typename Real>
__global__ void sigmoid_kernel(int ncase, const int *method, const double *dtau, const double *shift, double *E)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncase) return;
    const int m = method[k];
    const double hd = dtau[k], s = shift[k];
    const int n = (int)floor((24.0 - s) / hd + 1e-9) + 1;
    const double z0 = -12.0 + s;
    const Real h = (Real)hd;
    // uniform grid: one optical path for every interval
    const Coef<Real> co = coefficients(h);
    Real I = (Real)sig_exact(z0);
    Real yM = sig_source((Real)z0);
    Real yO = n > 1 ? sig_source((Real)(z0 + hd)) : Real(0);
    double emax = 0.0;
    for (int i = 1; i < n; ++i) {
        const double zO = z0 + hd * i;
        const bool has_p = i + 1 < n;
        const Real yP = has_p ? sig_source((Real)(z0 + hd * (i + 1))) : Real(0);
        if (m == PORTA_SC_LINEAR) {
            I = co.e * I + co.pm * yM + co.po * yO;
        } else {
            const Real c = has_p ? upwind_control(m, yM, yO, yP, h, h) : Real(0.5) * (yM + yO);
            I = co.e * I + co.wm * yM + co.wo * yO + co.wc * c;
        }
        const double ia = sig_exact(zO);
        emax = fmax(emax, fabs(((double)I - ia) / ia));
        yM = yO;
        yO = yP;
    }
    E[k] = emax;
}

}  // namespace

}  // namespace porta

using namespace porta;

extern "C" int porta_sigmoid_error(int precision, int ncase, const int *method, const double *dtau,
                                   const double *shift, double *E)
{
    if (ncase < 1 || !method || !dtau || !shift || !E || (precision != PORTA_FP32 && precision != PORTA_FP64))
        return PORTA_EINVAL;
    for (int k = 0; k < ncase; ++k) {
        if (method[k] < PORTA_SC_BESSER || method[k] > PORTA_SC_CBEZIER) return PORTA_EINVAL;
        if (!(dtau[k] >= 1e-4 && dtau[k] <= 24.0) || !(shift[k] >= 0.0 && shift[k] < dtau[k])) return PORTA_EINVAL;
    }
    const size_t bi = sizeof(int) * (size_t)ncase, bd = sizeof(double) * (size_t)ncase;
    void *buf = nullptr;
    if (porta_api::pmalloc_bytes(&buf, bi + 3 * bd + 16) != cudaSuccess) return PORTA_ENOMEM;
    double *d_dtau = (double *)buf, *d_shift = d_dtau + ncase, *d_E = d_shift + ncase;
    int *d_m = (int *)(d_E + ncase);
    cudaError_t e = cudaMemcpy(d_m, method, bi, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_dtau, dtau, bd, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_shift, shift, bd, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const int bs = 128, nb = (ncase + bs - 1) / bs;
        if (precision == PORTA_FP32)
            sigmoid_kernel<float><<<nb, bs>>>(ncase, d_m, d_dtau, d_shift, d_E);
        else
            sigmoid_kernel<double><<<nb, bs>>>(ncase, d_m, d_dtau, d_shift, d_E);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(E, d_E, bd, cudaMemcpyDeviceToHost);
    porta_api::pfree(buf);
    return e == cudaSuccess ? PORTA_OK : PORTA_ECUDA;
}
