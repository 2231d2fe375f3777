// Device arithmetic of the formal solver (Sec. 3.2-3.3 of Stepan & Trujillo
// Bueno 2013): BESSER control points, the exponential-integral coefficients
// of the Bezier/DELO step, and the Hanle statistical-equilibrium solve (Eq. 2).
#pragma once
#include <cuda_runtime.h>

namespace porta {

// ---------------------------------------------------------------------------
// Coefficients of Eq. 7 for an upwind optical path t = tau_MO:
//   e = exp(-t),
//   psi'_M = (1 - e (1 + t)) / t,          psi'_O = (e + t - 1) / t,
//   w_M = (2 - e (t^2 + 2t + 2)) / t^2,    w_O = 1 - 2 (e + t - 1) / t^2,
//   w_C = 2 (t - 2 + e (t + 2)) / t^2      (Eqs. 8-12).
// Below a crossover the closed forms lose digits to cancellation and the
// Taylor series at t = 0 is used instead (Table 1 for double precision).
// Series coefficients of t^k, k >= 1, from expanding the closed forms:
//   psi'_M: (-1)^(k+1) k / (k+1)!        psi'_O: (-1)^(k+1) / (k+1)!
//   w_M:    (-1)^(k+1) k (k+1) / (k+2)!  w_O:    2 (-1)^(k+1) / (k+2)!
//   w_C:    2 (-1)^(k+1) k / (k+2)!
// ---------------------------------------------------------------------------
template <typename Real>
struct Coef {
    Real e, pm, po, wm, wo, wc;
};

__host__ __device__ constexpr double fact_d(int n) { return n <= 1 ? 1.0 : n * fact_d(n - 1); }
__host__ __device__ constexpr double sgn_d(int k) { return (k % 2) ? 1.0 : -1.0; }  // (-1)^(k+1)
__host__ __device__ constexpr double c_pm(int k) { return sgn_d(k) * k / fact_d(k + 1); }
__host__ __device__ constexpr double c_po(int k) { return sgn_d(k) / fact_d(k + 1); }
__host__ __device__ constexpr double c_wm(int k) { return sgn_d(k) * k * (k + 1.0) / fact_d(k + 2); }
__host__ __device__ constexpr double c_wo(int k) { return 2.0 * sgn_d(k) / fact_d(k + 2); }
__host__ __device__ constexpr double c_wc(int k) { return 2.0 * sgn_d(k) * k / fact_d(k + 2); }

// t * (a_1 + t (a_2 + ... + t a_N)) with a_k = coef(k), N = DEG
template <typename Real, int DEG, double (*COEF)(int)>
__device__ __forceinline__ Real horner(Real t)
{
    Real r = Real(COEF(DEG));
#pragma unroll
    for (int k = DEG - 1; k >= 1; --k) r = r * t + Real(COEF(k));
    return r * t;
}

// Double precision: degree 8 (the order of Table 1), crossovers of Table 1
// (w_M 0.14, w_O and w_C 0.18) and 0.1 for psi'.
__device__ __forceinline__ Coef<double> coefficients(double t)
{
    Coef<double> c;
    double e = exp(-t);
    c.e = e;
    double it = 1.0 / t, it2 = it * it;
    c.pm = t < 0.1 ? horner<double, 8, c_pm>(t) : (1.0 - e * (1.0 + t)) * it;
    c.po = t < 0.1 ? horner<double, 8, c_po>(t) : (e + t - 1.0) * it;
    c.wm = t < 0.14 ? horner<double, 8, c_wm>(t) : (2.0 - e * (t * t + 2.0 * t + 2.0)) * it2;
    c.wo = t < 0.18 ? horner<double, 8, c_wo>(t) : 1.0 - 2.0 * (e + t - 1.0) * it2;
    c.wc = t < 0.18 ? horner<double, 8, c_wc>(t) : 2.0 * (t - 2.0 + e * (t + 2.0)) * it2;
    return c;
}

// Single precision: degree-12 series; crossovers chosen where the series
// truncation error and the cancellation error of the closed form (evaluated
// in FP32) are equal, which keeps every coefficient within ~3e-7 relative
// of its exact value for all t > 0.
__device__ __forceinline__ Coef<float> coefficients(float t)
{
    Coef<float> c;
    float e = expf(-t);
    c.e = e;
    float it = 1.0f / t, it2 = it * it;
    c.pm = t < 0.95f ? horner<float, 12, c_pm>(t) : (1.0f - e * (1.0f + t)) * it;
    c.po = t < 0.95f ? horner<float, 12, c_po>(t) : (e + t - 1.0f) * it;
    c.wm = t < 1.55f ? horner<float, 12, c_wm>(t) : (2.0f - e * (t * t + 2.0f * t + 2.0f)) * it2;
    c.wo = t < 2.35f ? horner<float, 12, c_wo>(t) : 1.0f - 2.0f * (e + t - 1.0f) * it2;
    c.wc = t < 1.45f ? horner<float, 12, c_wc>(t) : 2.0f * (t - 2.0f + e * (t + 2.0f)) * it2;
    return c;
}

__device__ __forceinline__ double exp_dev(double x) { return exp(x); }
__device__ __forceinline__ float exp_dev(float x) { return expf(x); }

// ---------------------------------------------------------------------------
// BESSER upwind control point c_M of the quadratic Bezier spline on MO
// (Sec. 3.2, steps 1-9); ihM = 1/h_M, ihP = 1/h_P, ihMP = 1/(h_M + h_P).
// ---------------------------------------------------------------------------
template <typename Real>
__device__ __forceinline__ Real control_point(Real yM, Real yO, Real yP, Real hM, Real hP,
                                              Real ihM, Real ihP, Real ihMP)
{
    Real dM = (yO - yM) * ihM;                       // step 1
    Real dP = (yP - yO) * ihP;
    if (dM * dP <= Real(0)) return yO;               // step 2: extremum at O
    Real yp = (hM * dP + hP * dM) * ihMP;            // step 3 (Eq. 6)
    Real cM = yO - Real(0.5) * hM * yp;              // step 4
    Real cP = yO + Real(0.5) * hP * yp;
    if (cM < fmin(yM, yO) || cM > fmax(yM, yO))      // step 5
        return yM;                                   // step 6: overshoot in MO
    if (cP < fmin(yO, yP) || cP > fmax(yO, yP))      // step 7: overshoot in OP
        cP = yP;
    yp = (cP - yO) * Real(2) * ihP;                  // step 8
    return yO - Real(0.5) * hM * yp;                 // step 9
}

// ---------------------------------------------------------------------------
// Hanle statistical equilibrium for K = 2 of the upper level (Eq. 2):
//   S_Q + i Gamma sum_Q' K_QQ'(B) S_Q' = R_Q,
// written for the real unknowns x = (S^2_0, Re S^2_1, Im S^2_1, Re S^2_2, Im S^2_2)
// using S_{-Q} = (-1)^Q conj(S_Q). With g = Gamma * B / |B| the real matrix is
//   [ 1          sqrt6 gy  -sqrt6 gx  0      0     ]
//   [-sqrt6/2 gy  1         -gz        gy    -gx    ]
//   [ sqrt6/2 gx  gz         1         gx     gy    ]
//   [ 0          -gy        -gx        1     -2 gz  ]
//   [ 0           gx        -gy        2 gz   1     ]
// Scaling the Q != 0 unknowns and equations by sqrt(2) makes the matrix the
// identity plus an antisymmetric matrix, whose symmetric part is positive
// definite; Gaussian elimination without pivoting is then stable (FP64).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void hanle_solve5(double gx, double gy, double gz, const double r[5], double x[5])
{
    const double s6 = 2.449489742783178098197284;  // sqrt(6)
    double A[5][6] = {
        {1.0, s6 * gy, -s6 * gx, 0.0, 0.0, r[0]},
        {-0.5 * s6 * gy, 1.0, -gz, gy, -gx, r[1]},
        {0.5 * s6 * gx, gz, 1.0, gx, gy, r[2]},
        {0.0, -gy, -gx, 1.0, -2.0 * gz, r[3]},
        {0.0, gx, -gy, 2.0 * gz, 1.0, r[4]},
    };
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        double inv = 1.0 / A[c][c];
#pragma unroll
        for (int q = c + 1; q < 5; ++q) {
            double f = A[q][c] * inv;
#pragma unroll
            for (int s = c; s < 6; ++s) A[q][s] -= f * A[c][s];
        }
    }
#pragma unroll
    for (int q = 4; q >= 0; --q) {
        double s = A[q][5];
#pragma unroll
        for (int t = q + 1; t < 5; ++t) s -= A[q][t] * x[t];
        x[q] = s / A[q][q];
    }
}

}  // namespace porta
