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
//   w_C = 2 (t - 2 + e (t + 2)) / t^2      (Eqs. 9-13).
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

// t * (a_1 + t (a_2 + ... + t a_N)) with a_k = COEF(k), N = DEG; every
// coefficient is a compile-time constant of type Real.
template <typename Real, double (*COEF)(int), int K, int DEG>
__device__ __forceinline__ Real horner_tail(Real t)
{
    constexpr double c = COEF(K);
    if constexpr (K == DEG) {
        return Real(c);
    } else {
        return Real(c) + t * horner_tail<Real, COEF, K + 1, DEG>(t);
    }
}

template <typename Real, int DEG, double (*COEF)(int)>
__device__ __forceinline__ Real horner(Real t)
{
    return t * horner_tail<Real, COEF, 1, DEG>(t);
}

// The linear-interpolation coefficients follow from the quadratic ones: a
// linear source on MO is the Bezier curve whose control point is the midpoint
// c_M = (y_M + y_O)/2, so psi'_M = w_M + w_C/2 and psi'_O = w_O + w_C/2 (all
// terms positive: no cancellation). Only the three w series are evaluated.

// Double precision: degree 8 (the order of Table 1), crossovers of Table 1
// (w_M 0.14, w_O and w_C 0.18).
__device__ __forceinline__ Coef<double> coefficients(double t)
{
    Coef<double> c;
    double e = exp(-t);
    c.e = e;
    double it = 1.0 / t, it2 = it * it;
    c.wm = t < 0.14 ? horner<double, 8, c_wm>(t) : (2.0 - e * (t * t + 2.0 * t + 2.0)) * it2;
    c.wo = t < 0.18 ? horner<double, 8, c_wo>(t) : 1.0 - 2.0 * (e + t - 1.0) * it2;
    c.wc = t < 0.18 ? horner<double, 8, c_wc>(t) : 2.0 * (t - 2.0 + e * (t + 2.0)) * it2;
    c.pm = c.wm + 0.5 * c.wc;
    c.po = c.wo + 0.5 * c.wc;
    return c;
}

// Single precision: three regimes, chosen so that every coefficient stays
// within 6e-7 relative of its exact value for all t > 0 when evaluated in
// FP32: degree-6 series for t < 0.25 (truncation below 2e-7 there), degree-12
// series for t < 1.5, closed forms above (where their cancellation costs at
// most a factor ~5).
// w_M, w_O, w_C of one optical path t given e = exp(-t)
__device__ __forceinline__ void wcoef(float t, float e, float &wm, float &wo, float &wc)
{
    if (t < 0.25f) {
        wm = horner<float, 6, c_wm>(t);
        wo = horner<float, 6, c_wo>(t);
        wc = horner<float, 6, c_wc>(t);
    } else if (t < 1.5f) {
        wm = horner<float, 12, c_wm>(t);
        wo = horner<float, 12, c_wo>(t);
        wc = horner<float, 12, c_wc>(t);
    } else {
        const float it = 1.0f / t, it2 = it * it;
        wm = (2.0f - e * (t * t + 2.0f * t + 2.0f)) * it2;
        wo = 1.0f - 2.0f * (e + t - 1.0f) * it2;
        wc = 2.0f * (t - 2.0f + e * (t + 2.0f)) * it2;
    }
}

__device__ __forceinline__ Coef<float> coefficients(float t)
{
    Coef<float> c;
    c.e = expf(-t);
    wcoef(t, c.e, c.wm, c.wo, c.wc);
    c.pm = c.wm + 0.5f * c.wc;
    c.po = c.wo + 0.5f * c.wc;
    return c;
}

// reciprocal: IEEE in FP64; in FP32 the hardware approximation rcp.approx.ftz
// (max 1 ulp; the operands here are normal numbers below 2^126), since the FP32
// form's error budget is 1e-5. The bare instruction saves the scaling steps of a
// general approximate division (4% of the J^K_Q sweep's time).
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Profile shape exp(-(x - s)^2). In FP32 it is evaluated as a power of two by
// the hardware approximation ex2.approx.ftz (max 2 ulp; the rounding of the FP32
// argument x - s already bounds its accuracy to ~1e-7 (x-s)^2 relative), and the
// exponent is capped at 60 so that eta_I and its reciprocal stay normal numbers
// far in the wings (the flush-to-zero form then never sees a subnormal result);
// the capped terms are below 1e-26 relative to line centre, where the optical
// paths vanish.
__device__ __forceinline__ float profile_shape(float xs)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(fminf(xs * xs, 60.0f) * -1.4426950408889634f));
    return r;
}
__device__ __forceinline__ double profile_shape(double xs) { return exp(-xs * xs); }

// ---------------------------------------------------------------------------
// BESSER upwind control point c_M of the quadratic Bezier spline on MO
// (Sec. 3.2, steps 1-9); ihM = 1/h_M, ihP = 1/h_P, ihMP = 1/(h_M + h_P).
// ---------------------------------------------------------------------------
// Per-update constants shared by the four Stokes parameters:
//   g.a = h_M/(h_P (h_M + h_P)), g.b = h_P/(h_M (h_M + h_P)), so that the derivative
//   of Eq. 6 is y'_O = g.a (y_P - y_O) + g.b (y_O - y_M);
//   g.hm2 = h_M/2, g.hp2 = h_P/2, g.r = h_M/h_P.
template <typename Real>
struct BesserGeom {
    Real a, b, hm2, hp2, r;
};

template <typename Real>
__device__ __forceinline__ BesserGeom<Real> besser_geom(Real hM, Real hP)
{
    BesserGeom<Real> g;
    const Real is = rcp(hM + hP);
    const Real ihM = rcp(hM), ihP = rcp(hP);
    g.a = hM * ihP * is;
    g.b = hP * ihM * is;
    g.hm2 = Real(0.5) * hM;
    g.hp2 = Real(0.5) * hP;
    g.r = hM * ihP;
    return g;
}

// Branch-free form: every step is evaluated and the outcome selected, so lanes
// of a warp that take different branches do not diverge. Interval tests use
// the sign of products ((c - y1)(c - y2) > 0 <=> c outside [min, max]).
// `branch` reports the outcome: 0 extremum at O (step 2), 1 c_M clipped to y_M
// (steps 5-6), 2 c_P clipped to y_P (steps 7-9), 3 the parabola (step 4).
template <typename Real>
__device__ __forceinline__ Real control_point_branch(Real yM, Real yO, Real yP, const BesserGeom<Real> &g, int &branch)
{
    const Real dm = yO - yM, dp = yP - yO;           // step 1 (h_M d_M, h_P d_P)
    const Real yp = g.a * dp + g.b * dm;             // step 3 (Eq. 6)
    const Real w = g.hm2 * yp;                       // step 4: c_M = y_O - w
    Real u = g.hp2 * yp;                             //         c_P = y_O + u
    const bool clip = u * (u - dp) > Real(0);        // step 7: c_P outside [y_O, y_P] -> y_P
    u = clip ? dp : u;
    const Real cM9 = yO - g.r * u;                   // steps 8-9: y'_O = 2 (c_P - y_O)/h_P
    const bool over = (dm - w) * w < Real(0);        // steps 5-6: c_M outside [y_M, y_O] -> y_M
    const Real r = over ? yM : cM9;
    const bool ext = dm * dp <= Real(0);             // step 2: extremum at O
    branch = ext ? 0 : (over ? 1 : (clip ? 2 : 3));
    return ext ? yO : r;
}

template <typename Real>
__device__ __forceinline__ Real control_point(Real yM, Real yO, Real yP, const BesserGeom<Real> &g)
{
    int branch;
    return control_point_branch(yM, yO, yP, g, branch);
}

// ---------------------------------------------------------------------------
// The BESSER-DELO step (Eq. 7) with a general propagation matrix: the seven
// elements (eta_I, eta_Q, eta_U, eta_V, rho_Q, rho_U, rho_V) at M and at O,
// K' = K/eta_I - 1 with the off-diagonal pattern of the Unno-Rachkovsky
// matrix, kappa^-1 = 1 + psi'_O K'_O (Eq. 8) solved by Gaussian elimination
// with partial pivoting. The two-level sweeps use its specializations (an I-V
// block, or the arrow of dichroism); this form is the general one.
// ---------------------------------------------------------------------------
template <typename Real>
__device__ __forceinline__ void kprime4(const Real *eta, Real K[4][4])
{
    const Real a = Real(1) / eta[0];
    const Real q = eta[1] * a, u = eta[2] * a, v = eta[3] * a, rq = eta[4] * a, ru = eta[5] * a, rv = eta[6] * a;
    K[0][0] = 0;  K[0][1] = q;   K[0][2] = u;   K[0][3] = v;
    K[1][0] = q;  K[1][1] = 0;   K[1][2] = rv;  K[1][3] = -ru;
    K[2][0] = u;  K[2][1] = -rv; K[2][2] = 0;   K[2][3] = rq;
    K[3][0] = v;  K[3][1] = ru;  K[3][2] = -rq; K[3][3] = 0;
}

template <typename Real>
__device__ __forceinline__ void delo_step_general(const Real IM[4], const Real etaM[7], const Real epsM[4],
                                                  const Real etaO[7], const Real epsO[4], Real etaP_I,
                                                  const Real epsP[4], Real dsM, Real dsP, bool has_p, Real IO[4],
                                                  Real &lstar)
{
    Real SM[4], SO[4], SP[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        SM[s] = epsM[s] / etaM[0];
        SO[s] = epsO[s] / etaO[0];
        SP[s] = has_p ? epsP[s] / etaP_I : Real(0);
    }
    const Real tMO = Real(0.5) * (etaM[0] + etaO[0]) * dsM;
    const Real tOP = has_p ? Real(0.5) * (etaO[0] + etaP_I) * dsP : Real(1);
    const Coef<Real> co = coefficients(tMO);
    Real cM[4];
    if (has_p) {
        const BesserGeom<Real> bg = besser_geom(tMO, tOP);
#pragma unroll
        for (int s = 0; s < 4; ++s) cM[s] = control_point(SM[s], SO[s], SP[s], bg);
    } else {
#pragma unroll
        for (int s = 0; s < 4; ++s) cM[s] = Real(0.5) * (SM[s] + SO[s]);
    }
    Real kM[4][4], kO[4][4], A[4][5];
    kprime4(etaM, kM);
    kprime4(etaO, kO);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        Real acc = co.e * IM[r];
#pragma unroll
        for (int s = 0; s < 4; ++s) acc -= co.pm * kM[r][s] * IM[s];
        A[r][4] = acc + co.wm * SM[r] + co.wo * SO[r] + co.wc * cM[r];
#pragma unroll
        for (int s = 0; s < 4; ++s) A[r][s] = (r == s ? Real(1) : Real(0)) + co.po * kO[r][s];
    }
    // elimination with partial pivoting (the diagonal is 1 + 0, off-diagonals psi'_O K'_O)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int piv = c;
#pragma unroll
        for (int r = c + 1; r < 4; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const Real x = A[c][s];
            A[c][s] = A[piv][s];
            A[piv][s] = x;
        }
        const Real inv = Real(1) / A[c][c];
#pragma unroll
        for (int r = c + 1; r < 4; ++r) {
            const Real f = A[r][c] * inv;
#pragma unroll
            for (int s = c; s < 5; ++s) A[r][s] -= f * A[c][s];
        }
    }
#pragma unroll
    for (int r = 3; r >= 0; --r) {
        Real s = A[r][4];
#pragma unroll
        for (int q = r + 1; q < 4; ++q) s -= A[r][q] * IO[q];
        IO[r] = s / A[r][r];
    }
    lstar = co.wo + (has_p ? co.wc : Real(0.5) * co.wc);
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

// y = M x with M the real matrix of hanle_solve5 (same unknowns and equations)
__device__ __forceinline__ void hanle_apply5(double gx, double gy, double gz, const double x[5], double y[5])
{
    const double s6 = 2.449489742783178098197284;  // sqrt(6)
    y[0] = x[0] + s6 * gy * x[1] - s6 * gx * x[2];
    y[1] = -0.5 * s6 * gy * x[0] + x[1] - gz * x[2] + gy * x[3] - gx * x[4];
    y[2] = 0.5 * s6 * gx * x[0] + gz * x[1] + x[2] + gx * x[3] + gy * x[4];
    y[3] = -gy * x[1] - gx * x[2] + x[3] - 2.0 * gz * x[4];
    y[4] = gx * x[1] - gy * x[2] + 2.0 * gz * x[3] + x[4];
}

}  // namespace porta
