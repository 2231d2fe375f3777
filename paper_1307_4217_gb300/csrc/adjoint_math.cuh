// Derivatives of the formal-solver step for the adjoint sweep (adjoint.cu):
// t-derivatives of the Bezier/DELO coefficients (Eqs. 9-13) and the partial
// derivatives of the BESSER control point (Sec. 3.2) on the branch it takes.
#pragma once
#include "device_math.cuh"

namespace porta {

// ---------------------------------------------------------------------------
// Derivatives for the adjoint sweep.
// d/dt of the step coefficients (Eqs. 9-13), from differentiating the closed
// forms and writing the result through the coefficients themselves:
//   de = -e,              dpsi'_M = e - psi'_M/t,   dpsi'_O = psi'_M/t,
//   dw_M = e - 2 w_M/t,   dw_O = w_C/t,             dw_C = 2 (psi'_M - w_C)/t.
// The cancellation in these forms is at most a factor of a few for every
// t > 0, so they are as accurate as the coefficients (series or closed form).
// ---------------------------------------------------------------------------
template <typename Real>
struct CoefD {
    Real de, dpm, dpo, dwm, dwo, dwc;
};

template <typename Real>
__device__ __forceinline__ CoefD<Real> coefficient_derivs(Real t, const Coef<Real> &c)
{
    CoefD<Real> d;
    const Real it = rcp(t);
    d.de = -c.e;
    d.dpm = c.e - c.pm * it;
    d.dpo = c.pm * it;
    d.dwm = c.e - Real(2) * c.wm * it;
    d.dwo = c.wc * it;
    d.dwc = Real(2) * (c.pm - c.wc) * it;
    return d;
}

// Partial derivatives of the BESSER control point with respect to
// (y_M, y_O, y_P, h_M, h_P) on the branch it takes (Sec. 3.2):
//   step 2 (extremum at O): c = y_O;  step 6 (overshoot in MO): c = y_M;
//   steps 7-9 with c_P clipped: c = y_O - (h_M/h_P)(y_P - y_O);
//   otherwise (step 4): c = y_O - h_M^2 (y_P - y_O)/(2 h_P s) - h_P (y_O - y_M)/(2 s),
//   s = h_M + h_P.
// The branch comes from control_point_branch on the same BesserGeom, so the
// adjoint takes the branch the forward sweep took. The h-derivatives of the
// parabola are linear in (d_P, d_M) = (y_P - y_O, y_O - y_M) with per-update
// factors, computed once for the four Stokes parameters.
template <typename Real>
struct BesserGrad {
    BesserGeom<Real> g;
    Real dyM, dyP;          // parabola: dc/dy_M, dc/dy_P
    Real hMp, hMm, hPp, hPm; // parabola: dc/dh_M = hMp d_P + hMm d_M, dc/dh_P = hPp d_P + hPm d_M
    Real ihP;                // 1/h_P (clipped branch)
};

template <typename Real>
__device__ __forceinline__ BesserGrad<Real> besser_grad(Real hM, Real hP)
{
    BesserGrad<Real> b;
    b.g = besser_geom(hM, hP);
    const Real is = rcp(hM + hP);
    b.ihP = rcp(hP);
    b.dyM = b.g.b * b.g.hm2;
    b.dyP = -b.g.a * b.g.hm2;
    // grouped as bounded ratios times one reciprocal: optical paths reach 1e-28
    // in the far wings, where 1/(h_M + h_P)^2 alone would overflow FP32
    const Real fM = hM * is, fP = hP * is, fq = (hM + Real(2) * hP) * is;   // in [0, 1], [0, 1], [1, 2]
    b.hMp = -Real(0.5) * fM * fq * b.ihP;
    b.hMm = Real(0.5) * fP * is;
    b.hPp = Real(0.5) * fM * fq * b.g.r * b.ihP;
    b.hPm = -Real(0.5) * fM * is;
    return b;
}

// partial derivatives of the control point on the branch that
// control_point_branch reported, selected without divergence
template <typename Real>
struct CpGrad {
    Real dyM, dyO, dyP, dhM, dhP;
};

template <typename Real>
__device__ __forceinline__ CpGrad<Real> control_point_grad(int branch, Real yM, Real yO, Real yP, const BesserGrad<Real> &b)
{
    const Real dm = yO - yM, dp = yP - yO;
    const Real rdp = dp * b.ihP;
    const Real hM = b.hMp * dp + b.hMm * dm, hP = b.hPp * dp + b.hPm * dm;
    const Real r = b.g.r;
    const bool e = branch == 0, o = branch == 1, k = branch == 2, q = branch == 3;
    CpGrad<Real> d;
    d.dyM = o ? Real(1) : (q ? b.dyM : Real(0));
    d.dyO = e ? Real(1) : (k ? Real(1) + r : (q ? Real(1) - b.dyM - b.dyP : Real(0)));
    d.dyP = k ? -r : (q ? b.dyP : Real(0));
    d.dhM = k ? -rdp : (q ? hM : Real(0));
    d.dhP = k ? r * rdp : (q ? hP : Real(0));
    return d;
}

// Solve M^T x = r with M the real matrix of hanle_solve5 (same scaling
// argument: M^T is the identity minus the antisymmetric part after the sqrt(2)
// rescaling, so elimination without pivoting is stable).
__device__ __forceinline__ void hanle_solve5_t(double gx, double gy, double gz, const double r[5], double x[5])
{
    const double s6 = 2.449489742783178098197284;  // sqrt(6)
    const double M[5][5] = {
        {1.0, s6 * gy, -s6 * gx, 0.0, 0.0},
        {-0.5 * s6 * gy, 1.0, -gz, gy, -gx},
        {0.5 * s6 * gx, gz, 1.0, gx, gy},
        {0.0, -gy, -gx, 1.0, -2.0 * gz},
        {0.0, gx, -gy, 2.0 * gz, 1.0},
    };
    double A[5][6];
#pragma unroll
    for (int a = 0; a < 5; ++a) {
#pragma unroll
        for (int c = 0; c < 5; ++c) A[a][c] = M[c][a];
        A[a][5] = r[a];
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const double inv = 1.0 / A[c][c];
#pragma unroll
        for (int q = c + 1; q < 5; ++q) {
            const double f = A[q][c] * inv;
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
