// Short characteristics that end on the first cell face they cross (Sec. 3.1:
// the upwind and downwind points M and P may lie on a vertical plane of the
// grid), for the J^K_Q formal solution of a set of boxes (one box, the line boxes
// of a multilevel atom, or independent boxes).
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
// One CTA of two warps per (box, ray, frequency group) item (a grid-stride loop over
// the items, about eight CTAs per SM: the line passes are bound by the latency of
// their dependent loads, so many small CTAs), the group's frequencies in order, the
// planes in sweep order; the CTA's Stokes planes (upwind and current), its
// Lambda* plane and the per-frequency transfer coefficients of the planes ku, k
// and kd (each computed once per plane and frequency) live in global scratch
// memory, laid out per ray so that the points of a line are adjacent (columns
// first for the rays whose face planes are swept in columns); each item's partial sums (stored on its first
// frequency, added on the later ones) are added over the groups in group order
// into the general sweep's per-ray partials, which the J^K_Q finalize sums over
// rays in ray order. A face plane's passes stop when no intensity changes by more
// than tol of the plane's largest, or, where a pass shrinks the change at least
// fourfold, once the change stops halving within 8 tol (the rounding floor); a
// plane that does neither within maxpass passes sets bit 2 of the error flag and
// keeps its last pass.
#include <algorithm>

#include "device_math.cuh"
#include "faces_kernels.cuh"
#include "sweep_common.cuh"

namespace porta {

namespace {

// The interpolation stencil of M (or P), the same for every point of a plane (the
// offset (f_x, f_y) of a layer is uniform): per corner its node offset from the
// point, taken modulo the grid (>= 0), and its weight; on a vertical face corners
// 0, 1 lie on the point's own plane (weight 1 - s) and 2, 3 on the neighbouring one
// (weight s), else all four lie on the neighbouring plane (bilinear). ds = s times
// the layer's path length (s = 1 off the faces).
template <typename Real>
struct Sten {
    int ox[4], oy[4];
    Real w[4];
    Real ds;
    double s;
    bool vert;
    bool xface;        // a vertical face x = const (|f_x| >= |f_y|), else y = const
    int step;          // order of the plane's lines in a pass: -1 where f > 0 (upwind first)
};

__device__ __forceinline__ int pmod(int i, int n) { return ((i % n) + n) % n; }

template <typename Real>
__device__ __forceinline__ Sten<Real> make_sten(int nx, int ny, double fx, double fy, double ds, bool planes)
{
    Sten<Real> st;
    int di[4], dj[4];
    double w[4], s = 1.0;
    // planes: M and P on the neighbouring horizontal planes at any offset (bilinear, periodic)
    st.vert = !planes && (fabs(fx) > 1.0 || fabs(fy) > 1.0);
    st.xface = fabs(fx) >= fabs(fy);
    st.step = (st.xface ? fx : fy) > 0 ? -1 : 1;
    if (st.vert) {
        // the first face crossed: x = x_(i + sgn f_x) where |f_x| >= |f_y|, at s = 1 / max(|f_x|, |f_y|)
        const double ax = fabs(fx), ay = fabs(fy);
        s = 1.0 / (ax >= ay ? ax : ay);
        const int sx = fx > 0 ? 1 : (fx < 0 ? -1 : 0), sy = fy > 0 ? 1 : (fy < 0 ? -1 : 0);
        double g;
        if (ax >= ay) {
            di[0] = di[1] = sx;
            dj[0] = 0;
            dj[1] = sy != 0 ? sy : 1;
            g = ay * s;
        } else {
            dj[0] = dj[1] = sy;
            di[0] = 0;
            di[1] = sx != 0 ? sx : 1;
            g = ax * s;
        }
        di[2] = di[0]; dj[2] = dj[0];
        di[3] = di[1]; dj[3] = dj[1];
        w[0] = (1 - g) * (1 - s); w[1] = g * (1 - s);
        w[2] = (1 - g) * s;       w[3] = g * s;
    } else {
        const double x0 = floor(fx), y0 = floor(fy), gx = fx - x0, gy = fy - y0;
        const int i0 = (int)x0, j0 = (int)y0;
        di[0] = i0; dj[0] = j0; di[1] = i0 + 1; dj[1] = j0;
        di[2] = i0; dj[2] = j0 + 1; di[3] = i0 + 1; dj[3] = j0 + 1;
        w[0] = (1 - gx) * (1 - gy); w[1] = gx * (1 - gy);
        w[2] = (1 - gx) * gy;       w[3] = gx * gy;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        st.ox[c] = pmod(di[c], nx);
        st.oy[c] = pmod(dj[c], ny);
        st.w[c] = (Real)w[c];
    }
    st.ds = (Real)(s * ds);
    st.s = s;
    return st;
}

// The BESSER-DELO step (Eq. 7) where the propagation matrix holds eta_I and eta_V
// only (the two-level atoms' weak-field Zeeman term): kappa^-1 = 1 + psi'_O K'_O
// (Eq. 8) couples I and V alone and is inverted in closed form; Q and U are the
// scalar step. Lambda* as in Eq. 14 (w_O + w_C/2 on the last plane).
template <typename Real>
__device__ __forceinline__ void delo_step_iv(const Real IM[4], Real etaM, Real etaVM, const Real epsM[4], Real etaO,
                                             Real etaVO, const Real epsO[4], Real etaP, const Real epsP[4], Real dM,
                                             Real dP, bool has_p, Real IO[4], Real &ls)
{
    const Real iM = Real(1) / etaM, iO = Real(1) / etaO, iP = has_p ? Real(1) / etaP : Real(0);
    Real SM[4], SO[4], SP[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        SM[s] = epsM[s] * iM;
        SO[s] = epsO[s] * iO;
        SP[s] = epsP[s] * iP;
    }
    const Real tMO = Real(0.5) * (etaM + etaO) * dM;
    const Coef<Real> co = coefficients(tMO);
    Real cM[4];
    if (has_p) {
        const BesserGeom<Real> bg = besser_geom(tMO, Real(0.5) * (etaO + etaP) * dP);
#pragma unroll
        for (int s = 0; s < 4; ++s) cM[s] = control_point(SM[s], SO[s], SP[s], bg);
    } else {
#pragma unroll
        for (int s = 0; s < 4; ++s) cM[s] = Real(0.5) * (SM[s] + SO[s]);
    }
    Real r[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) r[s] = co.e * IM[s] + co.wm * SM[s] + co.wo * SO[s] + co.wc * cM[s];
    const Real pk = co.pm * (etaVM * iM);
    r[0] -= pk * IM[3];
    r[3] -= pk * IM[0];
    const Real av = co.po * (etaVO * iO), idet = Real(1) / (Real(1) - av * av);
    IO[0] = (r[0] - av * r[3]) * idet;
    IO[3] = (r[3] - av * r[0]) * idet;
    IO[1] = r[1];
    IO[2] = r[2];
    ls = co.wo + (has_p ? co.wc : Real(0.5) * co.wc);
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

// Media of the sweep: the two-level atoms (I-V coupling by the weak-field Zeeman
// term), a polarized multilevel line (dichroism), or an explicit medium (a general
// propagation matrix given per voxel).
enum FaceMedium { FM_PLAIN = 0, FM_DICH = 1, FM_GEN = 2 };

// Coefficient words per node: eta_I, eta_V, eps (NS); with dichroism: eta_I, eta_Q,
// eta_U, eta_V, eps (4); explicit medium: eta_I, eta_Q, eta_U, eta_V, rho_Q, rho_U,
// rho_V, eps (4).
template <int NS, int FM>
struct CW {
    static constexpr int n = FM == FM_GEN ? 11 : (FM == FM_DICH ? 8 : NS + 2);
    static constexpr int ev = FM == FM_PLAIN ? 1 : 3;                       // eta_V
    static constexpr int eps = FM == FM_GEN ? 7 : (FM == FM_DICH ? 4 : 2);  // first emission word
};

// The line's dichroism and orientation terms at node v for the ray (a polarized
// multilevel line, Sec. 2): eta_i / (chi phi) = 1 + d_i(Omega) from the lower-level
// multipoles D^2_Q (i = I, Q, U) and D^1_Q (V); the node's opacity is rescaled by
// 1 + d_I, its source terms and Zeeman factor by 1 / (1 + d_I); returns the ratios
// eta_Q / eta_I, eta_U / eta_I, the orientation term of eta_V / eta_I and the
// orientation emission of S_V (the emission multipoles S^1_Q projected on V).
template <typename Real>
__device__ __forceinline__ void dich_terms(const SweepArgs<Real> &a, const RayDev<Real> &ray, long long v,
                                           Node<Real, 4> &n, Real &dq, Real &du, Real &dv, Real &sv)
{
    const long long nv = a.nvox;
    const Real d20 = a.dich[v], d21r = a.dich[nv + v], d21i = a.dich[2 * nv + v];
    const Real d22r = a.dich[3 * nv + v], d22i = a.dich[4 * nv + v];
    Real dd[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const Real *t = ray.t + 6 * i;
        dd[i] = t[1] * d20 + Real(2) * (t[2] * d21r + t[3] * d21i) + Real(2) * (t[4] * d22r + t[5] * d22i);
    }
    // T^1_Q(V, Omega) = sqrt(3/2) Omega_Q: T10 = sqrt(3/2) Omega_z, T11 = -sqrt(3/4) (Omega_x + i Omega_y)
    const Real t10 = Real(1.2247448713915890491) * ray.oz;
    const Real t11r = Real(-0.86602540378443864676) * ray.ox, t11i = Real(-0.86602540378443864676) * ray.oy;
    const Real dvr = t10 * a.dich[5 * nv + v] + Real(2) * (t11r * a.dich[6 * nv + v] + t11i * a.dich[7 * nv + v]);
    const Real svr = t10 * a.dich[8 * nv + v] + Real(2) * (t11r * a.dich[9 * nv + v] + t11i * a.dich[10 * nv + v]);
    const Real f = Real(1) + dd[0], inv = Real(1) / f;
    n.chi *= f;
    n.SI *= inv;
    n.SQ *= inv;
    n.SU *= inv;
    n.b *= inv;
    dq = dd[1] * inv;
    du = dd[2] * inv;
    dv = dvr * inv;
    sv = svr * inv;
}

// A ray's planes in scratch memory: row-major (p = j nx + i), or column-major
// (p = i ny + j) for the rays whose face planes are swept in columns (x faces),
// so that the points of a line lie together in both cases.
struct Layout {
    int nx, ny;
    bool col;
    __device__ __forceinline__ int at(int i, int j) const { return col ? i * ny + j : j * nx + i; }
};

// the transfer coefficients of every node of plane k at frequency x, word c of
// node (i, j) at cw[(c * nxy) + L.at(i, j)] (the nodes read in the atmosphere's order)
template <typename Real, int NS, int FM>
__device__ __forceinline__ void plane_coefs(const SweepArgs<Real> &a, const RayDev<Real> &ray, int m, long long base,
                                            const Layout &L, Real x, Real *cw)
{
    using C = CW<NS, FM>;
    constexpr bool DI = FM == FM_DICH;
    const int nxy = L.nx * L.ny;
    for (int p = threadIdx.x; p < nxy; p += blockDim.x) {
        Node<Real, NS> n = make_node<Real, NS>(a, ray, base + p, m, false);
        Real w[C::n];
        const Real xs = x - n.s;
        if constexpr (NS == 1) {
            w[0] = n.chi * profile_shape(xs);
            w[1] = Real(0);
            w[2] = w[0] * n.S;
        } else if constexpr (FM == FM_GEN) {
            // explicit medium: K'/eta_I (eta_Q, eta_U, eta_V, rho_Q, rho_U, rho_V) and S per voxel
            const long long v = base + p, nv = a.nvox;
            const Real eI = n.chi * profile_shape(xs);
            w[0] = eI;
#pragma unroll
            for (int k = 0; k < 6; ++k) w[1 + k] = eI * (Real)a.kexpl[k * nv + v];
#pragma unroll
            for (int i = 0; i < 4; ++i) w[7 + i] = eI * (Real)a.sexpl[i * nv + v];
        } else {
            Real dq = 0, du = 0, dv = 0, sv = 0;
            if constexpr (DI) dich_terms<Real>(a, ray, base + p, n, dq, du, dv, sv);
            const Real eI = n.chi * profile_shape(xs), bx = n.b * xs;
            w[0] = eI;
            if constexpr (DI) {
                w[1] = eI * dq;
                w[2] = eI * du;
            }
            w[C::ev] = eI * (bx + dv);
            w[C::eps] = eI * n.SI;
            w[C::eps + 1] = eI * n.SQ;
            w[C::eps + 2] = eI * n.SU;
            w[C::eps + 3] = eI * (bx * n.S00 + sv);
        }
        const int jy = p / L.nx, lp = L.at(p - jy * L.nx, jy);
#pragma unroll
        for (int c = 0; c < C::n; ++c) cw[c * nxy + lp] = w[c];
    }
}

// The BESSER-DELO step (Eq. 7) of a polarized multilevel line: K' holds eta_Q,
// eta_U (dichroism) and eta_V over eta_I, so kappa^-1 = 1 + psi'_O K'_O (Eq. 8) is an
// arrow matrix (first row and column, unit diagonal), inverted in closed form.
template <typename Real>
__device__ __forceinline__ void delo_step_arrow(const Real IM[4], const Real eM[8], const Real eO[8], Real etaP,
                                                const Real epsP[4], Real dM, Real dP, bool has_p, Real IO[4], Real &ls)
{
    const Real iM = Real(1) / eM[0], iO = Real(1) / eO[0], iP = has_p ? Real(1) / etaP : Real(0);
    Real SM[4], SO[4], SP[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        SM[s] = eM[4 + s] * iM;
        SO[s] = eO[4 + s] * iO;
        SP[s] = epsP[s] * iP;
    }
    const Real tMO = Real(0.5) * (eM[0] + eO[0]) * dM;
    const Coef<Real> co = coefficients(tMO);
    Real cM[4];
    if (has_p) {
        const BesserGeom<Real> bg = besser_geom(tMO, Real(0.5) * (eO[0] + etaP) * dP);
#pragma unroll
        for (int s = 0; s < 4; ++s) cM[s] = control_point(SM[s], SO[s], SP[s], bg);
    } else {
#pragma unroll
        for (int s = 0; s < 4; ++s) cM[s] = Real(0.5) * (SM[s] + SO[s]);
    }
    const Real qM = eM[1] * iM, uM = eM[2] * iM, vM = eM[3] * iM;
    Real r[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) r[s] = co.e * IM[s] + co.wm * SM[s] + co.wo * SO[s] + co.wc * cM[s];
    r[0] -= co.pm * (qM * IM[1] + uM * IM[2] + vM * IM[3]);
    r[1] -= co.pm * qM * IM[0];
    r[2] -= co.pm * uM * IM[0];
    r[3] -= co.pm * vM * IM[0];
    const Real aq = co.po * (eO[1] * iO), au = co.po * (eO[2] * iO), av = co.po * (eO[3] * iO);
    IO[0] = (r[0] - aq * r[1] - au * r[2] - av * r[3]) / (Real(1) - aq * aq - au * au - av * av);
    IO[1] = r[1] - aq * IO[0];
    IO[2] = r[2] - au * IO[0];
    IO[3] = r[3] - av * IO[0];
    ls = co.wo + (has_p ? co.wc : Real(0.5) * co.wc);
}

// One CTA per (box, ray, frequency group). Per frequency and plane: the coefficients of
// the downwind plane kd (those of the planes ku and k carried over from the two
// planes before), then the plane's points. Where M lies on the upwind plane (offset
// within a cell) one parallel pass is exact; where it lies on vertical faces the
// plane is swept line by line in the upwind order (columns for x faces, rows for y
// faces: a line's points depend only on the line before), in place, and the pass is
// repeated until no intensity changes by more than tol of the plane's largest (the
// first line of a pass reads the last line of the previous one: the periodic chain).
// (FP32: eight CTAs of 64 threads per SM, i.e. at most 128 registers a thread)
template <typename Real, int NS, int FM>
__global__ void __launch_bounds__(64, sizeof(Real) == 4 ? 8 : 3) faces_kernel(const SweepArgs<Real> a, Real *scratch, long long cta_words,
                                                  Real *gpart, Real *gpartv, int nbox, int ngroups, const double *dxy,
                                                  int maxpass, Real tol, int *err, int emergent, int planes)
{
    using C = CW<NS, FM>;
    constexpr bool DI = FM == FM_DICH;
    constexpr int NC = C::n;                      // coefficient words per node
    __shared__ Real red[2];
    const int fper = (a.nnu + ngroups - 1) / ngroups;
    const int per_box = a.nray * ngroups;
    // work items: (box, ray, frequency group), each CTA with its own scratch slot
    for (int item = blockIdx.x; item < nbox * per_box; item += gridDim.x) {
        const int box = item / per_box, r = item - box * per_box;
        const int m = r / ngroups, grp = r - m * ngroups;
        const BoxDev B = a.boxes[box];
        const int nx = B.nx, ny = B.ny, nz = B.nz;
        const long long nxy = (long long)nx * ny;
        const double dx = dxy[2 * box], dy = dxy[2 * box + 1];
        const RayDev<Real> ray = a.rays[m];
        const PlaneGeom<Real> *G = a.geom + B.geom0 + (long long)m * nz;
        const bool upward = ray.mu > Real(0);
        const Layout L = {nx, ny, fabs((double)ray.ox / dx) >= fabs((double)ray.oy / dy)};
        // scratch of the CTA: two Stokes planes (upwind and current, swapped per
        // plane), Lambda*, three coefficient planes (ku, k, kd, rotated per plane)
        Real *Iu = scratch + (long long)blockIdx.x * cta_words;
        Real *Ik = Iu + NS * nxy;
        Real *lsb = Ik + NS * nxy;
        Real *cu = lsb + nxy, *ck = cu + NC * nxy, *cd = ck + NC * nxy;
        // this item's partial sums over its frequencies: [ray][group][nvox] (the box's
        // voxels); with dichroism also the integral of Stokes V (J^1_Q)
        Real *part = gpart + ((long long)m * ngroups + grp) * a.nvox * (NS == 1 ? 2 : 4);
        Real *partv = DI ? gpartv + ((long long)m * ngroups + grp) * a.nvox : nullptr;
        const int jb = grp * fper, je = min(a.nnu, jb + fper);
        for (int j = jb; j < je; ++j) {
            const Real x = a.xf[j], wf = a.wf[j];
            for (int q = 0; q < nz; ++q) {
                const int k = G[q].kz;
                const long long base = B.vox0 + (long long)k * nxy;
                if (q == 0) {
                    for (int p = threadIdx.x; p < nxy; p += blockDim.x) {
                        const long long v = base + p;
                        const int jy = p / nx, lp = L.at(p - jy * nx, jy);
                        Real I0[NS];
#pragma unroll
                        for (int s = 0; s < NS; ++s) I0[s] = Real(0);
                        if (upward) I0[0] = a.bpl[v];
#pragma unroll
                        for (int s = 0; s < NS; ++s) Ik[s * nxy + lp] = I0[s];
                        lsb[lp] = Real(0);
                    }
                } else {
                    const int ku = G[q - 1].kz;
                    const bool has_p = q + 1 < nz;
                    const int kd = has_p ? G[q + 1].kz : k;
                    const double dsM = (double)G[q].ds, dsP = has_p ? (double)G[q + 1].ds : 0.0;
                    const Sten<Real> sm =
                        make_sten<Real>(nx, ny, -dsM * (double)ray.ox / dx, -dsM * (double)ray.oy / dy, dsM, planes != 0);
                    const Sten<Real> sp =
                        make_sten<Real>(nx, ny, dsP * (double)ray.ox / dx, dsP * (double)ray.oy / dy, dsP, planes != 0);
                    const bool vertP = has_p && sp.vert;
                    // the finished plane becomes the upwind one; the coefficients of
                    // ku and k are those of the previous step's k and kd
                    {
                        Real *t = Iu;
                        Iu = Ik;
                        Ik = t;
                    }
                    if (q >= 2) {
                        Real *t = cu;
                        cu = ck;
                        ck = cd;
                        cd = t;
                    }
                    // a face plane's passes start from zero intensities
                    if (sm.vert)
                        for (long long e = threadIdx.x; e < NS * nxy; e += blockDim.x) Ik[e] = Real(0);
                    if (q == 1) {
                        plane_coefs<Real, NS, FM>(a, ray, m, B.vox0 + (long long)ku * nxy, L, x, cu);
                        plane_coefs<Real, NS, FM>(a, ray, m, base, L, x, ck);
                    }
                    if (has_p) plane_coefs<Real, NS, FM>(a, ray, m, B.vox0 + (long long)kd * nxy, L, x, cd);
                    __syncthreads();
                    // one point's update (in place into Ik); returns the change of its Stokes vector
                    auto update = [&](int ix, int jy, Real &chg, Real &mag) {
                        const int p = L.at(ix, jy);
                        // M: every coefficient word and the Stokes vector, interpolated
                        Real eM[NC], IM[NS];
#pragma unroll
                        for (int w = 0; w < NC; ++w) eM[w] = Real(0);
#pragma unroll
                        for (int s = 0; s < NS; ++s) IM[s] = Real(0);
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            int ia = ix + sm.ox[c], ja = jy + sm.oy[c];
                            ia -= ia >= nx ? nx : 0;
                            ja -= ja >= ny ? ny : 0;
                            const bool own = sm.vert && c < 2;
                            const Real *cc = own ? ck : cu;
                            const Real *Ib = own ? Ik : Iu;
                            const int pc = L.at(ia, ja);
                            const Real wc = sm.w[c];
#pragma unroll
                            for (int w = 0; w < NC; ++w) eM[w] += wc * cc[w * nxy + pc];
#pragma unroll
                            for (int s = 0; s < NS; ++s) IM[s] += wc * Ib[s * nxy + pc];
                        }
                        Real eO[NC];
#pragma unroll
                        for (int w = 0; w < NC; ++w) eO[w] = ck[w * nxy + p];
                        // P: eta_I and the emission
                        Real etaP = 0, epsP[NS];
#pragma unroll
                        for (int s = 0; s < NS; ++s) epsP[s] = Real(0);
                        if (has_p) {
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                int ia = ix + sp.ox[c], ja = jy + sp.oy[c];
                                ia -= ia >= nx ? nx : 0;
                                ja -= ja >= ny ? ny : 0;
                                const Real *cc = vertP && c < 2 ? ck : cd;
                                const int pc = L.at(ia, ja);
                                const Real wc = sp.w[c];
                                etaP += wc * cc[pc];
#pragma unroll
                                for (int s = 0; s < NS; ++s) epsP[s] += wc * cc[(C::eps + s) * nxy + pc];
                            }
                        }
                        const Real dM = sm.ds, dP = sp.ds;
                        Real IO[NS], ls;
                        if constexpr (NS == 1) {
                            const Real SM = eM[2] / eM[0], SO = eO[2] / eO[0];
                            const Real tMO = Real(0.5) * (eM[0] + eO[0]) * dM;
                            const Coef<Real> co = coefficients(tMO);
                            Real cM;
                            if (has_p) {
                                const Real SP = epsP[0] / etaP, tOP = Real(0.5) * (eO[0] + etaP) * dP;
                                cM = control_point(SM, SO, SP, besser_geom(tMO, tOP));
                            } else {
                                cM = Real(0.5) * (SM + SO);
                            }
                            IO[0] = co.e * IM[0] + co.wm * SM + co.wo * SO + co.wc * cM;
                            ls = co.wo + (has_p ? co.wc : Real(0.5) * co.wc);
                        } else if constexpr (DI) {
                            delo_step_arrow<Real>(IM, eM, eO, etaP, epsP, dM, dP, has_p, IO, ls);
                        } else if constexpr (FM == FM_GEN) {
                            // the seven elements of K' (Eqs. 7-8), pivoted elimination
                            delo_step_general<Real>(IM, eM, eM + 7, eO, eO + 7, etaP, epsP, dM, dP, has_p, IO, ls);
                        } else {
                            delo_step_iv<Real>(IM, eM[0], eM[1], eM + 2, eO[0], eO[1], eO + 2, etaP, epsP, dM, dP, has_p, IO, ls);
                        }
#pragma unroll
                        for (int s = 0; s < NS; ++s) {
                            chg = fmax(chg, fabs(IO[s] - Ik[s * nxy + p]));
                            mag = fmax(mag, fabs(IO[s]));
                            Ik[s * nxy + p] = IO[s];
                        }
                        lsb[p] = ls;
                    };
                    if (!sm.vert) {
                        Real chg = 0, mag = 0;
                        // the points in the layout's order
                        const int n_in = L.col ? ny : nx;
                        for (int p = threadIdx.x; p < nxy; p += blockDim.x) {
                            const int o = p / n_in, r = p - o * n_in;
                            if (L.col) update(o, r, chg, mag);
                            else update(r, o, chg, mag);
                        }
                    } else {
                        // lines in the upwind order: a point depends on the line at +sgn(f)
                        const bool xface = sm.xface;
                        const int n_lines = xface ? nx : ny, n_pts = xface ? ny : nx;
                        const int step = sm.step;
                        // (1 - s)^n bounds the factor by which a pass shrinks the change of
                        // the plane (the chain's own-plane weight 1 - s over n lines, times
                        // transmissions e^-tau <= 1); where it is below 1/4, a change that no
                        // longer halves from one pass to the next is rounding noise
                        const bool fast = pow(1.0 - sm.s, (double)n_lines) <= 0.25;
                        Real prev = 0;
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
                            if (fast && pass >= 1 && chg >= Real(0.5) * prev && chg <= Real(8) * tol * mag) break;
                            prev = chg;
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
                        for (int p = threadIdx.x; p < nxy; p += blockDim.x) {
                            const int jy = p / nx, lp = L.at(p - jy * nx, jy);
#pragma unroll
                            for (int s = 0; s < NS; ++s)
                                a.out[(((long long)m * a.nnu + j) * nxy + p) * NS + s] = (double)Ik[s * nxy + lp];
                        }
                    __syncthreads();
                    continue;
                }
                // the plane's sums: w_j phi_O / N (I, Q, U, Lambda*) added to the ray's partials
                for (int p = threadIdx.x; p < nxy; p += blockDim.x) {
                    const long long vO = base + p;
                    const int jy = p / nx, lp = L.at(p - jy * nx, jy);
                    const Real wt = wf * profile_shape(x - a.vel[vO] * ray.mu) * a.invn[(long long)m * a.nvox + vO];
                    if constexpr (NS == 1) {
                        R2<Real> *pp = reinterpret_cast<R2<Real> *>(part) + vO;
                        R2<Real> o = {wt * Ik[lp], wt * lsb[lp]};
                        if (j > jb) { const R2<Real> old = *pp; o.x += old.x; o.y += old.y; }
                        *pp = o;
                    } else {
                        R4<Real> *pp = reinterpret_cast<R4<Real> *>(part) + vO;
                        R4<Real> o = {wt * Ik[lp], wt * Ik[nxy + lp], wt * Ik[2 * nxy + lp], wt * lsb[lp]};
                        if (j > jb) { const R4<Real> old = *pp; o.x += old.x; o.y += old.y; o.z += old.z; o.w += old.w; }
                        *pp = o;
                        if constexpr (DI) partv[vO] = (j > jb ? partv[vO] : Real(0)) + wt * Ik[3 * nxy + lp];
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

// frequency groups: enough (box, ray, group) items for ~8 CTAs per SM
static int faces_groups(int nbox, int nray, int nnu)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long base = std::max(1LL, (long long)nbox * nray);
    return (int)std::max(1LL, std::min<long long>(nnu, 8LL * std::max(1, nsm) / base));
}

static int faces_ctas(long long items)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return (int)std::max(1LL, std::min<long long>(items, 8LL * std::max(1, nsm)));
}

template <typename Real, int NS>
size_t faces_scratch_bytes(int nbox, int nray, int nnu, long long nxy_max, long long nvox, int medium)
{
    const int ng = faces_groups(nbox, nray, nnu);
    const int ctas = faces_ctas((long long)nbox * nray * ng);
    const bool di = NS == 4 && medium == FM_DICH;
    const int nc = NS == 4 && medium == FM_GEN ? 11 : (di ? 8 : NS + 2);
    // with one group the items write the per-ray partials directly
    const size_t na = (NS == 1 ? 2 : 4) + (di ? 1 : 0);
    const size_t gpart = ng > 1 ? (size_t)nray * ng * nvox * na : 0;
    return sizeof(Real) * ((size_t)ctas * (2 * NS + 1 + 3 * nc) * nxy_max + gpart);
}

template <typename Real, int NS, int FM>
static cudaError_t launch_faces_k(const SweepArgs<Real> &a, Real *scratch, int nbox, long long nxy_max,
                                  const double *dxy, int maxpass, int *err, cudaStream_t st, bool emergent, bool planes)
{
    const Real tol = sizeof(Real) == 8 ? Real(1e-15) : Real(2e-7);
    const int ng = faces_groups(nbox, a.nray, a.nnu);
    const int ctas = faces_ctas((long long)nbox * a.nray * ng);
    constexpr bool DI = FM == FM_DICH;
    const long long cta_words = (long long)(2 * NS + 1 + 3 * CW<NS, FM>::n) * nxy_max;
    constexpr int NA = NS == 1 ? 2 : 4;
    Real *gpart = ng > 1 ? scratch + (size_t)ctas * cta_words : (Real *)a.part;
    Real *gpartv = ng > 1 ? gpart + (size_t)a.nray * ng * a.nvox * NA : a.partv;
    faces_kernel<Real, NS, FM><<<ctas, 64, 0, st>>>(a, scratch, cta_words, gpart, gpartv, nbox, ng, dxy, maxpass, tol,
                                                    err, emergent ? 1 : 0, planes ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || emergent || ng == 1) return e;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long n = (long long)a.nray * a.nvox;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 16LL * std::max(1, nsm));
    faces_group_sum_kernel<Real, NA><<<blocks, 256, 0, st>>>(gpart, ng, a.nvox, a.nray, (Real *)a.part);
    e = cudaGetLastError();
    if (e == cudaSuccess && DI) {
        faces_group_sum_kernel<Real, 1><<<blocks, 256, 0, st>>>(gpartv, ng, a.nvox, a.nray, a.partv);
        e = cudaGetLastError();
    }
    return e;
}

template <typename Real, int NS>
cudaError_t launch_faces(const SweepArgs<Real> &a, Real *scratch, int nbox, long long nxy_max, const double *dxy,
                         int maxpass, int *err, cudaStream_t st, bool emergent, bool planes)
{
    if constexpr (NS == 4) {
        if (a.dich)
            return launch_faces_k<Real, 4, FM_DICH>(a, scratch, nbox, nxy_max, dxy, maxpass, err, st, emergent, planes);
        if (a.kexpl)
            return launch_faces_k<Real, 4, FM_GEN>(a, scratch, nbox, nxy_max, dxy, maxpass, err, st, emergent, planes);
    }
    return launch_faces_k<Real, NS, FM_PLAIN>(a, scratch, nbox, nxy_max, dxy, maxpass, err, st, emergent, planes);
}

#define PORTA_FACES_INST(R, N)                                                                              \
    template cudaError_t launch_faces<R, N>(const SweepArgs<R> &, R *, int, long long, const double *, int, int *, \
                                            cudaStream_t, bool, bool);                                           \
    template size_t faces_scratch_bytes<R, N>(int, int, int, long long, long long, int);
PORTA_FACES_INST(float, 1)
PORTA_FACES_INST(float, 4)
PORTA_FACES_INST(double, 1)
PORTA_FACES_INST(double, 4)
#undef PORTA_FACES_INST

}  // namespace porta
