// Formal solution for the radiation-field tensors (Sec. 3 of Stepan & Trujillo
// Bueno 2013): the short-characteristics BESSER sweep of every ray direction
// and frequency, fused with the frequency integration of the Stokes parameters
// and Lambda* that feeds J^K_Q (Eq. 1, Eq. 14) and the Jacobi update.
//
// The decomposition is that of the general sweep (sweep.cu): one thread-block
// cluster per ray at a time, the plane split into strips of sheared rows, one
// per CTA, with the first row of the next strip read through DSMEM after a
// cluster barrier, and the stencils of the bilinear interpolation at the
// upwind point M and downwind point P fixed nearest-neighbour accesses in the
// frame sheared along the characteristics.
//
// What this kernel does differently. The transfer coefficients of a node
// depend on the frequency only through the profile, eta_I = chi phi(x - s) and
// eta_V = b (x - s) eta_I, while its source vector S(Omega) does not (CRD).
// When a plane enters the 3-slot ring, its nodes' frequency-independent data
// (S_I, S_Q, S_U, S^0_0 | chi, s, b, 1/N) are staged once, and then, for every
// frequency of the pass, the node's (eta_I, eta_V) are computed once and kept
// in shared memory. A point update then interpolates eps = sum_k w_k eta_k S_k
// and eta = sum_k w_k eta_k from its 4 upwind and 4 downwind corners without
// evaluating a profile: the corners' source vectors are read once per point
// (registers across the frequency loop), their (eta_I, eta_V) once per
// frequency. Only the point O itself evaluates its profile (for Lambda* and
// the frequency-integration weight).
//
// Shared memory per CTA:
//   ring[3][NCH][nodes]   frequency-independent node data (16-byte chunks)
//   coef[3][F][nodes]     (eta_I, eta_V) (NS = 4) or eta_I (NS = 1) per frequency
//   ibuf[2][F][...][pts]  Stokes vectors of planes q-1 and q
//   lane[threads][NA]     fixed-order frequency-lane reduction
// with nodes = (rows + 2) nx (one halo row on each side, recomputed locally).
#include <cooperative_groups.h>

#include "device_math.cuh"
#include "porta_internal.cuh"
#include "sweep_common.cuh"

namespace cg = cooperative_groups;

namespace porta {

namespace {

// Shared-memory words per node: the ring holds the frequency-independent source
// vector (NS = 4: S_I, S_Q, S_U, S^0_0 as 16-byte chunks; NS = 1: S as a scalar
// plane); the transient staging area holds (chi, s[, b]) of the plane being
// filled, for the per-frequency coefficients.
template <typename Real, int NS>
struct JW {
    static constexpr int per = 16 / (int)sizeof(Real);        // Reals per 16-byte chunk
    static constexpr int s_words = NS == 1 ? 1 : 4;            // source words per node
    static constexpr int s_chunks = NS == 1 ? 0 : 4 / per;     // 16-byte chunks per node (NS = 4)
    static constexpr int g_words = NS == 1 ? 2 : 3;            // staged geometry words per node
    static constexpr int cw = NS == 1 ? 1 : 2;                 // coefficient words per node and frequency
    static constexpr int na = NS == 1 ? 2 : 4;                 // accumulated quantities per point
    static constexpr int nacc = NS == 1 ? 2 : 7;               // fixed-point accumulators per voxel
};

template <typename Real>
__device__ __forceinline__ void chunk_put(typename V16<Real>::T *p, const Real *w)
{
    if constexpr (sizeof(Real) == 4) *p = make_float4(w[0], w[1], w[2], w[3]);
    else *p = make_double2(w[0], w[1]);
}
template <typename Real>
__device__ __forceinline__ void chunk_get(const typename V16<Real>::T *p, Real *w)
{
    if constexpr (sizeof(Real) == 4) {
        const float4 v = *p;
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else {
        const double2 v = *p;
        w[0] = v.x; w[1] = v.y;
    }
}

constexpr int kJFrac = 46;   // fixed-point fraction bits below a voxel's reference value

// 2^e as an exact floating-point value (e within the type's normal exponent range)
__device__ __forceinline__ float pow2(float, int e) { return __int_as_float((e + 127) << 23); }
__device__ __forceinline__ double pow2(double, int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// one term of the fixed-point sum: x * 2^e (exact) rounded to an integer. Integer
// additions are exact and commute, so the sums do not depend on the order in which
// rays, frequency passes and concurrent launches add their terms. A term beyond
// 2^62 (or not finite) sets the overflow flag instead.
__device__ __forceinline__ void jadd(unsigned long long *p, float y, int *err)
{
    if (!(fabsf(y) < 4.6116860e18f)) {
        atomicOr(err, 1);
        return;
    }
    // y = +-m 2^ex with the 24-bit significand m: the integer nearest to y from
    // integer operations (halves away from zero; |y| < 2^-1 gives 0)
    const unsigned b = __float_as_uint(y);
    const int ex = (int)((b >> 23) & 0xffu) - 150;
    const unsigned m = (b & 0x7fffffu) | 0x800000u;
    long long n = 0;
    if (ex >= 0) n = (long long)((unsigned long long)m << ex);
    else if (ex > -25) n = (long long)((m + (1u << (-ex - 1))) >> (-ex));
    if (b >> 31) n = -n;
    atomicAdd(p, (unsigned long long)n);
}
__device__ __forceinline__ void jadd(unsigned long long *p, double y, int *err)
{
    if (!(fabs(y) < 4.611686018427387904e18)) {
        atomicOr(err, 1);
        return;
    }
    atomicAdd(p, (unsigned long long)__double2ll_rn(y));
}

// per-ray partial integrals of a point (the FP64 form: summed over rays in ray
// order afterwards): store on the first frequency pass, add on later ones
template <typename Real, int NS>
__device__ __forceinline__ void store_partial(const SweepArgs<Real> &a, int m, long long v, int g, const Real *acc)
{
    if constexpr (NS == 1) {
        R2<Real> *pp = reinterpret_cast<R2<Real> *>(a.part) + (long long)m * a.nvox + v;
        R2<Real> o = {acc[0], acc[1]};
        if (g > 0) { R2<Real> old = *pp; o.x += old.x; o.y += old.y; }
        *pp = o;
    } else {
        R4<Real> *pp = reinterpret_cast<R4<Real> *>(a.part) + (long long)m * a.nvox + v;
        R4<Real> o = {acc[0], acc[1], acc[2], acc[3]};
        if (g > 0) { R4<Real> old = *pp; o.x += old.x; o.y += old.y; o.z += old.z; o.w += old.w; }
        *pp = o;
    }
}

}  // namespace

template <typename Real, int NS>
int jsweep_smem_bytes(int nodes, int ipts, int F, int threads)
{
    using W = JW<Real, NS>;
    (void)threads;
    const int ring = (3 * nodes * W::s_words * (int)sizeof(Real) + 15) / 16 * 16;
    const int coef = (3 * F * jsweep_stride(nodes * W::cw, (int)sizeof(Real)) * (int)sizeof(Real) + 15) / 16 * 16;
    const int stokes = 2 * F * jsweep_stride(ipts * NS, (int)sizeof(Real)) * (int)sizeof(Real);
    const int stage = W::g_words * nodes * (int)sizeof(Real);
    const int freq = 2 * F * (int)sizeof(Real);
    return ring + coef + stokes + stage + freq;
}

// Pairs of Reals: the Stokes vector of the polarized atom is handled as the pairs
// (I, Q) and (U, V), whose arithmetic shares every coefficient. In FP32 a pair
// op is one packed instruction (FFMA2, FMUL2, FADD2: each lane rounds exactly
// as the scalar op); in FP64 it is two scalar ops.
template <typename Real> struct PairT;
template <> struct PairT<float> { using T = float2; };
template <> struct PairT<double> { using T = double2; };

__device__ __forceinline__ float2 pmk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 pmk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 psub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// BESSER control points (Sec. 3.2, steps 1-9) of two Stokes parameters at once;
// the same steps and selections as control_point (device_math.cuh)
template <typename P2, typename Real>
__device__ __forceinline__ P2 control_point2(P2 yM, P2 yO, P2 yP, const BesserGeom<Real> &g)
{
    const P2 dm = psub(yO, yM), dp = psub(yP, yO);                      // step 1
    const P2 yp = pfma(pmk(g.a, g.a), dp, pmul(pmk(g.b, g.b), dm));     // step 3 (Eq. 6)
    const P2 w = pmul(pmk(g.hm2, g.hm2), yp);                            // step 4: c_M = y_O - w
    P2 u = pmul(pmk(g.hp2, g.hp2), yp);                                  //         c_P = y_O + u
    const P2 tc = pmul(u, psub(u, dp));                                  // step 7: c_P outside [y_O, y_P]
    u.x = tc.x > Real(0) ? dp.x : u.x;
    u.y = tc.y > Real(0) ? dp.y : u.y;
    const P2 c9 = pfma(pmk(-g.r, -g.r), u, yO);                          // steps 8-9
    const P2 to = pmul(psub(dm, w), w);                                  // steps 5-6: c_M outside [y_M, y_O]
    const P2 te = pmul(dm, dp);                                          // step 2: extremum at O
    P2 r;
    r.x = te.x <= Real(0) ? yO.x : (to.x < Real(0) ? yM.x : c9.x);
    r.y = te.y <= Real(0) ? yO.y : (to.y < Real(0) ? yM.y : c9.y);
    return r;
}

template <typename Real, int NS, bool PROBE>
__device__ __forceinline__ void jsweep_item(const SweepArgs<Real> &a, cg::cluster_group &cluster, Real *ring,
                                            Real *coef, Real *ibuf, Real *scratch, Real *sray, Real *sfreq,
                                            int box, int m, int g, int rank, int C)
{
    using V = typename V16<Real>::T;
    using P2 = typename PairT<Real>::T;
    using W = JW<Real, NS>;
    constexpr int NA = W::na;
    constexpr int CW = W::cw;
    const BoxDev B = a.boxes[box];
    const int nx = B.nx, ny = B.ny, nz = B.nz, F = a.F;
    const int row0 = (int)(((long long)rank * ny) / C);
    const int R = (int)(((long long)(rank + 1) * ny) / C) - row0;
    const int next_row = (row0 + R) % ny;
    const int next_owner = (int)(((long long)(next_row + 1) * C + ny - 1) / ny) - 1;
    const Real *ibuf_next = cluster.map_shared_rank(ibuf, next_owner);
    const int j0 = g * F;
    const int nf = min(F, a.nnu - j0);
    const PlaneGeom<Real> *G = a.geom + B.geom0 + (long long)m * nz;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nodes = a.ring_plane;                  // node capacity of a ring slot
    const int nn = (R + 2) * nx;                     // nodes of this strip's slot
    const int iplane = a.istride;                    // Reals per (buf, f) Stokes plane
    const int cplane = a.cstride;                    // Reals per (slot, f) coefficient plane
    const int ipts = a.ipts_max;
    const int npts = R * nx;
    // voxel indices fit in 32 bits (porta_create limits nvox to 2^31)
    const int nvox = (int)a.nvox, vox0 = (int)B.vox0;
    const Real *__restrict__ chi = a.chi, *__restrict__ vel = a.vel, *__restrict__ rho = a.rho;
    const Real *__restrict__ invn = a.invn + (long long)m * a.nvox;

    // the ray's constants and this pass's frequency nodes and weights, staged in
    // shared memory (the previous item ended at a cluster barrier: no reader is left)
    if (tid < 24) {
        const Real *rp = reinterpret_cast<const Real *>(a.rays + m);
        sray[tid] = rp[tid];                         // mu, ox, oy, oz, T[18], w, pad
    }
    for (int f = tid; f < nf; f += nt) {
        sfreq[f] = a.xf[j0 + f];
        sfreq[F + f] = a.wf[j0 + f];
    }
    __syncthreads();
    const Real mu = sray[0];
    const bool upward = mu > Real(0);

    // Frequency lanes: when the strip has fewer points than threads, L = 2 or 4
    // adjacent threads share a point and take frequencies lane, lane + L, ...;
    // their sums meet by warp shuffles in a fixed order.
    const int lmax = npts > 0 ? min(nf, nt / npts) : 1;
    const int L = lmax >= 4 ? 4 : (lmax >= 2 ? 2 : 1);
    const int lane = tid & (L - 1);
    const int pfirst = tid / L;
    const int pstep = nt / L;
    const int dl = nt / nx, dc = nt - dl * nx;
    const int pl_ = pstep / nx, pc_ = pstep - pl_ * nx;

    V *const ringv = reinterpret_cast<V *>(ring);
    Real *const stage = scratch;

    // Stage plane q into ring slot q % 3: source vectors, then per-frequency (eta_I, eta_V).
    auto fill = [&](int q) {
        const PlaneGeom<Real> gq = G[q];
        const int s = q % 3;
        const int kbase = gq.kz * ny;
        Real T[18], ox = 0, oy = 0, oz = 0;
        if constexpr (NS == 4) {
#pragma unroll
            for (int i = 0; i < 18; ++i) T[i] = sray[4 + i];
            ox = sray[1]; oy = sray[2]; oz = sray[3];
        }
        int lr = tid / nx, c = tid - (tid / nx) * nx;
        for (int idx = tid; idx < nn; idx += nt) {
            int pi = c + gq.ax;
            pi -= pi >= nx ? nx : 0;
            int pj = row0 + lr - 1 + gq.ay;
            pj += pj < 0 ? ny : 0;
            pj -= pj >= ny ? ny : 0;
            pj -= pj >= ny ? ny : 0;
            const int v = vox0 + (kbase + pj) * nx + pi;
            stage[idx] = chi[v];
            stage[nodes + idx] = vel[v] * mu;
            if constexpr (NS == 1) {
                ring[s * nodes + idx] = rho[v];
            } else {
                const Real s00 = rho[v], s20 = rho[nvox + v], s21r = rho[2 * nvox + v], s21i = rho[3 * nvox + v];
                const Real s22r = rho[4 * nvox + v], s22i = rho[5 * nvox + v];
                Real w[4];
                // S_i(Omega) = sum_KQ (-1)^Q T^K_Q(i, Omega) S^K_-Q (Eq. 1 tensors, two-level emissivity)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const Real *t = T + 6 * i;
                    w[i] = t[0] * s00 + t[1] * s20 + Real(2) * (t[2] * s21r + t[3] * s21i) +
                           Real(2) * (t[4] * s22r + t[5] * s22i);
                }
                w[3] = s00;
#pragma unroll
                for (int h = 0; h < W::s_chunks; ++h) chunk_put<Real>(ringv + (s * W::s_chunks + h) * nodes + idx, w + h * W::per);
                stage[2 * nodes + idx] = a.bfac * (a.bx[v] * ox + a.by[v] * oy + a.bz[v] * oz);
            }
            c += dc;
            lr += dl;
            if (c >= nx) { c -= nx; ++lr; }
        }
        __syncthreads();
        // per node its coefficients at every frequency of the pass (a warp writes
        // consecutive nodes); when the slot has fewer nodes than threads, the
        // frequencies are split between nt / nn thread groups
        const int ngrp = max(1, min(nf, nt / nn));
        const int grp = tid / nn;
        for (int idx = tid - grp * nn; grp < ngrp && idx < nn; idx += nt) {
            const Real chi_n = stage[idx], s_n = stage[nodes + idx];
            Real b_n = 0;
            if constexpr (NS == 4) b_n = stage[2 * nodes + idx];
            Real *cp = coef + (s * F + grp) * cplane + idx * CW;
            for (int f = grp; f < nf; f += ngrp, cp += ngrp * cplane) {
                const Real xs = sfreq[f] - s_n;
                const Real eta = chi_n * profile_shape(xs);
                if constexpr (NS == 1) {
                    cp[0] = eta;
                } else {
                    R2<Real> e2 = {eta, b_n * xs * eta};
                    *reinterpret_cast<R2<Real> *>(cp) = e2;
                }
            }
        }
    };

    // the fixed-point terms of a point's frequency-integrated Stokes parameters and
    // Lambda* for this pass: J^K_Q += w_m sum_p T^K_Q(p, m) I_p, Lambda-bar* += w_m L
    // (the ray's weight and tensors in the sweep's precision; FP32 terms convert
    // to fixed point without rounding). The L frequency lanes of a point hold the
    // same totals and share the terms: lane k adds the components c = k mod L.
    auto add_terms = [&](int v, const Real *tot) {
        const Real scale = pow2(Real(0), a.jexp[v]);
        const Real w = sray[22];
        unsigned long long *acc = a.jacc + v;
        if constexpr (NS == 1) {
            if (lane == 0) jadd(acc, w * tot[0] * scale, a.jerr);
            if (lane == (L > 1 ? 1 : 0)) jadd(acc + nvox, w * tot[1] * scale, a.jerr);
        } else {
            const Real pI = w * tot[0] * scale, pQ = w * tot[1] * scale, pU = w * tot[2] * scale;
            for (int k = lane; k < 6; k += L)
                jadd(acc + (size_t)k * nvox, sray[4 + k] * pI + sray[10 + k] * pQ + sray[16 + k] * pU, a.jerr);
            if (lane == 6 % L) jadd(acc + (size_t)6 * nvox, w * tot[3] * scale, a.jerr);
        }
    };

    fill(0);
    __syncthreads();
    if (nz > 1) fill(1);
    __syncthreads();
    for (int q = 0; q < nz; ++q) {
        const PlaneGeom<Real> gq = G[q];
        const bool has_p = q + 1 < nz;
        const PlaneGeom<Real> gp = has_p ? G[q + 1] : gq;
        const int sM = (q + 2) % 3, sO = q % 3, sP = (q + 1) % 3;
        Real *iw = ibuf + (q & 1) * F * iplane;
        const int ro = ((q + 1) & 1) * F * iplane;
        const Real *ir = ibuf + ro;
        const Real *irn = ibuf_next + ro;
        const Real mx1 = gq.tx, mx0 = Real(1) - gq.tx, my1 = gq.ty, my0 = Real(1) - gq.ty;
        const Real px0 = gp.tx, px1 = Real(1) - gp.tx, py0 = gp.ty, py1 = Real(1) - gp.ty;
        const Real dsM = Real(0.5) * gq.ds, dsP = has_p ? Real(0.5) * gp.ds : Real(0);
        const Real wM[4] = {mx0 * my0, mx1 * my0, mx0 * my1, mx1 * my1};
        const Real wP[4] = {px0 * py0, px1 * py0, px0 * py1, px1 * py1};
        // the weights as pairs (both lanes equal), for the pair arithmetic
        P2 wM2[4], wP2[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            wM2[k] = pmk(wM[k], wM[k]);
            wP2[k] = pmk(wP[k], wP[k]);
        }
        const Real *cMb = coef + sM * F * cplane, *cPb = coef + sP * F * cplane;
        const V *rMb = ringv + sM * W::s_chunks * nodes, *rOb = ringv + sO * W::s_chunks * nodes;
        const V *rPb = ringv + sP * W::s_chunks * nodes;

        Real acc[NA], accp[NA];
        bool pend = false, row0_written = false;
        int vpend = 0;
        int l = pfirst / nx, c = pfirst - (pfirst / nx) * nx;
        // every warp takes the same number of point rounds (the lane shuffles below)
        for (int pb = 0; pb < npts; pb += pstep) {
            const int p = pb + pfirst;
            if (pb > 0) {
                c += pc_;
                l += pl_;
                if (c >= nx) { c -= nx; ++l; }
            }
            const bool active = p < npts;
            row0_written |= active && l == 0;
#pragma unroll
            for (int s = 0; s < NA; ++s) acc[s] = Real(0);
            int v = 0;
            if (active) {
                int pi = c + gq.ax;
                pi -= pi >= nx ? nx : 0;
                int pj = row0 + l + gq.ay;
                pj -= pj >= ny ? ny : 0;
                pj -= pj >= ny ? ny : 0;
                v = vox0 + (gq.kz * ny + pj) * nx + pi;
                // the point's own data: source vector from the ring, the rest from global memory
                const int io = (l + 1) * nx + c;
                Real SO[NS];
                if constexpr (NS == 1) {
                    SO[0] = ring[sO * nodes + io];
                } else {
#pragma unroll
                    for (int h = 0; h < W::s_chunks; ++h) chunk_get<Real>(rOb + h * nodes + io, SO + h * W::per);
                }
                const Real chiO = chi[v], sO_ = vel[v] * mu, invnO = invn[v];
                Real bO = 0;
                if constexpr (NS == 4) bO = a.bfac * (a.bx[v] * sray[1] + a.by[v] * sray[2] + a.bz[v] * sray[3]);

                if (q == 0) {
                    // boundary plane: I = (B, 0, 0, 0) entering at the bottom, 0 at the top; Lambda* = 0
                    Real I0[NS];
#pragma unroll
                    for (int s = 0; s < NS; ++s) I0[s] = Real(0);
                    if (upward) I0[0] = a.bpl[v];
                    for (int f = lane; f < nf; f += L) {
                        StokesIO<Real, NS>::store(iw + f * iplane, ipts, l * nx + c, I0);
                        const Real wt = sfreq[F + f] * profile_shape(sfreq[f] - sO_) * invnO;
                        acc[0] += wt * I0[0];
                        if (PROBE && a.probe_ray == m) {
                            const int j = j0 + f;
#pragma unroll
                            for (int s = 0; s < NS; ++s) a.probe[((long long)j * a.nvox + v) * NS + s] = I0[s];
                            a.probe_ls[(long long)j * a.nvox + v] = Real(0);
                        }
                    }
                } else {
                    const int c1 = (c + 1 == nx) ? 0 : c + 1;
                    const int cm = (c == 0) ? nx - 1 : c - 1;
                    const int rM[4] = {(l + 1) * nx + c, (l + 1) * nx + c1, (l + 2) * nx + c, (l + 2) * nx + c1};
                    const int rP[4] = {l * nx + cm, l * nx + c, (l + 1) * nx + cm, (l + 1) * nx + c};
                    // upwind corners' source vectors times their bilinear weights, held
                    // across the frequency loop (the downwind corners' sources are read
                    // again for each frequency: holding both spills at the register cap)
                    Real SMk[4][W::s_words];
                    P2 A01[4], A23[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if constexpr (NS == 1) {
                            SMk[k][0] = wM[k] * ring[sM * nodes + rM[k]];
                        } else {
#pragma unroll
                            for (int h = 0; h < W::s_chunks; ++h) chunk_get<Real>(rMb + h * nodes + rM[k], SMk[k] + h * W::per);
                            A01[k] = pmul(wM2[k], pmk(SMk[k][0], SMk[k][1]));
                            A23[k] = pmul(wM2[k], pmk(SMk[k][2], SMk[k][3]));
                        }
                    }
                    const bool last_row = (l + 1 == R);
                    const int ilo = l * nx;
                    const Real *ihi_base = last_row ? irn : ir;
                    const int ihi = last_row ? 0 : (l + 1) * nx;

                    for (int f = lane; f < nf; f += L) {
                        const Real x = sfreq[f];
                        const Real *pl = ir + f * iplane;
                        const Real *ph = ihi_base + f * iplane;
                        const Real *cM = cMb + f * cplane;
                        const Real *cP = cPb + f * cplane;
                        // the point O: its own profile (optical paths, Lambda*, integration weight)
                        const Real xsO = x - sO_;
                        const Real phO = profile_shape(xsO);
                        const Real etaO = chiO * phO;
                        if constexpr (NS == 1) {
                            // a3: upwind intensity and transfer coefficients at M and P (bilinear)
                            const Real IM = wM[0] * pl[ilo + c] + wM[1] * pl[ilo + c1] + wM[2] * ph[ihi + c] +
                                            wM[3] * ph[ihi + c1];
                            Real etaM = 0, epsM = 0, etaP = 0, epsP = 0;
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const Real ek = cM[rM[k]];
                                etaM += wM[k] * ek;
                                epsM += SMk[k][0] * ek;           // (w S)_k eta_k
                            }
                            if (has_p) {
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    const Real we = wP[k] * cP[rP[k]];
                                    etaP += we;
                                    epsP += we * ring[sP * nodes + rP[k]];
                                }
                            }
                            const Real SM = epsM * rcp(etaM), SOs = SO[0];
                            const Real tMO = (etaM + etaO) * dsM;
                            const Coef<Real> co = coefficients(tMO);
                            Real cMs, SP = 0;
                            if (has_p) {
                                SP = epsP * rcp(etaP);
                                const Real tOP = (etaO + etaP) * dsP;
                                cMs = control_point(SM, SOs, SP, besser_geom(tMO, tOP));
                            } else {
                                cMs = Real(0.5) * (SM + SOs);
                            }
                            const Real IO = co.e * IM + co.wm * SM + co.wo * SOs + co.wc * cMs;
                            iw[f * iplane + l * nx + c] = IO;
                            const Real ls = co.wo + (has_p ? co.wc : Real(0.5) * co.wc);
                            const Real wt = sfreq[F + f] * phO * invnO;
                            acc[0] += wt * IO;
                            acc[1] += wt * ls;
                            if (PROBE && a.probe_ray == m) {
                                const int j = j0 + f;
                                a.probe[(long long)j * a.nvox + v] = IO;
                                a.probe_ls[(long long)j * a.nvox + v] = ls;
                            }
                        } else {
                            // a3: upwind Stokes vector (bilinear), as the pairs (I, Q), (U, V)
                            P2 IM01, IM23;
                            {
                                Real t[4][4];
                                StokesIO<Real, 4>::load(pl, ipts, ilo + c, t[0]);
                                StokesIO<Real, 4>::load(pl, ipts, ilo + c1, t[1]);
                                // the row after the strip's last is the next CTA's row 0 (DSMEM, a
                                // generic load); the others are local (shared-memory loads)
                                if (last_row) {
                                    StokesIO<Real, 4>::load(ph, ipts, c, t[2]);
                                    StokesIO<Real, 4>::load(ph, ipts, c1, t[3]);
                                } else {
                                    StokesIO<Real, 4>::load(pl, ipts, ilo + nx + c, t[2]);
                                    StokesIO<Real, 4>::load(pl, ipts, ilo + nx + c1, t[3]);
                                }
                                IM01 = pmul(wM2[0], pmk(t[0][0], t[0][1]));
                                IM23 = pmul(wM2[0], pmk(t[0][2], t[0][3]));
#pragma unroll
                                for (int k = 1; k < 4; ++k) {
                                    IM01 = pfma(wM2[k], pmk(t[k][0], t[k][1]), IM01);
                                    IM23 = pfma(wM2[k], pmk(t[k][2], t[k][3]), IM23);
                                }
                            }
                            // a2-a3: transfer coefficients at M and P from the corners' (eta_I, eta_V):
                            // (eta, eta_V) += w (eta_k, eta_V,k); (eps_I, eps_Q) += eta_k w (S_I, S_Q)_k;
                            // (eps_U, eps_V) += (eta_k, eta_V,k) w (S_U, S^0_0)_k
                            P2 eM = pmk(Real(0), Real(0)), eM01 = eM, eM23 = eM;
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const P2 e2 = reinterpret_cast<const P2 *>(cM)[rM[k]];
                                eM = pfma(wM2[k], e2, eM);
                                eM01 = pfma(A01[k], pmk(e2.x, e2.x), eM01);
                                eM23 = pfma(A23[k], e2, eM23);
                            }
                            P2 eP = pmk(Real(0), Real(0)), eP01 = eP, eP23 = eP;
                            if (has_p) {
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    Real sp[4];
#pragma unroll
                                    for (int h = 0; h < W::s_chunks; ++h) chunk_get<Real>(rPb + h * nodes + rP[k], sp + h * W::per);
                                    const P2 e2 = reinterpret_cast<const P2 *>(cP)[rP[k]];
                                    const P2 wk = pmul(wP2[k], e2);
                                    eP = padd(eP, wk);
                                    eP01 = pfma(pmk(wk.x, wk.x), pmk(sp[0], sp[1]), eP01);
                                    eP23 = pfma(wk, pmk(sp[2], sp[3]), eP23);
                                }
                            }
                            const Real kvO = bO * xsO;
                            const P2 SO01 = pmk(SO[0], SO[1]), SO23 = pmk(SO[2], kvO * SO[3]);
                            const Real iM = rcp(eM.x);
                            const P2 SM01 = pmul(eM01, pmk(iM, iM)), SM23 = pmul(eM23, pmk(iM, iM));
                            // a4: optical paths (trapezoid along MO and OP)
                            const Real tMO = (eM.x + etaO) * dsM;
                            // a6: exponential-integral coefficients (Eqs. 9-13)
                            const Coef<Real> co = coefficients(tMO);
                            // a5: BESSER control points per Stokes parameter
                            P2 cM01, cM23;
                            if (has_p) {
                                const Real iP = rcp(eP.x);
                                const P2 SP01 = pmul(eP01, pmk(iP, iP)), SP23 = pmul(eP23, pmk(iP, iP));
                                const Real tOP = (etaO + eP.x) * dsP;
                                const BesserGeom<Real> bg = besser_geom(tMO, tOP);
                                cM01 = control_point2(SM01, SO01, SP01, bg);
                                cM23 = control_point2(SM23, SO23, SP23, bg);
                            } else {
                                cM01 = pmul(pmk(Real(0.5), Real(0.5)), padd(SM01, SO01));
                                cM23 = pmul(pmk(Real(0.5), Real(0.5)), padd(SM23, SO23));
                            }
                            // a7: BESSER-DELO step (Eq. 7); kappa^-1 = 1 + psi'_O K'_O (Eq. 8)
                            // couples I and V only
                            P2 r01 = pmul(pmk(co.e, co.e), IM01), r23 = pmul(pmk(co.e, co.e), IM23);
                            r01 = pfma(pmk(co.wm, co.wm), SM01, r01);
                            r23 = pfma(pmk(co.wm, co.wm), SM23, r23);
                            r01 = pfma(pmk(co.wo, co.wo), SO01, r01);
                            r23 = pfma(pmk(co.wo, co.wo), SO23, r23);
                            r01 = pfma(pmk(co.wc, co.wc), cM01, r01);
                            r23 = pfma(pmk(co.wc, co.wc), cM23, r23);
                            const Real kvM = eM.y * iM;
                            const Real pk = co.pm * kvM;
                            const Real rI = r01.x - pk * IM23.y, rV = r23.y - pk * IM01.x;
                            const Real av = co.po * kvO;
                            const Real idet = rcp(Real(1) - av * av);
                            Real IO[4];
                            IO[0] = (rI - av * rV) * idet;
                            IO[3] = (rV - av * rI) * idet;
                            IO[1] = r01.y;
                            IO[2] = r23.x;
                            StokesIO<Real, 4>::store(iw + f * iplane, ipts, l * nx + c, IO);
                            // a8: Lambda* (Eq. 14; w_O + w_C/2 on the last plane) and accumulation
                            const Real ls = co.wo + (has_p ? co.wc : Real(0.5) * co.wc);
                            const Real wt = sfreq[F + f] * phO * invnO;
                            const P2 a01 = pfma(pmk(wt, wt), pmk(IO[0], IO[1]), pmk(acc[0], acc[1]));
                            const P2 a23 = pfma(pmk(wt, wt), pmk(IO[2], ls), pmk(acc[2], acc[3]));
                            acc[0] = a01.x; acc[1] = a01.y; acc[2] = a23.x; acc[3] = a23.y;
                            if (PROBE && a.probe_ray == m) {
                                const int j = j0 + f;
#pragma unroll
                                for (int s = 0; s < 4; ++s) a.probe[((long long)j * a.nvox + v) * 4 + s] = IO[s];
                                a.probe_ls[(long long)j * a.nvox + v] = ls;
                            }
                        }
                    }
                }
            }   // active
            // fixed-order sum over the frequency lanes of each point (adjacent threads;
            // every lane ends with the same totals, the additions being commutative)
            for (int o = 1; o < L; o <<= 1) {
#pragma unroll
                for (int s = 0; s < NA; ++s) acc[s] += __shfl_xor_sync(0xffffffffu, acc[s], o);
            }
            if (active && (a.jacc || lane == 0)) {
                if (pb + pstep < npts) {
                    if (a.jacc) add_terms(v, acc);
                    else store_partial<Real, NS>(a, m, v, g, acc);
                } else {
                    pend = true;
                    vpend = v;
#pragma unroll
                    for (int s = 0; s < NA; ++s) accp[s] = acc[s];
                }
            }
        }
        // plane q done here: arrive (release), stage plane q+2, wait (acquire). The
        // last point round's sums go to global memory after the arrive, so that its
        // release does not wait for them (nothing in the sweep reads them).
        __syncthreads();
        // release by the warps that wrote row 0 (the only Stokes vectors another CTA
        // reads, through DSMEM); the others' plane data are read in this CTA only
        if (__any_sync(0xffffffffu, row0_written)) cluster_arrive_release();
        else cluster_arrive_relaxed();
        if (pend) {
            if (a.jacc) add_terms(vpend, accp);
            else store_partial<Real, NS>(a, m, vpend, g, accp);
        }
        if (q + 2 < nz) fill(q + 2);
        __syncthreads();
        cluster_wait_acquire();
    }
}

template <typename Real, int NS, bool PROBE>
__global__ void __launch_bounds__(512, 1) jsweep_kernel(const SweepArgs<Real> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Real sray[24];
    using W = JW<Real, NS>;
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int cid = blockIdx.x / C;
    const int ncl = gridDim.x / C;
    Real *ring = reinterpret_cast<Real *>(smem_raw);
    const int ring_bytes = (3 * a.ring_plane * W::s_words * (int)sizeof(Real) + 15) / 16 * 16;
    Real *coef = reinterpret_cast<Real *>(smem_raw + ring_bytes);
    const int coef_bytes = (3 * a.F * a.cstride * (int)sizeof(Real) + 15) / 16 * 16;
    Real *ibuf = reinterpret_cast<Real *>(smem_raw + ring_bytes + coef_bytes);
    Real *scratch = ibuf + 2 * a.F * a.istride;
    Real *sfreq = scratch + W::g_words * a.ring_plane;
    cluster.sync();
    if (a.next_item) {
        __shared__ int s_item[2];
        for (int k = 0;; ++k) {
            if (rank == 0 && threadIdx.x == 0) {
                const int it = atomicAdd(a.next_item, 1);
                for (int r = 0; r < C; ++r) *cluster.map_shared_rank(s_item + (k & 1), r) = it;
            }
            cluster.sync();
            const int item = s_item[k & 1];
            if (item >= a.nitems) break;
            const int code = a.items ? a.items[item] : item;
            const int box = code / a.nray, m = code - box * a.nray;
            for (int g = 0; g < a.ngroups; ++g)
                jsweep_item<Real, NS, PROBE>(a, cluster, ring, coef, ibuf, scratch, sray, sfreq, box, m, g, rank, C);
        }
        return;
    }
    for (int item = cid; item < a.nitems; item += ncl) {
        const int code = a.items ? a.items[item] : item;
        const int box = code / a.nray, m = code - box * a.nray;
        for (int g = 0; g < a.ngroups; ++g)
            jsweep_item<Real, NS, PROBE>(a, cluster, ring, coef, ibuf, scratch, sray, sfreq, box, m, g, rank, C);
    }
}

// Fixed-point scale of each voxel: 2^e with e = 46 - ilogb(max(|S^0_0|, |B|)),
// so that a term of the size of the voxel's source function or Planck function
// carries 46 fraction bits and the accumulator has 2^16 of headroom above it
// (an FP32 term then converts without rounding; an FP64 term rounds at 2^-47 of
// the reference value).
template <typename Real, int NS>
__global__ void jacc_prepare_kernel(long long nvox, const Real *rho, const Real *bpl, int *jexp,
                                    unsigned long long *jacc)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const double ref = fmax(fmax(fabs((double)rho[v]), fabs((double)bpl[v])), 1e-30);
    // kept within the FP32 exponent range, where the sweep forms 2^e exactly
    jexp[v] = min(max(kJFrac - ilogb(ref), -100), 126);
#pragma unroll
    for (int k = 0; k < JW<Real, NS>::nacc; ++k) jacc[k * nvox + v] = 0ULL;
}

template <int NS>
__global__ void jacc_finalize_kernel(long long nvox, const unsigned long long *jacc, const int *jexp, double *jkq,
                                     double *lstar)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const double inv = ldexp(1.0, -jexp[v]);
    constexpr int NJ = NS == 1 ? 1 : 6;
#pragma unroll
    for (int k = 0; k < NJ; ++k) jkq[v * NJ + k] = (double)(long long)jacc[k * nvox + v] * inv;
    lstar[v] = (double)(long long)jacc[NJ * nvox + v] * inv;
}

template <typename Real, int NS>
cudaError_t launch_jacc_prepare(const SweepArgs<Real> &a, cudaStream_t st)
{
    const int bs = 256;
    const long long nb = (a.nvox + bs - 1) / bs;
    jacc_prepare_kernel<Real, NS><<<(unsigned)nb, bs, 0, st>>>(a.nvox, a.rho, a.bpl, const_cast<int *>(a.jexp), a.jacc);
    return cudaGetLastError();
}

template <int NS>
cudaError_t launch_jacc_finalize(long long nvox, const unsigned long long *jacc, const int *jexp, double *jkq,
                                 double *lstar, cudaStream_t st)
{
    const int bs = 256;
    const long long nb = (nvox + bs - 1) / bs;
    jacc_finalize_kernel<NS><<<(unsigned)nb, bs, 0, st>>>(nvox, jacc, jexp, jkq, lstar);
    return cudaGetLastError();
}

template <typename Real, int NS, bool PROBE>
static cudaError_t jprepare(int cluster, int smem)
{
    void *k = (void *)jsweep_kernel<Real, NS, PROBE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (cluster > 8) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <typename Real, int NS>
cudaError_t jsweep_max_active_clusters(int cluster, int smem, int threads, int *out)
{
    cudaError_t e = jprepare<Real, NS, false>(cluster, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cluster);
    lc.blockDim = dim3(threads);
    lc.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(out, jsweep_kernel<Real, NS, false>, &lc);
}

// the probe variant writes one ray's Stokes vectors and Lambda* at every node and
// frequency (porta_probe_ray); the plain one keeps no trace of that in its loop
template <typename Real, int NS>
cudaError_t launch_jsweep(const SweepArgs<Real> &a, LaunchCfg &cfg, cudaStream_t st)
{
    const bool probe = a.probe_ray >= 0;
    cudaError_t e = probe ? jprepare<Real, NS, true>(cfg.cluster, cfg.smem) : jprepare<Real, NS, false>(cfg.cluster, cfg.smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cfg.clusters * cfg.cluster);
    lc.blockDim = dim3(cfg.threads);
    lc.dynamicSmemBytes = cfg.smem;
    lc.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cfg.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    if (cfg.priority != 0) {
        at[1].id = cudaLaunchAttributePriority;
        at[1].val.priority = cfg.priority;
        lc.numAttrs = 2;
    }
    if (probe) return cudaLaunchKernelEx(&lc, jsweep_kernel<Real, NS, true>, a);
    return cudaLaunchKernelEx(&lc, jsweep_kernel<Real, NS, false>, a);
}

#define PORTA_JINST(R, N)                                                                    \
    template int jsweep_smem_bytes<R, N>(int, int, int, int);                                \
    template cudaError_t jsweep_max_active_clusters<R, N>(int, int, int, int *);             \
    template cudaError_t launch_jsweep<R, N>(const SweepArgs<R> &, LaunchCfg &, cudaStream_t);          \
    template cudaError_t launch_jacc_prepare<R, N>(const SweepArgs<R> &, cudaStream_t);
PORTA_JINST(float, 1)
PORTA_JINST(float, 4)
PORTA_JINST(double, 1)
PORTA_JINST(double, 4)
#undef PORTA_JINST
template cudaError_t launch_jacc_finalize<1>(long long, const unsigned long long *, const int *, double *, double *,
                                             cudaStream_t);
template cudaError_t launch_jacc_finalize<4>(long long, const unsigned long long *, const int *, double *, double *,
                                             cudaStream_t);

}  // namespace porta
