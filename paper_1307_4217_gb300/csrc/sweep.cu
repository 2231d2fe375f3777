// Short-characteristics BESSER formal solution on sm_103a (Sec. 3 of Stepan &
// Trujillo Bueno 2013), fused with the frequency integration of the Stokes
// parameters and Lambda* that feeds J^K_Q (Eq. 1) and the Jacobi update.
//
// Decomposition. One thread-block cluster owns one ray direction at a time
// (persistent loop over rays) and sweeps the planes of the grid in topological
// order. The plane is split into contiguous strips of sheared rows, one strip
// per CTA of the cluster. Because the grid is uniform and periodic
// horizontally, the upwind/downwind interpolation stencil of every point of a
// plane has the same fractional weights; working in a frame sheared along the
// characteristics (see PlaneGeom) turns the bilinear stencils into fixed
// nearest-neighbour accesses, however far a grazing ray travels horizontally
// between planes. The only cross-CTA data is the first sheared row of the next
// strip, read from that CTA's shared memory (DSMEM) after a cluster barrier.
//
// Shared memory per CTA (planes of 16-byte chunks, [chunk][row][col], so that
// neighbouring threads read neighbouring 16-byte words):
//   ring[3][NW/chunk][rows+2][nx]  frequency-independent node data of planes
//                             q-1, q, q+1 (own rows plus one halo row on each
//                             side, recomputed locally from global memory);
//   ibuf[2][F][NS/chunk][rows][nx] Stokes vectors of planes q-1 and q for F
//                             frequencies.
// Each thread owns points of its strip and loops over the F frequencies of the
// pass, reading the data of its 8 stencil corners from the node ring for each
// frequency, and accumulates the
// frequency-integrated Stokes I, Q, U and Lambda* of its point in registers;
// one store (or read-modify-write for later frequency passes) per point and
// plane writes the per-ray partial integrals.
#include <cooperative_groups.h>

#include "device_math.cuh"
#include "porta_internal.cuh"
#include "sweep_common.cuh"

namespace cg = cooperative_groups;

namespace porta {

template <typename Real, int NS>
int sweep_smem_bytes(int ring_plane, int ipts_max, int F, int threads, int na)
{
    return 3 * ring_plane * 16 + (2 * F * ipts_max * NS + threads * na) * (int)sizeof(Real);
}


// per-ray partial integrals of a point: store on the first frequency pass,
// read-modify-write on later passes; PV: also the integral of Stokes V (acc[4])
template <typename Real, int NS, bool PV = false>
__device__ __forceinline__ void accumulate_partial(const SweepArgs<Real> &a, int m, long long v, int g, const Real *acc)
{
    if constexpr (PV) {
        Real *pv = a.partv + (long long)m * a.nvox + v;
        *pv = g > 0 ? *pv + acc[4] : acc[4];
    }
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

// Lagrange weights at offset f of the quadratic through nodes -1, 0, 1
template <typename Real>
__device__ __forceinline__ void quad3(Real f, Real w[3])
{
    w[0] = Real(0.5) * f * (f - Real(1));
    w[1] = (Real(1) - f) * (Real(1) + f);
    w[2] = Real(0.5) * f * (f + Real(1));
}

// BQ: biquadratic (9-point) interpolation at M and P instead of bilinear (Sec. 3.1);
// the ring then keeps two halo rows on each side of the strip
// GK: an explicit medium (a general propagation matrix, per voxel K'/eta_I and S
// independent of direction and frequency; emergent mode, NS = 4, bilinear)
template <typename Real, int NS, int MODE, bool DI, bool BQ, bool GK>
__device__ __forceinline__ void sweep_item(const SweepArgs<Real> &a, cg::cluster_group &cluster,
                                           typename V16<Real>::T *ring, Real *ibuf, Real *lane_buf, int box, int m,
                                           int g, int rank, int C, int dir_out)
{
    using V = typename V16<Real>::T;
    // accumulated quantities per point: (I, Lambda*), (I, Q, U, Lambda*), and for polarized
    // lines of the multilevel atom also V (for J^1_Q)
    constexpr int NA = NS == 1 ? 2 : (DI ? 5 : 4);
    const BoxDev B = a.boxes[box];
    const int nx = B.nx, ny = B.ny, nz = B.nz, F = a.F;
    const int rmax = (ny + C - 1) / C;
    const int row0 = (int)(((long long)rank * ny) / C);
    const int R = (int)(((long long)(rank + 1) * ny) / C) - row0;
    // The sheared row after this strip, (row0 + R) mod ny, is row 0 of the CTA
    // that owns it: the largest rank k with floor(k ny / C) <= row (CTAs own no
    // rows when ny < C).
    const int next_row = (row0 + R) % ny;
    const int next_owner = (int)(((long long)(next_row + 1) * C + ny - 1) / ny) - 1;
    const Real *ibuf_next = cluster.map_shared_rank(ibuf, next_owner);
    // the sheared row before this strip (biquadratic stencils reach it): the last row
    // of the CTA that owns it
    const int prev_row = (row0 + ny - 1) % ny;
    const int prev_owner = (int)(((long long)(prev_row + 1) * C + ny - 1) / ny) - 1;
    const int prev_local = prev_row - (int)(((long long)prev_owner * ny) / C);
    const Real *ibuf_prev = cluster.map_shared_rank(ibuf, prev_owner);
    static_assert(!(BQ && DI), "the biquadratic variant has no dichroism");
    static_assert(!GK || (NS == 4 && !DI && !BQ && MODE == MODE_EMERGENT), "explicit media: emergent, bilinear");
    constexpr int H = BQ ? 2 : 1;                   // halo rows of the ring on each side
    const int j0 = g * F;
    const int nf = min(F, a.nnu - j0);
    const PlaneGeom<Real> *G = a.geom + B.geom0 + (long long)m * nz;
    const RayDev<Real> ray = a.rays[m];
    const bool upward = ray.mu > Real(0);
    const long long nxy = (long long)nx * ny;
    const bool jmode = (MODE == MODE_JKQ);
    const int tid = threadIdx.x, nt = blockDim.x;
    constexpr int NCH = node_words<NS>() * (int)sizeof(Real) / 16;
    const int chunk = (rmax + 2 * H) * nx;          // ring chunk-plane stride (16-byte chunks)
    const int plane = NCH * chunk;                  // ring plane stride
    // dichroism and orientation (polarized lines of the multilevel atom): the node's
    // opacity, source terms and Zeeman factor are rescaled by eta_I / (chi phi) =
    // 1 + d_I(Omega); eta_Q / eta_I takes the node's profile-normalization word (the
    // normalization is then read from global memory at O); a second 3-slot ring after
    // the node ring (the launch reserves it) holds per node eta_U / eta_I, the
    // orientation emission term of S_V and the orientation term of eta_V / eta_I
    // (both independent of frequency): words 0, 1, 2 at stride dstride
    constexpr bool dich = NS == 4 && DI;
    Real *dring = reinterpret_cast<Real *>(ring + 3 * plane);
    const int dstride = (chunk * (int)sizeof(Real) + 15) / 16 * 16 / (int)sizeof(Real);
    const int ipts = rmax * nx;                     // points per Stokes plane
    const int ichunk = ipts;                        // Stokes chunk-plane stride (16-byte chunks)
    const int iplane = NS * ipts;                   // Reals per (buf, f) Stokes plane
    const int npts = R * nx;

    // Frequency lanes: when the strip has fewer points than threads, threads
    // tid = lane * npts + p share point p and take frequencies lane, lane + L, ...
    const int L = npts > 0 ? max(1, min(nf, nt / npts)) : 1;
    const int lane = L > 1 ? tid / npts : 0;
    const int pstart = L > 1 ? (lane < L ? tid - lane * npts : npts) : tid;
    const int pstep = L > 1 ? npts : nt;

    // thread -> (row, column) stepping without integer division in the loops
    const int dl = nt / nx, dc = nt - dl * nx;

    auto fill = [&](int q) {
        const PlaneGeom<Real> gq = G[q];
        const int nn = (R + 2 * H) * nx;
        const long long kbase = (long long)gq.kz * ny;
        int lr = tid / nx, c = tid - (tid / nx) * nx;      // lr = ring row (local row + 1)
        for (int idx = tid; idx < nn; idx += nt) {
            int pi = c + gq.ax;
            pi -= pi >= nx ? nx : 0;
            int pj = row0 + lr - H + gq.ay;                  // in [-H, 2 ny + H)
            if constexpr (BQ) {
                pj = ((pj % ny) + ny) % ny;
            } else {
                pj += pj < 0 ? ny : 0;
                pj -= pj >= ny ? ny : 0;
                pj -= pj >= ny ? ny : 0;
            }
            const long long v = B.vox0 + (kbase + pj) * nx + pi;
            Node<Real, NS> n = make_node<Real, NS>(a, ray, v, m, jmode);
            if constexpr (GK) {
                // the node's S (S_V in the S^0_0 word) and its K'/eta_I in the second ring
                const long long nv = a.nvox;
                n.SI = (Real)a.sexpl[v];
                n.SQ = (Real)a.sexpl[nv + v];
                n.SU = (Real)a.sexpl[2 * nv + v];
                n.S00 = (Real)a.sexpl[3 * nv + v];
                n.b = Real(0);
                Real *gk = dring + (q % 3) * 6 * dstride + idx;
#pragma unroll
                for (int k = 0; k < 6; ++k) gk[k * dstride] = (Real)a.kexpl[k * nv + v];
            }
            if constexpr (NS == 4) {
                if constexpr (dich) {
                    const long long nv = a.nvox;
                    const Real d20 = a.dich[v], d21r = a.dich[nv + v], d21i = a.dich[2 * nv + v];
                    const Real d22r = a.dich[3 * nv + v], d22i = a.dich[4 * nv + v];
                    Real dd[3];
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const Real *t = ray.t + 6 * i;
                        dd[i] = t[1] * d20 + Real(2) * (t[2] * d21r + t[3] * d21i) + Real(2) * (t[4] * d22r + t[5] * d22i);
                    }
                    // orientation: sum_Q (-1)^Q T^1_Q(V, Omega) X^1_-Q = T10 X10 + 2 (ReT11 ReX11 + ImT11 ImX11)
                    // with T^1_Q(V, Omega) = sqrt(3/2) Omega_Q: T10 = sqrt(3/2) Omega_z,
                    // T11 = -sqrt(3/4) (Omega_x + i Omega_y)
                    const Real t10 = Real(1.2247448713915890491) * ray.oz;
                    const Real t11r = Real(-0.86602540378443864676) * ray.ox, t11i = Real(-0.86602540378443864676) * ray.oy;
                    const Real dv = t10 * a.dich[5 * nv + v] + Real(2) * (t11r * a.dich[6 * nv + v] + t11i * a.dich[7 * nv + v]);
                    const Real sv = t10 * a.dich[8 * nv + v] + Real(2) * (t11r * a.dich[9 * nv + v] + t11i * a.dich[10 * nv + v]);
                    const Real f = Real(1) + dd[0], inv = Real(1) / f;
                    n.chi *= f;
                    n.SI *= inv;
                    n.SQ *= inv;
                    n.SU *= inv;
                    n.b *= inv;
                    n.invn = dd[1] * inv;
                    Real *dr = dring + (q % 3) * 3 * dstride + idx;
                    dr[0] = dd[2] * inv;
                    dr[dstride] = sv * inv;
                    dr[2 * dstride] = dv * inv;
                }
            }
            ring_store<Real, NS>(ring, plane, chunk, q % 3, idx, n);
            c += dc;
            lr += dl;
            if (c >= nx) { c -= nx; ++lr; }
        }
    };

    fill(0);
    if (nz > 1) fill(1);
    __syncthreads();
    for (int q = 0; q < nz; ++q) {
        const PlaneGeom<Real> gq = G[q];
        const bool has_p = q + 1 < nz;
        const PlaneGeom<Real> gp = has_p ? G[q + 1] : gq;
        const int sM = (q + 2) % 3, sO = q % 3, sP = (q + 1) % 3;
        Real *iw = ibuf + (q & 1) * F * iplane;              // write plane q
        const int ro = ((q + 1) & 1) * F * iplane;           // read plane q-1
        const Real *ir = ibuf + ro;
        const Real *irn = ibuf_next + ro;
        // interpolation weights (uniform over the plane)
        const Real mx1 = gq.tx, mx0 = Real(1) - gq.tx, my1 = gq.ty, my0 = Real(1) - gq.ty;
        const Real px0 = gp.tx, px1 = Real(1) - gp.tx, py0 = gp.ty, py1 = Real(1) - gp.ty;
        const Real dsM = gq.ds, dsP = has_p ? gp.ds : Real(0);

        long long v_lane = 0;
        int p_lane = 0;
        Real acc[NA];
        int l = pstart / nx, c = pstart - (pstart / nx) * nx;
        for (int p = pstart; p < npts; p += pstep) {
            if (p != pstart) {
                c += dc;
                l += dl;
                if (c >= nx) { c -= nx; ++l; }
            }
            int pi = c + gq.ax;
            pi -= pi >= nx ? nx : 0;
            int pj = row0 + l + gq.ay;           // in [0, 2 ny)
            pj -= pj >= ny ? ny : 0;
            pj -= pj >= ny ? ny : 0;
            const long long vloc = ((long long)gq.kz * ny + pj) * nx + pi;
            const long long v = B.vox0 + vloc;
            const Node<Real, NS> nO = ring_load<Real, NS>(ring, plane, chunk, sO, (l + H) * nx + c);
            // profile normalization at O (in the ring, except for the dichroism variant)
            Real invnO = nO.invn;
            if constexpr (dich) invnO = jmode ? a.invn[(long long)m * a.nvox + v] : Real(1);
#pragma unroll
            for (int s = 0; s < NA; ++s) acc[s] = Real(0);

            if (q == 0) {
                // boundary plane: I = (B, 0, 0, 0) entering at the bottom, 0 at the top; Lambda* = 0
                Real I0[NS];
#pragma unroll
                for (int s = 0; s < NS; ++s) I0[s] = Real(0);
                if (upward) I0[0] = a.bpl[v];
                for (int f = lane; f < nf; f += L) {
                    const int j = j0 + f;
                    StokesIO<Real, NS>::store(iw + f * iplane, ichunk, l * nx + c, I0);
                    if constexpr (MODE == MODE_EMERGENT) {
                        if (a.store) {
                            Real *o = a.store + (((long long)dir_out * a.nnu + j) * a.nvox + v) * NS;
#pragma unroll
                            for (int s = 0; s < NS; ++s) o[s] = I0[s];
                        }
                    }
                    if constexpr (MODE == MODE_JKQ) {
                        const Real wt = a.wf[j] * profile_shape(a.xf[j] - nO.s) * invnO;
                        acc[0] += wt * I0[0];
                        if (a.probe_ray == m) {
#pragma unroll
                            for (int s = 0; s < NS; ++s) a.probe[((long long)j * a.nvox + v) * NS + s] = I0[s];
                            a.probe_ls[(long long)j * a.nvox + v] = Real(0);
                        }
                    }
                }
            } else {
                const int c1 = (c + 1 == nx) ? 0 : c + 1;
                const int cm = (c == 0) ? nx - 1 : c - 1;
                // upwind corners (c|c1, l|l+1) on plane q-1; downwind (cm|c, l-1|l) on plane q+1
                // ring positions and bilinear weights of the corners; their node data
                // are read again for every frequency (shared-memory loads instead of
                // ~50 registers held across the frequency loop)
                const int rM[4] = {(l + 1) * nx + c, (l + 1) * nx + c1, (l + 2) * nx + c, (l + 2) * nx + c1};
                const int rP[4] = {l * nx + cm, l * nx + c, (l + 1) * nx + cm, (l + 1) * nx + c};
                const Real wM[4] = {mx0 * my0, mx1 * my0, mx0 * my1, mx1 * my1};
                const Real wP[4] = {px0 * py0, px1 * py0, px0 * py1, px1 * py1};
                // dichroism ratios and orientation terms of the upwind corners, of O and
                // (emission only) of the downwind corners
                Real mdq[4] = {0, 0, 0, 0}, mdu[4] = {0, 0, 0, 0}, msv[4] = {0, 0, 0, 0}, mdv[4] = {0, 0, 0, 0};
                Real psv[4] = {0, 0, 0, 0}, odq = 0, odu = 0, osv = 0, odv = 0;
                if constexpr (dich) {
                    const Real *dm = dring + sM * 3 * dstride;
                    const int ix[4] = {(l + 1) * nx + c, (l + 1) * nx + c1, (l + 2) * nx + c, (l + 2) * nx + c1};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        mdq[k] = ring_load<Real, NS>(ring, plane, chunk, sM, ix[k]).invn;
                        mdu[k] = dm[ix[k]];
                        msv[k] = dm[dstride + ix[k]];
                        mdv[k] = dm[2 * dstride + ix[k]];
                    }
                    odq = nO.invn;
                    const Real *dO = dring + sO * 3 * dstride + (l + 1) * nx + c;
                    odu = dO[0];
                    osv = dO[dstride];
                    odv = dO[2 * dstride];
                    if (has_p) {
                        const Real *dp = dring + sP * 3 * dstride + dstride;
#pragma unroll
                        for (int k = 0; k < 4; ++k) psv[k] = dp[rP[k]];
                    }
                }
                const Real wI[4] = {mx0 * my0, mx1 * my0, mx0 * my1, mx1 * my1};
                const bool last_row = (l + 1 == R);
                const int ilo = l * nx;                               // row l in this CTA
                const Real *ihi_base = last_row ? irn : ir;          // row l+1 (next CTA's row 0)
                const int ihi = last_row ? 0 : (l + 1) * nx;
                // biquadratic stencils: per axis the quadratic through the nearest node and
                // its two neighbours; M at (c + t_x, l + t_y) on plane q-1, P at
                // (c - t'_x, l - t'_y) on plane q+1 (sheared frame). Upwind Stokes rows
                // before the strip are the previous CTA's, after it the next CTA's.
                int bqM[9], bqP[9], bqI[3], bqC[3];
                Real bwM[9], bwP[9];
                const Real *bqB[3];
                if constexpr (BQ) {
                    const int oxm = gq.tx >= Real(0.5) ? 1 : 0, oym = gq.ty >= Real(0.5) ? 1 : 0;
                    const int oxp = gp.tx > Real(0.5) ? -1 : 0, oyp = gp.ty > Real(0.5) ? -1 : 0;
                    Real qxm[3], qym[3], qxp[3], qyp[3];
                    quad3<Real>(gq.tx - Real(oxm), qxm);
                    quad3<Real>(gq.ty - Real(oym), qym);
                    quad3<Real>(-gp.tx - Real(oxp), qxp);
                    quad3<Real>(-gp.ty - Real(oyp), qyp);
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const int cmx = ((c + oxm - 1 + a) % nx + nx) % nx, cpx = ((c + oxp - 1 + a) % nx + nx) % nx;
                        bqC[a] = cmx;
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            bqM[3 * b + a] = (l + oym - 1 + b + H) * nx + cmx;
                            bwM[3 * b + a] = qxm[a] * qym[b];
                            bqP[3 * b + a] = (l + oyp - 1 + b + H) * nx + cpx;
                            bwP[3 * b + a] = qxp[a] * qyp[b];
                        }
                    }
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const int r = l + oym - 1 + b;                     // in [-1, R + 1]
                        bqB[b] = r < 0 ? ibuf_prev + ro : (r >= R ? irn : ir);
                        bqI[b] = (r < 0 ? prev_local : (r >= R ? r - R : r)) * nx;
                    }
                }

                for (int f = lane; f < nf; f += L) {
                    const int j = j0 + f;
                    const Real x = a.xf[j];
                    const Real *pl = ir + f * iplane;
                    const Real *ph = ihi_base + f * iplane;
                    // a3: upwind Stokes vector (bilinear or biquadratic)
                    Real IM[NS];
                    if constexpr (BQ) {
#pragma unroll
                        for (int s = 0; s < NS; ++s) IM[s] = Real(0);
#pragma unroll
                        for (int b = 0; b < 3; ++b)
#pragma unroll
                            for (int a2 = 0; a2 < 3; ++a2) {
                                Real t[NS];
                                StokesIO<Real, NS>::load(bqB[b] + f * iplane, ichunk, bqI[b] + bqC[a2], t);
#pragma unroll
                                for (int s = 0; s < NS; ++s) IM[s] += bwM[3 * b + a2] * t[s];
                            }
                    } else {
                        Real t0[NS], t1[NS], t2[NS], t3[NS];
                        StokesIO<Real, NS>::load(pl, ichunk, ilo + c, t0);
                        StokesIO<Real, NS>::load(pl, ichunk, ilo + c1, t1);
                        StokesIO<Real, NS>::load(ph, ichunk, ihi + c, t2);
                        StokesIO<Real, NS>::load(ph, ichunk, ihi + c1, t3);
#pragma unroll
                        for (int s = 0; s < NS; ++s) IM[s] = wI[0] * t0[s] + wI[1] * t1[s] + wI[2] * t2[s] + wI[3] * t3[s];
                    }
                    Real IO[NS];
                    Coef<Real> co{};                          // (used by the J^K_Q sums below)
                    Real phO = Real(0);
                    if constexpr (GK) {
                        // explicit medium: eta = eta_I (1, K'/eta_I) and eps = eta_I S at the nodes, interpolated
                        // at M and P; the BESSER-DELO step with the full kappa^-1 = 1 + psi'_O K'_O (Eqs. 7-8)
                        Real etaM7[7], epsM4[4], etaO7[7], epsO4[4], epsP4[4], etaPI = 0;
#pragma unroll
                        for (int q = 0; q < 7; ++q) etaM7[q] = Real(0);
#pragma unroll
                        for (int s = 0; s < 4; ++s) epsM4[s] = epsP4[s] = Real(0);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const CornerM<Real, NS> km = corner_m<Real, NS>(ring_load<Real, NS>(ring, plane, chunk, sM, rM[k]), wM[k]);
                            const Real we = km.wchi * profile_shape(x - km.s);
                            const Real *gk = dring + sM * 6 * dstride + rM[k];
                            etaM7[0] += we;
#pragma unroll
                            for (int q = 1; q < 7; ++q) etaM7[q] += we * gk[(q - 1) * dstride];
                            epsM4[0] += we * km.SI;
                            epsM4[1] += we * km.SQ;
                            epsM4[2] += we * km.SU;
                            epsM4[3] += we * km.S00;
                        }
                        if (has_p) {
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const CornerM<Real, NS> kp = corner_m<Real, NS>(ring_load<Real, NS>(ring, plane, chunk, sP, rP[k]), wP[k]);
                                const Real we = kp.wchi * profile_shape(x - kp.s);
                                etaPI += we;
                                epsP4[0] += we * kp.SI;
                                epsP4[1] += we * kp.SQ;
                                epsP4[2] += we * kp.SU;
                                epsP4[3] += we * kp.S00;
                            }
                        }
                        const Real etaOI = nO.chi * profile_shape(x - nO.s);
                        const Real *gkO = dring + sO * 6 * dstride + (l + H) * nx + c;
                        etaO7[0] = etaOI;
#pragma unroll
                        for (int q = 1; q < 7; ++q) etaO7[q] = etaOI * gkO[(q - 1) * dstride];
                        epsO4[0] = etaOI * nO.SI;
                        epsO4[1] = etaOI * nO.SQ;
                        epsO4[2] = etaOI * nO.SU;
                        epsO4[3] = etaOI * nO.S00;
                        Real lsg;
                        delo_step_general<Real>(IM, etaM7, epsM4, etaO7, epsO4, etaPI, epsP4, dsM, dsP, has_p, IO, lsg);
                    } else {
                        // a2-a3: node transfer coefficients and bilinear interpolation at M and P
                        Real etaM = 0, etaVM = 0, etaQM = 0, etaUM = 0, epsM[NS];
    #pragma unroll
                        for (int s = 0; s < NS; ++s) epsM[s] = 0;
                        constexpr int NK = BQ ? 9 : 4;           // interpolation corners
    #pragma unroll
                        for (int k = 0; k < NK; ++k) {
                            const CornerM<Real, NS> km = corner_m<Real, NS>(
                                ring_load<Real, NS>(ring, plane, chunk, sM, BQ ? bqM[k] : rM[k]), BQ ? bwM[k] : wM[k]);
                            const Real xs = x - km.s;
                            const Real we = km.wchi * profile_shape(xs);
                            etaM += we;
                            if constexpr (dich) {
                                etaQM += we * mdq[k];
                                etaUM += we * mdu[k];
                                etaVM += we * mdv[k];
                                epsM[3] += we * msv[k];
                            }
                            if constexpr (NS == 1) {
                                epsM[0] += we * km.S;
                            } else {
                                const Real wkv = we * (km.b * xs);
                                etaVM += wkv;
                                epsM[0] += we * km.SI;
                                epsM[1] += we * km.SQ;
                                epsM[2] += we * km.SU;
                                epsM[3] += wkv * km.S00;
                            }
                        }
                        Real etaP = 0, epsP[NS];
    #pragma unroll
                        for (int s = 0; s < NS; ++s) epsP[s] = 0;
                        if (has_p) {
    #pragma unroll
                            for (int k = 0; k < NK; ++k) {
                                const CornerP<Real, NS> kp = corner_p<Real, NS>(
                                    ring_load<Real, NS>(ring, plane, chunk, sP, BQ ? bqP[k] : rP[k]), BQ ? bwP[k] : wP[k]);
                                const Real xs = x - kp.s;
                                const Real we = kp.wchi * profile_shape(xs);
                                etaP += we;
                                if constexpr (NS == 1) {
                                    epsP[0] += we * kp.S;
                                } else {
                                    epsP[0] += we * kp.SI;
                                    epsP[1] += we * kp.SQ;
                                    epsP[2] += we * kp.SU;
                                    epsP[3] += we * (kp.bS * xs);
                                    if constexpr (dich) epsP[3] += we * psv[k];
                                }
                            }
                        }
                        const Real xsO = x - nO.s;
                        phO = profile_shape(xsO);
                        const Real etaO = nO.chi * phO;
                        Real SO[NS], SM[NS], SP[NS];
                        const Real iM = rcp(etaM);
                        if constexpr (NS == 1) {
                            SO[0] = nO.S;
                        } else {
                            SO[0] = nO.SI; SO[1] = nO.SQ; SO[2] = nO.SU; SO[3] = nO.b * xsO * nO.S00;
                            if constexpr (dich) SO[3] += osv;
                        }
    #pragma unroll
                        for (int s = 0; s < NS; ++s) SM[s] = epsM[s] * iM;
                        // a4: optical paths (trapezoid along MO and OP)
                        const Real tMO = Real(0.5) * (etaM + etaO) * dsM;
                        Real tOP = Real(1);
                        if (has_p) {
                            const Real iP = rcp(etaP);
    #pragma unroll
                            for (int s = 0; s < NS; ++s) SP[s] = epsP[s] * iP;
                            tOP = Real(0.5) * (etaO + etaP) * dsP;
                        } else {
    #pragma unroll
                            for (int s = 0; s < NS; ++s) SP[s] = Real(0);
                        }
                        // a6: exponential-integral coefficients
                        co = coefficients(tMO);
                        // a5: BESSER control points per Stokes parameter
                        Real cM[NS];
                        if (has_p) {
                            const BesserGeom<Real> bg = besser_geom(tMO, tOP);
    #pragma unroll
                            for (int s = 0; s < NS; ++s) cM[s] = control_point(SM[s], SO[s], SP[s], bg);
                        } else {
    #pragma unroll
                            for (int s = 0; s < NS; ++s) cM[s] = Real(0.5) * (SM[s] + SO[s]);
                        }
                        // a7: BESSER-DELO step (Eq. 7)
                        if constexpr (NS == 1) {
                            IO[0] = co.e * IM[0] + co.wm * SM[0] + co.wo * SO[0] + co.wc * cM[0];
                        } else if constexpr (dich) {
                            // K' with eta_Q, eta_U (dichroism) and eta_V entries over eta_I:
                            // (K'I)_0 = q I_1 + u I_2 + v I_3, (K'I)_k = k_k I_0
                            const Real qM = etaQM * iM, uM = etaUM * iM, vM = etaVM * iM;
                            const Real qO = odq, uO = odu, vO = nO.b * xsO + odv;
                            Real rhs[4];
    #pragma unroll
                            for (int s = 0; s < 4; ++s) rhs[s] = co.e * IM[s] + co.wm * SM[s] + co.wo * SO[s] + co.wc * cM[s];
                            rhs[0] -= co.pm * (qM * IM[1] + uM * IM[2] + vM * IM[3]);
                            rhs[1] -= co.pm * qM * IM[0];
                            rhs[2] -= co.pm * uM * IM[0];
                            rhs[3] -= co.pm * vM * IM[0];
                            // (1 + psi'_O K'_O)^-1 of the arrow-shaped matrix
                            const Real aq = co.po * qO, au = co.po * uO, av = co.po * vO;
                            IO[0] = (rhs[0] - aq * rhs[1] - au * rhs[2] - av * rhs[3]) * rcp(Real(1) - aq * aq - au * au - av * av);
                            IO[1] = rhs[1] - aq * IO[0];
                            IO[2] = rhs[2] - au * IO[0];
                            IO[3] = rhs[3] - av * IO[0];
                        } else {
                            // K' has only the eta_V / eta_I entries (weak-field Zeeman)
                            const Real kvM = etaVM * iM;
                            const Real kvO = nO.b * xsO;
                            Real rhs[4];
    #pragma unroll
                            for (int s = 0; s < 4; ++s) rhs[s] = co.e * IM[s] + co.wm * SM[s] + co.wo * SO[s] + co.wc * cM[s];
                            rhs[0] -= co.pm * kvM * IM[3];
                            rhs[3] -= co.pm * kvM * IM[0];
                            // kappa^-1 = 1 + psi'_O K'_O couples I and V only
                            const Real av = co.po * kvO;
                            const Real idet = rcp(Real(1) - av * av);
                            IO[0] = (rhs[0] - av * rhs[3]) * idet;
                            IO[3] = (rhs[3] - av * rhs[0]) * idet;
                            IO[1] = rhs[1];
                            IO[2] = rhs[2];
                        }
                    }
                    StokesIO<Real, NS>::store(iw + f * iplane, ichunk, l * nx + c, IO);
                    // a8: Lambda* (Eq. 14; w_O + w_C/2 on the last plane) and accumulation
                    if constexpr (MODE == MODE_JKQ) {
                        const Real ls = co.wo + (has_p ? co.wc : Real(0.5) * co.wc);
                        const Real wt = a.wf[j] * phO * invnO;
                        if constexpr (NS == 1) {
                            acc[0] += wt * IO[0];
                            acc[1] += wt * ls;
                        } else {
                            acc[0] += wt * IO[0];
                            acc[1] += wt * IO[1];
                            acc[2] += wt * IO[2];
                            acc[3] += wt * ls;
                            if constexpr (NA == 5) acc[4] += wt * IO[3];
                        }
                        if (a.probe_ray == m) {
#pragma unroll
                            for (int s = 0; s < NS; ++s) a.probe[((long long)j * a.nvox + v) * NS + s] = IO[s];
                            a.probe_ls[(long long)j * a.nvox + v] = ls;
                        }
                    } else {
                        if (q == nz - 1) {
                            double *o = a.out + (((long long)dir_out * a.nnu + j) * nxy + (long long)pj * nx + pi) * NS;
#pragma unroll
                            for (int s = 0; s < NS; ++s) o[s] = (double)IO[s];
                        }
                        if (a.store) {
                            Real *o = a.store + (((long long)dir_out * a.nnu + j) * a.nvox + v) * NS;
#pragma unroll
                            for (int s = 0; s < NS; ++s) o[s] = IO[s];
                        }
                    }
                }
            }
            if constexpr (MODE == MODE_JKQ) {
                if (L == 1) {
                    accumulate_partial<Real, NS, NA == 5>(a, m, v, g, acc);
                } else {
#pragma unroll
                    for (int s = 0; s < NA; ++s) lane_buf[(s * L + lane) * npts + p] = acc[s];
                    v_lane = v;
                    p_lane = p;
                }
            }
        }
        if constexpr (MODE == MODE_JKQ) {
            if (L > 1) {
                // fixed-order sum over the frequency lanes of each point
                __syncthreads();
                if (lane == 0 && pstart < npts) {
                    Real tot[NA];
#pragma unroll
                    for (int s = 0; s < NA; ++s) {
                        tot[s] = Real(0);
                        for (int k = 0; k < L; ++k) tot[s] += lane_buf[(s * L + k) * npts + p_lane];
                    }
                    accumulate_partial<Real, NS, NA == 5>(a, m, v_lane, g, tot);
                }
            }
        }
        // Plane q is done in this CTA: nobody here reads ring slot (q-1)%3 or
        // the Stokes plane of q-1 any more. Arrive on the cluster barrier
        // (release: the new Stokes plane becomes visible to the neighbour CTA),
        // refill the free ring slot with plane q+2 while the other CTAs
        // finish, then wait (acquire) before plane q+1 reads the neighbour's data.
        __syncthreads();
        cluster_arrive_release();
        if (q + 2 < nz) fill(q + 2);
        __syncthreads();
        cluster_wait_acquire();
    }
}

template <typename Real, int NS, int MODE, bool DI = false, bool BQ = false, bool GK = false>
__global__ void __launch_bounds__(512, 1) sweep_kernel(const SweepArgs<Real> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int cid = blockIdx.x / C;
    const int ncl = gridDim.x / C;
    using V = typename V16<Real>::T;
    V *ring = reinterpret_cast<V *>(smem_raw);
    Real *ibuf = reinterpret_cast<Real *>(ring + 3 * a.ring_plane);
    Real *lane_buf = ibuf + 2 * a.F * NS * a.ipts_max;
    cluster.sync();
    if constexpr (MODE == MODE_JKQ) {
        if (a.next_item) {
            // dynamic work list: CTA 0 of the cluster takes the next item from the
            // launch's counter and writes it into every CTA's shared memory before
            // the cluster barrier (slot k & 1: a slot is rewritten only after every
            // CTA has passed the barrier that followed its last read)
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
                    sweep_item<Real, NS, MODE, DI, BQ, GK>(a, cluster, ring, ibuf, lane_buf, box, m, g, rank, C, 0);
            }
            return;
        }
    }
    for (int item = cid; item < a.nitems; item += ncl) {
        if constexpr (MODE == MODE_JKQ) {
            const int code = a.items ? a.items[item] : item;
            const int box = code / a.nray, m = code - box * a.nray;
            for (int g = 0; g < a.ngroups; ++g)
                sweep_item<Real, NS, MODE, DI, BQ, GK>(a, cluster, ring, ibuf, lane_buf, box, m, g, rank, C, 0);
        } else {
            const int d = item / a.ngroups, g = item - d * a.ngroups;
            sweep_item<Real, NS, MODE, DI, BQ, GK>(a, cluster, ring, ibuf, lane_buf, 0, d, g, rank, C, d);
        }
    }
}

template <typename Real, int NS>
static void *kernel_ptr(int mode, bool dich = false, bool bq = false, bool gk = false)
{
    // the explicit medium (general propagation matrix), emergent mode
    if constexpr (NS == 4)
        if (gk) return (void *)sweep_kernel<Real, NS, MODE_EMERGENT, false, false, true>;
    // the dichroism variant (polarized lines of the multilevel atom)
    if (NS == 4 && dich)
        return mode == MODE_JKQ ? (void *)sweep_kernel<Real, NS, MODE_JKQ, NS == 4>
                                : (void *)sweep_kernel<Real, NS, MODE_EMERGENT, NS == 4>;
    // biquadratic interpolation
    if (bq)
        return mode == MODE_JKQ ? (void *)sweep_kernel<Real, NS, MODE_JKQ, false, true>
                                : (void *)sweep_kernel<Real, NS, MODE_EMERGENT, false, true>;
    return mode == MODE_JKQ ? (void *)sweep_kernel<Real, NS, MODE_JKQ> : (void *)sweep_kernel<Real, NS, MODE_EMERGENT>;
}

template <typename Real, int NS>
static cudaError_t prepare(int mode, int cluster, int smem, bool dich = false, bool bq = false, bool gk = false)
{
    void *k = kernel_ptr<Real, NS>(mode, dich, bq, gk);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (cluster > 8) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <typename Real, int NS>
cudaError_t max_active_clusters(int cluster, int smem, int threads, int *out, bool dich, bool bq, bool gk)
{
    cudaError_t e = prepare<Real, NS>(gk ? MODE_EMERGENT : MODE_JKQ, cluster, smem, dich, bq, gk);
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
    return cudaOccupancyMaxActiveClusters(
        out, (void (*)(SweepArgs<Real>))kernel_ptr<Real, NS>(gk ? MODE_EMERGENT : MODE_JKQ, dich, bq, gk), &lc);
}

template <typename Real, int NS>
cudaError_t launch_sweep(const SweepArgs<Real> &a, int mode, LaunchCfg &cfg, cudaStream_t st)
{
    const bool dich = NS == 4 && a.dich != nullptr;
    const bool gk = NS == 4 && a.kexpl != nullptr;
    const bool bq = !dich && !gk && a.interp == 2;
    if (gk && mode != MODE_EMERGENT) return cudaErrorInvalidValue;
    cudaError_t e = prepare<Real, NS>(mode, cfg.cluster, cfg.smem, dich, bq, gk);
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
    if constexpr (NS == 4)
        if (gk) return cudaLaunchKernelEx(&lc, sweep_kernel<Real, NS, MODE_EMERGENT, false, false, true>, a);
    if (dich)
        return mode == MODE_JKQ ? cudaLaunchKernelEx(&lc, sweep_kernel<Real, NS, MODE_JKQ, NS == 4>, a)
                                : cudaLaunchKernelEx(&lc, sweep_kernel<Real, NS, MODE_EMERGENT, NS == 4>, a);
    if (bq)
        return mode == MODE_JKQ ? cudaLaunchKernelEx(&lc, sweep_kernel<Real, NS, MODE_JKQ, false, true>, a)
                                : cudaLaunchKernelEx(&lc, sweep_kernel<Real, NS, MODE_EMERGENT, false, true>, a);
    if (mode == MODE_JKQ)
        return cudaLaunchKernelEx(&lc, sweep_kernel<Real, NS, MODE_JKQ>, a);
    return cudaLaunchKernelEx(&lc, sweep_kernel<Real, NS, MODE_EMERGENT>, a);
}

#define PORTA_INST(R, N)                                                                           \
    template int sweep_smem_bytes<R, N>(int, int, int, int, int);                                            \
    template cudaError_t max_active_clusters<R, N>(int, int, int, int *, bool, bool, bool);        \
    template cudaError_t launch_sweep<R, N>(const SweepArgs<R> &, int, LaunchCfg &, cudaStream_t);
PORTA_INST(float, 1)
PORTA_INST(float, 4)
PORTA_INST(double, 1)
PORTA_INST(double, 4)
#undef PORTA_INST

}  // namespace porta
