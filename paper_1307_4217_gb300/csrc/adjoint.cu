// Adjoint (reverse mode) of the emergent-Stokes formal solution (Sec. 3,
// Eq. 7 with the BESSER control points of Sec. 3.2) at fixed multipoles.
//
// Parameters per voxel: the line-centre opacity chi, the emission scale
// e = chi S^0_0 (the multipoles scale as e/chi with their ratios to S^0_0
// fixed) and b = bfac B.Omega (bfac = 2 gbar zeta), so that with
// phi = exp(-(x - s)^2) and xs = x - s the node coefficients are
//   eta_I = chi phi,        eta_V = b xs chi phi,
//   eps_i = e phi S_i/S00,  eps_V = b xs e phi      (unpolarized: eps = e phi).
// Given dL/dI of the top plane (all frequencies of the emergent directions),
// the kernel returns per (direction, frequency group) dL/dchi, dL/de and
// dL/db of every node; a second kernel sums the groups in a fixed order and
// turns dL/db into dL/dB = bfac sum_dir Omega dL/db.
//
// Decomposition: the forward sweep's. One thread-block cluster owns one
// (direction, frequency group); the planes are visited in reverse sweep order
// with the sheared rows split into strips, one per CTA. The forward Stokes
// vectors of every plane come from the forward emergent sweep's tape; each
// step is recomputed locally with the forward's arithmetic (so the control
// point takes the forward's branch) and differentiated by hand. Every
// transposed interpolation is a gather, not a scatter, so there are no atomics
// and the result does not depend on scheduling:
//   - the upwind Stokes adjoint of a node on plane q-1 gathers the dL/dI_M of
//     the 4 points of plane q whose upwind stencil holds it;
//   - the coefficient adjoint of a node on plane q collects its own term as O
//     (step q), the dL/d(M interpolants) of 4 points of plane q+1 and the
//     dL/d(P interpolants) of 4 points of plane q-1 (step q-1), and is turned
//     into parameter gradients once complete.
// In the sheared frame these stencils are the fixed neighbour offsets
// (0|-1, 0|-1) and (0|+1, 0|+1); the one row across a strip boundary is read
// from the neighbouring CTA's shared memory (DSMEM) after a cluster barrier.
#include <cooperative_groups.h>

#include <algorithm>

#include "adjoint_math.cuh"
#include "device_math.cuh"
#include "porta_internal.cuh"
#include "sweep_common.cuh"

namespace cg = cooperative_groups;

namespace porta {

// adjoint values stored per point and frequency:
//   NM: dL/d(eta_I, [eta_V], eps[NS]) of the M interpolants, and of the node as O
//   NP: dL/d(eta_I, eps[NS]) of the P interpolants (eta_V is not interpolated at P)
template <int NS>
__host__ __device__ constexpr int adj_nm() { return NS == 1 ? 2 : 6; }
template <int NS>
__host__ __device__ constexpr int adj_np() { return NS + 1; }

// bytes before the tape tile (16-byte aligned), and the whole shared memory:
// ring, gI, gM, gP, T (per point and frequency), then the staged tape rows
// of the upwind plane (tile_pts = (rows + 1) x nx points per frequency) and
// the reduced frequencies and quadrature weights of the group (2 F)
// points per adjoint plane: the strip's points rounded up to a multiple of 4,
// so that every vector plane below starts on a 16-byte boundary
__host__ __device__ constexpr int adj_ipa(int ipts) { return (ipts + 3) / 4 * 4; }

template <typename Real, int NS>
__host__ __device__ constexpr int adjoint_tile_offset(int ring_plane, int ipts, int F)
{
    return (3 * ring_plane * 16 +
            F * adj_ipa(ipts) * (2 * NS + adj_nm<NS>() + adj_np<NS>() + 2 * adj_nm<NS>()) * (int)sizeof(Real) + 15) /
           16 * 16;
}

template <typename Real, int NS>
int adjoint_smem_bytes(int ring_plane, int ipts, int tile_pts, int F)
{
    return adjoint_tile_offset<Real, NS>(ring_plane, ipts, F) + (F * tile_pts * NS + 2 * F) * (int)sizeof(Real);
}

// asynchronous global -> shared copy of one Stokes vector (cp.async, 4/8/16 bytes per instruction)
template <int BYTES>
__device__ __forceinline__ void cp_async_bytes(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}
template <typename Real, int NS>
__device__ __forceinline__ void copy_stokes_async(Real *dst, const Real *src)
{
    constexpr int B = NS * (int)sizeof(Real);
    if constexpr (B <= 16) {
        cp_async_bytes<B>(dst, src);
    } else {
        cp_async_bytes<16>(dst, src);
        cp_async_bytes<16>(dst + 16 / sizeof(Real), src + 16 / sizeof(Real));
    }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// one Stokes vector from shared memory (vector loads)
template <typename Real, int NS>
__device__ __forceinline__ void load_stokes(const Real *p, Real v[NS])
{
    if constexpr (NS == 4 && sizeof(Real) == 4) {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else if constexpr (NS == 4) {
        const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
        v[0] = p[0];
    }
}

// W Reals per point in shared memory: planes of 16-byte chunks ([chunk][p],
// consecutive points in consecutive 16-byte words) for the first
// W / (16 / sizeof(Real)) chunks and one narrower plane for the Reals left
// over; n = points per plane (a multiple of 4), so every plane is 16-byte aligned
template <typename Real, int W>
struct SVec {
    static constexpr int PER = 16 / (int)sizeof(Real);
    static constexpr int NC = W / PER, REM = W - NC * PER;
    static_assert(REM <= 2, "at most two Reals in the narrow plane");
    using V = typename V16<Real>::T;
    __device__ static __forceinline__ void load(const Real *b, int n, int p, Real v[W])
    {
#pragma unroll
        for (int h = 0; h < NC; ++h) {
            const V x = reinterpret_cast<const V *>(b + h * PER * n)[p];
            if constexpr (PER == 4) {
                v[4 * h] = x.x; v[4 * h + 1] = x.y; v[4 * h + 2] = x.z; v[4 * h + 3] = x.w;
            } else {
                v[2 * h] = x.x; v[2 * h + 1] = x.y;
            }
        }
        const Real *r = b + NC * PER * n;
        if constexpr (REM == 2) {
            const R2<Real> x = reinterpret_cast<const R2<Real> *>(r)[p];
            v[NC * PER] = x.x; v[NC * PER + 1] = x.y;
        } else if constexpr (REM == 1) {
            v[NC * PER] = r[p];
        }
    }
    __device__ static __forceinline__ void store(Real *b, int n, int p, const Real v[W])
    {
#pragma unroll
        for (int h = 0; h < NC; ++h) {
            V x;
            if constexpr (PER == 4) {
                x.x = v[4 * h]; x.y = v[4 * h + 1]; x.z = v[4 * h + 2]; x.w = v[4 * h + 3];
            } else {
                x.x = v[2 * h]; x.y = v[2 * h + 1];
            }
            reinterpret_cast<V *>(b + h * PER * n)[p] = x;
        }
        Real *r = b + NC * PER * n;
        if constexpr (REM == 2) {
            reinterpret_cast<R2<Real> *>(r)[p] = R2<Real>{v[NC * PER], v[NC * PER + 1]};
        } else if constexpr (REM == 1) {
            r[p] = v[NC * PER];
        }
    }
};

// CTA owning sheared row r when CTA k owns rows floor(k ny / C) .. floor((k+1) ny / C) - 1
__device__ __forceinline__ int row_owner(int r, int ny, int C)
{
    return (int)(((long long)(r + 1) * C + ny - 1) / ny) - 1;
}
__device__ __forceinline__ int row_start(int k, int ny, int C) { return (int)(((long long)k * ny) / C); }

// parameter gradients (chi, e, b) of one node at reduced frequency x from the
// node's total adjoint t = dL/d(eta_I, [eta_V], eps[NS])
template <typename Real, int NS>
__device__ __forceinline__ void node_param_grad(const Node<Real, NS> &n, Real x, const Real *t, Real &gchi, Real &ge,
                                                Real &gb)
{
    const Real xs = x - n.s;
    const Real ph = profile_shape(xs);
    if constexpr (NS == 1) {
        gchi += ph * t[0];
        ge += ph * t[1];
    } else {
        const Real bxs = n.b * xs;
        const Real iS = rcp(n.S00);
        gchi += ph * (t[0] + bxs * t[1]);
        ge += ph * ((n.SI * t[2] + n.SQ * t[3] + n.SU * t[4]) * iS + bxs * t[5]);
        gb += xs * ph * n.chi * (t[1] + n.S00 * t[5]);
    }
}

// the same in the unknowns: dL/dchi at fixed rho, dL/dB (3) and dL/drho (up to 6)
// added to o[10] (eps_i = chi phi S_i(rho), eps_V = S00 eta_V, S_i = sum_c T_ic rho_c
// with the real multipole layout's factor 2 for Q != 0); o in the sweep's precision
// over one frequency group (the per-cluster sums across items are FP64)
template <typename Real, int NS>
__device__ __forceinline__ void node_param_grad_rho(const Node<Real, NS> &n, const RayDev<Real> &ray, Real bfac, Real x,
                                                    const Real *t, Real *o)
{
    const Real xs = x - n.s;
    const Real ph = profile_shape(xs);
    if constexpr (NS == 1) {
        o[0] += ph * (t[0] + n.S * t[1]);
        o[4] += n.chi * ph * t[1];
    } else {
        const Real bxs = n.b * xs;
        o[0] += ph * (t[0] + bxs * t[1] + n.SI * t[2] + n.SQ * t[3] + n.SU * t[4] + bxs * n.S00 * t[5]);
        const Real gb = bfac * xs * ph * n.chi * (t[1] + n.S00 * t[5]);
        o[1] += gb * ray.ox;
        o[2] += gb * ray.oy;
        o[3] += gb * ray.oz;
        const Real cp = n.chi * ph;
        const Real gS[3] = {cp * t[2], cp * t[3], cp * t[4]};
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const Real f2 = c >= 2 ? Real(2) : Real(1);
            o[4 + c] += f2 * (ray.t[c] * gS[0] + ray.t[6 + c] * gS[1] + ray.t[12 + c] * gS[2]);
        }
        o[4] += cp * bxs * t[5];
    }
}

template <typename Real, int NS, int FORM>
__device__ __forceinline__ void adjoint_item(const SweepArgs<Real> &a, cg::cluster_group &cluster,
                                             typename V16<Real>::T *ring, Real *gI, Real *gM, Real *gP, Real *T,
                                             Real *tt, int d, int g, int rank, int C, int item, int cid)
{
    constexpr int NM = adj_nm<NS>(), NP = adj_np<NS>();
    constexpr int NCH = node_words<NS>() * (int)sizeof(Real) / 16;
    const BoxDev B = a.boxes[0];
    const int nx = B.nx, ny = B.ny, nz = B.nz, F = a.F;
    const int rmax = (ny + C - 1) / C;
    const int row0 = row_start(rank, ny, C);
    const int R = row_start(rank + 1, ny, C) - row0;
    // neighbours in the sheared frame: the owner of the row after the strip
    // (its row 0) and of the row before it (its last row)
    const int next_row = (row0 + R) % ny;
    const int next_owner = row_owner(next_row, ny, C);
    const int prev_row = (row0 + ny - 1) % ny;
    const int prev_owner = row_owner(prev_row, ny, C);
    const int prev_last = prev_row - row_start(prev_owner, ny, C);
    const int ipa = adj_ipa(a.ipts_max);                // points per adjoint plane
    const Real *gI_prev = cluster.map_shared_rank(gI, prev_owner);
    const Real *gM_prev = cluster.map_shared_rank(gM, prev_owner);
    const Real *gP_next = cluster.map_shared_rank(gP, next_owner);
    const int j0 = g * F;
    const int nf = min(F, a.nnu - j0);
    const PlaneGeom<Real> *G = a.geom + (long long)d * nz;
    const RayDev<Real> ray = a.rays[d];
    const long long nxy = (long long)nx * ny;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int chunk = (rmax + 2) * nx;
    const int plane = NCH * chunk;
    const int npts = R * nx;
    const int tile_pts = (rmax + 1) * nx;               // staged tape points per frequency
    Real *xsh = tt + (long long)F * tile_pts * NS;      // x_j and w_j of the group
    const Real *tape = a.store + (long long)d * a.nnu * a.nvox * NS;
    Real *gout_part = FORM == 0 ? a.gpart + (long long)item * 3 * a.nvox : nullptr;
    Real *acc = FORM != 0 ? reinterpret_cast<Real *>(a.gacc) + (long long)cid * 10 * a.nvox : nullptr;
    const int mglob = a.ray0 + d;                       // ray index for the J weights (form 2)
    const Real wray = FORM == 2 ? (Real)a.tw[19 * mglob] : Real(0);
    // offsets of the vector planes (SVec): gI[par][f], gM[f], gP[f], T[par][f]
    auto oI = [&](int par, int f) { return (par * F + f) * NS * ipa; };
    auto oM = [&](int f) { return f * NM * ipa; };
    auto oP = [&](int f) { return f * NP * ipa; };
    auto oT = [&](int par, int f) { return (par * F + f) * NM * ipa; };
    using VI = SVec<Real, NS>;
    using VM = SVec<Real, NM>;
    using VP = SVec<Real, NP>;

    // thread -> (row, column) of its first point, and the stride of the point
    // loops in rows and columns (no integer division inside the loops)
    const int tl0 = tid / nx, tc0 = tid - tl0 * nx;
    const int dl = nt / nx, dc = nt - dl * nx;
    auto step = [&](int &l, int &c) {
        c += dc;
        l += dl;
        if (c >= nx) { c -= nx; ++l; }
    };
    auto fill = [&](int q, const PlaneGeom<Real> &gq) {
        const int nn = (R + 2) * nx;
        const long long kb = (long long)gq.kz * ny;
        // voxel of ring node (lr, c), lr = ring row (local row + 1)
        auto ring_voxel = [&](int lr, int c) {
            int pi = c + gq.ax;
            pi -= pi >= nx ? nx : 0;
            int pj = row0 + lr - 1 + gq.ay;                  // in [-1, 2 ny)
            pj += pj < 0 ? ny : 0;
            pj -= pj >= ny ? ny : 0;
            return B.vox0 + (kb + pj) * nx + pi;
        };
        // two nodes per thread and round, so that their global loads are in
        // flight together
        int lr = tl0, c = tc0;
        for (int idx = tid; idx < nn; idx += 2 * nt) {
            int lr2 = lr, c2 = c;
            step(lr2, c2);
            const bool two = idx + nt < nn;
            const long long v = ring_voxel(lr, c);
            const long long v2 = two ? ring_voxel(lr2, c2) : v;
            const Node<Real, NS> n1 = make_node<Real, NS>(a, ray, v, mglob, FORM == 2);
            const Node<Real, NS> n2 = make_node<Real, NS>(a, ray, v2, mglob, FORM == 2);
            ring_store<Real, NS>(ring, plane, chunk, q % 3, idx, n1);
            if (two) ring_store<Real, NS>(ring, plane, chunk, q % 3, idx + nt, n2);
            lr = lr2;
            c = c2;
            step(lr, c);
        }
    };
    // physical voxel of sheared node (c, local row l) of plane q, l in [0, R]
    auto voxel = [&](const PlaneGeom<Real> &gq, int c, int l) {
        int pi = c + gq.ax;
        pi -= pi >= nx ? nx : 0;
        int pj = row0 + l + gq.ay;                           // in [0, 2 ny)
        pj -= pj >= ny ? ny : 0;
        return ((long long)gq.kz * ny + pj) * nx + pi;
    };
    // parameter gradients of the nodes of plane pq (ring slot `slot`) from the
    // adjoint totals T[par] plus, with_p, the P gathers of plane pq-1
    auto finalize_pt = [&](const PlaneGeom<Real> &gq, int slot, int par, bool with_p, const Real *wP, int p, int l,
                           int c) {
        {
            const int c1 = c + 1 == nx ? 0 : c + 1;
            const Node<Real, NS> n = ring_load<Real, NS>(ring, plane, chunk, slot, (l + 1) * nx + c);
            const bool last = l + 1 == R;
            const Real *ph = last ? gP_next : gP;
            const int lh = last ? 0 : (l + 1) * nx;
            Real gchi = 0, ge = 0, gb = 0;
            Real o[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int f = 0; f < nf; ++f) {
                Real t[NM];
                VM::load(T + oT(par, f), ipa, p, t);
                if (with_p) {
                    // node (c, l) of plane pq is corner (c-1|c, l-1|l) of the points
                    // (c+1|c, l+1|l) of plane pq-1
                    Real gp[NP], u0[NP], u1[NP], u2[NP], u3[NP];
                    VP::load(ph + oP(f), ipa, lh + c1, u0);
                    VP::load(ph + oP(f), ipa, lh + c, u1);
                    VP::load(gP + oP(f), ipa, l * nx + c1, u2);
                    VP::load(gP + oP(f), ipa, l * nx + c, u3);
#pragma unroll
                    for (int k = 0; k < NP; ++k) gp[k] = wP[0] * u0[k] + wP[1] * u1[k] + wP[2] * u2[k] + wP[3] * u3[k];
                    t[0] += gp[0];
#pragma unroll
                    for (int s = 0; s < NS; ++s) t[NM - NS + s] += gp[1 + s];
                }
                if constexpr (FORM == 0)
                    node_param_grad<Real, NS>(n, xsh[f], t, gchi, ge, gb);
                else
                    node_param_grad_rho<Real, NS>(n, ray, a.bfac, xsh[f], t, o);
            }
            const long long v = B.vox0 + voxel(gq, c, l);
            if constexpr (FORM == 0) {
                gout_part[v] = gchi;
                gout_part[a.nvox + v] = ge;
                gout_part[2 * a.nvox + v] = gb;
            } else {
                // this cluster's accumulators, as reductions performed in the L2 (no
                // load on this thread's path), in the sweep's precision (an FP32 sweep
                // adds FP32 terms: no conversions on the GPU's low-rate FP64 pipe). A
                // node is finalized by one thread per item and the cluster's items are
                // separated by cluster barriers (release / acquire), so the additions
                // into each accumulator happen in item order: the sums are reproducible.
#pragma unroll
                for (int k = 0; k < 10; ++k) atomicAdd(acc + k * a.nvox + v, o[k]);
            }
        }
    };
    auto finalize = [&](int pq, int slot, int par, bool with_p, const Real *wP) {
        const PlaneGeom<Real> gq = G[pq];
        int l = tl0, c = tc0;
        for (int p = tid; p < npts; p += nt) {
            finalize_pt(gq, slot, par, with_p, wP, p, l, c);
            step(l, c);
        }
    };

    // tape rows 0..R of the strip (sheared frame) of plane qq, all frequencies of the group
    auto stage = [&](const PlaneGeom<Real> &gg) {
        const int per = (R + 1) * nx;
        const Real *src0 = tape + (long long)j0 * a.nvox * NS;
        int lr = tl0, c = tc0;
        for (int r = tid; r < per; r += nt) {
            const Real *src = src0 + (B.vox0 + voxel(gg, c, lr)) * NS;
            Real *dst = tt + (long long)r * NS;
            for (int f = 0; f < nf; ++f)
                copy_stokes_async<Real, NS>(dst + (long long)f * tile_pts * NS, src + (long long)f * a.nvox * NS);
            step(lr, c);
        }
        cp_async_commit();
    };

    {
        const PlaneGeom<Real> g1 = G[nz - 1], g2 = G[nz - 2];
        fill(nz - 1, g1);
        fill(nz - 2, g2);
        stage(g2);
    }
    cp_async_wait_all();
    for (int f = tid; f < nf; f += nt) {
        xsh[f] = a.xf[j0 + f];
        xsh[F + f] = FORM == 2 ? (Real)a.wf[j0 + f] : Real(0);
    }
    for (int p = tid; p < npts; p += nt)
        for (int f = 0; f < nf; ++f) {
            Real z[NM];
#pragma unroll
            for (int k = 0; k < NM; ++k) z[k] = Real(0);
            VM::store(T + oT((nz - 1) & 1, f), ipa, p, z);
        }
    __syncthreads();
    cluster.sync();

    for (int q = nz - 1; q >= 1; --q) {
        const PlaneGeom<Real> gq = G[q];
        const bool has_p = q + 1 < nz;
        const PlaneGeom<Real> gp = has_p ? G[q + 1] : gq;
        const int sM = (q + 2) % 3, sO = q % 3, sP = (q + 1) % 3;
        const int par = q & 1, opar = par ^ 1;
        const Real mx1 = gq.tx, mx0 = Real(1) - gq.tx, my1 = gq.ty, my0 = Real(1) - gq.ty;
        const Real px0 = gp.tx, px1 = Real(1) - gp.tx, py0 = gp.ty, py1 = Real(1) - gp.ty;
        const Real wM[4] = {mx0 * my0, mx1 * my0, mx0 * my1, mx1 * my1};
        const Real wP[4] = {px0 * py0, px1 * py0, px0 * py1, px1 * py1};
        // weights of the upwind stencils of plane q+1 (Stokes adjoint gather)
        const Real nx1 = gp.tx, nx0 = Real(1) - gp.tx, ny1 = gp.ty, ny0 = Real(1) - gp.ty;
        const Real wN[4] = {nx0 * ny0, nx1 * ny0, nx0 * ny1, nx1 * ny1};
        const Real dsM = gq.ds, dsP = has_p ? gp.ds : Real(0);

        // ---- phase 1: local reverse step at every point of the strip ----
        int pl = tl0, pc = tc0;
        for (int p = tid; p < npts; p += nt, step(pl, pc)) {
            const int l = pl, c = pc;
            const int c1 = c + 1 == nx ? 0 : c + 1;
            const int cm = c == 0 ? nx - 1 : c - 1;
            const Node<Real, NS> nO = ring_load<Real, NS>(ring, plane, chunk, sO, (l + 1) * nx + c);
            // ring positions of the upwind (plane q-1) and downwind (plane q+1)
            // stencil corners; their node data are read again for every frequency
            // (shared-memory loads instead of ~50 live registers across the loop)
            const int rM[4] = {(l + 1) * nx + c, (l + 1) * nx + c1, (l + 2) * nx + c, (l + 2) * nx + c1};
            const int rP[4] = {l * nx + cm, l * nx + c, (l + 1) * nx + cm, (l + 1) * nx + c};
            const long long vO = voxel(gq, c, l);
            // form 2: dL/dI_p per unit J weight at O, sum_KQ T^K_Q(p, Omega) dL/dJ^K_Q, and dL/dLambda*
            Real gdir[3] = {0, 0, 0}, gLv = 0;
            if constexpr (FORM == 2) {
                const Real *gj = a.gjkq + (B.vox0 + vO) * (NS == 1 ? 1 : 6);
                if constexpr (NS == 1) {
                    gdir[0] = gj[0];
                } else {
#pragma unroll
                    for (int s = 0; s < 3; ++s) {
                        Real acc_s = 0;
#pragma unroll
                        for (int c6 = 0; c6 < 6; ++c6) acc_s += ray.t[6 * s + c6] * gj[c6];
                        gdir[s] = acc_s;
                    }
                }
                gLv = a.glstar[B.vox0 + vO];
            }
            // rows of the Stokes-adjoint gather from plane q+1: (c|c-1, l|l-1)
            const bool first = l == 0;
            const Real *glo = first ? gI_prev : gI;
            const int llo = first ? prev_last * nx : (l - 1) * nx;

            for (int f = 0; f < nf; ++f) {
                const int j = j0 + f;
                const Real x = xsh[f];
                Real lam[NS];
                if (q == nz - 1) {
                    if constexpr (FORM == 2) {
#pragma unroll
                        for (int s = 0; s < NS; ++s) lam[s] = Real(0);
                    } else {
                        const double *go = a.gout + (((long long)d * a.nnu + j) * nxy + (vO - (long long)gq.kz * nxy)) * NS;
#pragma unroll
                        for (int s = 0; s < NS; ++s) lam[s] = (Real)go[s];
                    }
                } else {
                    Real u0[NS], u1[NS], u2[NS], u3[NS];
                    VI::load(gI + oI(opar, f), ipa, l * nx + c, u0);
                    VI::load(gI + oI(opar, f), ipa, l * nx + cm, u1);
                    VI::load(glo + oI(opar, f), ipa, llo + c, u2);
                    VI::load(glo + oI(opar, f), ipa, llo + cm, u3);
#pragma unroll
                    for (int s = 0; s < NS; ++s) lam[s] = wN[0] * u0[s] + wN[1] * u1[s] + wN[2] * u2[s] + wN[3] * u3[s];
                }
                // ---- forward recomputation (the forward sweep's arithmetic) ----
                // upwind Stokes vector from the staged tape rows l, l+1 of plane q-1
                Real IM[NS];
                {
                    const Real *tf = tt + (long long)f * tile_pts * NS;
                    Real t0[NS], t1[NS], t2[NS], t3[NS];
                    load_stokes<Real, NS>(tf + (l * nx + c) * NS, t0);
                    load_stokes<Real, NS>(tf + (l * nx + c1) * NS, t1);
                    load_stokes<Real, NS>(tf + ((l + 1) * nx + c) * NS, t2);
                    load_stokes<Real, NS>(tf + ((l + 1) * nx + c1) * NS, t3);
#pragma unroll
                    for (int s = 0; s < NS; ++s) IM[s] = wM[0] * t0[s] + wM[1] * t1[s] + wM[2] * t2[s] + wM[3] * t3[s];
                }
                Real etaM = 0, etaVM = 0, epsM[NS];
#pragma unroll
                for (int s = 0; s < NS; ++s) epsM[s] = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const CornerM<Real, NS> km = corner_m<Real, NS>(ring_load<Real, NS>(ring, plane, chunk, sM, rM[k]), wM[k]);
                    const Real xs = x - km.s;
                    const Real we = km.wchi * profile_shape(xs);
                    etaM += we;
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
                    for (int k = 0; k < 4; ++k) {
                        const CornerP<Real, NS> kp =
                            corner_p<Real, NS>(ring_load<Real, NS>(ring, plane, chunk, sP, rP[k]), wP[k]);
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
                        }
                    }
                }
                const Real xsO = x - nO.s;
                const Real phO = profile_shape(xsO);
                const Real etaO = nO.chi * phO;
                Real SO[NS], SM[NS], SP[NS];
                const Real iM = rcp(etaM), iO = rcp(etaO);
                if constexpr (NS == 1) {
                    SO[0] = nO.S;
                } else {
                    SO[0] = nO.SI; SO[1] = nO.SQ; SO[2] = nO.SU; SO[3] = nO.b * xsO * nO.S00;
                }
#pragma unroll
                for (int s = 0; s < NS; ++s) SM[s] = epsM[s] * iM;
                const Real tMO = Real(0.5) * (etaM + etaO) * dsM;
                Real tOP = Real(1), iP = Real(0);
                if (has_p) {
                    iP = rcp(etaP);
#pragma unroll
                    for (int s = 0; s < NS; ++s) SP[s] = epsP[s] * iP;
                    tOP = Real(0.5) * (etaO + etaP) * dsP;
                } else {
#pragma unroll
                    for (int s = 0; s < NS; ++s) SP[s] = Real(0);
                }
                const Coef<Real> co = coefficients(tMO);
                // control points exactly as the forward sweep computes them; their
                // partial derivatives are formed per Stokes parameter where used
                BesserGrad<Real> bg{};
                int branches = 0;                  // control-point branch per Stokes parameter, 2 bits each
                Real cM[NS];
                if (has_p) {
                    bg = besser_grad(tMO, tOP);
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        int br;
                        cM[s] = control_point_branch(SM[s], SO[s], SP[s], bg.g, br);
                        branches |= br << (2 * s);
                    }
                } else {
#pragma unroll
                    for (int s = 0; s < NS; ++s) cM[s] = Real(0.5) * (SM[s] + SO[s]);
                }
                // form 2: the J^K_Q and Lambda-bar* sums weigh I_O and Lambda*_O by w_m w_j phi_O / N
                Real lw = 0;
                if constexpr (FORM == 2) {
                    const Real wt = wray * xsh[F + f] * phO * nO.invn;
                    lam[0] += wt * gdir[0];
                    if constexpr (NS == 4) {
                        lam[1] += wt * gdir[1];
                        lam[2] += wt * gdir[2];
                    }
                    lw = wt * gLv;
                }
                // ---- reverse step ----
                Real gr[NS], g_pm = 0, g_po = 0, g_kvM = 0, g_kvO = 0, kvM = 0, kvO = 0;
                if constexpr (NS == 1) {
                    gr[0] = lam[0];
                } else {
                    // I_O = kappa (rhs) with kappa^-1 = 1 + psi'_O K'_O coupling I and V
                    kvM = etaVM * iM;
                    kvO = nO.b * xsO;
                    Real rr[4];
#pragma unroll
                    for (int s = 0; s < 4; ++s) rr[s] = co.e * IM[s] + co.wm * SM[s] + co.wo * SO[s] + co.wc * cM[s];
                    rr[0] -= co.pm * kvM * IM[3];
                    rr[3] -= co.pm * kvM * IM[0];
                    const Real av = co.po * kvO;
                    const Real idet = rcp(Real(1) - av * av);
                    const Real IO0 = (rr[0] - av * rr[3]) * idet, IO3 = (rr[3] - av * rr[0]) * idet;
                    gr[0] = (lam[0] - av * lam[3]) * idet;
                    gr[3] = (lam[3] - av * lam[0]) * idet;
                    gr[1] = lam[1];
                    gr[2] = lam[2];
                    const Real ga = (lam[0] * (Real(2) * av * IO0 - rr[3]) + lam[3] * (Real(2) * av * IO3 - rr[0])) * idet;
                    g_po = ga * kvO;
                    g_kvO = ga * co.po;
                    const Real cr = gr[0] * IM[3] + gr[3] * IM[0];
                    g_pm = -kvM * cr;
                    g_kvM = -co.pm * cr;
                }
                Real g_e = 0, g_wm = 0, g_wo = 0, g_wc = 0, g_tM = 0, g_tP = 0;
                Real gIM[NS], gSM[NS], gSO[NS], gSP[NS];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    g_e += gr[s] * IM[s];
                    g_wm += gr[s] * SM[s];
                    g_wo += gr[s] * SO[s];
                    g_wc += gr[s] * cM[s];
                    gIM[s] = gr[s] * co.e;
                    const Real gc = gr[s] * co.wc;
                    CpGrad<Real> cp{Real(0.5), Real(0.5), Real(0), Real(0), Real(0)};
                    if (has_p) cp = control_point_grad((branches >> (2 * s)) & 3, SM[s], SO[s], SP[s], bg);
                    gSM[s] = gr[s] * co.wm + gc * cp.dyM;
                    gSO[s] = gr[s] * co.wo + gc * cp.dyO;
                    gSP[s] = gc * cp.dyP;
                    g_tM += gc * cp.dhM;
                    g_tP += gc * cp.dhP;
                }
                if constexpr (NS == 4) {
                    gIM[3] -= gr[0] * co.pm * kvM;
                    gIM[0] -= gr[3] * co.pm * kvM;
                }
                const CoefD<Real> cd = coefficient_derivs(tMO, co);
                g_tM += g_e * cd.de + g_pm * cd.dpm + g_po * cd.dpo + g_wm * cd.dwm + g_wo * cd.dwo + g_wc * cd.dwc;
                if constexpr (FORM == 2)   // Lambda* = w_O + w_C (w_C/2 on the last plane)
                    g_tM += lw * (cd.dwo + (has_p ? Real(1) : Real(0.5)) * cd.dwc);
                Real g_etaM = Real(0.5) * dsM * g_tM;
                Real g_etaO = Real(0.5) * dsM * g_tM + Real(0.5) * dsP * g_tP;
                Real g_etaP = Real(0.5) * dsP * g_tP;
                Real gout_m[NM], gout_o[NM], gout_p[NP];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    gout_m[NM - NS + s] = gSM[s] * iM;
                    g_etaM -= gSM[s] * SM[s] * iM;
                    gout_o[NM - NS + s] = gSO[s] * iO;
                    g_etaO -= gSO[s] * SO[s] * iO;
                    gout_p[1 + s] = gSP[s] * iP;
                    g_etaP -= gSP[s] * SP[s] * iP;
                }
                if constexpr (NS == 4) {
                    gout_m[1] = g_kvM * iM;
                    g_etaM -= g_kvM * kvM * iM;
                    gout_o[1] = g_kvO * iO;
                    g_etaO -= g_kvO * kvO * iO;
                }
                gout_m[0] = g_etaM;
                gout_o[0] = g_etaO;
                gout_p[0] = g_etaP;
                VI::store(gI + oI(par, f), ipa, p, gIM);
                VM::store(gM + oM(f), ipa, p, gout_m);
                VP::store(gP + oP(f), ipa, p, gout_p);
                {
                    Real t[NM];
                    VM::load(T + oT(par, f), ipa, p, t);
#pragma unroll
                    for (int k = 0; k < NM; ++k) t[k] += gout_o[k];
                    VM::store(T + oT(par, f), ipa, p, t);
                }
            }
        }
        // phase 1 -> phase 2: the strip's gI, gM, gP are published to the
        // neighbours (release); the rows that need none of the neighbours'
        // values are completed while the barrier is pending
        __syncthreads();
        cluster_arrive_release();

        // ---- phase 2: complete node adjoints ----
        // (a) plane q+1 is complete once the P gathers of plane q are added;
        //     its last row gathers row 0 of the next strip
        // (b) the M gathers of plane q start the totals of plane q-1 (same
        //     buffer and element as (a), read there before written here by the
        //     same thread); row 0 gathers the last row of the previous strip,
        //     and the last row waits for its own (a)
        auto phase2 = [&](bool remote) {
            int l = tl0, c = tc0;
            for (int p = tid; p < npts; p += nt) {
                const bool firstrow = l == 0, lastrow = l + 1 == R;
                if (has_p && lastrow == remote) finalize_pt(gp, sP, opar, true, wP, p, l, c);
                if ((firstrow || lastrow) == remote) {
                    const int cm = c == 0 ? nx - 1 : c - 1;
                    const Real *mlo = firstrow ? gM_prev : gM;
                    const int llo = firstrow ? prev_last * nx : (l - 1) * nx;
                    for (int f = 0; f < nf; ++f) {
                        Real u0[NM], u1[NM], u2[NM], u3[NM], t[NM];
                        VM::load(gM + oM(f), ipa, l * nx + c, u0);
                        VM::load(gM + oM(f), ipa, l * nx + cm, u1);
                        VM::load(mlo + oM(f), ipa, llo + c, u2);
                        VM::load(mlo + oM(f), ipa, llo + cm, u3);
#pragma unroll
                        for (int k = 0; k < NM; ++k) t[k] = wM[0] * u0[k] + wM[1] * u1[k] + wM[2] * u2[k] + wM[3] * u3[k];
                        VM::store(T + oT(opar, f), ipa, p, t);
                    }
                }
                step(l, c);
            }
        };
        phase2(false);
        cluster_wait_acquire();
        phase2(true);
        // (c) the boundary plane has no O or P terms: complete now
        if (q == 1) finalize(0, sM, opar, false, wP);
        // end of step: the DSMEM gathers of phase 2 have been consumed, so this
        // barrier only orders them before the next phase 1 overwrites gM and gP
        // (write after read): no release fence needed
        __syncthreads();
        cluster_arrive_relaxed();
        if (q - 2 >= 0) {
            const PlaneGeom<Real> g2 = G[q - 2];
            stage(g2);           // tape rows for step q-1, in flight during the refill and the barrier
            fill(q - 2, g2);
        }
        cp_async_wait_all();
        __syncthreads();
        cluster_wait_acquire();
    }
    // plane 1: no P terms (plane 0 is not swept)
    finalize(1, 1, 1, false, nullptr);
    __syncthreads();
}

template <typename Real, int NS, int FORM>
__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? 2 : 1) adjoint_kernel(const SweepArgs<Real> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NM = adj_nm<NS>(), NP = adj_np<NS>();
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int cid = blockIdx.x / C;
    const int ncl = gridDim.x / C;
    using V = typename V16<Real>::T;
    V *ring = reinterpret_cast<V *>(smem_raw);
    const int ipa = adj_ipa(a.ipts_max);
    Real *gI = reinterpret_cast<Real *>(ring + 3 * a.ring_plane);
    Real *gM = gI + 2 * a.F * NS * ipa;
    Real *gP = gM + a.F * NM * ipa;
    Real *T = gP + a.F * NP * ipa;
    Real *tt = reinterpret_cast<Real *>(smem_raw + adjoint_tile_offset<Real, NS>(a.ring_plane, a.ipts_max, a.F));
    cluster.sync();
    for (int item = cid; item < a.nitems; item += ncl) {
        const int d = item / a.ngroups, g = item - d * a.ngroups;
        adjoint_item<Real, NS, FORM>(a, cluster, ring, gI, gM, gP, T, tt, d, g, rank, C, item, cid);
        cluster.sync();
    }
}

// dL/dchi, dL/de, dL/dB of every voxel: the per-item partials summed in item order
template <typename Real>
__global__ void adjoint_reduce_kernel(const Real *gpart, int nitems, int ngroups, long long nvox,
                                      const RayDev<Real> *rays, double bfac, double *g_chi, double *g_e, double *g_b)
{
    const int ndir = nitems / ngroups;
    if constexpr (sizeof(Real) == 4) {
        // FP32 partials: compensated FP32 sums in the same order (no FP64 arithmetic,
        // which this GPU runs at a small fraction of the FP32 rate)
        auto kadd = [](float &s, float &c, float x) {
            const float y = x - c, t = s + y;
            c = (t - s) - y;
            s = t;
        };
        for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
            float sc = 0, cc = 0, se = 0, ce = 0, bx = 0, cx = 0, by = 0, cy = 0, bz = 0, cz = 0;
            for (int d = 0; d < ndir; ++d) {
                const Real *p0 = gpart + (long long)d * ngroups * 3 * nvox;
                float gb = 0, cb = 0;
#pragma unroll 4
                for (int g = 0; g < ngroups; ++g) {
                    const Real *p = p0 + (long long)g * 3 * nvox;
                    kadd(sc, cc, p[v]);
                    kadd(se, ce, p[nvox + v]);
                    kadd(gb, cb, p[2 * nvox + v]);
                }
                const RayDev<Real> &r = rays[d];
                kadd(bx, cx, gb * r.ox);
                kadd(by, cy, gb * r.oy);
                kadd(bz, cz, gb * r.oz);
            }
            g_chi[v] = sc;
            g_e[v] = se;
            if (g_b) {
                g_b[v] = bfac * bx;
                g_b[nvox + v] = bfac * by;
                g_b[2 * nvox + v] = bfac * bz;
            }
        }
        return;
    }
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        double sc = 0, se = 0, bx = 0, by = 0, bz = 0;
        // directions in order, the groups of a direction in order (loads of
        // several items in flight; the sums keep this fixed order)
        for (int d = 0; d < ndir; ++d) {
            const Real *p0 = gpart + (long long)d * ngroups * 3 * nvox;
            double gb = 0;
#pragma unroll 4
            for (int g = 0; g < ngroups; ++g) {
                const Real *p = p0 + (long long)g * 3 * nvox;
                sc += (double)p[v];
                se += (double)p[nvox + v];
                gb += (double)p[2 * nvox + v];
            }
            const RayDev<Real> &r = rays[d];
            bx += gb * (double)r.ox;
            by += gb * (double)r.oy;
            bz += gb * (double)r.oz;
        }
        g_chi[v] = sc;
        g_e[v] = se;
        if (g_b) {
            g_b[v] = bfac * bx;
            g_b[nvox + v] = bfac * by;
            g_b[2 * nvox + v] = bfac * bz;
        }
    }
}

template <typename Real, int NS>
static void *adjoint_ptr(int form)
{
    return form == 0 ? (void *)adjoint_kernel<Real, NS, 0>
                     : (form == 1 ? (void *)adjoint_kernel<Real, NS, 1> : (void *)adjoint_kernel<Real, NS, 2>);
}

template <typename Real, int NS>
static cudaError_t prepare_adjoint(int cluster, int smem, int form)
{
    const void *k = adjoint_ptr<Real, NS>(form);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (cluster > 8) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <typename Real, int NS>
cudaError_t adjoint_max_active_clusters(int cluster, int smem, int threads, int *out, int form)
{
    cudaError_t e = prepare_adjoint<Real, NS>(cluster, smem, form);
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
    return cudaOccupancyMaxActiveClusters(out, adjoint_ptr<Real, NS>(form), &lc);
}

template <typename Real, int NS>
cudaError_t launch_adjoint(const SweepArgs<Real> &a, const LaunchCfg &cfg, cudaStream_t st, int form)
{
    cudaError_t e = prepare_adjoint<Real, NS>(cfg.cluster, cfg.smem, form);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cfg.clusters * cfg.cluster);
    lc.blockDim = dim3(cfg.threads);
    lc.dynamicSmemBytes = cfg.smem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cfg.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    if (form == 0) return cudaLaunchKernelEx(&lc, adjoint_kernel<Real, NS, 0>, a);
    if (form == 1) return cudaLaunchKernelEx(&lc, adjoint_kernel<Real, NS, 1>, a);
    return cudaLaunchKernelEx(&lc, adjoint_kernel<Real, NS, 2>, a);
}

// per voxel: sum of the per-cluster accumulators in cluster order (FP64)
template <typename Real>
__global__ void adjoint_acc_reduce_kernel(const Real *gacc, int nclusters, long long nvox, int nl, double *g_chi,
                                          double *g_b, double *g_rho)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        double s[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int cl = 0; cl < nclusters; ++cl) {
            const Real *p = gacc + (long long)cl * 10 * nvox + v;
#pragma unroll
            for (int k = 0; k < 10; ++k) s[k] += (double)p[k * nvox];
        }
        g_chi[v] += s[0];
        if (g_b) {
            g_b[v] += s[1];
            g_b[nvox + v] += s[2];
            g_b[2 * nvox + v] += s[3];
        }
        for (int c = 0; c < nl; ++c) g_rho[v * nl + c] = s[4 + c];
    }
}

template <typename Real>
cudaError_t launch_adjoint_acc_reduce(const Real *gacc, int nclusters, long long nvox, int nl, double *g_chi,
                                      double *g_b, double *g_rho, cudaStream_t st)
{
    const int threads = 256;
    const long long blocks = std::min<long long>((nvox + threads - 1) / threads, 152LL * 16);
    adjoint_acc_reduce_kernel<Real><<<(int)blocks, threads, 0, st>>>(gacc, nclusters, nvox, nl, g_chi, g_b, g_rho);
    return cudaGetLastError();
}
template cudaError_t launch_adjoint_acc_reduce<float>(const float *, int, long long, int, double *, double *, double *,
                                                      cudaStream_t);
template cudaError_t launch_adjoint_acc_reduce<double>(const double *, int, long long, int, double *, double *, double *,
                                                       cudaStream_t);

template <typename Real>
cudaError_t launch_adjoint_reduce(const Real *gpart, int nitems, int ngroups, long long nvox, const RayDev<Real> *rays,
                                  double bfac, double *g_chi, double *g_e, double *g_b, cudaStream_t st)
{
    const int threads = 256;
    const long long blocks = std::min<long long>((nvox + threads - 1) / threads, 152LL * 16);
    adjoint_reduce_kernel<Real><<<(int)blocks, threads, 0, st>>>(gpart, nitems, ngroups, nvox, rays, bfac, g_chi, g_e, g_b);
    return cudaGetLastError();
}

#define PORTA_ADJ_INST(R, N)                                                                        \
    template int adjoint_smem_bytes<R, N>(int, int, int, int);                                      \
    template cudaError_t adjoint_max_active_clusters<R, N>(int, int, int, int *, int);              \
    template cudaError_t launch_adjoint<R, N>(const SweepArgs<R> &, const LaunchCfg &, cudaStream_t, int);
PORTA_ADJ_INST(float, 1)
PORTA_ADJ_INST(float, 4)
PORTA_ADJ_INST(double, 1)
PORTA_ADJ_INST(double, 4)
#undef PORTA_ADJ_INST
template cudaError_t launch_adjoint_reduce<float>(const float *, int, int, long long, const RayDev<float> *, double,
                                                  double *, double *, double *, cudaStream_t);
template cudaError_t launch_adjoint_reduce<double>(const double *, int, int, long long, const RayDev<double> *, double,
                                                   double *, double *, double *, cudaStream_t);

}  // namespace porta
