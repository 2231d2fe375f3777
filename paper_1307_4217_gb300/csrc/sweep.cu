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
// Shared memory per CTA:
//   ring[3][rows+2][nx][NW]   frequency-independent node data of planes q-1, q, q+1
//                             (own rows plus one halo row on each side, recomputed
//                             locally from global memory);
//   ibuf[2][F][rows][nx][NS]  Stokes vectors of planes q-1 and q for F frequencies.
// Each thread owns points of its strip and loops over the F frequencies of the
// pass, reusing the ring data of its 9 stencil nodes, and accumulates the
// frequency-integrated Stokes I, Q, U and Lambda* of its point in registers;
// one store (or read-modify-write for later frequency passes) per point and
// plane writes the per-ray partial integrals.
#include <cooperative_groups.h>

#include "device_math.cuh"
#include "porta_internal.cuh"

namespace cg = cooperative_groups;

namespace porta {

template <int NS>
__host__ __device__ constexpr int node_words() { return NS == 1 ? 4 : 8; }

template <typename Real, int NS>
int sweep_smem_bytes(int nx, int rmax, int F)
{
    return (3 * (rmax + 2) * nx * node_words<NS>() + 2 * F * rmax * nx * NS) * (int)sizeof(Real);
}

template <typename Real>
struct alignas(4 * sizeof(Real)) R4 { Real x, y, z, w; };
template <typename Real>
struct alignas(2 * sizeof(Real)) R2 { Real x, y; };

// ---- node data: chi, s (Doppler shift along the ray), [b = 2 gbar zeta B.Omega],
//      S_I, [S_Q, S_U, S^0_0], invN (profile normalization) -------------------
template <typename Real, int NS>
struct Node;

template <typename Real>
struct Node<Real, 1> {
    Real chi, s, S, invn;
};
template <typename Real>
struct Node<Real, 4> {
    Real chi, s, b, SI, SQ, SU, S00, invn;
};

template <typename Real, int NS>
__device__ __forceinline__ Node<Real, NS> load_node(const Real *p)
{
    Node<Real, NS> n;
    if constexpr (sizeof(Real) == 4) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
        float4 a = q[0];
        if constexpr (NS == 1) {
            n.chi = a.x; n.s = a.y; n.S = a.z; n.invn = a.w;
        } else {
            float4 b = q[1];
            n.chi = a.x; n.s = a.y; n.b = a.z; n.SI = a.w;
            n.SQ = b.x; n.SU = b.y; n.S00 = b.z; n.invn = b.w;
        }
    } else {
        const double2 *q = reinterpret_cast<const double2 *>(p);
        double2 a = q[0], b = q[1];
        if constexpr (NS == 1) {
            n.chi = a.x; n.s = a.y; n.S = b.x; n.invn = b.y;
        } else {
            double2 c = q[2], d = q[3];
            n.chi = a.x; n.s = a.y; n.b = b.x; n.SI = b.y;
            n.SQ = c.x; n.SU = c.y; n.S00 = d.x; n.invn = d.y;
        }
    }
    return n;
}

template <typename Real, int NS>
__device__ __forceinline__ void store_node(Real *p, const Node<Real, NS> &n)
{
    if constexpr (sizeof(Real) == 4) {
        float4 *q = reinterpret_cast<float4 *>(p);
        if constexpr (NS == 1) {
            q[0] = make_float4(n.chi, n.s, n.S, n.invn);
        } else {
            q[0] = make_float4(n.chi, n.s, n.b, n.SI);
            q[1] = make_float4(n.SQ, n.SU, n.S00, n.invn);
        }
    } else {
        double2 *q = reinterpret_cast<double2 *>(p);
        if constexpr (NS == 1) {
            q[0] = make_double2(n.chi, n.s);
            q[1] = make_double2(n.S, n.invn);
        } else {
            q[0] = make_double2(n.chi, n.s);
            q[1] = make_double2(n.b, n.SI);
            q[2] = make_double2(n.SQ, n.SU);
            q[3] = make_double2(n.S00, n.invn);
        }
    }
}

template <typename Real, int NS>
__device__ __forceinline__ void load_stokes(const Real *p, Real v[NS])
{
    if constexpr (NS == 1) {
        v[0] = p[0];
    } else if constexpr (sizeof(Real) == 4) {
        float4 a = *reinterpret_cast<const float4 *>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else {
        double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
}

template <typename Real, int NS>
__device__ __forceinline__ void store_stokes(Real *p, const Real v[NS])
{
    if constexpr (NS == 1) {
        p[0] = v[0];
    } else if constexpr (sizeof(Real) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
}

// Profile shape exp(-(x - s)^2). In FP32 the exponent is capped at 80 so that
// eta_I = chi * shape stays a nonzero (possibly subnormal) number far in the
// wings instead of underflowing to zero; the capped terms are below 2e-35
// relative to line centre.
__device__ __forceinline__ float profile_shape(float xs) { return expf(-fminf(xs * xs, 80.0f)); }
__device__ __forceinline__ double profile_shape(double xs) { return exp(-xs * xs); }

// ---- the per-ray, per-plane node data (a2: frequency-independent part) ----
template <typename Real, int NS>
__device__ __forceinline__ Node<Real, NS> make_node(const SweepArgs<Real> &a, const RayDev<Real> &ray,
                                                    long long v, int m, bool with_norm)
{
    Node<Real, NS> n;
    n.chi = a.chi[v];
    n.s = a.vel[v] * ray.mu;
    n.invn = with_norm ? a.invn[(long long)m * a.nvox + v] : Real(1);
    if constexpr (NS == 1) {
        n.S = a.rho[v];
    } else {
        const long long nv = a.nvox;
        Real s00 = a.rho[v], s20 = a.rho[nv + v], s21r = a.rho[2 * nv + v], s21i = a.rho[3 * nv + v];
        Real s22r = a.rho[4 * nv + v], s22i = a.rho[5 * nv + v];
        n.b = a.bfac * (a.bx[v] * ray.ox + a.by[v] * ray.oy + a.bz[v] * ray.oz);
        // S_i(Omega) = sum_KQ (-1)^Q T^K_Q(i, Omega) S^K_{-Q} (Eq. 1 tensors, two-level emissivity)
        Real S[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const Real *t = ray.t + 6 * i;
            S[i] = t[0] * s00 + t[1] * s20 + Real(2) * (t[2] * s21r + t[3] * s21i) +
                   Real(2) * (t[4] * s22r + t[5] * s22i);
        }
        n.SI = S[0]; n.SQ = S[1]; n.SU = S[2]; n.S00 = s00;
    }
    return n;
}

__device__ __forceinline__ int wrapi(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

template <typename Real, int NS, int MODE>
__device__ __forceinline__ void sweep_item(const SweepArgs<Real> &a, cg::cluster_group &cluster, Real *ring,
                                           Real *ibuf, Real *ibuf_next, int m, int g, int row0, int R, int dir_out)
{
    constexpr int NW = node_words<NS>();
    const int nx = a.nx, ny = a.ny, nz = a.nz, F = a.F, rmax = a.rmax;
    const int j0 = g * F;
    const int nf = min(F, a.nnu - j0);
    const PlaneGeom<Real> *G = a.geom + (long long)m * nz;
    const RayDev<Real> ray = a.rays[m];
    const bool upward = ray.mu > Real(0);
    const long long nxy = (long long)nx * ny;
    const bool jmode = (MODE == MODE_JKQ);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ring_plane = (rmax + 2) * nx * NW;
    const int npts = R * nx;

    auto fill = [&](int q) {
        const PlaneGeom<Real> gq = G[q];
        Real *slot = ring + (q % 3) * ring_plane;
        const int nn = (R + 2) * nx;
        for (int idx = tid; idx < nn; idx += nt) {
            int l = idx / nx - 1, c = idx - (idx / nx) * nx;
            int r = wrapi(row0 + l, ny);
            int pi = wrapi(c + gq.ax, nx), pj = wrapi(r + gq.ay, ny);
            long long v = ((long long)gq.kz * ny + pj) * nx + pi;
            store_node<Real, NS>(slot + ((l + 1) * nx + c) * NW, make_node<Real, NS>(a, ray, v, m, jmode));
        }
    };

    fill(0);
    for (int q = 0; q < nz; ++q) {
        if (q + 1 < nz) fill(q + 1);
        __syncthreads();
        const PlaneGeom<Real> gq = G[q];
        const bool has_p = q + 1 < nz;
        const PlaneGeom<Real> gp = has_p ? G[q + 1] : gq;
        const Real *rM = ring + ((q + 2) % 3) * ring_plane;   // plane q-1
        const Real *rO = ring + (q % 3) * ring_plane;
        const Real *rP = ring + ((q + 1) % 3) * ring_plane;   // plane q+1
        Real *iw = ibuf + (q & 1) * F * rmax * nx * NS;        // write plane q
        const int ro = ((q + 1) & 1) * F * rmax * nx * NS;     // read plane q-1
        const Real *ir = ibuf + ro;
        const Real *irn = ibuf_next + ro;
        // interpolation weights (uniform over the plane)
        const Real mx1 = gq.tx, mx0 = Real(1) - gq.tx, my1 = gq.ty, my0 = Real(1) - gq.ty;
        const Real px0 = gp.tx, px1 = Real(1) - gp.tx, py0 = gp.ty, py1 = Real(1) - gp.ty;
        const Real wM[4] = {mx0 * my0, mx1 * my0, mx0 * my1, mx1 * my1};
        const Real wP[4] = {px0 * py0, px1 * py0, px0 * py1, px1 * py1};
        const Real dsM = gq.ds, dsP = has_p ? gp.ds : Real(0);

        for (int p = tid; p < npts; p += nt) {
            const int l = p / nx, c = p - (p / nx) * nx;
            const int pi = wrapi(c + gq.ax, nx), pj = wrapi(row0 + l + gq.ay, ny);
            const long long v = ((long long)gq.kz * ny + pj) * nx + pi;
            const Node<Real, NS> nO = load_node<Real, NS>(rO + ((l + 1) * nx + c) * NW);
            Real acc[NS == 1 ? 2 : 4];
#pragma unroll
            for (int s = 0; s < (NS == 1 ? 2 : 4); ++s) acc[s] = Real(0);

            if (q == 0) {
                // boundary plane: I = (B, 0, 0, 0) entering at the bottom, 0 at the top; Lambda* = 0
                Real I0[NS];
#pragma unroll
                for (int s = 0; s < NS; ++s) I0[s] = Real(0);
                if (upward) I0[0] = a.bpl[v];
                for (int f = 0; f < nf; ++f) {
                    const int j = j0 + f;
                    store_stokes<Real, NS>(iw + ((f * rmax + l) * nx + c) * NS, I0);
                    if constexpr (MODE == MODE_JKQ) {
                        const Real wt = a.wf[j] * profile_shape(a.xf[j] - nO.s) * nO.invn;
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
                const Node<Real, NS> nM[4] = {
                    load_node<Real, NS>(rM + ((l + 1) * nx + c) * NW), load_node<Real, NS>(rM + ((l + 1) * nx + c1) * NW),
                    load_node<Real, NS>(rM + ((l + 2) * nx + c) * NW), load_node<Real, NS>(rM + ((l + 2) * nx + c1) * NW)};
                Node<Real, NS> nP[4];
                if (has_p) {
                    nP[0] = load_node<Real, NS>(rP + (l * nx + cm) * NW);
                    nP[1] = load_node<Real, NS>(rP + (l * nx + c) * NW);
                    nP[2] = load_node<Real, NS>(rP + ((l + 1) * nx + cm) * NW);
                    nP[3] = load_node<Real, NS>(rP + ((l + 1) * nx + c) * NW);
                } else {
                    nP[0] = nP[1] = nP[2] = nP[3] = nO;
                }
                const bool last_row = (l + 1 == R);
                const Real *ir_lo = ir + (l * nx) * NS;                              // row l
                const Real *ir_hi = last_row ? irn : ir + ((l + 1) * nx) * NS;      // row l+1

                for (int f = 0; f < nf; ++f) {
                    const int j = j0 + f;
                    const Real x = a.xf[j];
                    const int fo = f * rmax * nx * NS;
                    // upwind Stokes vectors at the 4 corners
                    Real IMc[4][NS];
                    load_stokes<Real, NS>(ir_lo + fo + c * NS, IMc[0]);
                    load_stokes<Real, NS>(ir_lo + fo + c1 * NS, IMc[1]);
                    load_stokes<Real, NS>(ir_hi + fo + c * NS, IMc[2]);
                    load_stokes<Real, NS>(ir_hi + fo + c1 * NS, IMc[3]);

                    // a2-a3: node transfer coefficients and bilinear interpolation at M and P
                    Real etaM = 0, etaVM = 0, epsM[NS], IM[NS];
#pragma unroll
                    for (int s = 0; s < NS; ++s) { epsM[s] = 0; IM[s] = 0; }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const Real xs = x - nM[k].s;
                        const Real we = wM[k] * nM[k].chi * profile_shape(xs);
                        etaM += we;
#pragma unroll
                        for (int s = 0; s < NS; ++s) IM[s] += wM[k] * IMc[k][s];
                        if constexpr (NS == 1) {
                            epsM[0] += we * nM[k].S;
                        } else {
                            const Real kv = nM[k].b * xs;
                            etaVM += we * kv;
                            epsM[0] += we * nM[k].SI;
                            epsM[1] += we * nM[k].SQ;
                            epsM[2] += we * nM[k].SU;
                            epsM[3] += we * kv * nM[k].S00;
                        }
                    }
                    Real etaP = 0, epsP[NS];
#pragma unroll
                    for (int s = 0; s < NS; ++s) epsP[s] = 0;
                    if (has_p) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const Real xs = x - nP[k].s;
                            const Real we = wP[k] * nP[k].chi * profile_shape(xs);
                            etaP += we;
                            if constexpr (NS == 1) {
                                epsP[0] += we * nP[k].S;
                            } else {
                                epsP[0] += we * nP[k].SI;
                                epsP[1] += we * nP[k].SQ;
                                epsP[2] += we * nP[k].SU;
                                epsP[3] += we * nP[k].b * xs * nP[k].S00;
                            }
                        }
                    }
                    const Real xsO = x - nO.s;
                    const Real phO = profile_shape(xsO);
                    const Real etaO = nO.chi * phO;
                    Real SO[NS], SM[NS], SP[NS];
                    const Real iM = Real(1) / etaM;
                    if constexpr (NS == 1) {
                        SO[0] = nO.S;
                    } else {
                        SO[0] = nO.SI; SO[1] = nO.SQ; SO[2] = nO.SU; SO[3] = nO.b * xsO * nO.S00;
                    }
#pragma unroll
                    for (int s = 0; s < NS; ++s) SM[s] = epsM[s] * iM;
                    // a4: optical paths (trapezoid along MO and OP)
                    const Real tMO = Real(0.5) * (etaM + etaO) * dsM;
                    Real tOP = Real(1), ihP = Real(1), ihMP = Real(1);
                    if (has_p) {
                        const Real iP = Real(1) / etaP;
#pragma unroll
                        for (int s = 0; s < NS; ++s) SP[s] = epsP[s] * iP;
                        tOP = Real(0.5) * (etaO + etaP) * dsP;
                        ihP = Real(1) / tOP;
                        ihMP = Real(1) / (tMO + tOP);
                    }
                    const Real ihM = Real(1) / tMO;
                    // a6: exponential-integral coefficients
                    const Coef<Real> co = coefficients(tMO);
                    // a5: BESSER control points per Stokes parameter
                    Real cM[NS];
#pragma unroll
                    for (int s = 0; s < NS; ++s)
                        cM[s] = has_p ? control_point(SM[s], SO[s], SP[s], tMO, tOP, ihM, ihP, ihMP)
                                      : Real(0.5) * (SM[s] + SO[s]);
                    // a7: BESSER-DELO step (Eq. 7)
                    Real IO[NS];
                    if constexpr (NS == 1) {
                        IO[0] = co.e * IM[0] + co.wm * SM[0] + co.wo * SO[0] + co.wc * cM[0];
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
                        const Real idet = Real(1) / (Real(1) - av * av);
                        IO[0] = (rhs[0] - av * rhs[3]) * idet;
                        IO[3] = (rhs[3] - av * rhs[0]) * idet;
                        IO[1] = rhs[1];
                        IO[2] = rhs[2];
                    }
                    store_stokes<Real, NS>(iw + ((f * rmax + l) * nx + c) * NS, IO);
                    // a8: Lambda* (Eq. 13; w_O + w_C/2 on the last plane) and accumulation
                    if constexpr (MODE == MODE_JKQ) {
                        const Real ls = co.wo + (has_p ? co.wc : Real(0.5) * co.wc);
                        const Real wt = a.wf[j] * phO * nO.invn;
                        if constexpr (NS == 1) {
                            acc[0] += wt * IO[0];
                            acc[1] += wt * ls;
                        } else {
                            acc[0] += wt * IO[0];
                            acc[1] += wt * IO[1];
                            acc[2] += wt * IO[2];
                            acc[3] += wt * ls;
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
                    }
                }
            }
            if constexpr (MODE == MODE_JKQ) {
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
        }
        cluster.sync();
    }
}

template <typename Real, int NS, int MODE>
__global__ void __launch_bounds__(256, 1) sweep_kernel(const SweepArgs<Real> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int cid = blockIdx.x / C;
    const int ncl = gridDim.x / C;
    const int row0 = (int)(((long long)rank * a.ny) / C);
    const int row1 = (int)(((long long)(rank + 1) * a.ny) / C);
    Real *ring = reinterpret_cast<Real *>(smem_raw);
    Real *ibuf = ring + 3 * (a.rmax + 2) * a.nx * node_words<NS>();
    Real *ibuf_next = cluster.map_shared_rank(ibuf, (rank + 1) % C);
    cluster.sync();
    for (int item = cid; item < a.nitems; item += ncl) {
        if constexpr (MODE == MODE_JKQ) {
            for (int g = 0; g < a.ngroups; ++g)
                sweep_item<Real, NS, MODE>(a, cluster, ring, ibuf, ibuf_next, item, g, row0, row1 - row0, 0);
        } else {
            const int d = item / a.ngroups, g = item - d * a.ngroups;
            sweep_item<Real, NS, MODE>(a, cluster, ring, ibuf, ibuf_next, d, g, row0, row1 - row0, d);
        }
    }
}

template <typename Real, int NS>
static void *kernel_ptr(int mode)
{
    return mode == MODE_JKQ ? (void *)sweep_kernel<Real, NS, MODE_JKQ> : (void *)sweep_kernel<Real, NS, MODE_EMERGENT>;
}

template <typename Real, int NS>
static cudaError_t prepare(int mode, int cluster, int smem)
{
    void *k = kernel_ptr<Real, NS>(mode);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (cluster > 8) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <typename Real, int NS>
cudaError_t max_active_clusters(int cluster, int smem, int threads, int *out)
{
    cudaError_t e = prepare<Real, NS>(MODE_JKQ, cluster, smem);
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
    return cudaOccupancyMaxActiveClusters(out, (void (*)(SweepArgs<Real>))kernel_ptr<Real, NS>(MODE_JKQ), &lc);
}

template <typename Real, int NS>
cudaError_t launch_sweep(const SweepArgs<Real> &a, int mode, LaunchCfg &cfg, cudaStream_t st)
{
    cudaError_t e = prepare<Real, NS>(mode, cfg.cluster, cfg.smem);
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
    if (mode == MODE_JKQ)
        return cudaLaunchKernelEx(&lc, sweep_kernel<Real, NS, MODE_JKQ>, a);
    return cudaLaunchKernelEx(&lc, sweep_kernel<Real, NS, MODE_EMERGENT>, a);
}

#define PORTA_INST(R, N)                                                                           \
    template int sweep_smem_bytes<R, N>(int, int, int);                                            \
    template cudaError_t max_active_clusters<R, N>(int, int, int, int *);                          \
    template cudaError_t launch_sweep<R, N>(const SweepArgs<R> &, int, LaunchCfg &, cudaStream_t);
PORTA_INST(float, 1)
PORTA_INST(float, 4)
PORTA_INST(double, 1)
PORTA_INST(double, 4)
#undef PORTA_INST

}  // namespace porta
