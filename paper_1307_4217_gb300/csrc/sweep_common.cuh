// Device pieces shared by the forward sweep (sweep.cu) and its adjoint
// (adjoint.cu): per-node data of the sheared-frame ring buffers in shared
// memory, the Stokes-plane chunk layout, the profile shape, the per-node
// transfer data and the split cluster barrier.
#pragma once
#include "device_math.cuh"
#include "porta_internal.cuh"

namespace porta {

template <int NS>
__host__ __device__ constexpr int node_words() { return NS == 1 ? 4 : 8; }

template <typename Real>
struct alignas(4 * sizeof(Real)) R4 { Real x, y, z, w; };
template <typename Real>
struct alignas(2 * sizeof(Real)) R2 { Real x, y; };

// 16-byte vector of the shared-memory layouts: all ring and Stokes planes are
// stored as planes of 16-byte chunks, [chunk][row][col], so that consecutive
// threads (consecutive columns) read consecutive 16-byte words (no bank conflicts).
template <typename Real> struct V16;
template <> struct V16<float> { using T = float4; };
template <> struct V16<double> { using T = double2; };

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
__device__ __forceinline__ Node<Real, NS> unpack_node(const Real *w)
{
    Node<Real, NS> n;
    if constexpr (NS == 1) {
        n.chi = w[0]; n.s = w[1]; n.S = w[2]; n.invn = w[3];
    } else {
        n.chi = w[0]; n.s = w[1]; n.b = w[2]; n.SI = w[3];
        n.SQ = w[4]; n.SU = w[5]; n.S00 = w[6]; n.invn = w[7];
    }
    return n;
}

template <typename Real, int NS>
__device__ __forceinline__ Node<Real, NS> ring_load(const typename V16<Real>::T *ring, int plane_stride,
                                                    int chunk_stride, int slot, int idx)
{
    constexpr int NW = node_words<NS>();
    constexpr int NCH = NW * (int)sizeof(Real) / 16;
    constexpr int PER = 16 / (int)sizeof(Real);
    Real w[NW];
    const typename V16<Real>::T *p = ring + slot * plane_stride + idx;
#pragma unroll
    for (int h = 0; h < NCH; ++h) {
        typename V16<Real>::T v = p[h * chunk_stride];
        if constexpr (PER == 4) {
            w[4 * h] = v.x; w[4 * h + 1] = v.y; w[4 * h + 2] = v.z; w[4 * h + 3] = v.w;
        } else {
            w[2 * h] = v.x; w[2 * h + 1] = v.y;
        }
    }
    return unpack_node<Real, NS>(w);
}

template <typename Real, int NS>
__device__ __forceinline__ void ring_store(typename V16<Real>::T *ring, int plane_stride, int chunk_stride, int slot,
                                           int idx, const Node<Real, NS> &n)
{
    constexpr int NW = node_words<NS>();
    constexpr int NCH = NW * (int)sizeof(Real) / 16;
    constexpr int PER = 16 / (int)sizeof(Real);
    Real w[NW];
    if constexpr (NS == 1) {
        w[0] = n.chi; w[1] = n.s; w[2] = n.S; w[3] = n.invn;
    } else {
        w[0] = n.chi; w[1] = n.s; w[2] = n.b; w[3] = n.SI; w[4] = n.SQ; w[5] = n.SU; w[6] = n.S00; w[7] = n.invn;
    }
    typename V16<Real>::T *p = ring + slot * plane_stride + idx;
#pragma unroll
    for (int h = 0; h < NCH; ++h) {
        typename V16<Real>::T v;
        if constexpr (PER == 4) {
            v.x = w[4 * h]; v.y = w[4 * h + 1]; v.z = w[4 * h + 2]; v.w = w[4 * h + 3];
        } else {
            v.x = w[2 * h]; v.y = w[2 * h + 1];
        }
        p[h * chunk_stride] = v;
    }
}

// Stokes-vector planes: NS = 4 as 16-byte chunk planes ([chunk][row][col]);
// NS = 1 as a plane of scalars.
template <typename Real, int NS>
struct StokesIO {
    static constexpr int ICH = NS == 1 ? 1 : 4 * (int)sizeof(Real) / 16;
    // element offset (in units of Real) of chunk 0 of point idx in plane (buf, f)
    __device__ static __forceinline__ void load(const Real *plane, int chunk_stride, int idx, Real v[NS])
    {
        if constexpr (NS == 1) {
            v[0] = plane[idx];
        } else if constexpr (sizeof(Real) == 4) {
            float4 a = reinterpret_cast<const float4 *>(plane)[idx];
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        } else {
            const double2 *p = reinterpret_cast<const double2 *>(plane);
            double2 a = p[idx], b = p[idx + chunk_stride];
            v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
        }
    }
    __device__ static __forceinline__ void store(Real *plane, int chunk_stride, int idx, const Real v[NS])
    {
        if constexpr (NS == 1) {
            plane[idx] = v[0];
        } else if constexpr (sizeof(Real) == 4) {
            reinterpret_cast<float4 *>(plane)[idx] = make_float4(v[0], v[1], v[2], v[3]);
        } else {
            double2 *p = reinterpret_cast<double2 *>(plane);
            p[idx] = make_double2(v[0], v[1]);
            p[idx + chunk_stride] = make_double2(v[2], v[3]);
        }
    }
    // Reals per (buf, f) plane
    __host__ __device__ static constexpr int plane_reals(int pts) { return NS * pts; }
};


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


// frequency-independent data of an interpolation corner, with the bilinear
// weight folded into the opacity: upwind corners keep b and S^0_0 separately
// (eta_V and eps_V are both interpolated), downwind corners only their product.
template <typename Real, int NS> struct CornerM;
template <typename Real> struct CornerM<Real, 1> { Real wchi, s, S; };
template <typename Real> struct CornerM<Real, 4> { Real wchi, s, b, SI, SQ, SU, S00; };
template <typename Real, int NS> struct CornerP;
template <typename Real> struct CornerP<Real, 1> { Real wchi, s, S; };
template <typename Real> struct CornerP<Real, 4> { Real wchi, s, bS, SI, SQ, SU; };

template <typename Real, int NS>
__device__ __forceinline__ CornerM<Real, NS> corner_m(const Node<Real, NS> &n, Real w)
{
    CornerM<Real, NS> c;
    c.wchi = w * n.chi;
    c.s = n.s;
    if constexpr (NS == 1) {
        c.S = n.S;
    } else {
        c.b = n.b; c.SI = n.SI; c.SQ = n.SQ; c.SU = n.SU; c.S00 = n.S00;
    }
    return c;
}

template <typename Real, int NS>
__device__ __forceinline__ CornerP<Real, NS> corner_p(const Node<Real, NS> &n, Real w)
{
    CornerP<Real, NS> c;
    c.wchi = w * n.chi;
    c.s = n.s;
    if constexpr (NS == 1) {
        c.S = n.S;
    } else {
        c.bS = n.b * n.S00; c.SI = n.SI; c.SQ = n.SQ; c.SU = n.SU;
    }
    return c;
}

// split cluster barrier (PTX barrier.cluster): arrive with release semantics,
// wait with acquire semantics; all threads of all CTAs of the cluster take part
__device__ __forceinline__ void cluster_arrive_release()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
// arrive without release semantics: for a barrier that only orders reads of
// other CTAs' shared memory (values already consumed) before later writes
__device__ __forceinline__ void cluster_arrive_relaxed()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire()
{
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

}  // namespace porta
