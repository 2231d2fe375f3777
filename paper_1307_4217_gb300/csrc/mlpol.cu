// Polarized multilevel atom: the multipolar components rho^K_Q(J) of every
// level (K = 0 .. 2J, no interference between levels) as the unknowns of
// Eq. 2, with the radiative rates of the multilevel atom (absorption,
// spontaneous and stimulated emission, relaxation; Wigner 3j, 6j and 9j
// symbols), the Hanle term and collisions on the line transitions.
//
// Host: the rate equations are linear in a short list of per-voxel sources
// (1, the radiation tensors J^K_Q of each line, the field B, the collisional
// excitation rates, and the Lambda-bar* terms of the preconditioned population
// equations), so they are tabulated once per atom as a sparse list of
// (row, column) cells, each a sum of (source, coefficient) terms, over the
// real unknowns (Q = 0 real parts, Q > 0 real and imaginary parts; the
// components Q < 0 follow from rho^K_-Q = (-1)^Q conj rho^K_Q).
//
// Device: mlpol_prepare_kernel writes each line's opacity, Planck function
// and emission multipoles S^K_Q = S_line w^(K) conj(rho^K_Q / rho^0_0)(J_u)
// (K = 0, 1, 2) and its dichroism multipoles D^K_Q (K = 1, 2) into the sweep
// arrays of the line's box (the polarized two-level formal solver, with the
// orientation terms in eps_V and eta_V, then solves every line; J^1_Q comes
// from Stokes V); mlpol_see_kernel assembles the real system of one voxel per
// CTA in shared memory over all multipoles (69 for J = 0, 1, 2, 1, 2),
// replaces the row of level 0's population by the trace
// sum_J sqrt(2J+1) rho^0_0(J) = 1, and solves it in FP64 in two blocks: the
// population rows (preconditioned) with the K > 0 multipoles at their old
// values, then the K > 0 rows (plain rates) with the new populations, by
// Gaussian elimination with partial pivoting.
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <vector>

#include "mlpol_kernels.cuh"

namespace porta {

// ---------------------------------------------------------------- Wigner symbols (Racah formulas)

namespace {

double fact(int n)
{
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= k;
    return f;
}

// arguments doubled (2j, 2m), so half-integers are integers
bool tri2(int a, int b, int c) { return a + b >= c && b + c >= a && c + a >= b && (a + b + c) % 2 == 0; }

double delta2(int a, int b, int c)
{
    return fact((a + b - c) / 2) * fact((a - b + c) / 2) * fact((-a + b + c) / 2) / fact((a + b + c) / 2 + 1);
}

double w3j2(int j1, int j2, int j3, int m1, int m2, int m3)
{
    if (m1 + m2 + m3 != 0 || !tri2(j1, j2, j3)) return 0.0;
    const int jm[3][2] = {{j1, m1}, {j2, m2}, {j3, m3}};
    for (auto &p : jm)
        if (std::abs(p[1]) > p[0] || (p[0] + p[1]) % 2) return 0.0;
    double pre = delta2(j1, j2, j3);
    for (auto &p : jm) pre *= fact((p[0] + p[1]) / 2) * fact((p[0] - p[1]) / 2);
    const int kmin = std::max({0, (j2 - j3 - m1) / 2, (j1 - j3 + m2) / 2});
    const int kmax = std::min({(j1 + j2 - j3) / 2, (j1 - m1) / 2, (j2 + m2) / 2});
    double s = 0.0;
    for (int k = kmin; k <= kmax; ++k) {
        const double d = fact(k) * fact((j3 - j2 + m1) / 2 + k) * fact((j3 - j1 - m2) / 2 + k) *
                         fact((j1 + j2 - j3) / 2 - k) * fact((j1 - m1) / 2 - k) * fact((j2 + m2) / 2 - k);
        s += (k % 2 ? -1.0 : 1.0) / d;
    }
    const int e = (j1 - j2 - m3) / 2;
    return ((e % 2 + 2) % 2 ? -1.0 : 1.0) * s * std::sqrt(pre);
}

double w6j2(int a, int b, int c, int d, int e, int f)
{
    if (!tri2(a, b, c) || !tri2(a, e, f) || !tri2(d, b, f) || !tri2(d, e, c)) return 0.0;
    const double pre = delta2(a, b, c) * delta2(a, e, f) * delta2(d, b, f) * delta2(d, e, c);
    const int t1 = (a + b + c) / 2, t2 = (a + e + f) / 2, t3 = (d + b + f) / 2, t4 = (d + e + c) / 2;
    const int u1 = (a + b + d + e) / 2, u2 = (b + c + e + f) / 2, u3 = (c + a + f + d) / 2;
    double s = 0.0;
    for (int k = std::max({t1, t2, t3, t4}); k <= std::min({u1, u2, u3}); ++k)
        s += (k % 2 ? -1.0 : 1.0) * fact(k + 1) /
             (fact(k - t1) * fact(k - t2) * fact(k - t3) * fact(k - t4) * fact(u1 - k) * fact(u2 - k) * fact(u3 - k));
    return s * std::sqrt(pre);
}

double w9j2(int a, int b, int c, int d, int e, int f, int g, int h, int i)
{
    const int lo = std::max({std::abs(a - i), std::abs(h - d), std::abs(b - f)});
    const int hi = std::min({a + i, h + d, b + f});
    double s = 0.0;
    for (int x = lo; x <= hi; x += 2)
        s += (x % 2 ? -1.0 : 1.0) * (x + 1) * w6j2(a, b, c, f, i, x) * w6j2(d, e, f, b, x, h) * w6j2(g, h, i, x, a, d);
    return s;
}

int two(double j) { return (int)std::lround(2.0 * j); }
double W3(double a, double b, double c, double d, double e, double f) { return w3j2(two(a), two(b), two(c), two(d), two(e), two(f)); }
double W6(double a, double b, double c, double d, double e, double f) { return w6j2(two(a), two(b), two(c), two(d), two(e), two(f)); }
double W9(double a, double b, double c, double d, double e, double f, double g, double h, double i)
{
    return w9j2(two(a), two(b), two(c), two(d), two(e), two(f), two(g), two(h), two(i));
}
double sgn(double e) { return (std::lround(e) % 2 + 2) % 2 ? -1.0 : 1.0; }

using cplx = std::complex<double>;
using CMat = std::vector<cplx>;     // n x n, row-major

}  // namespace

int mlpol_tables(const std::vector<double> &J, const std::vector<double> &E, const std::vector<int> &up,
                 const std::vector<int> &lo, const std::vector<double> &A, const std::vector<double> &eps,
                 MlPolTables &t)
{
    const int nlev = (int)J.size(), nline = (int)up.size();
    // complex basis (level, K, Q), Q = -K..K; real basis (level, K, Q >= 0, part)
    std::vector<int> cl, cK, cQ;
    std::map<long long, int> cidx;
    auto ckey = [](int i, int K, int Q) { return ((long long)i * 64 + K) * 64 + (Q + 32); };
    for (int i = 0; i < nlev; ++i)
        for (int K = 0; K <= two(J[i]); ++K)
            for (int Q = -K; Q <= K; ++Q) {
                cidx[ckey(i, K, Q)] = (int)cl.size();
                cl.push_back(i); cK.push_back(K); cQ.push_back(Q);
            }
    const int n = (int)cl.size();
    std::vector<int> rl, rK, rQ, rp;
    for (int i = 0; i < nlev; ++i)
        for (int K = 0; K <= two(J[i]); ++K) {
            rl.push_back(i); rK.push_back(K); rQ.push_back(0); rp.push_back(0);
            for (int Q = 1; Q <= K; ++Q)
                for (int p = 0; p < 2; ++p) {
                    rl.push_back(i); rK.push_back(K); rQ.push_back(Q); rp.push_back(p);
                }
        }
    const int nr = (int)rl.size();
    if (nr != n || n > kMlPolMaxUnk) return -1;
    // x = C r
    CMat Cm((size_t)n * nr, 0.0);
    for (int k = 0; k < nr; ++k) {
        const int i = rl[k], K = rK[k], Q = rQ[k];
        if (Q == 0) {
            Cm[(size_t)cidx[ckey(i, K, 0)] * nr + k] = 1.0;
            continue;
        }
        const cplx z = rp[k] == 0 ? cplx(1.0, 0.0) : cplx(0.0, 1.0);
        Cm[(size_t)cidx[ckey(i, K, Q)] * nr + k] += z;
        Cm[(size_t)cidx[ckey(i, K, -Q)] * nr + k] += sgn(Q) * std::conj(z);
    }
    std::vector<double> g(nlev);
    for (int i = 0; i < nlev; ++i) g[i] = 2.0 * J[i] + 1.0;
    // source layout: 0 const, 1 + 9 li + c (J real layout J00, J10, Re J11, Im J11, J20, Re J21,
    // Im J21, Re J22, Im J22), then B (3), C_lu per line, -Lambda* S_old per line, -Lambda* per line
    t.nline = nline;
    t.src_j = 1;
    t.src_b = 1 + 9 * nline;
    t.src_clu = t.src_b + 3;
    t.src_pop = t.src_clu + nline;
    t.src_spop = t.src_pop + nline;
    t.nsrc = t.src_spop + nline;
    std::vector<CMat> G(t.nsrc, CMat((size_t)n * n, 0.0));
    auto at = [n](CMat &M, int a, int b) -> cplx & { return M[(size_t)a * n + b]; };
    // radiative matrices per (Kr, Qr), Kr = 0, 1, 2
    for (int li = 0; li < nline; ++li) {
        const int u = up[li], l = lo[li];
        const double Ju = J[u], Jl = J[l];
        const double r = (E[u] - E[l]) / (E[up[0]] - E[lo[0]]);
        const double Bul = A[li] / (r * r * r), Blu = g[u] / g[l] * Bul;
        const double Cul = eps[li] / (1.0 - eps[li]) * A[li];
        std::map<int, CMat> Mr;          // key Kr * 8 + (Qr + 2)
        CMat Mpop((size_t)n * n, 0.0), Mspop((size_t)n * n, 0.0);
        auto mr = [&](int Kr, int Qr) -> CMat & {
            auto it = Mr.find(Kr * 8 + Qr + 2);
            if (it == Mr.end()) it = Mr.emplace(Kr * 8 + Qr + 2, CMat((size_t)n * n, 0.0)).first;
            return it->second;
        };
        for (int a = 0; a < n; ++a) {
            const int lev = cl[a], K = cK[a], Q = cQ[a];
            if (lev == u) {
                for (int Kl = 0; Kl <= two(Jl); ++Kl)
                    for (int Ql = -Kl; Ql <= Kl; ++Ql) {
                        const int b = cidx[ckey(l, Kl, Ql)];
                        for (int Kr = 0; Kr <= 2; ++Kr)
                            for (int Qr = -Kr; Qr <= Kr; ++Qr) {
                                const double v = (2 * Jl + 1) * Blu * std::sqrt(3.0 * (2 * K + 1) * (2 * Kl + 1) * (2 * Kr + 1)) *
                                                 sgn(Kl + Ql) * W9(Ju, Jl, 1, Ju, Jl, 1, K, Kl, Kr) * W3(K, Kl, Kr, -Q, Ql, -Qr);
                                if (v == 0.0) continue;
                                at(mr(Kr, Qr), a, b) += v;
                                if (K == 0 && Kl == 0 && Kr == 0) at(Mpop, a, b) += v;
                            }
                    }
                at(G[0], a, a) -= A[li];
                if (K == 0) at(Mspop, a, a) -= A[li];
                for (int Kp = 0; Kp <= two(Ju); ++Kp)
                    for (int Qp = -Kp; Qp <= Kp; ++Qp) {
                        const int b = cidx[ckey(u, Kp, Qp)];
                        for (int Kr = 0; Kr <= 2; ++Kr)
                            for (int Qr = -Kr; Qr <= Kr; ++Qr) {
                                if ((K + Kp + Kr) % 2) continue;
                                const double v = (2 * Ju + 1) * Bul * std::sqrt(3.0 * (2 * K + 1) * (2 * Kp + 1) * (2 * Kr + 1)) *
                                                 sgn(1 + Jl - Ju + Qp) * W6(K, Kp, Kr, Ju, Ju, Ju) * W6(1, 1, Kr, Ju, Ju, Jl) *
                                                 W3(K, Kp, Kr, Q, -Qp, Qr);
                                if (v == 0.0) continue;
                                at(mr(Kr, Qr), a, b) -= v;
                                if (K == 0 && Kp == 0 && Kr == 0) at(Mpop, a, b) -= v;
                            }
                    }
                at(G[0], a, a) -= Cul;
            }
            if (lev == l) {
                auto itb = cidx.find(ckey(u, K, Q));
                if (itb != cidx.end()) {
                    const double v = (2 * Ju + 1) * A[li] * sgn(1 + Ju + Jl + K) * W6(Ju, Ju, K, Jl, Jl, 1);
                    at(G[0], a, itb->second) += v;
                    if (K == 0) at(Mspop, a, itb->second) += v;
                }
                for (int Ku = 0; Ku <= two(Ju); ++Ku)
                    for (int Qu = -Ku; Qu <= Ku; ++Qu) {
                        const int b = cidx[ckey(u, Ku, Qu)];
                        for (int Kr = 0; Kr <= 2; ++Kr)
                            for (int Qr = -Kr; Qr <= Kr; ++Qr) {
                                const double v = (2 * Ju + 1) * Bul * std::sqrt(3.0 * (2 * K + 1) * (2 * Ku + 1) * (2 * Kr + 1)) *
                                                 sgn(Kr + Ku + Qu) * W9(Ju, Jl, 1, Ju, Jl, 1, Ku, K, Kr) * W3(K, Ku, Kr, -Q, Qu, -Qr);
                                if (v == 0.0) continue;
                                at(mr(Kr, Qr), a, b) += v;
                                if (K == 0 && Ku == 0 && Kr == 0) at(Mpop, a, b) += v;
                            }
                    }
                for (int Kp = 0; Kp <= two(Jl); ++Kp)
                    for (int Qp = -Kp; Qp <= Kp; ++Qp) {
                        const int b = cidx[ckey(l, Kp, Qp)];
                        for (int Kr = 0; Kr <= 2; ++Kr)
                            for (int Qr = -Kr; Qr <= Kr; ++Qr) {
                                if ((K + Kp + Kr) % 2) continue;
                                const double v = (2 * Jl + 1) * Blu * std::sqrt(3.0 * (2 * K + 1) * (2 * Kp + 1) * (2 * Kr + 1)) *
                                                 sgn(1 + Ju - Jl + Kr + Qp) * W6(K, Kp, Kr, Jl, Jl, Jl) * W6(1, 1, Kr, Jl, Jl, Ju) *
                                                 W3(K, Kp, Kr, Q, -Qp, Qr);
                                if (v == 0.0) continue;
                                at(mr(Kr, Qr), a, b) -= v;
                                if (K == 0 && Kp == 0 && Kr == 0) at(Mpop, a, b) -= v;
                            }
                    }
                // collisional excitation out of the lower level (unit C_lu; all multipoles relax)
                at(G[t.src_clu + li], a, a) -= 1.0;
            }
        }
        // collisional transfer of populations (n = sqrt(2J+1) rho^0_0)
        const int a0u = cidx[ckey(u, 0, 0)], a0l = cidx[ckey(l, 0, 0)];
        at(G[t.src_clu + li], a0u, a0l) += std::sqrt(g[l] / g[u]);
        at(G[0], a0l, a0u) += Cul * std::sqrt(g[u] / g[l]);
        // J sources of this line in the real layout
        auto addJ = [&](int s, int Kr, int Qr, cplx f) {
            auto it = Mr.find(Kr * 8 + Qr + 2);
            if (it == Mr.end()) return;
            for (size_t e = 0; e < it->second.size(); ++e) G[s][e] += f * it->second[e];
        };
        // (J^K_-Q = (-1)^Q conj J^K_Q: J^K_{+-1} = +-Re + i Im, J^2_{+-2} = Re +- i Im)
        const int s0 = t.src_j + 9 * li;
        addJ(s0 + 0, 0, 0, 1.0);
        addJ(s0 + 1, 1, 0, 1.0);
        addJ(s0 + 2, 1, 1, 1.0); addJ(s0 + 2, 1, -1, -1.0);
        addJ(s0 + 3, 1, 1, cplx(0, 1)); addJ(s0 + 3, 1, -1, cplx(0, 1));
        addJ(s0 + 4, 2, 0, 1.0);
        addJ(s0 + 5, 2, 1, 1.0); addJ(s0 + 5, 2, -1, -1.0);
        addJ(s0 + 6, 2, 1, cplx(0, 1)); addJ(s0 + 6, 2, -1, cplx(0, 1));
        addJ(s0 + 7, 2, 2, 1.0); addJ(s0 + 7, 2, -2, 1.0);
        addJ(s0 + 8, 2, 2, cplx(0, 1)); addJ(s0 + 8, 2, -2, cplx(0, -1));
        G[t.src_pop + li] = Mpop;
        G[t.src_spop + li] = Mspop;
    }
    // Hanle: -i w_J H^K(b) in d rho / dt (rho^K_Q turns as e^{-i Q w_J t} for b along z:
    // counterclockwise precession about the field), Lande factor 1, b in gauss
    const double wj = -2.0 * M_PI * kLarmorPerGauss;
    for (int a = 0; a < n; ++a) {
        const int lev = cl[a], K = cK[a], Q = cQ[a];
        at(G[t.src_b + 2], a, a) += cplx(0, wj * Q);
        if (Q - 1 >= -K) {
            const int b = cidx[ckey(lev, K, Q - 1)];
            const double f = 0.5 * std::sqrt((double)(K + Q) * (K - Q + 1));
            at(G[t.src_b + 0], a, b) += cplx(0, wj * f);
            at(G[t.src_b + 1], a, b) += cplx(wj * f, 0);      // i * (-i) = 1
        }
        if (Q + 1 <= K) {
            const int b = cidx[ckey(lev, K, Q + 1)];
            const double f = 0.5 * std::sqrt((double)(K - Q) * (K + Q + 1));
            at(G[t.src_b + 0], a, b) += cplx(0, wj * f);
            at(G[t.src_b + 1], a, b) += cplx(-wj * f, 0);     // i * i = -1
        }
    }
    // real system rows: (complex row, part); trace row
    t.nunk = nr;
    t.trace.assign(nr, 0.0);
    t.pop_idx.assign(nlev, -1);
    t.row0 = -1;
    for (int k = 0; k < nr; ++k)
        if (rK[k] == 0) {
            t.trace[k] = std::sqrt(g[rl[k]]);
            t.pop_idx[rl[k]] = k;
            if (rl[k] == 0) t.row0 = k;
        }
    // sparse cells of the real matrices R_s = select(G_s C)
    std::map<long long, std::vector<std::pair<int, double>>> cells;
    for (int s = 0; s < t.nsrc; ++s)
        for (int row = 0; row < nr; ++row) {
            if (row == t.row0) continue;
            const int ci = cidx[ckey(rl[row], rK[row], rQ[row])];
            for (int col = 0; col < nr; ++col) {
                cplx y = 0.0;
                for (int b = 0; b < n; ++b) {
                    const cplx m = G[s][(size_t)ci * n + b];
                    if (m != 0.0) y += m * Cm[(size_t)b * nr + col];
                }
                const double v = rp[row] == 0 ? y.real() : y.imag();
                if (std::abs(v) == 0.0) continue;
                cells[(long long)row * nr + col].emplace_back(s, v);
            }
        }
    t.cell_rc.clear(); t.cell_start.assign(1, 0); t.ent_src.clear(); t.ent_coef.clear();
    for (auto &c : cells) {
        t.cell_rc.push_back((int)(c.first / nr));
        t.cell_rc.push_back((int)(c.first % nr));
        for (auto &e : c.second) {
            t.ent_src.push_back(e.first);
            t.ent_coef.push_back(e.second);
        }
        t.cell_start.push_back((int)t.ent_src.size());
    }
    // per line the multipoles rho^0_0, rho^1_Q, rho^2_Q of the upper level (emission; stimulated
    // emission in the dichroism) and of the lower level (absorption), with
    // w^(K)_{J J'} = (-1)^(1+J+J') sqrt(3(2J+1)) {1 1 K; J J J'}
    t.upk.assign(9 * (size_t)nline, -1);
    t.lok.assign(9 * (size_t)nline, -1);
    t.wu.assign(2 * (size_t)nline, 0.0);
    t.wl.assign(2 * (size_t)nline, 0.0);
    auto ridx = [&](int i, int K, int Q, int p) {
        for (int k = 0; k < nr; ++k)
            if (rl[k] == i && rK[k] == K && rQ[k] == Q && rp[k] == p) return k;
        return -1;
    };
    auto fill9 = [&](int i, int *ix) {
        const int KQp[9][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {1, 1, 1}, {2, 0, 0},
                               {2, 1, 0}, {2, 1, 1}, {2, 2, 0}, {2, 2, 1}};
        for (int c = 0; c < 9; ++c)
            if (KQp[c][0] <= two(J[i])) ix[c] = ridx(i, KQp[c][0], KQp[c][1], KQp[c][2]);
    };
    for (int li = 0; li < nline; ++li) {
        const int u = up[li], l = lo[li];
        fill9(u, &t.upk[9 * (size_t)li]);
        fill9(l, &t.lok[9 * (size_t)li]);
        for (int K = 1; K <= 2; ++K) {
            if (two(J[u]) >= K)
                t.wu[2 * li + K - 1] = sgn(1 + J[l] + J[u]) * std::sqrt(3.0 * (2 * J[u] + 1)) * W6(1, 1, K, J[u], J[u], J[l]);
            if (two(J[l]) >= K)
                t.wl[2 * li + K - 1] = sgn(1 + J[l] + J[u]) * std::sqrt(3.0 * (2 * J[l] + 1)) * W6(1, 1, K, J[l], J[l], J[u]);
        }
    }
    return 0;
}

// ---------------------------------------------------------------- kernels

namespace {

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

template <typename Real>
__global__ void mlpol_prepare_kernel(const MlConst mc, MlPolDev T, long long nvox1, const double *x, const double *chis,
                                     const double *kT, Real *chi_out, Real *bpl_out, Real *S_out, double *S64_out,
                                     Real *pol_out, unsigned long long *bad)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= nvox1) return;
    const double *xv = x + v * T.nunk;
    double n[kMlMaxLevel];
    for (int i = 0; i < mc.nlev; ++i) n[i] = sqrt(mc.g[i]) * xv[T.pop_idx[i]];
    const long long nvox = nvox1 * mc.nline;
    const double chi = chis[v], t = kT[v];
    int nbad = 0;
    for (int k = 0; k < mc.nline; ++k) {
        const int u = mc.up[k], l = mc.lo[k];
        const double op = chi * mc.s[k] * (n[l] - n[u] * mc.g[l] / mc.g[u]);
        const double S = mc.r3[k] * n[u] / (n[l] * mc.g[u] / mc.g[l] - n[u]);
        const long long o = (long long)k * nvox1 + v;
        nbad += !(op > 0.0 && op < 1e300) || !(fabs(S) < 1e300);
        chi_out[o] = (Real)op;
        bpl_out[o] = (Real)(mc.r3[k] / expm1(mc.dE[k] / t));
        // S^K_Q = S w^(K) conj(rho^K_Q / rho^0_0)(upper): K = 0, 2 in the two-level real layout
        // (S00, S20, Re/Im S21, Re/Im S22), K = 1 as (S10, Re S11, Im S11); conjugation
        // negates the imaginary parts
        const int *iu = T.upk + 9 * k, *il = T.lok + 9 * k;
        const double *wu = T.wu + 2 * k, *wl = T.wl + 2 * k;
        double s6[6] = {S, 0, 0, 0, 0, 0}, s3[3] = {0, 0, 0};
        if (iu[4] >= 0) {
            const double f = S * wu[1] / xv[iu[0]];
            s6[1] = f * xv[iu[4]];
            s6[2] = f * xv[iu[5]];
            s6[3] = -f * xv[iu[6]];
            s6[4] = f * xv[iu[7]];
            s6[5] = -f * xv[iu[8]];
        }
        if (iu[1] >= 0) {
            const double f = S * wu[0] / xv[iu[0]];
            s3[0] = f * xv[iu[1]];
            s3[1] = f * xv[iu[2]];
            s3[2] = -f * xv[iu[3]];
        }
        for (int c = 0; c < 6; ++c) {
            S64_out[o * 6 + c] = s6[c];
            S_out[c * nvox + o] = (Real)s6[c];
        }
        // dichroism: D^K_Q = conj([(-1)^K B_lu sqrt(2Jl+1) w^(K)(l) rho^K_Q(l) - B_ul sqrt(2Ju+1) w^(K)(u) rho^K_Q(u)]
        //                        / [B_lu sqrt(2Jl+1) rho^0_0(l) - B_ul sqrt(2Ju+1) rho^0_0(u)]),
        // K = 2 (D20, Re/Im D21, Re/Im D22) then K = 1 (D10, Re/Im D11)
        const double al = mc.Blu[k] * sqrt(mc.g[l]), au = mc.Bul[k] * sqrt(mc.g[u]);
        const double den = al * xv[il[0]] - au * xv[iu[0]];
        double d8[8];
        for (int c = 0; c < 8; ++c) {
            const int j = c < 5 ? 4 + c : c - 4;           // component in the Kr = 0, 1, 2 layout
            const int K = c < 5 ? 2 : 1;
            const double sa = K == 2 ? 1.0 : -1.0;
            double num = 0.0;
            if (il[j] >= 0) num += sa * al * wl[K - 1] * xv[il[j]];
            if (iu[j] >= 0) num -= au * wu[K - 1] * xv[iu[j]];
            d8[c] = num / den;
        }
        d8[2] = -d8[2];
        d8[4] = -d8[4];
        d8[7] = -d8[7];
        for (int c = 0; c < 8; ++c) pol_out[c * nvox + o] = (Real)d8[c];
        for (int c = 0; c < 3; ++c) pol_out[(8 + c) * nvox + o] = (Real)s3[c];
    }
    if (nbad) atomicAdd(bad, (unsigned long long)nbad);
}

// One CTA of kVoxThreads threads per voxel (a persistent loop over voxels): the
// voxel's system lives in shared memory (40 KB for 69 unknowns), so an SM holds
// about five voxels; the warps of a CTA share its assembly, reductions and
// elimination, which keeps ~20 warps per SM in flight for the latency-bound
// shared-memory and table loads.
constexpr int kVoxThreads = 128;
constexpr int kVoxWarps = kVoxThreads / 32;

// sum over the CTA, the same value (and the same order of additions) in every thread
__device__ __forceinline__ double cta_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();                                  // red is free (its last readers passed here)
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kVoxWarps; ++w) t += red[w];
    return t;
}

__device__ __forceinline__ double cta_max(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = red[0];
    for (int w = 1; w < kVoxWarps; ++w) t = fmax(t, red[w]);
    return t;
}

// largest |value| with the smallest row among equal values (partial pivoting)
__device__ __forceinline__ void cta_argmax(double &bv, int &br, double *red, int *redi)
{
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int orr = __shfl_xor_sync(0xffffffffu, br, o);
        if (ov > bv || (ov == bv && orr < br)) { bv = ov; br = orr; }
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = bv;
        redi[threadIdx.x >> 5] = br;
    }
    __syncthreads();
    bv = red[0];
    br = redi[0];
    for (int w = 1; w < kVoxWarps; ++w)
        if (red[w] > bv || (red[w] == bv && redi[w] < br)) { bv = red[w]; br = redi[w]; }
}

// the same over FP32 values (FP32 compares: the FP64 pipe of this GPU is a small
// fraction of its FP32 rate, and compares occupy it like arithmetic)
__device__ __forceinline__ void cta_argmax(float &bv, int &br, float *red, int *redi)
{
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int orr = __shfl_xor_sync(0xffffffffu, br, o);
        if (ov > bv || (ov == bv && orr < br)) { bv = ov; br = orr; }
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = bv;
        redi[threadIdx.x >> 5] = br;
    }
    __syncthreads();
    bv = red[0];
    br = redi[0];
    for (int w = 1; w < kVoxWarps; ++w)
        if (red[w] > bv || (red[w] == bv && redi[w] < br)) { bv = red[w]; br = redi[w]; }
}

// the real system of voxel v into A [N][N + 1] (row of level 0's population =
// the trace), sources into s; xo holds the old unknowns; lstar null: the plain
// rates (no preconditioning). Called by all threads of the voxel's CTA.
__device__ void mlpol_assemble(const MlConst &mc, const MlPolDev &T, long long nvox1, long long v, const double *kT,
                               const double *jkq, const double *j1, const double *lstar, const double *bvec,
                               const double *xo, double *A, double *s)
{
    const int N = T.nunk, N1 = N + 1, tid = threadIdx.x;
    if (tid == 0) {
        s[0] = 1.0;
        s[T.src_b] = bvec[v];
        s[T.src_b + 1] = bvec[nvox1 * mc.nline + v];
        s[T.src_b + 2] = bvec[2 * nvox1 * mc.nline + v];
    }
    for (int k = tid; k < mc.nline; k += kVoxThreads) {
        const int u = mc.up[k], l = mc.lo[k];
        const long long o = (long long)k * nvox1 + v;
        double *sj = s + T.src_j + 9 * k;
        sj[0] = jkq[o * 6];
        for (int c = 0; c < 3; ++c) sj[1 + c] = j1[o * 3 + c];
        for (int c = 1; c < 6; ++c) sj[3 + c] = jkq[o * 6 + c];
        s[T.src_clu + k] = mc.g[u] / mc.g[l] * exp(-mc.dE[k] / kT[v]) * mc.Cul[k];
        if (lstar) {
            const double nu = sqrt(mc.g[u]) * xo[T.pop_idx[u]], nl = sqrt(mc.g[l]) * xo[T.pop_idx[l]];
            const double Sold = mc.r3[k] * nu / (nl * mc.g[u] / mc.g[l] - nu);
            const double ls = lstar[o];
            s[T.src_pop + k] = -ls * Sold;
            s[T.src_spop + k] = -ls;
        } else {
            s[T.src_pop + k] = 0.0;
            s[T.src_spop + k] = 0.0;
        }
    }
    for (int e = tid; e < N * N1; e += kVoxThreads) A[e] = 0.0;
    __syncthreads();
    for (int c = tid; c < T.ncell; c += kVoxThreads) {
        double val = 0.0;
        for (int e = T.cell_start[c]; e < T.cell_start[c + 1]; ++e) val += T.ent_coef[e] * s[T.ent_src[e]];
        A[T.cell_rc[2 * c] * N1 + T.cell_rc[2 * c + 1]] = val;
    }
    __syncthreads();
    for (int j = tid; j < N; j += kVoxThreads) A[T.row0 * N1 + j] = T.trace[j];
    __syncthreads();
}

// out = alpha A(x) + add + with_f e_row0 (full layout): A(x) the plain rate operator
// with the trace row; one CTA per voxel, shared memory as mlpol_see_kernel
__global__ void __launch_bounds__(kVoxThreads) mlpol_apply_kernel(const MlConst mc, MlPolDev T, long long nvox1,
                                                                  const double *kT, const double *jkq, const double *j1,
                                                                  const double *bvec, const double *x, double alpha,
                                                                  const double *add, int with_f, double *out)
{
    extern __shared__ double sm[];
    const int N = T.nunk, N1 = N + 1, tid = threadIdx.x;
    double *A = sm;
    double *xo = A + N * N1;
    double *s = xo + 2 * N;
    for (long long v = blockIdx.x; v < nvox1; v += gridDim.x) {
        for (int k = tid; k < N; k += kVoxThreads) xo[k] = x[v * N + k];
        __syncthreads();
        mlpol_assemble(mc, T, nvox1, v, kT, jkq, j1, nullptr, bvec, xo, A, s);
        for (int r = tid; r < N; r += kVoxThreads) {
            double y = 0.0;
            for (int c = 0; c < N; ++c) y += A[r * N1 + c] * xo[c];
            const long long o = v * N + r;
            out[o] = alpha * y + (add ? add[o] : 0.0) + (with_f && r == T.row0 ? 1.0 : 0.0);
        }
        __syncthreads();
    }
}

// Solve of the K > 0 block B x = b (B = A restricted to the M = N - L unknowns
// kidx[], b their right-hand sides; A itself is left unchanged) by LU factors in
// FP32 and iterative refinement with FP64 residuals: x = 0, r = b, then
// d = (LU)^-1 P r, x += d, r = b - B x until the correction is below 1e-13 of x
// (or has stopped shrinking below 1e-12 of it, the floor of FP64 residuals).
// The factorization costs a third of the FP64 elimination's M^3 operations in
// FP32 (64 times the FP64 rate on this GPU); each refinement step costs M^2 in
// FP64. Returns false (the same in every thread) when a pivot vanishes or the
// refinement does not converge: the caller then eliminates in FP64. On success
// xn[kidx[i]] = x_i.
__device__ bool mlpol_refine_solve(const double *A, int N, int M, const int *kidx, float *LU, float *y, int *piv,
                                   double *xr, double *rr, double *xn, double *red, float *redf, int *redi)
{
    const int N1 = N + 1, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int e = tid; e < M * M; e += kVoxThreads) {
        const int i = e / M, j = e - (e / M) * M;
        LU[e] = (float)A[kidx[i] * N1 + kidx[j]];
    }
    for (int i = tid; i < M; i += kVoxThreads) {
        rr[i] = A[kidx[i] * N1 + N];
        xr[i] = 0.0;
    }
    __syncthreads();
    // LU with partial pivoting (rows swapped in place, multipliers below the diagonal).
    // Step k: swap the pivot row in, then each warp updates its rows r = k+1+w (mod 4)
    // with the lanes over the columns, stores the row's multiplier, and lane 0 (which
    // holds column k+1) keeps the largest |value| of that column among the warp's rows:
    // the next pivot comes from the four warps' candidates after one barrier (two
    // barriers per step; the pivot is the largest |value|, the smallest row on ties).
    constexpr int kCols = (kMlPolMaxUnk + 31) / 32;     // column slots per lane
    float bv = -1.0f;
    int br = 0;
    for (int r = tid; r < M; r += kVoxThreads) {
        const float a = fabsf(LU[r * M]);
        if (a > bv) { bv = a; br = r; }
    }
    cta_argmax(bv, br, redf, redi);
    for (int k = 0; k < M; ++k) {
        if (!(bv > 0.0f)) return false;
        if (tid == 0) piv[k] = br;
        if (br != k)
            for (int j = tid; j < M; j += kVoxThreads) {
                const float tmp = LU[k * M + j];
                LU[k * M + j] = LU[br * M + j];
                LU[br * M + j] = tmp;
            }
        __syncthreads();
        const float inv = 1.0f / LU[k * M + k];
        float u[kCols];
#pragma unroll
        for (int m = 0; m < kCols; ++m) {
            const int j = k + 1 + lane + 32 * m;
            u[m] = j < M ? LU[k * M + j] : 0.0f;
        }
        float cv = -1.0f;
        int cr = M;
        for (int r = k + 1 + wid; r < M; r += kVoxWarps) {
            const float l = LU[r * M + k] * inv;
#pragma unroll
            for (int m = 0; m < kCols; ++m) {
                const int j = k + 1 + lane + 32 * m;
                if (j < M) LU[r * M + j] -= l * u[m];
            }
            if (lane == 0) {                // (r > k, so column k + 1 exists)
                const float a = fabsf(LU[r * M + k + 1]);
                if (a > cv) { cv = a; cr = r; }
            }
        }
        __syncwarp();
        for (int r = k + 1 + wid + kVoxWarps * lane; r < M; r += 32 * kVoxWarps) LU[r * M + k] *= inv;
        if (lane == 0) {
            redf[wid] = cv;
            redi[wid] = cr;
        }
        __syncthreads();
        bv = redf[0];
        br = redi[0];
        for (int w = 1; w < kVoxWarps; ++w)
            if (redf[w] > bv || (redf[w] == bv && redi[w] < br)) { bv = redf[w]; br = redi[w]; }
        // (the next step writes red only after its swap barrier)
    }
    double dprev = 1e300;
    for (int it = 0; it < 8; ++it) {
        // d = U^-1 L^-1 P r in FP32 (warp 0)
        if (wid == 0) {
            for (int i = lane; i < M; i += 32) y[i] = (float)rr[i];
            __syncwarp();
            if (lane == 0)
                for (int k = 0; k < M; ++k) {
                    const int p = piv[k];
                    if (p != k) {
                        const float t = y[k]; y[k] = y[p]; y[p] = t;
                    }
                }
            __syncwarp();
            for (int k = 0; k + 1 < M; ++k) {
                const float yk = y[k];
                for (int i = k + 1 + lane; i < M; i += 32) y[i] -= LU[i * M + k] * yk;
                __syncwarp();
            }
            for (int k = M - 1; k >= 0; --k) {
                const float yk = y[k] / LU[k * M + k];
                for (int i = lane; i < k; i += 32) y[i] -= LU[i * M + k] * yk;
                __syncwarp();
                if (lane == 0) y[k] = yk;
                __syncwarp();
            }
        }
        __syncthreads();
        double dm = 0.0, xm = 0.0;
        for (int i = tid; i < M; i += kVoxThreads) {
            xr[i] += (double)y[i];
            dm = fmax(dm, fabs((double)y[i]));
            xm = fmax(xm, fabs(xr[i]));
        }
        dm = cta_max(dm, red);
        xm = cta_max(xm, red);
        if (!(dm < 1e300 && xm < 1e300)) return false;
        if (dm <= 1e-13 * xm || (dm <= 1e-12 * xm && dm > 0.5 * dprev)) {
            for (int i = tid; i < M; i += kVoxThreads) xn[kidx[i]] = xr[i];
            __syncthreads();
            return true;
        }
        dprev = dm;
        // r = b - B x (FP64)
        for (int i = tid; i < M; i += kVoxThreads) {
            const double *Ar = A + kidx[i] * N1;
            double acc = Ar[N];
            for (int j = 0; j < M; ++j) acc -= Ar[kidx[j]] * xr[j];
            rr[i] = acc;
        }
        __syncthreads();
    }
    return false;
}

// one CTA per voxel; shared memory: A[nunk][nunk + 1], x_old, x_new, sources, and
// for the refinement solve FP64 x and r, the FP32 LU factors and work vector,
// pivots and the indices of the K > 0 unknowns
__global__ void __launch_bounds__(kVoxThreads) mlpol_see_kernel(const MlConst mc, MlPolDev T, long long nvox1,
                                                                const double *kT, const double *jkq, const double *j1,
                                                                const double *lstar, const double *bvec,
                                                                const double *src, double *x, unsigned long long *resid,
                                                                unsigned long long *bad)
{
    extern __shared__ double sm[];
    __shared__ double red[kVoxWarps];
    __shared__ float redf[kVoxWarps];
    __shared__ int redi[kVoxWarps];
    const int N = T.nunk, N1 = N + 1;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    double *A = sm;
    double *xo = A + N * N1;
    double *xn = xo + N;
    double *s = xn + N;
    double *xr = s + T.nsrc;
    double *rr = xr + N;
    float *LU = reinterpret_cast<float *>(rr + N);
    float *y = LU + N * N;
    int *kidx = reinterpret_cast<int *>(y + N);
    int *piv = kidx + N;
    // the K > 0 unknowns (all but the populations)
    const int M = N - mc.nlev;
    if (tid == 0) {
        int m = 0;
        for (int k = 0; k < N; ++k) {
            bool pop = false;
            for (int i = 0; i < mc.nlev; ++i) pop |= T.pop_idx[i] == k;
            if (!pop) kidx[m++] = k;
        }
    }
    double ch_max = 0.0;
    for (long long v = blockIdx.x; v < nvox1; v += gridDim.x) {
        for (int k = tid; k < N; k += kVoxThreads) xo[k] = x[v * N + k];
        __syncthreads();
        mlpol_assemble(mc, T, nvox1, v, kT, jkq, j1, lstar, bvec, xo, A, s);
        // right-hand side: (1, 0, ...) on the trace row, or the coarse-grid source
        for (int r = tid; r < N; r += kVoxThreads) A[r * N1 + N] = src ? src[v * N + r] : (r == T.row0 ? 1.0 : 0.0);
        __syncthreads();
        // block 1: the population rows (K = 0) with the K > 0 multipoles at their old values
        const int L = mc.nlev;
        auto is_k0 = [&](int c) {
            for (int i = 0; i < L; ++i)
                if (T.pop_idx[i] == c) return true;
            return false;
        };
        for (int i = 0; i < L; ++i) {
            const int r = T.pop_idx[i];
            double acc = 0.0;
            for (int c = tid; c < N; c += kVoxThreads)
                if (!is_k0(c)) acc += A[r * N1 + c] * xo[c];
            acc = cta_sum(acc, red);
            if (tid == 0) A[r * N1 + N] -= acc;
        }
        __syncthreads();
        if (tid == 0) {
            int ok1 = 1;
            double m[kMlMaxLevel][kMlMaxLevel + 1];
            for (int i = 0; i < L; ++i) {
                for (int j = 0; j < L; ++j) m[i][j] = A[T.pop_idx[i] * N1 + T.pop_idx[j]];
                m[i][L] = A[T.pop_idx[i] * N1 + N];
            }
            for (int c = 0; c < L && ok1; ++c) {
                int p = c;
                for (int r = c + 1; r < L; ++r)
                    if (fabs(m[r][c]) > fabs(m[p][c])) p = r;
                if (!(fabs(m[p][c]) > 0.0)) { ok1 = 0; break; }
                if (p != c)
                    for (int j = 0; j <= L; ++j) {
                        const double tmp = m[c][j]; m[c][j] = m[p][j]; m[p][j] = tmp;
                    }
                for (int r = c + 1; r < L; ++r) {
                    const double f = m[r][c] / m[c][c];
                    for (int j = c; j <= L; ++j) m[r][j] -= f * m[c][j];
                }
            }
            if (ok1)
                for (int i = L - 1; i >= 0; --i) {
                    double acc = m[i][L];
                    for (int j = i + 1; j < L; ++j) acc -= m[i][j] * xn[T.pop_idx[j]];
                    xn[T.pop_idx[i]] = acc / m[i][i];
                }
            redi[0] = ok1;
        }
        __syncthreads();
        const int ok1 = redi[0];
        // block 2: the K > 0 rows with the new populations; population rows become identities
        for (int r = tid; r < N; r += kVoxThreads) {
            if (is_k0(r)) {
                for (int c = 0; c < N; ++c) A[r * N1 + c] = c == r ? 1.0 : 0.0;
                A[r * N1 + N] = ok1 ? xn[r] : 1.0;
            } else {
                double bsub = 0.0;
                for (int i = 0; i < L; ++i) {
                    const int c = T.pop_idx[i];
                    bsub += A[r * N1 + c] * (ok1 ? xn[c] : 1.0);
                    A[r * N1 + c] = 0.0;
                }
                A[r * N1 + N] -= bsub;
            }
        }
        __syncthreads();
        // the K > 0 block by FP32 factors and FP64 refinement; if that fails, Gaussian
        // elimination in FP64 with partial pivoting on [A | b]: for pivot k the lanes
        // take the columns, the warps the rows of the trailing block
        bool ok = ok1 != 0;
        const bool refined =
            ok && M > 0 && T.solve == 0 && mlpol_refine_solve(A, N, M, kidx, LU, y, piv, xr, rr, xn, red, redf, redi);
        for (int k = 0; k < N && !refined; ++k) {
            double bv = -1.0;
            int br = k;
            for (int r = k + tid; r < N; r += kVoxThreads) {
                const double a = fabs(A[r * N1 + k]);
                if (a > bv) { bv = a; br = r; }
            }
            cta_argmax(bv, br, red, redi);
            if (!(bv > 0.0)) { ok = false; break; }
            if (br != k)
                for (int j = k + tid; j <= N; j += kVoxThreads) {
                    const double tmp = A[k * N1 + j];
                    A[k * N1 + j] = A[br * N1 + j];
                    A[br * N1 + j] = tmp;
                }
            __syncthreads();
            const double inv = 1.0 / A[k * N1 + k];
            for (int j = k + 1 + lane; j <= N; j += 32) {
                const double akj = A[k * N1 + j] * inv;
#pragma unroll 4
                for (int r = k + 1 + wid; r < N; r += kVoxWarps) A[r * N1 + j] -= A[r * N1 + k] * akj;
            }
            __syncthreads();
        }
        double ch = 0.0;
        if (ok) {
            // back substitution (warp 0)
            if (wid == 0 && !refined)
                for (int k = N - 1; k >= 0; --k) {
                    double acc = 0.0;
                    for (int j = k + 1 + lane; j < N; j += 32) acc += A[k * N1 + j] * xn[j];
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if (lane == 0) xn[k] = (A[k * N1 + N] - acc) / A[k * N1 + k];
                    __syncwarp();
                }
            __syncthreads();
            double nb = 0.0;
            for (int i = tid; i < mc.nlev; i += kVoxThreads) {
                const double p0 = xo[T.pop_idx[i]], p1 = xn[T.pop_idx[i]];
                nb += !(p1 > 0.0 && p1 < 1e300);
                ch = fmax(ch, fabs(p1 - p0) / fabs(p0));
            }
            for (int k = tid; k < N; k += kVoxThreads) nb += !(fabs(xn[k]) < 1e300);
            nb = cta_sum(nb, red);
            if (nb > 0.0) {
                ok = false;
            } else {
                for (int k = tid; k < N; k += kVoxThreads) x[v * N + k] = xn[k];
            }
        }
        if (!ok) {
            if (tid == 0) atomicAdd(bad, 1ull);
            ch = 1e300;
        }
        ch = cta_max(ch, red);
        ch_max = fmax(ch_max, ch);
        __syncthreads();
    }
    if (tid == 0 && ch_max > 0.0) atomicMax(resid, (unsigned long long)__double_as_longlong(fmin(ch_max, 1e300)));
}

}  // namespace

template <typename Real>
cudaError_t run_mlpol_prepare(const MlConst &mc, const MlPolDev &T, long long nvox1, const double *x, const double *chis,
                              const double *kT, Real *chi_out, Real *bpl_out, Real *S_out, double *S64_out,
                              Real *pol_out, unsigned long long *bad, cudaStream_t st)
{
    mlpol_prepare_kernel<Real><<<nblk(nvox1, 128), 128, 0, st>>>(mc, T, nvox1, x, chis, kT, chi_out, bpl_out, S_out,
                                                                 S64_out, pol_out, bad);
    return cudaGetLastError();
}
template cudaError_t run_mlpol_prepare<float>(const MlConst &, const MlPolDev &, long long, const double *, const double *,
                                              const double *, float *, float *, float *, double *, float *,
                                              unsigned long long *, cudaStream_t);
template cudaError_t run_mlpol_prepare<double>(const MlConst &, const MlPolDev &, long long, const double *, const double *,
                                               const double *, double *, double *, double *, double *, double *,
                                               unsigned long long *, cudaStream_t);

size_t mlpol_see_smem(const MlPolDev &T, int voxels)
{
    const size_t N = T.nunk;
    return (size_t)voxels * (sizeof(double) * (N * (N + 1) + 4 * N + T.nsrc) + sizeof(float) * (N * N + N) +
                             sizeof(int) * 2 * N);
}

namespace {

__global__ void mlpol_jbar9_kernel(long long n, const double *jkq, const double *j1, double *jbar)
{
    const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (o >= n) return;
    double *b = jbar + o * 9;
    b[0] = jkq[o * 6];
    for (int c = 0; c < 3; ++c) b[1 + c] = j1[o * 3 + c];
    for (int c = 1; c < 6; ++c) b[3 + c] = jkq[o * 6 + c];
}

}  // namespace

cudaError_t run_mlpol_jbar9(long long n, const double *jkq, const double *j1, double *jbar, cudaStream_t st)
{
    mlpol_jbar9_kernel<<<nblk(n, 256), 256, 0, st>>>(n, jkq, j1, jbar);
    return cudaGetLastError();
}

// max relative change of the populations between two vectors of unknowns
__global__ void mlpol_change_kernel(const MlConst mc, MlPolDev T, long long nvox1, const double *old, const double *cur,
                                    unsigned long long *resid)
{
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double ch = 0.0;
    if (v < nvox1)
        for (int i = 0; i < mc.nlev; ++i) {
            const long long o = v * T.nunk + T.pop_idx[i];
            ch = fmax(ch, fabs(cur[o] - old[o]) / fabs(old[o]));
        }
    if (!(ch <= 1e300)) ch = 1e300;
    for (int s = 16; s > 0; s >>= 1) ch = fmax(ch, __shfl_xor_sync(0xffffffffu, ch, s));
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = ch;
    __syncthreads();
    if (wid == 0) {
        ch = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int s = 16; s > 0; s >>= 1) ch = fmax(ch, __shfl_xor_sync(0xffffffffu, ch, s));
        if (lane == 0) atomicMax(resid, (unsigned long long)__double_as_longlong(ch));
    }
}

cudaError_t run_mlpol_change(const MlConst &mc, const MlPolDev &T, long long nvox1, const double *old, const double *cur,
                             unsigned long long *resid, cudaStream_t st)
{
    mlpol_change_kernel<<<nblk(nvox1, 256), 256, 0, st>>>(mc, T, nvox1, old, cur, resid);
    return cudaGetLastError();
}

// persistent launch shape of the CTA-per-voxel kernels: as many CTAs as fit on the GPU
template <typename K>
static cudaError_t voxel_launch_shape(K kernel, const MlPolDev &T, long long nvox1, size_t &smem, int &blocks)
{
    int dev = 0, nsm = 0, per_sm = 1, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    smem = mlpol_see_smem(T, 1);
    if (smem > (size_t)optin) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kVoxThreads, smem);
    blocks = (int)std::max<long long>(1, std::min<long long>(nvox1, (long long)std::max(1, per_sm) * nsm));
    return cudaSuccess;
}

cudaError_t run_mlpol_see(const MlConst &mc, const MlPolDev &T, long long nvox1, const double *kT, const double *jkq,
                          const double *j1, const double *lstar, const double *bvec, double *x, unsigned long long *resid,
                          unsigned long long *bad, cudaStream_t st, const double *src)
{
    size_t smem = 0;
    int blocks = 1;
    cudaError_t e = voxel_launch_shape(mlpol_see_kernel, T, nvox1, smem, blocks);
    if (e != cudaSuccess) return e;
    mlpol_see_kernel<<<blocks, kVoxThreads, smem, st>>>(mc, T, nvox1, kT, jkq, j1, lstar, bvec, src, x, resid, bad);
    return cudaGetLastError();
}

cudaError_t run_mlpol_apply(const MlConst &mc, const MlPolDev &T, long long nvox1, const double *kT, const double *jkq,
                            const double *j1, const double *bvec, const double *x, double alpha, const double *add,
                            int with_f, double *out, cudaStream_t st)
{
    size_t smem = 0;
    int blocks = 1;
    cudaError_t e = voxel_launch_shape(mlpol_apply_kernel, T, nvox1, smem, blocks);
    if (e != cudaSuccess) return e;
    mlpol_apply_kernel<<<blocks, kVoxThreads, smem, st>>>(mc, T, nvox1, kT, jkq, j1, bvec, x, alpha, add, with_f, out);
    return cudaGetLastError();
}

}  // namespace porta
