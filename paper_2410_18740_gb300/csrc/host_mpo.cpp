// Host-side problem set-up for the GBS parent Hamiltonian.
//
//  * coefficients: H = R^T G R - N/2 with G = V^{-1}/4 (Eq. GBSHamiltonian).  Since the
//    covariance is V = 1/2 O diag(e^{-2r}, e^{2r}) O^T with O orthogonal (the passive
//    interferometer acting on xxpp quadratures), G is formed in closed form as
//    1/2 O diag(e^{2r}, e^{-2r}) O^T -- no matrix inverse.
//  * optimal local basis (Sec. "Optimal Local Basis for Gaussian States"): per mode the
//    2x2 reduced covariance V_i = S_i nu_i S_i^T (Eq. WilliamsonDecomposition), with the
//    symmetric choice S_i = (V_i/nu_i)^{1/2} written in closed form (A + I)/sqrt(tr A + 2)
//    for a 2x2 positive matrix of unit determinant (Cayley-Hamilton).  The Hamiltonian
//    becomes R^T S^T G S R (Eq. OLB), and the D x d read-out isometry
//    V_nm = <n|S_i^dag|m> (Eq. InverseBasisTransformation) is obtained from the Bogoliubov
//    action of S_i^dag on the ladder operators: S^dag|0> from its annihilation condition
//    (a two-term recurrence), S^dag|m> by m applications of the transformed creation
//    operator.
//  * local operators: exactly projected X, P, X^2, P^2, XP+PX (P H P of Eq.
//    ProjectionOperator; same-mode products carry the entries of the infinite operators,
//    which SM Sec. 5 obtains by building in a larger space and truncating).
//  * MPO: the centre-collapsed finite-state machine of SM Sec. 8 for the Gaussian part:
//    cuts left of the centre carry the raw quadratures of the left block, cuts right of
//    it carry, for every quadrature a still to come, the combination
//    sum_b 2 G_ab R_b of the left block's quadratures; the transition core couples the
//    two with scalar entries 2 G_ab.  Bond dimension w_s = 2 min(s, M - s) + 2.
#include "host_mpo.h"

#include <algorithm>
#include <cmath>
#include <cstdio>

namespace vtn {

LocalOps make_local_ops(int d) {
    LocalOps o;
    o.d = d;
    auto Z = [&]() { return std::vector<cplx>((size_t)d * d, cplx(0, 0)); };
    o.I = Z(); o.X = Z(); o.P = Z(); o.X2 = Z(); o.P2 = Z(); o.XPPX = Z();
    const double is2 = 1.0 / std::sqrt(2.0);
    for (int n = 0; n < d; ++n) {
        o.I[n * d + n] = 1.0;
        o.X2[n * d + n] = n + 0.5;
        o.P2[n * d + n] = n + 0.5;
        if (n + 1 < d) {
            double s = std::sqrt((double)(n + 1)) * is2;
            o.X[n * d + n + 1] = s;
            o.X[(n + 1) * d + n] = s;
            o.P[n * d + n + 1] = cplx(0, -s);
            o.P[(n + 1) * d + n] = cplx(0, s);
        }
        if (n + 2 < d) {
            double s = std::sqrt((double)(n + 1) * (n + 2));
            o.X2[n * d + n + 2] = 0.5 * s;
            o.X2[(n + 2) * d + n] = 0.5 * s;
            o.P2[n * d + n + 2] = -0.5 * s;
            o.P2[(n + 2) * d + n] = -0.5 * s;
            o.XPPX[n * d + n + 2] = cplx(0, -s);
            o.XPPX[(n + 2) * d + n] = cplx(0, s);
        }
    }
    return o;
}

std::vector<cplx> lbo_isometry(const double S[4], int D, int d) {
    // U_g = S_hat^dag with U_g^dag R U_g = S R, so U_g^dag a U_g = mu a + nu a^dag with
    // mu = (S00 + S11)/2, nu = (S00 - S11)/2 + i S01 for symmetric S; |mu|^2 - |nu|^2 = 1.
    // U_g a U_g^dag = conj(mu) a - nu a^dag annihilates U_g|0>, and
    // U_g a^dag U_g^dag = mu a^dag - conj(nu) a raises it.
    const cplx mu(0.5 * (S[0] + S[3]), 0.5 * (S[2] - S[1]));
    const cplx nu(0.5 * (S[0] - S[3]), 0.5 * (S[1] + S[2]));
    const int Dt = D + d + 2;
    std::vector<cplx> col((size_t)Dt, cplx(0, 0)), nxt((size_t)Dt);
    col[0] = 1.0 / std::sqrt(std::abs(mu));
    const cplx ratio = nu / std::conj(mu);
    for (int n = 1; n + 1 < Dt; ++n) {
        col[n + 1] = ratio * std::sqrt((double)n / (n + 1)) * col[n - 1];
    }
    std::vector<cplx> V((size_t)D * d, cplx(0, 0));
    for (int m = 0; m < d; ++m) {
        if (m > 0) {
            const double inv = 1.0 / std::sqrt((double)m);
            const int valid = Dt - m;  // rows still exact after m applications
            for (int n = 0; n < valid; ++n) {
                cplx v = cplx(0, 0);
                if (n > 0) v += mu * std::sqrt((double)n) * col[n - 1];
                v -= std::conj(nu) * std::sqrt((double)(n + 1)) * col[n + 1];
                nxt[n] = v * inv;
            }
            for (int n = valid; n < Dt; ++n) nxt[n] = 0.0;
            col.swap(nxt);
        }
        for (int n = 0; n < D; ++n) V[(size_t)n * d + m] = col[n];
    }
    return V;
}

namespace {

// Channel layout of cut s (0..M) for the centre-collapsed MPO with transition site t.
struct Cuts {
    int M, t;
    int width(int s) const {
        if (s == 0 || s == M) return 1;
        return s <= t ? 2 * s + 2 : 2 * (M - s) + 2;
    }
    bool raw(int s) const { return s <= t; }
    // -1 if the channel does not exist at this cut
    int start(int s) const { return s == M ? -1 : 0; }
    int done(int s) const {
        if (s == 0) return -1;
        if (s == M) return 0;
        return 1;
    }
    // raw open channel of quadrature q (mode j = q % M, kind = q / M) at cut s (needs j < s)
    int open(int s, int j, int kind) const {
        if (s == 0 || s == M || !raw(s) || j >= s) return -1;
        return 2 + 2 * j + kind;
    }
    // combo channel of quadrature of mode j at cut s (needs j >= s)
    int combo(int s, int j, int kind) const {
        if (s == 0 || s == M || raw(s) || j < s) return -1;
        return 2 + 2 * (j - s) + kind;
    }
};

struct CoreBuilder {
    HostCore c;
    const LocalOps* ops;
    int d;
    void add(int a, int b, const std::vector<cplx>& op, cplx scale, bool identity) {
        if (a < 0 || b < 0 || std::abs(scale) == 0.0) return;
        c.rows.push_back(a);
        c.cols.push_back(b);
        for (int i = 0; i < d * d; ++i) c.ops.push_back(scale * op[i]);
        c.ident.push_back(identity ? 1 : 0);
    }
    void add_lin(int a, int b, double cx, double cp) {  // cx X + cp P
        if (a < 0 || b < 0 || (cx == 0.0 && cp == 0.0)) return;
        c.rows.push_back(a);
        c.cols.push_back(b);
        for (int i = 0; i < d * d; ++i) c.ops.push_back(cx * ops->X[i] + cp * ops->P[i]);
        c.ident.push_back(0);
    }
};

}  // namespace

std::string build_problem(int M, const double* r, const double* U, int D, int d, bool force_lbo,
                          HostProblem& out) {
    char msg[256];
    if (M < 1) return "M must be >= 1";
    if (D < 2) return "D must be >= 2";
    if (d < 1 || d > D) return "need 1 <= d <= D";
    if (d > 16) return "d > 16 is not supported by this build";
    for (int i = 0; i < M; ++i)
        if (!std::isfinite(r[i])) return "non-finite squeezing parameter";
    // unitarity of U (row-major, interleaved)
    auto Ue = [&](int i, int j) { return cplx(U[2 * (i * M + j)], U[2 * (i * M + j) + 1]); };
    double dev = 0.0;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            cplx s = 0.0;
            for (int k = 0; k < M; ++k) s += std::conj(Ue(k, i)) * Ue(k, j);
            dev = std::max(dev, std::abs(s - (i == j ? 1.0 : 0.0)));
        }
    if (!(dev <= 1e-10)) {
        std::snprintf(msg, sizeof msg, "U is not unitary: max |U^dag U - I| = %.3e > 1e-10", dev);
        return msg;
    }
    const int n2 = 2 * M;
    HostProblem P;
    P.M = M; P.D = D; P.d = d;
    P.lbo = force_lbo || d < D;
    P.r.assign(r, r + M);
    // O = [[Re U, -Im U], [Im U, Re U]]
    std::vector<double> O((size_t)n2 * n2);
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            cplx u = Ue(i, j);
            O[(size_t)i * n2 + j] = u.real();
            O[(size_t)i * n2 + M + j] = -u.imag();
            O[(size_t)(M + i) * n2 + j] = u.imag();
            O[(size_t)(M + i) * n2 + M + j] = u.real();
        }
    std::vector<double> ev(n2), gv(n2);
    for (int k = 0; k < M; ++k) {
        ev[k] = 0.5 * std::exp(-2 * r[k]);
        ev[M + k] = 0.5 * std::exp(2 * r[k]);
        gv[k] = 0.5 * std::exp(2 * r[k]);
        gv[M + k] = 0.5 * std::exp(-2 * r[k]);
    }
    P.V.assign((size_t)n2 * n2, 0.0);
    std::vector<double> G((size_t)n2 * n2, 0.0);
    for (int i = 0; i < n2; ++i)
        for (int j = 0; j < n2; ++j) {
            double sv = 0, sg = 0;
            for (int k = 0; k < n2; ++k) {
                sv += O[(size_t)i * n2 + k] * ev[k] * O[(size_t)j * n2 + k];
                sg += O[(size_t)i * n2 + k] * gv[k] * O[(size_t)j * n2 + k];
            }
            P.V[(size_t)i * n2 + j] = sv;
            G[(size_t)i * n2 + j] = sg;
        }
    // symmetrise (exact in exact arithmetic)
    for (int i = 0; i < n2; ++i)
        for (int j = 0; j < i; ++j) {
            double a = 0.5 * (G[(size_t)i * n2 + j] + G[(size_t)j * n2 + i]);
            G[(size_t)i * n2 + j] = G[(size_t)j * n2 + i] = a;
        }
    P.iso.assign((size_t)M * D * d, cplx(0, 0));
    P.nu.assign(M, 0.5);
    if (P.lbo) {
        std::vector<double> S((size_t)n2 * n2, 0.0);
        for (int i = 0; i < M; ++i) {
            double v00 = P.V[(size_t)i * n2 + i], v01 = P.V[(size_t)i * n2 + M + i];
            double v11 = P.V[(size_t)(M + i) * n2 + M + i];
            double det = v00 * v11 - v01 * v01;
            if (!(det > 0)) return "reduced covariance is not positive definite";
            double nu = std::sqrt(det);
            P.nu[i] = nu;
            double a00 = v00 / nu, a01 = v01 / nu, a11 = v11 / nu;
            double sc = 1.0 / std::sqrt(a00 + a11 + 2.0);
            double s[4] = {(a00 + 1.0) * sc, a01 * sc, a01 * sc, (a11 + 1.0) * sc};
            S[(size_t)i * n2 + i] = s[0];
            S[(size_t)i * n2 + M + i] = s[1];
            S[(size_t)(M + i) * n2 + i] = s[2];
            S[(size_t)(M + i) * n2 + M + i] = s[3];
            std::vector<cplx> Vi = lbo_isometry(s, D, d);
            std::copy(Vi.begin(), Vi.end(), P.iso.begin() + (size_t)i * D * d);
        }
        // G' = S^T G S (S is block-diagonal per mode; dense product is fine at set-up)
        std::vector<double> T((size_t)n2 * n2, 0.0), Gr((size_t)n2 * n2, 0.0);
        for (int i = 0; i < n2; ++i)
            for (int j = 0; j < n2; ++j) {
                double s = 0;
                for (int k = 0; k < n2; ++k) s += G[(size_t)i * n2 + k] * S[(size_t)k * n2 + j];
                T[(size_t)i * n2 + j] = s;
            }
        for (int i = 0; i < n2; ++i)
            for (int j = 0; j < n2; ++j) {
                double s = 0;
                for (int k = 0; k < n2; ++k) s += S[(size_t)k * n2 + i] * T[(size_t)k * n2 + j];
                Gr[(size_t)i * n2 + j] = s;
            }
        for (int i = 0; i < n2; ++i)
            for (int j = 0; j < i; ++j) {
                double a = 0.5 * (Gr[(size_t)i * n2 + j] + Gr[(size_t)j * n2 + i]);
                Gr[(size_t)i * n2 + j] = Gr[(size_t)j * n2 + i] = a;
            }
        G.swap(Gr);
    } else {
        for (int i = 0; i < M; ++i)
            for (int n = 0; n < d; ++n) P.iso[(size_t)i * D * d + (size_t)n * d + n] = 1.0;
    }
    P.G = G;
    // lambda_max(G) by power iteration (G is positive definite)
    {
        std::vector<double> x(n2, 1.0), y(n2);
        double lam = 0;
        for (int it = 0; it < 2000; ++it) {
            double nrm = 0;
            for (int i = 0; i < n2; ++i) {
                double s = 0;
                for (int j = 0; j < n2; ++j) s += G[(size_t)i * n2 + j] * x[j];
                y[i] = s;
                nrm += s * s;
            }
            nrm = std::sqrt(nrm);
            double l2 = 0;
            for (int i = 0; i < n2; ++i) { x[i] = y[i] / nrm; }
            for (int i = 0; i < n2; ++i) l2 += x[i] * y[i];
            // Rayleigh quotient of the previous iterate times growth
            if (std::abs(nrm - lam) <= 1e-14 * nrm) { lam = nrm; break; }
            lam = nrm;
        }
        P.norm_bound = lam * M * (2.0 * d - 1.0);
    }
    // ---------------------------------------------------------------- MPO cores
    LocalOps ops = make_local_ops(d);
    Cuts cuts{M, M / 2};
    P.w.resize(M + 1);
    for (int s = 0; s <= M; ++s) P.w[s] = cuts.width(s);
    auto g = [&](int a, int b) { return G[(size_t)a * n2 + b]; };
    const int t = cuts.t;
    for (int k = 0; k < M; ++k) {
        CoreBuilder cb;
        cb.ops = &ops;
        cb.d = d;
        cb.c.wl = P.w[k];
        cb.c.wr = P.w[k + 1];
        cb.c.d = d;
        const int L = k, R = k + 1;
        const int xk = k, pk = M + k;
        // local term h_k = G_xx X^2 + G_pp P^2 + G_xp (XP + PX) - 1/2
        std::vector<cplx> h((size_t)d * d);
        for (int i = 0; i < d * d; ++i)
            h[i] = g(xk, xk) * ops.X2[i] + g(pk, pk) * ops.P2[i] + g(xk, pk) * ops.XPPX[i] - 0.5 * ops.I[i];
        cb.add(cuts.start(L), cuts.start(R), ops.I, 1.0, true);
        cb.add(cuts.start(L), cuts.done(R), h, 1.0, false);
        cb.add(cuts.done(L), cuts.done(R), ops.I, 1.0, true);
        if (k < t) {
            // raw -> raw
            cb.add(cuts.start(L), cuts.open(R, k, 0), ops.X, 1.0, false);
            cb.add(cuts.start(L), cuts.open(R, k, 1), ops.P, 1.0, false);
            for (int j = 0; j < k; ++j)
                for (int kind = 0; kind < 2; ++kind) {
                    int b = j + kind * M;
                    cb.add(cuts.open(L, j, kind), cuts.open(R, j, kind), ops.I, 1.0, true);
                    cb.add_lin(cuts.open(L, j, kind), cuts.done(R), 2.0 * g(b, xk), 2.0 * g(b, pk));
                }
        } else if (k == t) {
            // transition: raw (cut k) -> combo (cut k + 1)
            for (int j = 0; j < k; ++j)
                for (int kind = 0; kind < 2; ++kind) {
                    int b = j + kind * M;
                    cb.add_lin(cuts.open(L, j, kind), cuts.done(R), 2.0 * g(b, xk), 2.0 * g(b, pk));
                    for (int jj = k + 1; jj < M; ++jj)
                        for (int kk = 0; kk < 2; ++kk) {
                            int a = jj + kk * M;
                            cb.add(cuts.open(L, j, kind), cuts.combo(R, jj, kk), ops.I, 2.0 * g(a, b), true);
                        }
                }
            for (int jj = k + 1; jj < M; ++jj)
                for (int kk = 0; kk < 2; ++kk) {
                    int a = jj + kk * M;
                    cb.add_lin(cuts.start(L), cuts.combo(R, jj, kk), 2.0 * g(a, xk), 2.0 * g(a, pk));
                }
        } else {
            // combo -> combo
            for (int jj = k + 1; jj < M; ++jj)
                for (int kk = 0; kk < 2; ++kk) {
                    int a = jj + kk * M;
                    cb.add(cuts.combo(L, jj, kk), cuts.combo(R, jj, kk), ops.I, 1.0, true);
                    cb.add_lin(cuts.start(L), cuts.combo(R, jj, kk), 2.0 * g(a, xk), 2.0 * g(a, pk));
                }
            cb.add(cuts.combo(L, k, 0), cuts.done(R), ops.X, 1.0, false);
            cb.add(cuts.combo(L, k, 1), cuts.done(R), ops.P, 1.0, false);
        }
        P.cores.push_back(std::move(cb.c));
    }
    out = std::move(P);
    return "";
}

// ------------------------------------------------------------------------------------
// Non-Gaussian workload (Sec. "Beyond GBS: fully connected CZ-gate", Eqs. GlobalCZgate,
// nonGBSHamiltonian): H = R'^T G R' - N/2 with R' = (X, P + xi), xi_i = kappa Xi_i,
// Xi_i = prod_{n != i} X_n.  Expanded with G symmetric:
//   H = H_G + kappa sum_{a,i} G_{a p_i} (R_a Xi_i + Xi_i R_a) + kappa^2 sum_{i,j} G_{p_i p_j} Xi_i Xi_j,
// every term a product over all modes of one exactly projected single-mode operator (the
// bulk X for the kappa terms, X^2 for the kappa^2 terms, and at most two special modes).
// The MPO is the Gaussian one with extra channels appended at every inner cut s:
//   +0 bulk-X so far, +1 kappa term complete (bulk X continues), +2 bulk-X^2 so far,
//   +3 kappa^2 term complete (bulk X^2 continues), +4+3f+t first special of type t
//   (I, X^2, XP+PX) at site f < s (bulk X), +4+3s+f first special X at site f < s (bulk X^2).
// A pair's coefficient is applied at its second special site; at cut 0 the bulk states are
// the Gaussian start channel and at cut M every complete term lands in the final channel.
std::string build_problem_cz(int M, const double* r, const double* U, int D, double kappa, HostProblem& out) {
    if (!std::isfinite(kappa)) return "non-finite kappa";
    if (M < 2) return "the global CZ workload needs M >= 2";
    HostProblem P;
    std::string e = build_problem(M, r, U, D, D, false, P);
    if (!e.empty()) return e;
    P.kappa = kappa;
    const int d = D, n2 = 2 * M;
    if (kappa == 0.0) {
        out = std::move(P);
        return "";
    }
    const LocalOps ops = make_local_ops(d);
    auto g = [&](int a, int b) { return P.G[(size_t)a * n2 + b]; };
    const std::vector<int> base = P.w;
    auto inner = [&](int s) { return s > 0 && s < M; };
    auto SX = [&](int s) { return s == 0 ? 0 : (inner(s) ? base[s] + 0 : -1); };
    auto DX = [&](int s) { return s == M ? 0 : (inner(s) ? base[s] + 1 : -1); };
    auto SX2 = [&](int s) { return s == 0 ? 0 : (inner(s) ? base[s] + 2 : -1); };
    auto DX2 = [&](int s) { return s == M ? 0 : (inner(s) ? base[s] + 3 : -1); };
    auto MX = [&](int s, int f, int t) { return (inner(s) && f < s) ? base[s] + 4 + 3 * f + t : -1; };
    auto MX2 = [&](int s, int f) { return (inner(s) && f < s) ? base[s] + 4 + 3 * s + f : -1; };
    const std::vector<cplx>* T1[3] = {&ops.I, &ops.X2, &ops.XPPX};
    double sum_xp = 0.0;
    for (int i = 0; i < M; ++i) sum_xp += 2.0 * g(i, M + i);
    for (int s = 1; s < M; ++s) P.w[s] = base[s] + 4 + 4 * s;
    for (int k = 0; k < M; ++k) {
        CoreBuilder cb;
        cb.ops = &ops;
        cb.d = d;
        cb.c = P.cores[k];
        cb.c.wl = P.w[k];
        cb.c.wr = P.w[k + 1];
        const int L = k, R = k + 1;
        const int xk = k, pk = M + k;
        // ---- kappa terms, bulk X
        cb.add(SX(L), SX(R), ops.X, 1.0, false);
        for (int t = 0; t < 3; ++t) cb.add(SX(L), MX(R, k, t), *T1[t], 1.0, t == 0);
        {
            std::vector<cplx> single((size_t)d * d);
            for (int i = 0; i < d * d; ++i)
                single[i] = kappa * 2.0 * g(pk, pk) * ops.P[i] + (k == 0 ? kappa * sum_xp * ops.X[i] : cplx(0, 0));
            cb.add(SX(L), DX(R), single, 1.0, false);
        }
        for (int f = 0; f < k; ++f) {
            for (int t = 0; t < 3; ++t) cb.add(MX(L, f, t), MX(R, f, t), ops.X, 1.0, false);
            // first special I at f: second X^2 (2 kappa G_{x_k p_f}) and XP+PX (kappa G_{p_k p_f}) at k
            std::vector<cplx> op((size_t)d * d);
            for (int i = 0; i < d * d; ++i)
                op[i] = kappa * (2.0 * g(xk, M + f) * ops.X2[i] + g(pk, M + f) * ops.XPPX[i]);
            cb.add(MX(L, f, 0), DX(R), op, 1.0, false);
            // first special X^2 / XP+PX at f: identity at k
            cb.add(MX(L, f, 1), DX(R), ops.I, kappa * 2.0 * g(f, pk), true);
            cb.add(MX(L, f, 2), DX(R), ops.I, kappa * g(M + f, pk), true);
        }
        cb.add(DX(L), DX(R), ops.X, 1.0, false);
        // ---- kappa^2 terms, bulk X^2
        cb.add(SX2(L), SX2(R), ops.X2, 1.0, false);
        cb.add(SX2(L), MX2(R, k), ops.X, 1.0, false);
        cb.add(SX2(L), DX2(R), ops.I, kappa * kappa * g(pk, pk), true);
        for (int f = 0; f < k; ++f) {
            cb.add(MX2(L, f), MX2(R, f), ops.X2, 1.0, false);
            cb.add(MX2(L, f), DX2(R), ops.X, kappa * kappa * 2.0 * g(M + f, pk), false);
        }
        cb.add(DX2(L), DX2(R), ops.X2, 1.0, false);
        P.cores[k] = std::move(cb.c);
    }
    // |H| bound for tolerances: lambda_max(G) sum_a |R'_a|^2 + N/2 with |X|, |P| <= sqrt(2d)
    const double cx = std::sqrt(2.0 * d);
    const double cxi = std::abs(kappa) * std::pow(cx, M - 1);
    const double lam = P.norm_bound / (M * (2.0 * d - 1.0));
    P.norm_bound = lam * (M * cx * cx + M * (cx + cxi) * (cx + cxi)) + 0.5 * M;
    out = std::move(P);
    return "";
}

}  // namespace vtn
