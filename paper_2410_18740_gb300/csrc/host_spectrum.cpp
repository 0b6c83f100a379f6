// Closed-form bond spectra of a Gaussian state (host, plain C++17).
//
// The reduced state of modes 0..s-1 of a pure Gaussian state is, after a symplectic
// (Williamson) transformation of the block, a product of thermal states with mean photon
// numbers nbar_j = nu_j - 1/2, where nu_j are the symplectic eigenvalues of the block's
// covariance (the multi-mode form of the thermal reduced states the paper derives for the
// optimal local basis, Eq. diagReducedGaussianDM).  Its eigenvalues -- the squared Schmidt
// values of the cut -- are the products prod_j (1 - q_j) q_j^{n_j}, q_j = nbar_j / (nbar_j + 1).
// Local basis changes do not alter them; the Fock cutoff does (this is the infinite-cutoff
// spectrum, which the truncated ground state approaches as the cutoff grows).  The state is
// pure, so the smaller of the two blocks of a cut gives the spectrum.
//
// nu_j: with K = V^{1/2} (i Omega) V^{1/2} Hermitian, K^2 = -V^{1/2} Omega V Omega V^{1/2} is real
// symmetric with eigenvalues nu_j^2, each twice.  Both symmetric eigenproblems are solved by
// cyclic Jacobi rotations.
#include <algorithm>
#include <cmath>
#include <functional>
#include <queue>
#include <utility>
#include <string>
#include <vector>

#include "host_spectrum.h"

namespace vtn {
namespace {

// Eigenvalues (and, if Q != null, eigenvectors as columns of Q) of a symmetric n x n matrix.
void jacobi_eigh(std::vector<double> A, int n, std::vector<double>& w, std::vector<double>* Q) {
    if (Q) {
        Q->assign((size_t)n * n, 0.0);
        for (int i = 0; i < n; ++i) (*Q)[(size_t)i * n + i] = 1.0;
    }
    auto at = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
    double scale = 0.0;
    for (double x : A) scale = std::max(scale, std::fabs(x));
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off = std::max(off, std::fabs(at(i, j)));
        if (off <= 1e-17 * scale || scale == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = at(p, q);
                if (std::fabs(apq) <= 1e-300) continue;
                // rotation that zeroes A[p][q]
                const double theta = (at(q, q) - at(p, p)) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double akp = at(k, p), akq = at(k, q);
                    at(k, p) = c * akp - s * akq;
                    at(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double apk = at(p, k), aqk = at(q, k);
                    at(p, k) = c * apk - s * aqk;
                    at(q, k) = s * apk + c * aqk;
                }
                if (Q)
                    for (int k = 0; k < n; ++k) {
                        double& qkp = (*Q)[(size_t)k * n + p];
                        double& qkq = (*Q)[(size_t)k * n + q];
                        const double a = qkp, b = qkq;
                        qkp = c * a - s * b;
                        qkq = s * a + c * b;
                    }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = at(i, i);
}

}  // namespace

std::vector<double> symplectic_eigenvalues(const std::vector<double>& Vb, int m) {
    const int n = 2 * m;
    std::vector<double> w, Q;
    jacobi_eigh(Vb, n, w, &Q);
    // S = V^{1/2} = Q diag(sqrt w) Q^T
    std::vector<double> S((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += Q[(size_t)i * n + k] * std::sqrt(std::max(w[k], 0.0)) * Q[(size_t)j * n + k];
            S[(size_t)i * n + j] = acc;
        }
    // Omega (xxpp): Omega[i][m + i] = 1, Omega[m + i][i] = -1; (Omega X)[i][.] = X[m + i][.],
    // (Omega X)[m + i][.] = -X[i][.]
    auto omega_left = [&](const std::vector<double>& X) {
        std::vector<double> Y((size_t)n * n);
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) {
                Y[(size_t)i * n + j] = X[(size_t)(m + i) * n + j];
                Y[(size_t)(m + i) * n + j] = -X[(size_t)i * n + j];
            }
        return Y;
    };
    auto matmul = [&](const std::vector<double>& A, const std::vector<double>& B) {
        std::vector<double> C((size_t)n * n, 0.0);
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < n; ++k) {
                const double a = A[(size_t)i * n + k];
                for (int j = 0; j < n; ++j) C[(size_t)i * n + j] += a * B[(size_t)k * n + j];
            }
        return C;
    };
    // K2 = -S Omega V Omega S
    std::vector<double> OS = omega_left(S);            // Omega S
    std::vector<double> VOS = matmul(Vb, OS);          // V Omega S
    std::vector<double> OVOS = omega_left(VOS);        // Omega V Omega S
    std::vector<double> K2 = matmul(S, OVOS);
    for (double& x : K2) x = -x;
    for (int i = 0; i < n; ++i)  // symmetrise the rounding
        for (int j = i + 1; j < n; ++j) {
            const double a = 0.5 * (K2[(size_t)i * n + j] + K2[(size_t)j * n + i]);
            K2[(size_t)i * n + j] = K2[(size_t)j * n + i] = a;
        }
    std::vector<double> ev;
    jacobi_eigh(K2, n, ev, nullptr);
    std::sort(ev.begin(), ev.end());
    std::vector<double> nu(m);
    for (int j = 0; j < m; ++j) nu[j] = std::sqrt(std::max(0.0, 0.5 * (ev[2 * j] + ev[2 * j + 1])));
    return nu;
}

std::vector<double> gaussian_bond_spectrum(const std::vector<double>& V, int M, int cut, int k) {
    std::vector<double> spec(1, 1.0);
    if (cut > 0 && cut < M) {
        // a pure state's two sides share their spectrum: use the smaller block
        const int first = 2 * cut <= M ? 0 : cut;
        const int m = 2 * cut <= M ? cut : M - cut, n = 2 * m;
        std::vector<double> Vb((size_t)n * n);
        auto idx = [&](int a) { return a < m ? first + a : M + first + (a - m); };
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) Vb[(size_t)a * n + b] = V[(size_t)idx(a) * 2 * M + idx(b)];
        const std::vector<double> nu = symplectic_eigenvalues(Vb, m);
        for (double v : nu) {
            const double nbar = std::max(v - 0.5, 0.0), q = nbar / (nbar + 1.0);
            // top k of {spec[i] (1 - q) q^n}: only the top k partial products can contribute;
            // every row i is descending in n, so a k-way merge with a heap finds them
            using Item = std::pair<double, std::pair<int, int>>;  // (value, (i, n))
            std::priority_queue<Item> heap;
            for (int i = 0; i < (int)spec.size(); ++i) heap.push({spec[i] * (1.0 - q), {i, 0}});
            std::vector<double> next;
            next.reserve((size_t)k);
            while ((int)next.size() < k && !heap.empty()) {
                const Item top = heap.top();
                heap.pop();
                if (top.first <= 0.0) break;
                next.push_back(top.first);
                heap.push({top.first * q, {top.second.first, top.second.second + 1}});
            }
            spec.swap(next);
            if (spec.empty()) spec.push_back(0.0);
        }
    }
    spec.resize(k, 0.0);
    return spec;
}

}  // namespace vtn
