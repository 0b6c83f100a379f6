// Host-side problem set-up: Hamiltonian coefficients, Gaussian optimal local basis,
// exactly projected local operators and the centre-collapsed MPO of the GBS parent
// Hamiltonian.  Plain C++17, no CUDA; runs once per problem before anything is uploaded.
#pragma once

#include <complex>
#include <string>
#include <vector>

namespace vtn {

using cplx = std::complex<double>;

struct HostCore {
    int wl = 0, wr = 0, d = 0;
    std::vector<int> rows, cols;
    std::vector<cplx> ops;          // nnz * d * d, ops[k][s'][s]
    std::vector<unsigned char> ident;  // 1 if ops[k] = s * I (scalar in ops[k][0][0])
    int nnz() const { return (int)rows.size(); }
};

struct HostProblem {
    int M = 0, D = 0, d = 0;
    bool lbo = false;
    std::vector<double> r;          // [M]
    std::vector<double> V;          // covariance, 2M x 2M, xxpp
    std::vector<double> G;          // coefficients actually used (G or S^T G S), 2M x 2M
    std::vector<double> nu;         // symplectic eigenvalues (LBO) [M]
    std::vector<cplx> iso;          // M * D * d isometries V_nm (row n, col m)
    std::vector<int> w;             // bond dims, M + 1
    std::vector<HostCore> cores;    // M cores
    double norm_bound = 0.0;
    double kappa = 0.0;             // non-Gaussian workload only
};

// Builds everything; returns "" on success, otherwise the validation error message.
std::string build_problem(int M, const double* r, const double* U_interleaved, int D, int d,
                          bool force_lbo, HostProblem& out);

// The non-Gaussian (global CZ) workload in the Fock basis (d = D): the Gaussian MPO with the
// channels of the kappa and kappa^2 terms appended.
std::string build_problem_cz(int M, const double* r, const double* U_interleaved, int D, double kappa,
                             HostProblem& out);

// Exactly projected single-mode operators of dimension d (closed-form entries).
struct LocalOps {
    int d;
    std::vector<cplx> I, X, P, X2, P2, XPPX;
};
LocalOps make_local_ops(int d);

// D x d isometry <n|S^dag|m> for a symmetric symplectic 2x2 S (row-major s00 s01 s10 s11).
std::vector<cplx> lbo_isometry(const double S[4], int D, int d);

}  // namespace vtn
