// Closed-form bond spectra of a Gaussian state (host, plain C++17; see host_spectrum.cpp).
#pragma once

#include <vector>

namespace vtn {

// Symplectic eigenvalues (ascending, m of them) of a 2m x 2m covariance in xxpp order.
std::vector<double> symplectic_eigenvalues(const std::vector<double>& Vb, int m);

// The k largest eigenvalues (descending, zero-padded) of the reduced state of modes 0..cut-1
// of the pure Gaussian state with covariance V (2M x 2M, xxpp, row-major).
std::vector<double> gaussian_bond_spectrum(const std::vector<double>& V, int M, int cut, int k);

}  // namespace vtn
