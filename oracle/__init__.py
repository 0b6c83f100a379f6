"""CPU FP64 oracle for the variational tensor-network simulation of GBS (arXiv 2410.18740).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately unoptimised
restatement of the method in numpy/scipy double precision.  Only the test-suite, the
package's ``smoke()`` check and the benchmark's CPU-baseline leg may import it; the CUDA
library never links, imports or calls anything here, and the two share no code.  The
only shared module is ``paper_2410_18740_gb300.inputs`` (seeded random instances), which
carries none of the method's arithmetic.

Modules (each function cites the passage of the paper it follows):

* ``philox``      -- Philox4x32-10 counter-based generator (Salmon et al., SC'11), used
                     where the method draws random numbers (initial MPS, sampling).
* ``gbs``         -- covariance matrix and Hamiltonian coefficients (Eq. GBSHamiltonian),
                     exactly projected local operators (Eq. ProjectionOperator, SM Sec. 5),
                     Gaussian optimal local basis and its isometry (Eqs. WilliamsonDecomposition,
                     OLB, InverseBasisTransformation, Effectivecutoff), and the closed-form
                     Gaussian bond spectra (symplectic eigenvalues of a block's covariance).
* ``mpo``         -- matrix product operator of the Gaussian Hamiltonian (SM Sec. 8), built
                     with a plain "carry every quadrature" state machine (w = 2N + 2).
* ``dense``       -- dense Fock-space P H P and its exact ground state for tiny N, and
                     brute-force hafnian amplitudes of the GBS state.
* ``dmrg``        -- two-site DMRG (Sec. "Matrix Product States"): environments, effective
                     Hamiltonian product, Lanczos, truncation, sweeps, energy (Eq. MagOfSimError).
* ``dmrg1``       -- single-site DMRG with subspace expansion (Secs. "Results" and
                     "Discussion"): single-site effective Hamiltonian, expansion, sweeps.
* ``nongauss``    -- the global-CZ (non-Gaussian) parent Hamiltonian (Eq. nonGBSHamiltonian):
                     definition, term expansion and its MPO.
* ``mlp``         -- the warm start's multilayer perceptron: forward, MSE gradient, Adam.
* ``observables`` -- Fock-basis marginals after the inverse basis transformation and
                     sequential conditional sampling.

Parity status of each function is listed in its docstring; functions without an
independent pin say "parity unpinned".
"""
