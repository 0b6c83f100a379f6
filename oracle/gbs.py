"""GBS Hamiltonian coefficients, exactly projected local operators and the Gaussian
optimal local basis -- oracle (test infrastructure only; see ``oracle/__init__``).

Conventions (hbar = 1, vacuum quadrature variance 1/2, Sec. "Deriving the Hamiltonian"):
quadrature vector R = (X_1..X_N, P_1..P_N) ("xxpp"), a = (X + iP)/sqrt(2),
output modes a_out = U a_in, single-mode squeezers squeeze X: Var X_k = exp(-2 r_k)/2.
"""
import numpy as np
import scipy.linalg as sla


# ----------------------------------------------------------------------------------
# Covariance and Hamiltonian coefficients (Sec. "Gaussian Boson Sampling",
# Eq. GBSHamiltonian): V = 1/2 O D^2 O^T, H = R^T (V^{-1}/4) R - N/2.
# ----------------------------------------------------------------------------------

def quadrature_orthogonal(U):
    """O with R_out = O R_in for the passive transformation a_out = U a_in."""
    U = np.asarray(U, dtype=np.complex128)
    return np.block([[U.real, -U.imag], [U.imag, U.real]])


def covariance(r, U):
    """V = O (1/2 diag(e^{-2r}, e^{2r})) O^T -- the D matrix of Eq. (D = diag(e^{-r},e^{r}))
    squared and rotated by the interferometer.  Pinned: tr V = sum cosh 2r, 4 G V = I."""
    r = np.asarray(r, dtype=np.float64)
    O = quadrature_orthogonal(U)
    Vin = 0.5 * np.diag(np.concatenate([np.exp(-2 * r), np.exp(2 * r)]))
    return O @ Vin @ O.T


def hamiltonian_coefficients(r, U):
    """G = V^{-1}/4 (Eq. GBSHamiltonian), computed as the matrix inverse of the covariance
    (a library primitive) so that it is independent of any closed form."""
    return np.linalg.inv(covariance(r, U)) / 4.0


# ----------------------------------------------------------------------------------
# Local operators in the truncated Fock basis.  The paper keeps P H P (Eq.
# ProjectionOperator and the text after Eq. EffectiveHamiltonian) and builds operator
# products in a larger space before truncating (SM Sec. 5, "D+4 then truncate").
# ----------------------------------------------------------------------------------

def ladder(dim):
    a = np.zeros((dim, dim), dtype=np.complex128)
    for n in range(1, dim):
        a[n - 1, n] = np.sqrt(n)
    return a


def local_ops(d, pad=4):
    """Exactly projected single-mode operators of dimension d.

    Returns dict with X, P (truncations of the infinite operators) and X2, P2, XPPX
    (= X^2, P^2, XP + PX) computed as matrix products in dimension d + pad and then
    truncated to d x d, which equals the exact projection P A P for products of two
    quadratures when pad >= 1.  Pinned: X2 + P2 = diag(2n+1) exactly; X2 differs from
    (X_d)^2 only at entry (d-1, d-1) (SM Sec. 5)."""
    big = d + pad
    a = ladder(big)
    ad = a.conj().T
    X = (a + ad) / np.sqrt(2.0)
    P = -1j * (a - ad) / np.sqrt(2.0)
    cut = lambda A: np.ascontiguousarray(A[:d, :d])
    return {
        "I": np.eye(d, dtype=np.complex128),
        "X": cut(X),
        "P": cut(P),
        "X2": cut(X @ X),
        "P2": cut(P @ P),
        "XPPX": cut(X @ P + P @ X),
        "N": cut(ad @ a),
    }


# ----------------------------------------------------------------------------------
# Gaussian optimal local basis (Sec. "Optimal Local Basis for Gaussian States").
# ----------------------------------------------------------------------------------

def reduced_covariance(V, i):
    """2x2 covariance of mode i (rows/cols x_i, p_i of the xxpp matrix)."""
    N = V.shape[0] // 2
    idx = [i, N + i]
    return V[np.ix_(idx, idx)]


def williamson_single(Vi):
    """Eq. WilliamsonDecomposition for one mode: V_i = S_i nu_i I S_i^T.

    nu_i = sqrt(det V_i) (= nbar_i + 1/2 of Eq. diagReducedGaussianDM).  The rotation
    freedom S_i -> S_i R(theta) is fixed by the symmetric choice S_i = (V_i / nu_i)^{1/2},
    computed here through an eigendecomposition (library primitive).  Returns (S_i, nu_i).
    """
    nu = np.sqrt(np.linalg.det(Vi))
    w, Q = np.linalg.eigh(Vi / nu)
    S = Q @ np.diag(np.sqrt(w)) @ Q.T
    return S, nu


def lbo_transform(r, U):
    """Per-mode symplectics S_i, symplectic eigenvalues nu_i and the rotated coefficient
    matrix G' = S^T G S (Eq. OLB: H -> S_i H S_i^dagger acts on the quadratures of mode i
    by S_i, so R^T G R -> R^T S^T G S R).  Returns (S_list, nu, G_rot)."""
    V = covariance(r, U)
    G = hamiltonian_coefficients(r, U)
    N = V.shape[0] // 2
    S_full = np.zeros_like(V)
    S_list, nus = [], []
    for i in range(N):
        S, nu = williamson_single(reduced_covariance(V, i))
        S_list.append(S)
        nus.append(nu)
        idx = [i, N + i]
        S_full[np.ix_(idx, idx)] = S
    return S_list, np.array(nus), S_full.T @ G @ S_full


def quadratic_generator_ops(dim, pad=4):
    ops = local_ops(dim, pad)
    return ops["X2"], ops["P2"], ops["XPPX"]


def lbo_isometry(S, D, d, big=None):
    """V_nm = <n| S_hat^dagger |m>, n < D, m < d (Eq. InverseBasisTransformation).

    S_hat^dagger is the single-mode Gaussian unitary U_g with U_g^dagger R U_g = S R.
    Written as U_g = exp(-i R^T Q R / 2) with exp(Omega Q) = S, i.e.
    Q = -Omega log(S) (Omega = [[0,1],[-1,0]], [X, P] = i).  The exponential is taken with
    scipy's expm (library primitive) in a Fock space of dimension ``big`` >> D, then cut.
    Pinned: V^dagger V = I_d (Eq. Effectivecutoff) and |V[:,0]|^2 = squeezed-vacuum
    photon statistics."""
    if big is None:
        big = D + d + 320
    Om = np.array([[0.0, 1.0], [-1.0, 0.0]])
    w, Qs = np.linalg.eigh(S)
    logS = Qs @ np.diag(np.log(w)) @ Qs.T
    Q = -Om @ logS
    Q = 0.5 * (Q + Q.T)
    X2, P2, XPPX = quadratic_generator_ops(big)
    Hg = 0.5 * (Q[0, 0] * X2 + Q[1, 1] * P2 + Q[0, 1] * XPPX)
    Ug = sla.expm(-1j * Hg)
    return np.ascontiguousarray(Ug[:D, :d])


def truncation_epsilon(nu, d):
    """Eq. SpecWfromSDsums: eps = 1 - (1/N) sum_i sum_{k<d} nbar^k/(nbar+1)^{k+1},
    nbar_i = nu_i - 1/2 (the thermal occupations of Eq. diagReducedGaussianDM)."""
    nbar = np.asarray(nu) - 0.5
    k = np.arange(d)
    kept = np.sum(nbar[:, None] ** k[None, :] / (nbar[:, None] + 1.0) ** (k[None, :] + 1), axis=1)
    return 1.0 - np.mean(kept)


def norm_bound(G, N, d):
    """Deterministic bound on ||P H P||: P H P + N/2 <= lambda_max(G) sum_i P(X_i^2+P_i^2)P
    = lambda_max(G) sum_i (2 n_i + 1) <= lambda_max(G) N (2d - 1)."""
    return float(np.max(np.linalg.eigvalsh(G))) * N * (2 * d - 1)


# ----------------------------------------------------------------------------------
# Bond spectra of the Gaussian state (the multi-mode form of Eq. diagReducedGaussianDM):
# the reduced state of modes 0..s-1 is, after a Williamson transformation, a product of
# thermal states with nbar_j = nu_j - 1/2, nu_j the symplectic eigenvalues of the block's
# covariance.  Its eigenvalues -- the squared Schmidt values of the cut -- are the products
# prod_j (1 - q_j) q_j^{n_j}, q_j = nbar_j / (nbar_j + 1).  This is the infinite-cutoff
# spectrum; the truncated P H P ground state approaches it as d grows.
# ----------------------------------------------------------------------------------

def symplectic_eigenvalues(Vsub):
    """nu_j >= 1/2 of a 2m x 2m covariance (xxpp): the moduli of the eigenvalues of
    i Omega V (library eigvals), each appearing twice; returned ascending, m of them."""
    m = Vsub.shape[0] // 2
    Om = np.block([[np.zeros((m, m)), np.eye(m)], [-np.eye(m), np.zeros((m, m))]])
    ev = np.linalg.eigvals(1j * Om @ Vsub)
    return np.sort(np.abs(ev.real))[::2]


def gaussian_schmidt_spectrum(V, s, k, n_max=24):
    """The k largest eigenvalues of the reduced state of modes 0..s-1 (descending)."""
    N = V.shape[0] // 2
    idx = list(range(s)) + [N + j for j in range(s)]
    nu = symplectic_eigenvalues(V[np.ix_(idx, idx)])
    nbar = np.maximum(nu - 0.5, 0.0)
    q = nbar / (nbar + 1.0)
    spec = np.ones(1)
    for qj in q:
        p = (1.0 - qj) * qj ** np.arange(n_max + 1)
        spec = np.outer(spec, p).reshape(-1)
        spec = np.sort(spec)[::-1][: max(k, 1) * 64]    # keep a generous head
    return np.sort(spec)[::-1][:k]
