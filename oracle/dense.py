"""Dense Fock-space checks for tiny N -- oracle (test infrastructure only).

* ``dense_hamiltonian``: P H P on the full d^N space, assembled term by term from
  Eq. GBSHamiltonian with Kronecker products (mode 0 is the most significant index,
  matching the MPS ordering c_{n_1 n_2 ... n_N} of Eq. MPSAnsatz).
* ``ground_state``: lowest eigenpair of P H P (library eigensolver), the "dense exact
  solve" the paper delegates to thewalrus for D^N <~ 1e6 (Sec. "Gaussian Boson Sampling").
* ``gbs_amplitudes``: <n|psi> from brute-force hafnians, written from the GBS amplitude
  formula of the literature the paper builds on: |psi> = prod_k cosh(r_k)^{-1/2}
  exp(1/2 a^dag^T B a^dag)|0>, B = -U diag(tanh r) U^T, so
  <n|psi> = Haf(B_n) / sqrt(prod n_k! prod cosh r_k).
"""
import itertools
from functools import lru_cache

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import gbs


def _embed(op_list, N, d):
    """Kronecker product with op_list[i] (or identity) on mode i."""
    out = None
    for i in range(N):
        A = op_list.get(i, None)
        A = sp.identity(d, dtype=np.complex128, format="csr") if A is None else sp.csr_matrix(A)
        out = A if out is None else sp.kron(out, A, format="csr")
    return out


def dense_hamiltonian(G, d):
    """Sparse (d^N x d^N) P H P with H = sum_{ab} G_ab R_a R_b - N/2, same-mode products
    exactly projected, cross-mode products as tensor products."""
    G = np.asarray(G, dtype=np.float64)
    N = G.shape[0] // 2
    ops = gbs.local_ops(d)
    R = lambda a: ops["X"] if a < N else ops["P"]
    dim = d ** N
    H = sp.csr_matrix((dim, dim), dtype=np.complex128)
    for i in range(N):
        xi, pi = i, N + i
        hi = G[xi, xi] * ops["X2"] + G[pi, pi] * ops["P2"] + G[xi, pi] * ops["XPPX"] - 0.5 * ops["I"]
        H = H + _embed({i: hi}, N, d)
    for a in range(2 * N):
        for b in range(2 * N):
            ma, mb = a % N, b % N
            if ma == mb or G[a, b] == 0.0:
                continue
            H = H + G[a, b] * _embed({ma: R(a), mb: R(b)}, N, d)
    return H


def ground_state(G, d, k=1):
    """Lowest k eigenpairs of P H P (dense eigh below 4096 states, else Lanczos from scipy)."""
    H = dense_hamiltonian(G, d)
    if H.shape[0] <= 4096:
        w, v = np.linalg.eigh(H.toarray())
        return w[:k], v[:, :k]
    w, v = spla.eigsh(H, k=k, which="SA", tol=1e-14)
    order = np.argsort(w)
    return w[order], v[:, order]


def hafnian(A):
    """Hafnian by the perfect-matching recursion: Haf(A) = sum_{j>0} A_{0j} Haf(A without
    rows/cols 0, j).  Exponential; for <= 12 rows."""
    A = np.asarray(A)
    n = A.shape[0]
    if n == 0:
        return 1.0 + 0j
    if n % 2:
        return 0.0 + 0j

    @lru_cache(maxsize=None)
    def rec(mask):
        if mask == 0:
            return 1.0 + 0j
        idx = [i for i in range(n) if mask >> i & 1]
        i0 = idx[0]
        total = 0.0 + 0j
        for j in idx[1:]:
            total += A[i0, j] * rec(mask & ~(1 << i0) & ~(1 << j))
        return total

    return rec((1 << n) - 1)


def _fact(k):
    out = 1.0
    for j in range(2, k + 1):
        out *= j
    return out


def gbs_amplitudes(r, U, D):
    """Tensor of <n|psi> for all n with n_k < D (tiny N only)."""
    N = len(r)
    out = np.zeros((D,) * N, dtype=np.complex128)
    for n in itertools.product(range(D), repeat=N):
        if sum(n) % 2:
            continue
        out[n] = gbs_amplitude(r, U, n)
    return out


def gbs_amplitude(r, U, n):
    """<n|psi> for photon pattern n (tuple of ints)."""
    r = np.asarray(r, dtype=np.float64)
    U = np.asarray(U, dtype=np.complex128)
    B = -U @ np.diag(np.tanh(r)) @ U.T
    rows = [k for k, nk in enumerate(n) for _ in range(nk)]
    Bn = B[np.ix_(rows, rows)]
    norm = np.sqrt(np.prod([_fact(nk) for nk in n]) * np.prod(np.cosh(r)))
    return hafnian(Bn) / norm


def marginals_from_vector(psi, N, d, modes):
    """Joint Fock marginal of the listed modes from a dense normalised vector."""
    p = np.abs(np.asarray(psi).reshape((d,) * N)) ** 2
    p = p / p.sum()
    other = tuple(i for i in range(N) if i not in modes)
    m = p.sum(axis=other)
    # axes of m are in increasing mode order; reorder to the requested order
    order = np.argsort(np.argsort(modes))
    return np.transpose(m, axes=order) if len(modes) > 1 else m
