"""Observables of a variational MPS -- oracle (test infrastructure only).

* ``fock_tensors``: the inverse basis transformation of Eq. InverseBasisTransformation
  applied to every physical leg, A^F[a, n, b] = sum_m V_nm A[a, m, b] (n < D).
* ``marginal``: joint photon-number distribution P(n_{i1}, ..., n_{ik}) of the listed
  modes (the P(n) of Sec. "Main Methodology"): the partial trace over every other mode
  (taken in the solver basis, which is complete for the variational state), then the
  inverse basis transformation on the listed modes only.  Normalised by <psi|psi>, so
  with a local basis the probabilities of n < D sum to at most one.  Computed by
  brute-force transfer contractions carrying the open photon numbers.
* ``reduced_density``: the single-mode reduced density matrix rho_i (d x d, solver basis) of
  the variational state -- the partial trace over every other mode -- normalised by
  <psi|psi>; its diagonal in the Fock basis is the marginal P_i(n).
* ``sample``: sequential conditional sampling in the Fock basis,
  p(n_i | n_<i) proportional to || l_{i-1} A^F_i[n_i] ||^2 weighted by the right
  environment, inverse-CDF pick with a Philox uniform per (sample, mode).  The paper
  states that all of P(n) is available but gives no sampling algorithm; this is the
  standard chain-rule sampler for MPS, stated in the design notes as a reading.
"""
import numpy as np

from . import philox


def fock_tensors(mps, isometries):
    if isometries is None:
        return [A.copy() for A in mps]
    return [np.einsum("nm,amb->anb", V, A, optimize=True) for A, V in zip(mps, isometries)]


def _right_envs(mps):
    """Right transfer environments (ket, bra) of <psi|psi> in the solver basis."""
    N = len(mps)
    E = [None] * (N + 1)
    E[N] = np.ones((1, 1), dtype=np.complex128)
    for s in range(N - 1, -1, -1):
        A = mps[s]
        E[s] = np.einsum("asb,csb->ac", A, np.einsum("csd,bd->csb", A.conj(), E[s + 1], optimize=True), optimize=True)
    return E


def norm2_solver_basis(mps):
    E = np.ones((1, 1), dtype=np.complex128)
    for A in mps:
        E = np.einsum("isk,isl->kl", A.conj(), np.einsum("ij,jsl->isl", E, A, optimize=True), optimize=True)
    return float(E[0, 0].real)


def marginal(mps, isometries, modes):
    """Joint Fock-basis marginal of ``modes`` (list of distinct ints), shape (D,)*k,
    axes in the order given."""
    mpsF = fock_tensors(mps, isometries)
    N = len(mpsF)
    modes = list(modes)
    pos = {m: j for j, m in enumerate(sorted(modes))}
    # state: dict tuple(n for processed selected modes, ascending mode order) -> env (bra, ket)
    envs = {(): np.ones((1, 1), dtype=np.complex128)}
    for s in range(N):
        A = mpsF[s]
        new = {}
        for key, E in envs.items():
            if s in pos:
                for n in range(A.shape[1]):
                    An = A[:, n, :]
                    new[key + (n,)] = An.conj().T @ E @ An
            else:
                As = mps[s]   # traced mode: solver basis
                new[key] = np.einsum("isk,isl->kl", As.conj(), np.einsum("ij,jsl->isl", E, As, optimize=True), optimize=True)
        envs = new
    D = mpsF[0].shape[1]
    out = np.zeros((D,) * len(modes))
    for key, E in envs.items():
        out[key] = E[0, 0].real
    out /= norm2_solver_basis(mps)
    order = [pos[m] for m in modes]
    return np.transpose(out, axes=order) if len(modes) > 1 else out


def all_single_marginals(mps, isometries):
    return np.array([marginal(mps, isometries, [i]) for i in range(len(mps))])


def sample(mps, isometries, seed, n_samples):
    """int32 array [n_samples, N] of photon numbers."""
    mpsF = fock_tensors(mps, isometries)
    N = len(mpsF)
    Er = _right_envs(mps)
    out = np.zeros((n_samples, N), dtype=np.int32)
    for t in range(n_samples):
        l = np.ones((1,), dtype=np.complex128)
        for s in range(N):
            A = mpsF[s]
            cand = np.einsum("a,anb->nb", l, A, optimize=True)
            p = np.real(np.einsum("nb,nb->n", cand @ Er[s + 1], cand.conj(), optimize=True))
            p = np.maximum(p, 0.0)
            cdf = np.cumsum(p)
            u = float(philox.sample_uniforms(seed, np.array([t], dtype=np.uint64), s)[0])
            target = u * cdf[-1]
            n = int(np.searchsorted(cdf, target, side="right"))
            n = min(n, A.shape[1] - 1)
            out[t, s] = n
            l = cand[n] / np.sqrt(p[n])
    return out


def reduced_density(mps, site):
    """rho[s, s'] = <psi| (|s'><s| on ``site``) |psi> / <psi|psi>: the left transfer environment of
    sites < site, the site tensor, the right transfer environment of sites > site."""
    E = np.ones((1, 1), dtype=np.complex128)          # (bra, ket)
    for A in mps[:site]:
        E = np.einsum("isk,isl->kl", A.conj(), np.einsum("ij,jsl->isl", E, A, optimize=True), optimize=True)
    Er = _right_envs(mps)[site + 1]                    # (ket, bra)
    A = mps[site]
    rho = np.einsum("ij,jsb,bc,itc->st", E, A, Er, A.conj(), optimize=True)
    return rho / norm2_solver_basis(mps)
