"""Single-site DMRG with subspace expansion -- oracle (test infrastructure only).

Sec. "Results" finds the GBS ground state with single-site DMRG, and Sec. "Discussion" grows
the bond dimension from O(1) to its final value during the sweeps, citing the strictly
single-site algorithm with subspace expansion (Hubig, McCulloch, Schollwoeck and Wolf,
Phys. Rev. B 91, 155115 (2015)) for it.  A single-site update cannot enlarge a bond by
itself; the expansion does, by appending to the optimised tensor the action of the left
block of H on it.  This restatement, step by step in plain numpy, at site i sweeping right
(the left sweep is the mirror image):

1. Lanczos (``dmrg.lanczos_lowest``) on the single-site effective Hamiltonian
       y[l, t, r'] = sum L_i[a, l, l'] W_i[a, b, t, s] A[l', s, r] R_{i+1}[b, r, r']
   for the centre tensor A = A_i (chi_l, d, chi_r).
2. Expansion: P[(l, t), (b, r)] = sum L_i[a, l, l'] W_i[a, b, t, s] A[l', s, r] and
   Mx = [A | alpha P], a (chi_l d) x chi_r (1 + w_r) matrix; the next tensor B_{i+1}
   gains w_r chi_r zero rows, so Mx [B_{i+1}; 0] = A B_{i+1} and the state is unchanged.
3. Truncation of Mx by the eigendecomposition of Mx Mx^dag (``dmrg.truncate``): keep
   k = min(chi, chi_l d, chi_r (1 + w_r), d chi_{i+2}) eigenpairs of largest eigenvalue (the
   last bound: the bond cannot usefully exceed what the next site spans), then drop those
   with lambda <= cutoff * lambda_max -- the numerical null space of Mx, whose basis is
   arbitrary (the identity channel of W makes one block of P a copy of A, so Mx is rank
   deficient by construction).
4. A_i <- U_k (left-canonical); the centre moves on: A_{i+1} <- (U_k^dag A) B_{i+1};
   L_{i+1} from A_i.

Sweep: sites 0 .. N-2 to the right, then N-1 .. 1 to the left, with the centre ending on
site 0; the energy after each sweep is ``dmrg.energy`` of the whole MPS.  The expansion
weight of sweep t is alpha * alpha_decay^t.  Readings (the paper fixes none of them): this
fixed schedule instead of the adaptive alpha of the cited algorithm, the cutoff rule of step
3, and the sweep order.

Parity: pinned by the dense projected Hamiltonian (H_eff of step 1 equals Phi^dag H Phi for
the isometry Phi from the centre tensor to the state), by the invariance of the state under
the expansion, by the identity sum_b P[:, (b, r)] R[b, r, r'] = H_eff A (step 2 against
step 1), and by convergence to the dense ground energy from a product state (bond
dimension 1), which single-site DMRG cannot leave without the expansion.
"""
from dataclasses import dataclass, field

import numpy as np

from . import dmrg


def heff1_apply(L, W, R, A):
    """y[l, t, r'] = sum L[a, l, l'] W[a, b, t, s] A[l', s, r] R[b, r, r'] (step 1), one
    index group at a time (L, then W, then R)."""
    T = np.einsum("aij,jsk->aisk", L, A, optimize=True)
    U = np.einsum("abts,aisk->bitk", W, T, optimize=True)
    return np.einsum("bitk,bkl->itl", U, R, optimize=True)


def expand_right(L, W, A, alpha):
    """Mx = [A | alpha P] of step 2 as a (chi_l d) x chi_r (1 + w_r) matrix, columns ordered
    (block, r) with block 0 = A and block 1 + b = alpha P[:, b, :]."""
    cl, d, cr = A.shape
    T = np.einsum("aij,jsk->aisk", L, A, optimize=True)
    P = np.einsum("abts,aisk->itbk", W, T, optimize=True)          # (l, t, b, r)
    wr = W.shape[1]
    Mx = np.empty((cl * d, (1 + wr) * cr), dtype=np.complex128)
    Mx[:, :cr] = A.reshape(cl * d, cr)
    Mx[:, cr:] = alpha * P.reshape(cl * d, wr * cr)
    return Mx


def expand_left(R, W, A, alpha):
    """Mirror of ``expand_right``: Mx = [A; alpha P] with
    P[(a, l), (t, r')] = sum W[a, b, t, s] A[l, s, r] R[b, r, r'], a chi_l (1 + w_l) x (d chi_r)
    matrix, rows ordered (block, l) with block 0 = A and block 1 + a = alpha P[a]."""
    cl, d, cr = A.shape
    T = np.einsum("jsg,cgp->cjsp", A, R, optimize=True)
    P = np.einsum("bcts,cjsp->bjtp", W, T, optimize=True)          # (a, l, t, r')
    wl = W.shape[0]
    Mx = np.empty(((1 + wl) * cl, d * cr), dtype=np.complex128)
    Mx[:cl] = A.reshape(cl, d * cr)
    Mx[cl:] = alpha * P.reshape(wl * cl, d * cr)
    return Mx


def _keep(w, cutoff):
    """Number of leading eigenvalues (descending) above cutoff * the largest (at least 1)."""
    if w.size == 0:
        return 0
    return max(1, int(np.count_nonzero(w > cutoff * w[0])))


@dataclass
class SweepReport1:
    energies: list = field(default_factory=list)
    max_discarded: list = field(default_factory=list)
    dims: list = field(default_factory=list)
    matvecs: int = 0
    not_converged: int = 0


def dmrg1(cores, d, chi_max, n_sweeps, seed, chi_schedule=(), lanczos=None, alpha=1e-2,
          alpha_decay=0.5, cutoff=1e-12, mps=None, chi0=None):
    """Single-site DMRG with subspace expansion (module docstring).  The initial MPS is
    ``dmrg.initial_mps`` with bond dimension chi0 (default: the first schedule entry).
    Returns (mps, report)."""
    N = len(cores)
    p = lanczos or dmrg.LanczosParams()
    sched = list(chi_schedule) if chi_schedule else [chi_max]
    if mps is None:
        mps = dmrg.initial_mps(N, d, sched[0] if chi0 is None else chi0, seed)
    mps = [A.copy() for A in mps]
    Lenv = [None] * (N + 1)
    Renv = [None] * (N + 1)
    Lenv[0] = np.ones((1, 1, 1), dtype=np.complex128)
    Renv[N] = np.ones((1, 1, 1), dtype=np.complex128)
    for s in range(N - 1, 0, -1):
        Renv[s] = dmrg.env_right(Renv[s + 1], mps[s], cores[s])
    rep = SweepReport1()

    def optimise(i):
        A = mps[i]
        shape = A.shape
        L, W, R = Lenv[i], cores[i], Renv[i + 1]
        mv = lambda x: heff1_apply(L, W, R, x.reshape(shape)).reshape(-1)
        _, x, nmv, conv = dmrg.lanczos_lowest(mv, A.reshape(-1), p)
        rep.matvecs += nmv
        rep.not_converged += 0 if conv else 1
        return x.reshape(shape)

    for sweep in range(n_sweeps):
        chi_s = sched[min(sweep, len(sched) - 1)]
        a_s = alpha * alpha_decay ** sweep
        disc_max = 0.0
        if N == 1:
            mps[0] = optimise(0)
        for i in range(0, N - 1):                       # to the right
            A = optimise(i)
            cl, _, cr = A.shape
            Mx = expand_right(Lenv[i], cores[i], A, a_s)
            kmax = min(chi_s, d * mps[i + 1].shape[2])  # no more than the next site can hold
            left, right, w, disc = dmrg.truncate(Mx.reshape(cl, d, 1, Mx.shape[1]), "right", kmax)
            k = _keep(w, cutoff)
            disc_max = max(disc_max, disc)
            mps[i] = left[:, :, :k]
            C = right[:k, 0, :cr]                       # U_k^dag A
            B = mps[i + 1]
            mps[i + 1] = np.einsum("kr,rsn->ksn", C, B, optimize=True)
            Lenv[i + 1] = dmrg.env_left(Lenv[i], mps[i], cores[i])
        for i in range(N - 1, 0, -1):                   # to the left
            A = optimise(i)
            cl, _, cr = A.shape
            Mx = expand_left(Renv[i + 1], cores[i], A, a_s)
            kmax = min(chi_s, mps[i - 1].shape[0] * d)
            left, right, w, disc = dmrg.truncate(Mx.reshape(Mx.shape[0], 1, d, cr), "left", kmax)
            k = _keep(w, cutoff)
            disc_max = max(disc_max, disc)
            mps[i] = right[:k]
            C = left[:cl, 0, :k]                        # A V_k restricted to the original rows
            Aprev = mps[i - 1]
            mps[i - 1] = np.einsum("psl,lk->psk", Aprev, C, optimize=True)
            Renv[i] = dmrg.env_right(Renv[i + 1], mps[i], cores[i])
        rep.energies.append(dmrg.energy(mps, cores))
        rep.max_discarded.append(disc_max)
        rep.dims.append([1] + [A.shape[2] for A in mps])
    return mps, rep
