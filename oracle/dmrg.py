"""Two-site DMRG for the GBS parent Hamiltonian -- oracle (test infrastructure only).

The paper solves min <H> over matrix product states (Eq. MPSAnsatz, open boundaries)
with DMRG (Sec. "Matrix Product States"; single-site DMRG via quimb in Sec. "Results").
This restatement is the two-site variant, step by step in plain numpy:

* MPS tensors A[s] with shape (chi_s, d, chi_{s+1}); chi_0 = chi_N = 1.
* environments L[s] (sites 0..s-1) with index order (channel, bra, ket) and
  R[s] (sites s..N-1) with index order (channel, ket, bra); L[0] = R[N] = 1.
* two-site effective Hamiltonian product (the contraction
  Y = sum L W_i W_{i+1} Theta R, evaluated one index group at a time),
* Lanczos with full re-orthogonalisation (classical Gram-Schmidt, two passes) and
  explicit restarts; the Ritz pair of the tridiagonal matrix by scipy's
  ``eigh_tridiagonal`` (library primitive),
* truncation by the eigendecomposition of the reduced density matrix (library
  ``eigh``), keeping k = min(chi, chi_l d, d chi_r) largest eigenpairs -- the squared
  Schmidt values of Eq. SurrogateEpsChi -- and reporting the discarded weight,
* energy <psi|H|psi>/<psi|psi> (Eq. MagOfSimError) by a full left-to-right contraction.

Readings where the paper is silent (recorded in the design notes): Lanczos tolerance,
restart rule, initial state (Philox Gaussian entries, rows orthonormalised in order so
the initial MPS is right-canonical), sweep order (all N-1 bonds left-to-right, then all
N-1 bonds right-to-left), and chi schedule (Discussion: chi grown from O(1)).

Parity: pinned at the plain workload by the dense exact ground state (chi = d^2 makes
the MPS exact), by the product-state special case U = I, and by E >= 0.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from . import philox


def bond_dims(N, d, chi):
    """chi_s = min(chi, d^s, d^(N-s)) for the cuts s = 0..N (Python integers, no overflow)."""
    return [int(min(chi, d ** s, d ** (N - s))) for s in range(N + 1)]


def orthonormal_rows(M):
    """Gram-Schmidt of the rows of M in order (equivalently the Q factor of the LQ
    decomposition with a positive diagonal)."""
    Q, R = np.linalg.qr(M.conj().T)
    ph = np.diag(R).copy()
    ph = np.where(np.abs(ph) > 0, ph / np.abs(ph), 1.0)
    Q = Q * ph[None, :]
    return Q.conj().T


def initial_mps(N, d, chi0, seed, center=0):
    """Philox normals per site; sites s >= center get their rows orthonormalised in order
    (right-canonical), sites s < center the columns of the (chi_l d) x chi_r matrix
    (left-canonical); the centre site is divided by sqrt(chi_center) so that <psi|psi> = 1.
    center = 0 is the right-canonical initial state of the sweeps."""
    dims = bond_dims(N, d, chi0)
    mps = []
    for s in range(N):
        cl, cr = dims[s], dims[s + 1]
        z = philox.complex_normals(seed, s, cl * d * cr)
        if s >= center:
            A = orthonormal_rows(z.reshape(cl, d * cr)).reshape(cl, d, cr)
            if s == center:
                A = A / np.sqrt(cl)
        else:
            A = orthonormal_rows(z.reshape(cl * d, cr).conj().T).conj().T.reshape(cl, d, cr)
        mps.append(A)
    return mps


def move_center(mps, src, dst):
    """Move the orthogonality centre of a mixed-canonical MPS from site src to site dst by exact
    splits of theta = A_i A_i+1 (``truncate`` keeping the current bond dimension, so nothing
    is dropped).  Returns the new list of tensors."""
    mps = [A.copy() for A in mps]
    c = src
    while c < dst:
        th = np.einsum("asb,btc->astc", mps[c], mps[c + 1], optimize=True)
        mps[c], mps[c + 1], _, _ = truncate(th, "right", mps[c].shape[2])
        c += 1
    while c > dst:
        th = np.einsum("asb,btc->astc", mps[c - 1], mps[c], optimize=True)
        mps[c - 1], mps[c], _, _ = truncate(th, "left", mps[c].shape[0])
        c -= 1
    return mps


# ---------------------------------------------------------------- contractions
def env_left(L, A, W):
    """L'[b, l, k] = sum conj(A[i,t,l]) L[a,i,j] W[a,b,t,s] A[j,s,k], evaluated pairwise."""
    T = np.einsum("aij,jsk->aisk", L, A, optimize=True)
    U = np.einsum("abts,aisk->bitk", W, T, optimize=True)
    return np.einsum("itl,bitk->blk", A.conj(), U, optimize=True)


def env_right(R, A, W):
    """R'[b, j, i] = sum W[b,c,t,s] A[j,s,g] conj(A[i,t,p]) R[c,g,p], evaluated pairwise."""
    T = np.einsum("jsg,cgp->cjsp", A, R, optimize=True)
    U = np.einsum("bcts,cjsp->bjtp", W, T, optimize=True)
    return np.einsum("bjtp,itp->bji", U, A.conj(), optimize=True)


def heff_apply(L, W1, W2, R, theta):
    """Y[i,t,u,l] = sum L[a,i,j] W1[a,b,t,s] W2[b,c,u,v] theta[j,s,v,k] R[c,k,l],
    evaluated one index group at a time (L, then W1, then W2, then R)."""
    T1 = np.einsum("aij,jsvk->aisvk", L, theta, optimize=True)
    T2 = np.einsum("abts,aisvk->bitvk", W1, T1, optimize=True)
    T3 = np.einsum("bcuv,bitvk->cituk", W2, T2, optimize=True)
    return np.einsum("cituk,ckl->itul", T3, R, optimize=True)


def heff_apply_columns(L, W1, W2, R, theta, cols):
    """Y[:, :, :, cols] of ``heff_apply``: the same sum with the output index l restricted to
    ``cols``, evaluated from the right (R first, then W2, W1, L) so that a few output columns
    of a large product cost only their share of the work (sampled checks at full size)."""
    Rc = R[:, :, list(cols)]
    Z = np.einsum("jsvk,ckl->jsvcl", theta, Rc, optimize=True)
    Z = np.einsum("bcuv,jsvcl->jsbul", W2, Z, optimize=True)
    Z = np.einsum("abts,jsbul->jatul", W1, Z, optimize=True)
    return np.einsum("aij,jatul->itul", L, Z, optimize=True)


# ---------------------------------------------------------------- Lanczos
@dataclass
class LanczosParams:
    krylov_max: int = 32
    max_restarts: int = 4
    tol: float = 1e-10          # absolute residual ||H x - theta x||
    breakdown: float = 1e-14


def lanczos_lowest(matvec, x0, p: LanczosParams):
    """Lowest eigenpair of a Hermitian operator.  Returns (theta, x, n_matvec, converged)."""
    v = x0 / np.linalg.norm(x0)
    n_mv = 0
    theta, x, converged = None, v, False
    for _ in range(p.max_restarts + 1):
        V = [v]
        alpha, beta = [], []
        resid = np.inf
        for j in range(p.krylov_max):
            w = matvec(V[j])
            n_mv += 1
            Vm = np.array(V)
            c = Vm.conj() @ w
            alpha.append(float(c[j].real))
            w = w - Vm.T @ c
            c2 = Vm.conj() @ w
            w = w - Vm.T @ c2
            b = float(np.linalg.norm(w))
            if j == 0:
                th, y = np.array([alpha[0]]), np.ones((1, 1))
            else:
                th, y = sla.eigh_tridiagonal(np.array(alpha), np.array(beta),
                                             select="i", select_range=(0, 0))
            theta, ycol = float(th[0]), y[:, 0]
            resid = b * abs(ycol[-1])
            if resid <= p.tol or b <= p.breakdown or j == p.krylov_max - 1:
                break
            beta.append(b)
            V.append(w / b)
        Vm = np.array(V)
        x = Vm.T @ ycol
        x = x / np.linalg.norm(x)
        v = x
        if resid <= p.tol or b <= p.breakdown:
            converged = True
            break
    return theta, x, n_mv, converged


# ---------------------------------------------------------------- truncation
def truncate(theta, direction, chi_max):
    """Split a two-site tensor (chi_l, d, d, chi_r).  direction 'right': returns
    (A_left_canonical, centre, kept_eigs, discarded); 'left': (centre, B_right_canonical,
    kept_eigs, discarded)."""
    cl, d1, d2, cr = theta.shape
    Tm = theta.reshape(cl * d1, d2 * cr)
    nL, nR = Tm.shape
    k = min(chi_max, nL, nR)
    if direction == "right":
        rho = Tm @ Tm.conj().T
        w, U = np.linalg.eigh(rho)
        total = float(np.real(np.trace(rho)))
        w, U = w[::-1][:k], U[:, ::-1][:, :k]
        A = U.reshape(cl, d1, k)
        C = (U.conj().T @ Tm).reshape(k, d2, cr)
        return A, C, w, 1.0 - float(np.sum(w)) / total
    rho = Tm.conj().T @ Tm
    w, V = np.linalg.eigh(rho)
    total = float(np.real(np.trace(rho)))
    w, V = w[::-1][:k], V[:, ::-1][:, :k]
    B = V.conj().T.reshape(k, d2, cr)
    C = (Tm @ V).reshape(cl, d1, k)
    return C, B, w, 1.0 - float(np.sum(w)) / total


def truncate_warm(theta, direction, chi_max, Q0, q=1, p=8, seed=0, bond=0):
    """The same split as ``truncate`` with the kept subspace found by block subspace iteration
    on rho from a warm start instead of a full eigendecomposition (not in the paper: a
    cheaper truncation whose energies are compared with the exact one).  Steps:
      m = min(nL, nR, k + p) start vectors: the columns of Q0 (the current centre tensor spans the
      previous kept subspace), then rho * Omega with Omega from the Philox TRUNC stream of
      (seed, bond); Gram-Schmidt; q times Q <- orth(rho Q); Rayleigh-Ritz: the k largest
      eigenpairs (w, Y) of Q^dag rho Q give U = Q Y.  rho = T T^dag ('right') or T^dag T
      ('left') is applied as T (T^dag X), never formed.  Returns what ``truncate`` returns,
      with the Ritz values in place of the eigenvalues."""
    cl, d1, d2, cr = theta.shape
    Tm = theta.reshape(cl * d1, d2 * cr)
    nL, nR = Tm.shape
    k = min(chi_max, nL, nR)
    if direction == "right":
        n = nL
        apply = lambda X: Tm @ (Tm.conj().T @ X)
    else:
        n = nR
        apply = lambda X: Tm.conj().T @ (Tm @ X)
    m = min(nL, nR, k + p)       # no more vectors than the rank of rho can hold
    k0 = 0 if Q0 is None else min(Q0.shape[1], m)
    S = np.empty((n, m), dtype=np.complex128)
    if k0:
        S[:, :k0] = Q0[:, :k0]
    if m > k0:
        Om = philox.complex_normals(seed, bond, n * (m - k0), stream=philox.STREAM_TRUNC)
        S[:, k0:] = apply(Om.reshape(n, m - k0))
    orth = lambda X: orthonormal_rows(X.conj().T).conj().T
    Q = orth(S)
    for _ in range(q):
        Q = orth(apply(Q))
    Bm = Q.conj().T @ apply(Q)
    w, Y = np.linalg.eigh(0.5 * (Bm + Bm.conj().T))
    w, Y = w[::-1][:k], Y[:, ::-1][:, :k]
    U = Q @ Y
    total = float(np.linalg.norm(Tm) ** 2)
    if direction == "right":
        return U.reshape(cl, d1, k), (U.conj().T @ Tm).reshape(k, d2, cr), w, 1.0 - float(np.sum(w)) / total
    return (Tm @ U).reshape(cl, d1, k), U.conj().T.reshape(k, d2, cr), w, 1.0 - float(np.sum(w)) / total


# ---------------------------------------------------------------- energy
def norm2(mps):
    E = np.ones((1, 1), dtype=np.complex128)
    for A in mps:
        E = np.einsum("isk,isl->kl", A.conj(), np.einsum("ij,jsl->isl", E, A, optimize=True), optimize=True)
    return float(E[0, 0].real)


def energy(mps, cores):
    """<psi|H|psi>/<psi|psi> by a full left-to-right environment contraction."""
    L = np.ones((1, 1, 1), dtype=np.complex128)
    for A, W in zip(mps, cores):
        L = env_left(L, A, W)
    return float(L[0, 0, 0].real) / norm2(mps)


def env_left_h2(L2, A, W):
    """Two-layer left environment of <psi|H H|psi> (Sec. "Assessing the error from finite bond
    dimension": the variance of the variational state with respect to P H P):
    L2'[c, b, l, k] = sum conj(A[i,u,l]) W[a,c,u,t] W[a',b,t,s] L2[a, a', i, j] A[j,s,k];
    index a of L2 belongs to the H next to the bra, a' to the H next to the ket.  Evaluated
    pairwise."""
    T = np.einsum("xyij,jsk->xyisk", L2, A, optimize=True)
    U = np.einsum("ybts,xyisk->xbitk", W, T, optimize=True)    # H next to the ket: s -> t
    V = np.einsum("xcut,xbitk->cbiuk", W, U, optimize=True)    # H next to the bra: t -> u
    return np.einsum("iul,cbiuk->cblk", A.conj(), V, optimize=True)


def energy_variance(mps, cores):
    """(E, <H^2>, sigma_H) with E = <psi|H|psi>/<psi|psi>, <H^2> = <psi|H H|psi>/<psi|psi> and
    sigma_H = sqrt(max(0, <H^2> - E^2)) (Sec. "Assessing the error from finite bond
    dimension"); H is the MPO's operator (the projected P H P)."""
    L2 = np.ones((1, 1, 1, 1), dtype=np.complex128)
    for A, W in zip(mps, cores):
        L2 = env_left_h2(L2, A, W)
    n2 = norm2(mps)
    e = energy(mps, cores)
    h2 = float(L2[0, 0, 0, 0].real) / n2
    return e, h2, float(np.sqrt(max(0.0, h2 - e * e)))


# ---------------------------------------------------------------- sweeps
@dataclass
class SweepReport:
    energies: list = field(default_factory=list)
    max_discarded: list = field(default_factory=list)
    matvecs: int = 0
    not_converged: int = 0


def centre_energy(mps, cores, Lenv, Renv, lo):
    """Rayleigh quotient <theta|H_eff theta>/<theta|theta> of theta = A_lo A_lo+1 under the
    two-site effective Hamiltonian of bond (lo, lo+1): <psi|H|psi>/<psi|psi> of a state whose
    sites < lo are left-canonical and sites > lo+1 right-canonical (Eq. MagOfSimError)."""
    th = np.einsum("asb,btc->astc", mps[lo], mps[lo + 1], optimize=True)
    y = heff_apply(Lenv[lo], cores[lo], cores[lo + 1], Renv[lo + 2], th)
    return float(np.real(np.vdot(th, y))) / float(np.real(np.vdot(th, th)))


def dmrg(cores, d, chi_max, n_sweeps, seed, chi_schedule=(), lanczos=None,
         e_tol=0.0, e_target=None, mps=None, max_bonds=None, warm_q=None, window=None,
         energy_mode="full"):
    """Two-site DMRG sweeps.  Returns (mps, report).  ``max_bonds`` stops after that
    many bond optimisations (used only to time a bounded sample).  ``warm_q`` = None: exact
    truncation; an integer: ``truncate_warm`` with that many iterations, started from the
    current centre tensor (site i sweeping right, site i+1 sweeping left).
    ``window`` = (lo, hi): each sweep optimises bonds lo .. hi-1 left to right and back; the
    given ``mps`` must have its centre at site lo (sites < lo left-canonical, > lo
    right-canonical) and the sweep energy is then the centre Rayleigh quotient.
    ``energy_mode`` = "full": the sweep energy is the full contraction; "centre": the Rayleigh
    quotient of the final centre tensor (``centre_energy``)."""
    N = len(cores)
    p = lanczos or LanczosParams()
    sched = list(chi_schedule) if chi_schedule else [chi_max]
    lo, hi = (0, N - 1) if window is None else window
    if window is not None:
        energy_mode = "centre"
    if mps is None:
        mps = initial_mps(N, d, sched[0], seed, center=lo)
    mps = [A.copy() for A in mps]
    Lenv = [None] * (N + 1)
    Renv = [None] * (N + 1)
    Lenv[0] = np.ones((1, 1, 1), dtype=np.complex128)
    Renv[N] = np.ones((1, 1, 1), dtype=np.complex128)
    for s in range(0, lo):
        Lenv[s + 1] = env_left(Lenv[s], mps[s], cores[s])
    for s in range(N - 1, lo + 1, -1):
        Renv[s] = env_right(Renv[s + 1], mps[s], cores[s])
    rep = SweepReport()
    bonds_done = 0
    prev = None
    for sweep in range(n_sweeps):
        chi_s = sched[min(sweep, len(sched) - 1)]
        disc_max = 0.0
        for direction, bonds in (("right", range(lo, hi)), ("left", range(hi - 1, lo - 1, -1))):
            for i in bonds:
                theta = np.einsum("asb,btc->astc", mps[i], mps[i + 1], optimize=True)
                shape = theta.shape
                L, R, W1, W2 = Lenv[i], Renv[i + 2], cores[i], cores[i + 1]
                mv = lambda x: heff_apply(L, W1, W2, R, x.reshape(shape)).reshape(-1)
                _, x, nmv, conv = lanczos_lowest(mv, theta.reshape(-1), p)
                rep.matvecs += nmv
                rep.not_converged += 0 if conv else 1
                theta = x.reshape(shape)
                if warm_q is None:
                    left, right, _, disc = truncate(theta, direction, chi_s)
                else:
                    if direction == "right":
                        Q0 = mps[i].reshape(-1, mps[i].shape[2])
                    else:
                        Q0 = mps[i + 1].reshape(mps[i + 1].shape[0], -1).conj().T
                    left, right, _, disc = truncate_warm(theta, direction, chi_s, Q0, q=warm_q, seed=seed, bond=i)
                disc_max = max(disc_max, disc)
                mps[i], mps[i + 1] = left, right
                if direction == "right":
                    Lenv[i + 1] = env_left(Lenv[i], mps[i], cores[i])
                else:
                    Renv[i + 1] = env_right(Renv[i + 2], mps[i + 1], cores[i + 1])
                bonds_done += 1
                if max_bonds is not None and bonds_done >= max_bonds:
                    return mps, rep
        E = energy(mps, cores) if energy_mode == "full" else centre_energy(mps, cores, Lenv, Renv, lo)
        rep.energies.append(E)
        rep.max_discarded.append(disc_max)
        if e_target is not None and E <= e_target:
            break
        if prev is not None and e_tol > 0 and abs(E - prev) <= e_tol:
            break
        prev = E
    return mps, rep
