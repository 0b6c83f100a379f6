"""Pins of the oracle's single-site DMRG with subspace expansion (CPU only).

Each pin ties a step to something the oracle does not compute the same way: the dense
projected Hamiltonian (Kronecker products, term by term), the invariance of the state under
the expansion, the identity linking the expansion term to the effective Hamiltonian, and the
dense ground energy reached from a product state.
"""
import numpy as np
import pytest

from oracle import dense, dmrg, dmrg1, gbs, mpo
from paper_2410_18740_gb300 import inputs


def _left_canonical(cl, d, cr, rng):
    Z = inputs.random_complex((cl * d, cr), rng)
    Q, _ = np.linalg.qr(Z)
    return Q[:, :cr].reshape(cl, d, cr)


def _mixed_mps(N, d, chi, i, rng):
    """Sites < i left-canonical, sites > i right-canonical, random centre at i."""
    dims = dmrg.bond_dims(N, d, chi)
    sites = []
    for s in range(N):
        cl, cr = dims[s], dims[s + 1]
        if s < i:
            sites.append(_left_canonical(cl, d, cr, rng))
        elif s > i:
            B = _left_canonical(cr, d, cl, rng)          # (cr, d, cl) with orthonormal columns
            sites.append(np.transpose(B, (2, 1, 0)).conj())  # rows orthonormal over (s, r)
        else:
            sites.append(inputs.random_complex((cl, d, cr), rng))
    return sites


def _state(sites):
    psi = np.ones((1, 1), dtype=np.complex128)
    for A in sites:
        psi = np.einsum("xl,lsr->xsr", psi, A).reshape(-1, A.shape[2])
    return psi.reshape(-1)


@pytest.mark.parametrize("seed,i", [(0, 0), (1, 1), (2, 2), (3, 3)])
def test_heff1_is_the_projected_dense_hamiltonian(seed, i):
    """Phi maps the centre tensor to the state; y = Phi^dag H Phi x for the dense P H P."""
    N, d, chi = 4, 3, 5
    rng = inputs.rng_for(seed)
    w = inputs.workload("plain", seed, M=N, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    cores = mpo.build_mpo(G, d)
    H = dense.dense_hamiltonian(G, d).toarray()
    sites = _mixed_mps(N, d, chi, i, rng)
    cl, _, cr = sites[i].shape
    n = cl * d * cr
    Phi = np.empty((d ** N, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        Phi[:, j] = _state(sites[:i] + [e.reshape(cl, d, cr)] + sites[i + 1:])
    assert np.abs(Phi.conj().T @ Phi - np.eye(n)).max() < 1e-12
    L = np.ones((1, 1, 1), dtype=np.complex128)
    for s in range(i):
        L = dmrg.env_left(L, sites[s], cores[s])
    R = np.ones((1, 1, 1), dtype=np.complex128)
    for s in range(N - 1, i, -1):
        R = dmrg.env_right(R, sites[s], cores[s])
    x = inputs.random_complex((cl, d, cr), rng)
    y = dmrg1.heff1_apply(L, cores[i], R, x)
    ref = Phi.conj().T @ (H @ (Phi @ x.reshape(-1)))
    assert np.abs(y.reshape(-1) - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("seed", [0, 1])
def test_expansion_keeps_the_state_and_carries_heff(seed):
    """[A | alpha P] [B; 0] = A B, and contracting P's (b, r) columns with R gives H_eff A
    (likewise for the left expansion with L)."""
    rng = inputs.rng_for(seed + 10)
    w = inputs.workload("plain", seed, M=5, d=3, D=3)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    cores = mpo.build_mpo(G, 3)
    W = cores[2]
    wl, wr = W.shape[:2]
    cl, d, cr, cn = 4, 3, 5, 2
    L = inputs.random_complex((wl, cl, cl), rng)
    R = inputs.random_complex((wr, cr, cr), rng)
    A = inputs.random_complex((cl, d, cr), rng)
    alpha = 0.37
    y = dmrg1.heff1_apply(L, W, R, A)
    # right
    Mx = dmrg1.expand_right(L, W, A, alpha)
    assert Mx.shape == (cl * d, cr * (1 + wr))
    B = inputs.random_complex((cr, d * cn), rng)
    Bx = np.vstack([B, np.zeros((wr * cr, d * cn))])
    assert np.abs(Mx @ Bx - A.reshape(cl * d, cr) @ B).max() < 1e-12
    P = Mx[:, cr:].reshape(cl * d, wr, cr) / alpha
    assert np.abs(np.einsum("xbr,brq->xq", P, R) - y.reshape(cl * d, cr)).max() < 1e-11
    # left
    Mx = dmrg1.expand_left(R, W, A, alpha)
    assert Mx.shape == (cl * (1 + wl), d * cr)
    Aprev = inputs.random_complex((cn * d, cl), rng)
    Ax = np.hstack([Aprev, np.zeros((cn * d, wl * cl))])
    assert np.abs(Ax @ Mx - Aprev @ A.reshape(cl, d * cr)).max() < 1e-12
    P = Mx[cl:].reshape(wl, cl, d * cr) / alpha
    assert np.abs(np.einsum("alm,amx->lx", L, P) - y.reshape(cl, d * cr)).max() < 1e-11


@pytest.mark.parametrize("seed", [0, 1])
def test_dmrg1_from_a_product_state_reaches_the_dense_ground_energy(seed):
    """chi = 9 is exact for N = 4, d = 3; starting from bond dimension 1 only the expansion
    can grow the bonds.  Without it (alpha = 0) the bonds stay at 1."""
    N, d = 4, 3
    w = inputs.workload("plain", seed, M=N, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, N, d)
    e0 = dense.ground_state(G, d)[0][0]
    cores = mpo.build_mpo(G, d)
    lp = dmrg.LanczosParams(krylov_max=32, max_restarts=8, tol=1e-12)
    mps, rep = dmrg1.dmrg1(cores, d, 9, 8, seed=seed + 5, chi0=1, lanczos=lp, alpha=0.1, alpha_decay=0.5)
    assert rep.dims[-1] == [1, 3, 9, 3, 1]
    assert abs(rep.energies[-1] - e0) <= 1e-9 * Hn
    assert min(rep.energies) >= e0 - 1e-10 * Hn
    assert abs(dmrg.energy(mps, cores) - rep.energies[-1]) <= 1e-12 * Hn
    _, rep0 = dmrg1.dmrg1(cores, d, 9, 2, seed=seed + 5, chi0=1, lanczos=lp, alpha=0.0)
    assert rep0.dims[-1] == [1, 1, 1, 1, 1]
    assert rep0.energies[-1] > e0 + 1e-6


def test_dmrg1_single_mode():
    """N = 1: the sweep reduces to the Lanczos ground state of the single-mode H."""
    w = inputs.workload("plain", 3, M=1, d=6, D=6)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    e0 = dense.ground_state(G, 6)[0][0]
    cores = mpo.build_mpo(G, 6)
    _, rep = dmrg1.dmrg1(cores, 6, 4, 1, seed=1, lanczos=dmrg.LanczosParams(tol=1e-13))
    assert abs(rep.energies[-1] - e0) <= 1e-11
