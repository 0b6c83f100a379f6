"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every test here runs on the CPU (no GPU marker).  Each pin is chosen so that a
plausible mistake in the oracle (a dropped term, a wrong sign or index, a transposed
operand) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.stats

from oracle import dense, dmrg, gbs, mpo, observables, philox, warm
from paper_2410_18740_gb300 import inputs
from tests.conftest import GOLDEN


# ------------------------------------------------------------------ Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(np.array(v[0:4], dtype=np.uint64), np.array(v[4:6], dtype=np.uint64))
        assert [int(x) for x in out] == v[6:10]


def test_philox_uniform_range_and_moments():
    u = philox.sample_uniforms(7, np.arange(200000, dtype=np.uint64), 3)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 3e-3


# ------------------------------------------------------------------ covariance, G
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_covariance_invariants(seed):
    w = inputs.workload("plain", seed, M=5)
    V = gbs.covariance(w.r, w.U)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    N = w.M
    # trace: tr V = sum cosh 2r (invariant under the passive interferometer)
    assert abs(np.trace(V) - np.sum(np.cosh(2 * w.r))) < 1e-12
    # Fock-basis mean photon number sum <n_i> = tr V / 2 - N/2 = sum sinh^2 r
    assert abs(0.5 * np.trace(V) - N / 2 - np.sum(np.sinh(w.r) ** 2)) < 1e-12
    # pure state: 2V is symplectic
    Om = np.block([[np.zeros((N, N)), np.eye(N)], [-np.eye(N), np.zeros((N, N))]])
    assert np.abs((2 * V) @ Om @ (2 * V).T - Om).max() < 1e-12
    # G = V^{-1}/4 equals the closed form 1/2 O diag(e^{2r}, e^{-2r}) O^T (different route)
    O = gbs.quadrature_orthogonal(w.U)
    Gc = 0.5 * O @ np.diag(np.concatenate([np.exp(2 * w.r), np.exp(-2 * w.r)])) @ O.T
    assert np.abs(G - Gc).max() < 1e-12
    assert abs(np.max(np.linalg.eigvalsh(G)) - 0.5 * np.exp(2 * np.max(w.r))) < 1e-12


# ------------------------------------------------------------------ local operators
@pytest.mark.parametrize("d", [2, 3, 4, 6, 9])
def test_local_ops_exact_projection(d):
    ops = gbs.local_ops(d)
    n = np.arange(d)
    assert np.abs(ops["X2"] + ops["P2"] - np.diag(2 * n + 1.0)).max() < 1e-13
    # exactly projected X^2 differs from (P X P)^2 only at (d-1, d-1) (SM Sec. 5)
    diff = ops["X2"] - ops["X"] @ ops["X"]
    mask = np.ones((d, d), bool)
    mask[d - 1, d - 1] = False
    assert np.abs(diff[mask]).max() < 1e-13
    assert abs(diff[d - 1, d - 1] - d / 2.0) < 1e-13
    # XP + PX = i (a^dag^2 - a^2): entries -+ i sqrt((n+1)(n+2))
    for m in range(d - 2):
        v = math.sqrt((m + 1) * (m + 2))
        assert abs(ops["XPPX"][m, m + 2] + 1j * v) < 1e-13
        assert abs(ops["XPPX"][m + 2, m] - 1j * v) < 1e-13
    assert np.abs(ops["XPPX"] - ops["XPPX"].conj().T).max() < 1e-14


def test_commutator_defect_golden():
    for line in open(os.path.join(GOLDEN, "commutator_defect.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        vals = [int(x) for x in line.split()]
        d, diag = vals[0], np.array(vals[1:], dtype=float)
        ops = gbs.local_ops(d)
        C = ops["X"] @ ops["P"] - ops["P"] @ ops["X"]
        assert np.abs(C - 1j * np.diag(diag)).max() < 1e-13


# ------------------------------------------------------------------ optimal local basis
@pytest.mark.parametrize("seed", [3, 4])
def test_williamson_and_rotated_blocks(seed):
    w = inputs.workload("large", seed, M=6)
    S_list, nu, Grot = gbs.lbo_transform(w.r, w.U)
    V = gbs.covariance(w.r, w.U)
    N = w.M
    for i, S in enumerate(S_list):
        Vi = gbs.reduced_covariance(V, i)
        assert abs(np.linalg.det(S) - 1.0) < 1e-12
        assert np.abs(S @ (nu[i] * np.eye(2)) @ S.T - Vi).max() < 1e-12
    # (4 G')^{-1} is the rotated covariance with nu_i I diagonal blocks (text after Eq. WilliamsonDecomposition)
    Vrot = np.linalg.inv(4 * Grot)
    for i in range(N):
        blk = gbs.reduced_covariance(Vrot, i)
        assert np.abs(blk - nu[i] * np.eye(2)).max() < 1e-11
    # nu_i >= 1/2, and the thermal occupation is at most the Fock occupation
    nfock = 0.5 * (np.diag(V)[:N] + np.diag(V)[N:]) - 0.5
    assert np.all(nu >= 0.5 - 1e-12) and np.all(nu - 0.5 <= nfock + 1e-12)


@pytest.mark.parametrize("seed", [5, 6])
def test_lbo_isometry(seed):
    """Eq. Effectivecutoff: V^dagger V -> I_d as the Fock cutoff D grows; at D = 100 it
    holds to 1e-10 for the squeezing of the large workload (at D = 24 it need not: the
    cutoff can lie below the effective cutoff, and the lost tail is what marginals miss)."""
    w = inputs.workload("large", seed, M=3)
    S_list, nu, _ = gbs.lbo_transform(w.r, w.U)
    d = 6
    for S in S_list:
        errs = []
        for D in (24, 40, 100):
            Viso = gbs.lbo_isometry(S, D, d)
            G = Viso.conj().T @ Viso
            errs.append(np.abs(G - np.eye(d)).max())
            # the deficit is a loss of norm only: the Gram matrix stays <= I
            assert np.max(np.linalg.eigvalsh(G)) <= 1 + 1e-12
        assert errs[2] < 1e-10
        assert errs[0] + 1e-15 >= errs[1] >= errs[2] - 1e-15


def test_lbo_isometry_squeezed_vacuum_statistics():
    w = inputs.workload("large", 11, M=3)
    S_list, _, _ = gbs.lbo_transform(w.r, w.U)
    D = 40
    for S in S_list:
        Viso = gbs.lbo_isometry(S, D, 4)
        r_loc = math.log(np.max(np.linalg.eigvalsh(S)))
        t = math.tanh(r_loc)
        p = np.abs(Viso[:, 0]) ** 2
        for k in range(D):
            if k % 2:
                assert p[k] < 1e-24
            else:
                m = k // 2
                exact = math.factorial(2 * m) / (4 ** m * math.factorial(m) ** 2) * t ** (2 * m) / math.cosh(r_loc)
                assert abs(p[k] - exact) < 1e-12
        # covariance of S^dagger|0> equals S S^T / 2
        Db = 120
        ops = gbs.local_ops(Db)
        c = gbs.lbo_isometry(S, Db, 1)[:, 0]
        cov = np.array([[np.vdot(c, ops["X2"] @ c).real, 0.5 * np.vdot(c, ops["XPPX"] @ c).real],
                        [0.0, np.vdot(c, ops["P2"] @ c).real]])
        cov[1, 0] = cov[0, 1]
        assert np.abs(cov - 0.5 * S @ S.T).max() < 1e-10


def test_truncation_bound_eps_le_epsD_le_Neps():
    """Eq. SpecWfromSDsums: eps <= eps_D <= N eps, eps_D from the (large-cutoff) ground
    state in the optimal local basis."""
    for seed in (20, 21):
        w = inputs.workload("plain", seed, M=3, r_lo=0.4, r_hi=0.9)
        _, nu, Grot = gbs.lbo_transform(w.r, w.U)
        dbig = 12
        e0, v0 = dense.ground_state(Grot, dbig)
        assert e0[0] < 1e-5          # cutoff 12 leaves ~1e-6 of the state out; tolerances below
        psi = v0[:, 0].reshape((dbig,) * 3)
        for d in (2, 3, 4):
            epsD = 1.0 - np.sum(np.abs(psi[:d, :d, :d]) ** 2)
            eps = gbs.truncation_epsilon(nu, d)
            assert eps <= epsD + 1e-5
            assert epsD <= 3 * eps + 1e-5
            assert epsD > 1.5 * eps     # neither bound is trivially saturated here


def test_lbo_reduced_density_is_thermal():
    """In the optimal local basis the single-mode reduced density matrix is diagonal with
    weights nbar^k/(nbar+1)^(k+1) (Eq. diagReducedGaussianDM)."""
    w = inputs.workload("plain", 30, M=2, r_lo=0.3, r_hi=0.6)
    _, nu, Grot = gbs.lbo_transform(w.r, w.U)
    dbig = 24
    _, v0 = dense.ground_state(Grot, dbig)
    psi = v0[:, 0].reshape(dbig, dbig)
    rho0 = psi @ psi.conj().T
    nbar = nu[0] - 0.5
    k = np.arange(8)
    thermal = nbar ** k / (nbar + 1) ** (k + 1)
    assert np.abs(np.diag(rho0)[:8].real - thermal).max() < 1e-8
    off = rho0[:8, :8] - np.diag(np.diag(rho0[:8, :8]))
    assert np.abs(off).max() < 1e-8


# ------------------------------------------------------------------ MPO vs dense
@pytest.mark.parametrize("seed,M,d", [(0, 3, 3), (1, 4, 3), (2, 3, 4)])
def test_mpo_contracts_to_dense_hamiltonian(seed, M, d):
    w = inputs.workload("plain", seed, M=M)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    H1 = mpo.contract_dense(mpo.build_mpo(G, d))
    H2 = dense.dense_hamiltonian(G, d).toarray()
    assert np.abs(H1 - H2).max() < 1e-12
    assert np.abs(H1 - H1.conj().T).max() < 1e-12


# ------------------------------------------------------------------ hafnian amplitudes
def test_hafnian_closed_forms():
    for m in range(1, 6):
        assert abs(dense.hafnian(np.ones((2 * m, 2 * m))) - math.prod(range(1, 2 * m, 2))) < 1e-9
    A = np.array([[0, 2.0], [2.0, 0]])
    assert abs(dense.hafnian(A) - 2.0) < 1e-15
    rng = np.random.default_rng(0)
    B = rng.standard_normal((4, 4)); B = B + B.T
    expect = B[0, 1] * B[2, 3] + B[0, 2] * B[1, 3] + B[0, 3] * B[1, 2]
    assert abs(dense.hafnian(B) - expect) < 1e-12


def test_single_mode_amplitudes_textbook():
    r = np.array([0.7])
    U = np.eye(1, dtype=complex)
    t = math.tanh(0.7)
    for m in range(6):
        a = dense.gbs_amplitude(r, U, (2 * m,))
        exact = (-t) ** m * math.sqrt(math.factorial(2 * m)) / (2 ** m * math.factorial(m)) / math.sqrt(math.cosh(0.7))
        assert abs(a - exact) < 1e-13
        assert abs(dense.gbs_amplitude(r, U, (2 * m + 1,))) == 0.0


def test_vacuum_probability_and_normalisation():
    w = inputs.workload("plain", 4, M=3)
    amp = dense.gbs_amplitudes(w.r, w.U, 9)
    assert abs(abs(amp[0, 0, 0]) ** 2 - 1.0 / np.prod(np.cosh(w.r))) < 1e-13
    assert 0.99 < np.sum(np.abs(amp) ** 2) <= 1.0 + 1e-12


# ------------------------------------------------------------------ dense spectrum
def test_dense_ground_state_matches_hafnian_state():
    """The ground state of P H P approaches the GBS state as d grows; this fixes the
    U -> O map and the sign of B together."""
    w = inputs.workload("plain", 2, M=2, r_lo=0.3, r_hi=0.5)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    prev = None
    for d in (6, 10, 14):
        e0, v0 = dense.ground_state(G, d)
        amp = dense.gbs_amplitudes(w.r, w.U, d).reshape(-1)
        F = abs(np.vdot(amp, v0[:, 0])) ** 2 / np.vdot(amp, amp).real
        assert e0[0] >= -1e-12
        if prev is not None:
            assert 1 - F <= prev + 1e-12
        prev = 1 - F
    assert prev < 1e-6


def test_interlacing_monotone_and_spectrum_near_integers():
    w = inputs.workload("plain", 8, M=2, r_lo=0.2, r_hi=0.4)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    energies = []
    for d in range(2, 13):
        energies.append(dense.ground_state(G, d)[0][0])
    assert all(e >= -1e-12 for e in energies)
    assert all(energies[k + 1] <= energies[k] + 1e-12 for k in range(len(energies) - 1))
    wl = np.linalg.eigvalsh(dense.dense_hamiltonian(G, 16).toarray())[:4]
    assert np.abs(wl - np.array([0, 1, 1, 2])).max() < 1e-3


def test_fidelity_bound_F_ge_1_minus_E():
    """|<psi|phi>|^2 >= 1 - <phi|PHP|phi> for any normalised phi in the truncated space
    (text after Eq. MagOfSimError), with psi the exact (untruncated) GBS state."""
    w = inputs.workload("plain", 9, M=3, r_lo=0.3, r_hi=0.6)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    d = 4
    H = dense.dense_hamiltonian(G, d).toarray()
    amp = dense.gbs_amplitudes(w.r, w.U, d).reshape(-1)
    rng = np.random.default_rng(1)
    _, v0 = dense.ground_state(G, d)
    cands = [v0[:, 0]] + [v0[:, 0] + 0.3 * inputs.random_complex(d ** 3, rng) for _ in range(5)]
    for phi in cands:
        phi = phi / np.linalg.norm(phi)
        E = np.vdot(phi, H @ phi).real
        F = abs(np.vdot(amp, phi)) ** 2
        assert F >= 1 - E - 1e-12


def test_product_state_U_identity():
    """U = I: H decouples, the ground state is a product and each mode's energy is the
    lowest eigenvalue of its d x d single-mode problem; marginals tend to the squeezed
    vacuum (2n)!/(4^n n!^2) tanh^{2n} r / cosh r."""
    w = inputs.workload("plain", 12, M=3, identity_U=True, r_lo=0.3, r_hi=0.5)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    d = 10
    ops = gbs.local_ops(d)
    e_single = []
    for i in range(3):
        h = G[i, i] * ops["X2"] + G[3 + i, 3 + i] * ops["P2"] + G[i, 3 + i] * ops["XPPX"] - 0.5 * ops["I"]
        e_single.append(np.linalg.eigvalsh(h)[0])
    cores = mpo.build_mpo(G, d)
    mps, rep = dmrg.dmrg(cores, d, 1, 3, seed=3, lanczos=dmrg.LanczosParams(tol=1e-12))
    assert abs(rep.energies[-1] - sum(e_single)) < 1e-10
    marg = observables.marginal(mps, None, [1])
    t = math.tanh(w.r[1])
    for m in range(3):
        exact = math.factorial(2 * m) / (4 ** m * math.factorial(m) ** 2) * t ** (2 * m) / math.cosh(w.r[1])
        assert abs(marg[2 * m] - exact) < 1e-4
        assert marg[2 * m + 1] < 1e-12


# ------------------------------------------------------------------ DMRG
@pytest.mark.parametrize("seed", [0, 1])
def test_dmrg_plain_is_exact(seed):
    """Plain workload (M=4, d=4, chi=16 = d^2): the MPS is exact, so two-site DMRG must
    reach the dense ground energy to 1e-12 ||H||."""
    w = inputs.workload("plain", seed)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, w.M, w.d)
    e0, v0 = dense.ground_state(G, w.d)
    cores = mpo.build_mpo(G, w.d)
    mps, rep = dmrg.dmrg(cores, w.d, w.chi, 4, seed=seed + 100, lanczos=dmrg.LanczosParams(tol=1e-12))
    assert abs(rep.energies[-1] - e0[0]) <= 1e-12 * Hn
    assert rep.energies[-1] >= -1e-12
    for i in range(w.M):
        m = observables.marginal(mps, None, [i])
        md = dense.marginals_from_vector(v0[:, 0], w.M, w.d, [i])
        assert np.abs(m - md).max() < 1e-10
    m2 = observables.marginal(mps, None, [3, 1])
    md2 = dense.marginals_from_vector(v0[:, 0], w.M, w.d, [3, 1])
    assert np.abs(m2 - md2).max() < 1e-10


def test_truncation_weights_and_reconstruction():
    rng = np.random.default_rng(5)
    th = inputs.random_complex((3, 4, 4, 5), rng)
    th /= np.linalg.norm(th)
    A, C, w, disc = dmrg.truncate(th, "right", 100)
    assert abs(disc) < 1e-14 and abs(w.sum() - 1) < 1e-13
    assert np.abs(np.einsum("asb,btc->astc", A, C) - th).max() < 1e-13
    Al = A.reshape(12, -1)
    assert np.abs(Al.conj().T @ Al - np.eye(Al.shape[1])).max() < 1e-13
    C2, B, w2, disc2 = dmrg.truncate(th, "left", 5)
    assert abs(disc2 - (1 - w2.sum())) < 1e-14 and disc2 > 0
    Bm = B.reshape(5, -1)
    assert np.abs(Bm @ Bm.conj().T - np.eye(5)).max() < 1e-13
    # kept weight of the best rank-5 approximation equals the reconstruction overlap
    approx = np.einsum("asb,btc->astc", C2, B)
    assert abs(np.linalg.norm(th - approx) ** 2 - disc2) < 1e-12


def test_heff_columns_match_the_full_product():
    """The column-sampled H_eff product is the full product's columns (a different
    association of the same sum, used for checks at the large workload's shapes)."""
    rng = inputs.rng_for(606)
    cl, cr, d, (wl, wm, wr) = 5, 7, 3, (4, 5, 3)
    W1 = inputs.random_sparse_core(wl, wm, d, rng).dense()
    W2 = inputs.random_sparse_core(wm, wr, d, rng).dense()
    L = inputs.random_complex((wl, cl, cl), rng)
    R = inputs.random_complex((wr, cr, cr), rng)
    th = inputs.random_complex((cl, d, d, cr), rng)
    Y = dmrg.heff_apply(L, W1, W2, R, th)
    cols = [6, 0, 3]
    Yc = dmrg.heff_apply_columns(L, W1, W2, R, th, cols)
    assert np.abs(Yc - Y[..., cols]).max() <= 1e-13 * np.abs(Y).max()


def test_lanczos_against_dense_eigh():
    rng = np.random.default_rng(7)
    A = inputs.random_complex((60, 60), rng)
    H = A + A.conj().T
    lam, vec = np.linalg.eigh(H)
    th, x, nmv, conv = dmrg.lanczos_lowest(lambda v: H @ v, inputs.random_complex(60, rng),
                                           dmrg.LanczosParams(krylov_max=30, max_restarts=10, tol=1e-11))
    assert conv and abs(th - lam[0]) < 1e-10
    assert abs(abs(np.vdot(vec[:, 0], x)) - 1) < 1e-10


def test_initial_mps_right_canonical():
    mps = dmrg.initial_mps(5, 3, 7, seed=11)
    assert [A.shape for A in mps][2] == (7, 3, 7)
    for A in mps:
        Am = A.reshape(A.shape[0], -1)
        assert np.abs(Am @ Am.conj().T - np.eye(A.shape[0])).max() < 1e-13
    assert abs(dmrg.norm2(mps) - 1) < 1e-12


def _dense_vector(mps):
    v = mps[0]
    for A in mps[1:]:
        v = np.einsum("...a,asb->...sb", v, A)
    return v.reshape(-1)


@pytest.mark.parametrize("center", [0, 2, 4])
def test_initial_mps_mixed_canonical(center):
    """Sites left of the centre are left isometries, sites right of it right isometries, the
    state is normalised, and centre 0 is the right-canonical start state."""
    mps = dmrg.initial_mps(5, 3, 7, seed=11, center=center)
    for s, A in enumerate(mps):
        if s < center:
            Am = A.reshape(-1, A.shape[2])
            assert np.abs(Am.conj().T @ Am - np.eye(A.shape[2])).max() < 1e-13
        elif s > center:
            Am = A.reshape(A.shape[0], -1)
            assert np.abs(Am @ Am.conj().T - np.eye(A.shape[0])).max() < 1e-13
    assert abs(dmrg.norm2(mps) - 1) < 1e-12
    assert abs(np.linalg.norm(_dense_vector(mps)) - 1) < 1e-12
    if center == 0:
        for a, b in zip(mps, dmrg.initial_mps(5, 3, 7, seed=11)):
            assert np.array_equal(a, b)


def test_move_center_keeps_the_state():
    """Exact splits only change the gauge: the dense vector is unchanged and the canonical
    conditions hold around the new centre."""
    mps = dmrg.initial_mps(6, 3, 9, seed=4, center=1)
    v0 = _dense_vector(mps)
    for dst in (4, 0, 3):
        mps = dmrg.move_center(mps, {4: 1, 0: 4, 3: 0}[dst], dst)
        assert np.abs(_dense_vector(mps) - v0).max() < 1e-12
        for s, A in enumerate(mps):
            if s < dst:
                Am = A.reshape(-1, A.shape[2])
                assert np.abs(Am.conj().T @ Am - np.eye(A.shape[2])).max() < 1e-12
            elif s > dst:
                Am = A.reshape(A.shape[0], -1)
                assert np.abs(Am @ Am.conj().T - np.eye(A.shape[0])).max() < 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_centre_energy_equals_full_contraction(seed):
    """The centre Rayleigh quotient (one H_eff product) equals <psi|H|psi>/<psi|psi> from the
    full left-to-right contraction on canonical states, so both sweep-energy modes agree."""
    w = inputs.workload("split", seed, M=6, d=3, D=3)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, 6, 3)
    cores = mpo.build_mpo(G, 3)
    lp = dmrg.LanczosParams(krylov_max=20, max_restarts=2, tol=1e-11)
    _, full = dmrg.dmrg(cores, 3, 6, 2, seed=seed + 5, lanczos=lp)
    _, cen = dmrg.dmrg(cores, 3, 6, 2, seed=seed + 5, lanczos=lp, energy_mode="centre")
    for a, b in zip(full.energies, cen.energies):
        assert abs(a - b) <= 1e-10 * Hn


@pytest.mark.parametrize("window", [(0, 5), (1, 4), (2, 3)])
def test_windowed_sweep(window):
    """A windowed sweep on a state centred at the window's first site: the full window (0, N-1)
    repeats the full sweep; any window reports the full contraction energy of the state it
    returns, and with a bond dimension that truncates nothing the energy never rises."""
    lo, hi = window
    N, d = 6, 3
    w = inputs.workload("split", 7, M=N, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, N, d)
    cores = mpo.build_mpo(G, d)
    lp = dmrg.LanczosParams(krylov_max=24, max_restarts=3, tol=1e-11)
    start = dmrg.initial_mps(N, d, 27, seed=3, center=lo)
    e0 = dmrg.energy(start, cores)
    mps, rep = dmrg.dmrg(cores, d, 27, 2, seed=3, lanczos=lp, mps=start, window=window)
    assert abs(rep.energies[-1] - dmrg.energy(mps, cores)) <= 1e-10 * Hn
    assert rep.energies[0] <= e0 + 1e-10 * Hn
    assert rep.energies[1] <= rep.energies[0] + 1e-10 * Hn
    if window == (0, N - 1):
        _, full = dmrg.dmrg(cores, d, 27, 2, seed=3, lanczos=lp, mps=start)
        for a, b in zip(rep.energies, full.energies):
            assert abs(a - b) <= 1e-10 * Hn


def test_reduced_density_matches_marginals_and_product_states():
    """rho_i is Hermitian, positive, of unit trace, its diagonal is the Fock marginal computed
    by the marginal routine, and on a product state it is the projector on the local state."""
    w = inputs.workload("plain", 1, M=4)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    cores = mpo.build_mpo(G, 4)
    mps, _ = dmrg.dmrg(cores, 4, 16, 2, seed=3, lanczos=dmrg.LanczosParams(tol=1e-11))
    for i in range(4):
        rho = observables.reduced_density(mps, i)
        assert np.abs(rho - rho.conj().T).max() < 1e-13
        assert np.linalg.eigvalsh(rho).min() > -1e-13 and abs(np.trace(rho) - 1) < 1e-12
        assert np.abs(np.diag(rho).real - observables.marginal(mps, None, [i])).max() < 1e-12
    rng = inputs.rng_for(77)
    phis = [inputs.random_complex(3, rng) for _ in range(5)]
    prod = [(2.0 * phi).reshape(1, 3, 1) for phi in phis]
    for i, phi in enumerate(phis):
        u = phi / np.linalg.norm(phi)
        assert np.abs(observables.reduced_density(prod, i) - np.outer(u, u.conj())).max() < 1e-13


def test_warm_start_features_and_targets_closed_forms():
    """U = I: mode i is a single-mode squeezed vacuum with V_i = diag(e^{-2r}, e^{2r}) / 2, so its
    features are [-2r - log 2, 2r - log 2, 0, -log 2]; the ground state is a product, and each
    mode's target is its local ground state, whose vacuum weight approaches the textbook
    |<0|S(r)|0>|^2 = 1 / cosh r as the cutoff grows."""
    w = inputs.workload("plain", 2, M=3, identity_U=True)
    V = gbs.covariance(w.r, w.U)
    f = warm.features(V)
    for i, r in enumerate(w.r):
        assert np.abs(f[i] - [-2 * r - np.log(2), 2 * r - np.log(2), 0.0, -np.log(2)]).max() < 1e-12
    d = 14
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    cores = mpo.build_mpo(G, d)
    mps, _ = dmrg.dmrg(cores, d, 1, 2, seed=1, lanczos=dmrg.LanczosParams(tol=1e-12, krylov_max=40))
    t = warm.targets(mps)
    for i, r in enumerate(w.r):
        u = t[i, 0::2] + 1j * t[i, 1::2]
        assert abs(np.linalg.norm(u) - 1) < 1e-12 and u[0].real > 0 and abs(u[0].imag) < 1e-12
        assert abs(abs(u[0]) ** 2 - 1 / np.cosh(r)) < 2e-3
        assert np.abs(u[1::2]).max() < 1e-10          # squeezed vacuum: even photon numbers only


# ------------------------------------------------------------------ sampler
def test_sampler_goodness_of_fit():
    w = inputs.workload("plain", 1, M=3)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    cores = mpo.build_mpo(G, 3)
    mps, _ = dmrg.dmrg(cores, 3, 9, 3, seed=2, lanczos=dmrg.LanczosParams(tol=1e-12))
    joint = observables.marginal(mps, None, [0, 1, 2]).reshape(-1)
    smp = observables.sample(mps, None, seed=99, n_samples=4000)
    idx = smp[:, 0] * 9 + smp[:, 1] * 3 + smp[:, 2]
    counts = np.bincount(idx, minlength=27)
    keep = joint * 4000 > 5
    exp = joint[keep] * 4000
    obs = counts[keep]
    stat = np.sum((obs - exp) ** 2 / exp)
    pval = scipy.stats.chi2.sf(stat, df=keep.sum() - 1)
    assert pval > 1e-4


def test_lbo_marginals_mean_photon_number():
    """With the optimal local basis at small d, the Fock-basis marginals after the inverse
    basis transformation give <n_i> = (V_xixi + V_pipi)/2 - 1/2 (closed form of the
    covariance), and each marginal sums to at most one."""
    w = inputs.workload("plain", 40, M=3, r_lo=0.3, r_hi=0.6)
    S_list, nu, Grot = gbs.lbo_transform(w.r, w.U)
    d, D = 6, 40
    cores = mpo.build_mpo(Grot, d)
    mps, rep = dmrg.dmrg(cores, d, 36, 3, seed=5, lanczos=dmrg.LanczosParams(tol=1e-12))
    isos = [gbs.lbo_isometry(S, D, d) for S in S_list]
    V = gbs.covariance(w.r, w.U)
    for i in range(3):
        p = observables.marginal(mps, isos, [i])
        assert p.sum() <= 1 + 1e-12 and p.sum() > 1 - 1e-6
        nmean = float(np.sum(np.arange(D) * p))
        exact = 0.5 * (V[i, i] + V[3 + i, 3 + i]) - 0.5
        assert abs(nmean - exact) < 2e-4
    # Fock-basis marginal agrees with a large-cutoff Fock-basis dense solve
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    _, v0 = dense.ground_state(G, 14)
    pd = dense.marginals_from_vector(v0[:, 0], 3, 14, [1])
    p1 = observables.marginal(mps, isos, [1])
    assert np.abs(p1[:8] - pd[:8]).max() < 1e-4


# ------------------------------------------------------------------ energy variance
def _mps_to_vector(mps):
    v = mps[0].reshape(-1, mps[0].shape[-1])
    for A in mps[1:]:
        v = (v @ A.reshape(A.shape[0], -1)).reshape(-1, A.shape[-1])
    return v[:, 0]


def _vector_to_mps(v, N, d):
    """Exact MPS of a d^N vector by successive SVDs (no truncation)."""
    sites, rest, cl = [], v.reshape(1, -1), 1
    for s in range(N - 1):
        U, S, Vh = np.linalg.svd(rest.reshape(cl * d, -1), full_matrices=False)
        sites.append(U.reshape(cl, d, -1))
        rest = (S[:, None] * Vh)
        cl = U.shape[1]
    sites.append(rest.reshape(cl, d, 1))
    return sites


@pytest.mark.parametrize("seed,M,d", [(0, 3, 3), (1, 4, 3), (2, 3, 4)])
def test_energy_variance_matches_dense(seed, M, d):
    """<H^2> by the two-layer environment contraction equals ||H v||^2 / ||v||^2 of the dense
    vector of the same (non-canonical) MPS; E likewise; sigma_H > 0 off an eigenstate."""
    w = inputs.workload("plain", seed, M=M, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    rng = inputs.rng_for(900 + seed)
    dims = [1] + [min(5, d ** s, d ** (M - s)) for s in range(1, M)] + [1]
    mps = [inputs.random_complex((dims[s], d, dims[s + 1]), rng) for s in range(M)]
    v = _mps_to_vector(mps)
    H = dense.dense_hamiltonian(G, d)
    Hv = H @ v
    n2 = np.vdot(v, v).real
    e, h2, sig = dmrg.energy_variance(mps, mpo.build_mpo(G, d))
    Hn = gbs.norm_bound(G, M, d)
    assert abs(h2 - np.vdot(Hv, Hv).real / n2) <= 1e-12 * Hn * Hn
    assert abs(e - np.vdot(v, Hv).real / n2) <= 1e-12 * Hn
    assert sig > 1e-3


@pytest.mark.parametrize("seed", [0, 1])
def test_energy_variance_vanishes_on_the_ground_state(seed):
    """The exact ground state (an eigenstate of P H P) has sigma_H = 0: <H^2> = E0^2."""
    w = inputs.workload("plain", seed, M=3, d=4, D=4)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    e0, v0 = dense.ground_state(G, w.d)
    mps = _vector_to_mps(v0[:, 0], w.M, w.d)
    e, h2, sig = dmrg.energy_variance(mps, mpo.build_mpo(G, w.d))
    Hn = gbs.norm_bound(G, w.M, w.d)
    assert abs(e - e0[0]) <= 1e-12 * Hn
    assert abs(h2 - e0[0] ** 2) <= 1e-12 * Hn * Hn
    assert sig <= 1e-6 * Hn


# ------------------------------------------------------------------ non-Gaussian (global CZ) workload
from oracle import nongauss  # noqa: E402


@pytest.mark.parametrize("seed,N,d,kappa", [(0, 3, 3, 0.3), (1, 4, 3, 0.2), (2, 3, 4, 0.5), (3, 2, 4, 0.7)])
def test_nongauss_expansion_and_mpo_match_definition(seed, N, d, kappa):
    """P H P of Eq. nonGBSHamiltonian three ways: from its definition (R' = (X, P + xi) as
    padded-space operators, products as written, then restricted), from the term expansion,
    and from the FSM MPO contracted to a matrix."""
    w = inputs.workload("plain", seed, M=N, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hdef = nongauss.hamiltonian_definition(G, d, kappa).toarray()
    Hexp = nongauss.dense_hamiltonian(G, d, kappa).toarray()
    Hmpo = mpo.contract_dense(nongauss.build_mpo(G, d, kappa))
    scale = np.abs(Hdef).max()
    assert np.abs(Hdef - Hdef.conj().T).max() <= 1e-14 * scale
    assert np.abs(Hexp - Hdef).max() <= 1e-13 * scale
    assert np.abs(Hmpo - Hdef).max() <= 1e-13 * scale


def test_nongauss_kappa_zero_is_gbs():
    w = inputs.workload("plain", 0, M=3, d=4, D=4)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    H0 = nongauss.hamiltonian_definition(G, 4, 0.0).toarray()
    assert np.abs(H0 - dense.dense_hamiltonian(G, 4).toarray()).max() < 1e-13


def test_nongauss_transformed_gaussian_state_has_zero_energy():
    """exp(-i kappa X1 X2 X3) applied to the Gaussian state (Eq. GlobalCZgate) is the zero-energy
    state of Eq. nonGBSHamiltonian: its <H> falls geometrically with the Fock cutoff, while the
    same state has O(kappa^2) energy under the Hamiltonian with the sign of xi flipped."""
    import scipy.linalg as sla
    w = inputs.workload("plain", 4, M=3, r_lo=0.15, r_hi=0.25)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    kappa = 0.1
    es = []
    for D in (6, 8, 10):
        _, v0 = dense.ground_state(G, D)
        X = gbs.local_ops(D)["X"]
        psi = sla.expm(-1j * kappa * np.kron(np.kron(X, X), X)) @ v0[:, 0]
        H = nongauss.hamiltonian_definition(G, D, kappa)
        es.append(np.vdot(psi, H @ psi).real / np.vdot(psi, psi).real)
        if D == 10:
            Hm = nongauss.hamiltonian_definition(G, D, -kappa)
            e_wrong = np.vdot(psi, Hm @ psi).real / np.vdot(psi, psi).real
    assert es[0] > es[1] > es[2] > 0
    assert es[2] < 1e-7
    assert e_wrong > 1e3 * es[2] and e_wrong > 1e-4


# ------------------------------------------------------------------ bond spectra (a6)
def test_symplectic_eigenvalues_special_cases():
    """Product state (U = I): every block has nu = 1/2.  Pure state: a block and its
    complement have the same symplectic spectrum beyond the vacuum values.  One mode:
    nu = sqrt(det V_i), the Williamson value."""
    w = inputs.workload("plain", 0, M=5, identity_U=True)
    V = gbs.covariance(w.r, w.U)
    assert np.abs(gbs.symplectic_eigenvalues(V[np.ix_([0, 1, 5, 6], [0, 1, 5, 6])]) - 0.5).max() < 1e-12
    w = inputs.workload("plain", 1, M=5)
    V = gbs.covariance(w.r, w.U)
    a = gbs.symplectic_eigenvalues(V[np.ix_([0, 1, 5, 6], [0, 1, 5, 6])])
    b = gbs.symplectic_eigenvalues(V[np.ix_([2, 3, 4, 7, 8, 9], [2, 3, 4, 7, 8, 9])])
    assert np.abs(np.sort(b)[-2:] - np.sort(a)).max() < 1e-10 and abs(np.sort(b)[0] - 0.5) < 1e-10
    for i in range(5):
        Vi = gbs.reduced_covariance(V, i)
        assert abs(gbs.symplectic_eigenvalues(Vi)[0] - gbs.williamson_single(Vi)[1]) < 1e-12


@pytest.mark.parametrize("seed,N,d,cut", [(0, 3, 12, 1), (1, 3, 12, 2), (2, 2, 24, 1)])
def test_bond_spectrum_of_the_ground_state_is_gaussian(seed, N, d, cut):
    """The squared Schmidt values of the P H P ground state at a cut against the closed-form
    Gaussian spectrum: with F >= 1 - E (Eq. MagOfSimError) and the contraction of the trace
    norm under the partial trace, sum_i |lambda_i - mu_i| <= 2 sqrt(1 - F) <= 2 sqrt(E)."""
    w = inputs.workload("plain", seed, M=N, r_lo=0.3, r_hi=0.5)
    V = gbs.covariance(w.r, w.U)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    e0, v0 = dense.ground_state(G, d)
    psi = v0[:, 0].reshape(d ** cut, d ** (N - cut))
    lam = np.linalg.svd(psi, compute_uv=False) ** 2
    lam /= lam.sum()
    k = 12
    mu = gbs.gaussian_schmidt_spectrum(V, cut, k)
    assert np.sum(np.abs(lam[:k] - mu)) <= 2.0 * np.sqrt(max(e0[0], 0.0)) + 1e-12


# ------------------------------------------------------------------ warm-started truncation
def _theta_with_spectrum(rng, cl, d1, d2, cr, decay):
    th = inputs.random_complex((cl, d1, d2, cr), rng)
    Tm = th.reshape(cl * d1, d2 * cr)
    U, s, Vh = np.linalg.svd(Tm, full_matrices=False)
    s = decay ** np.arange(s.size)
    return ((U * s) @ Vh).reshape(th.shape) / np.linalg.norm(s)


def _projector(A):
    M = A.reshape(-1, A.shape[-1])
    return M @ M.conj().T


@pytest.mark.parametrize("direction", ["right", "left"])
def test_truncate_warm_full_space_and_exact_start_are_exact(direction):
    """Rayleigh-Ritz over the whole space (k + p >= n), or started from the exact kept
    eigenvectors with no iteration, reproduces the eigendecomposition: same eigenvalues,
    same kept subspace, same truncated theta."""
    rng = inputs.rng_for(41)
    th = _theta_with_spectrum(rng, 3, 2, 2, 5, 0.7)
    n = 6 if direction == "right" else 10
    for chi, Q0, q, p in ((n, None, 0, 8), (4, "exact", 0, 0)):
        l0, r0, w0, disc0 = dmrg.truncate(th, direction, chi)
        if Q0 == "exact":
            T = th.reshape(6, 10)
            rho = T @ T.conj().T if direction == "right" else T.conj().T @ T
            _, V = np.linalg.eigh(rho)
            Q0 = V[:, ::-1][:, :chi]
        l1, r1, w1, disc1 = dmrg.truncate_warm(th, direction, chi, Q0, q=q, p=p, seed=3, bond=1)
        assert np.abs(w1 - w0).max() < 1e-12 and abs(disc1 - disc0) < 1e-12
        kept0, kept1 = (l0, l1) if direction == "right" else (np.transpose(r0.conj(), (2, 1, 0)),
                                                               np.transpose(r1.conj(), (2, 1, 0)))
        assert np.abs(_projector(kept1) - _projector(kept0)).max() < 1e-10
        rec0 = np.einsum("asb,btc->astc", l0, r0)
        rec1 = np.einsum("asb,btc->astc", l1, r1)
        assert np.abs(rec1 - rec0).max() < 1e-10


def test_truncate_warm_ritz_values_interlace_and_converge():
    """Ritz values from any subspace lie below the eigenvalues of the same rank (Cauchy
    interlacing); subspace iteration drives them to the eigenvalues."""
    rng = inputs.rng_for(42)
    th = _theta_with_spectrum(rng, 8, 4, 4, 8, 0.85)
    _, _, lam, _ = dmrg.truncate(th, "right", 10)
    Q0 = inputs.random_complex((32, 10), rng)
    for q in (0, 1, 3):
        _, _, w, _ = dmrg.truncate_warm(th, "right", 10, Q0, q=q, p=4, seed=5, bond=2)
        assert np.all(w <= lam + 1e-13)
    _, _, w, _ = dmrg.truncate_warm(th, "right", 10, Q0, q=60, p=4, seed=5, bond=2)
    assert np.abs(w - lam).max() < 1e-10


def test_dmrg_with_warm_truncation_plain_is_exact():
    """chi = d^2 covers the plain workload: the warm truncation works on the full space and the
    sweep reaches the dense ground energy."""
    w = inputs.workload("plain", 1)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, w.M, w.d)
    e0 = dense.ground_state(G, w.d)[0][0]
    cores = mpo.build_mpo(G, w.d)
    _, rep = dmrg.dmrg(cores, w.d, 16, 4, seed=3, warm_q=1,
                       lanczos=dmrg.LanczosParams(krylov_max=32, max_restarts=8, tol=1e-12))
    assert abs(rep.energies[-1] - e0) <= 1e-10 * Hn
