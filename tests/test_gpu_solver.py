"""GPU solver parity against the CPU oracle (dense exact solve, hafnians, oracle DMRG).

Bars (FP64 path): |dE| <= 1e-10 ||H|| with ||H|| = lambda_max(G) M (2d - 1), marginal
probabilities within 1e-9, samples bit-identical to the oracle's sampler run on the same
MPS with the same Philox stream.
"""
import math
import os

import numpy as np
import pytest

from oracle import dense, dmrg as odmrg, gbs, mpo as ompo, nongauss, observables as oobs, philox
from paper_2410_18740_gb300 import inputs, vtn

pytestmark = pytest.mark.gpu


def gpu_sites(ctx, mps):
    M, _, _ = vtn.vtn_mps_info(mps)
    return [vtn.vtn_mps_get_site(ctx, mps, s) for s in range(M)]


def solve(ctx, w, chi, n_sweeps, seed, tol=1e-12, sched=None, lbo=False):
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, w.D, w.d, vtn.VTN_FLAG_LBO if lbo else 0)
    opts = vtn.vtn_sweep_opts_default(chi_max=chi, n_sweeps=n_sweeps, seed=seed, lanczos_tol=tol,
                                      krylov_max=32, lanczos_max_restarts=8,
                                      **({"chi_schedule": sched} if sched else {}))
    st, mps, rep = vtn.vtn_sweep(ctx, m, None, opts)
    return m, mps, rep, st


def test_initial_mps_matches_oracle(ctx):
    w = inputs.workload("plain", 0, M=5, d=3, D=3)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, 3, 3)
    mps = vtn.vtn_mps_random(ctx, m, 7, seed=11)
    osites = odmrg.initial_mps(5, 3, 7, seed=11)
    for a, b in zip(gpu_sites(ctx, mps), osites):
        assert a.shape == b.shape
        assert np.abs(a - b).max() < 1e-13
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_initial_mps_large_bonds_matches_oracle(ctx):
    """Bond dimension 512 at d = 6 (the large workload's shape): the site matrices of 216 x 3072
    and 512 x 1296 are orthonormalised by CholeskyQR2 on the GEMM; the rows must be the
    Gram-Schmidt rows of the oracle (numpy Householder QR with a positive diagonal)."""
    w = inputs.workload("plain", 0, M=8, d=6, D=6)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, 6, 6)
    mps = vtn.vtn_mps_random(ctx, m, 512, seed=23)
    osites = odmrg.initial_mps(8, 6, 512, seed=23)
    for a, b in zip(gpu_sites(ctx, mps), osites):
        assert a.shape == b.shape
        assert np.abs(a - b).max() < 1e-13
        rows = a.reshape(a.shape[0], -1)
        assert np.abs(rows @ rows.conj().T - np.eye(rows.shape[0])).max() < 1e-13
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_plain_workload_energy_and_marginals(ctx, seed):
    """Plain workload (M=4, d=4, chi=16): the MPS is exact, so the GPU energy must equal
    the dense exact ground energy, and marginals the dense ones."""
    w = inputs.workload("plain", seed)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, w.M, w.d)
    e0, v0 = dense.ground_state(G, w.d)
    m, mps, rep, st = solve(ctx, w, 16, 4, seed + 100)
    assert st == vtn.VTN_OK
    E = vtn.vtn_energy(ctx, m, mps)
    assert abs(E - e0[0]) <= 1e-10 * Hn
    assert abs(rep["energy"][-1] - E) <= 1e-12 * Hn
    assert E >= -1e-10 * Hn
    marg = vtn.vtn_marginals_all(ctx, m, mps)
    for i in range(w.M):
        assert np.abs(marg[i] - dense.marginals_from_vector(v0[:, 0], w.M, w.d, [i])).max() <= 1e-9
    for modes in ([0, 2], [3, 1], [2, 1, 0]):
        p = vtn.vtn_marginals(ctx, m, mps, modes)
        assert np.abs(p - dense.marginals_from_vector(v0[:, 0], w.M, w.d, modes)).max() <= 1e-9
    # fidelity bound F >= 1 - <H> against the exact (hafnian) GBS state
    sites = gpu_sites(ctx, mps)
    psi = sites[0]
    for A in sites[1:]:
        psi = np.tensordot(psi, A, axes=([-1], [0]))
    psi = psi.reshape(-1) / np.linalg.norm(psi)
    amp = dense.gbs_amplitudes(w.r, w.U, w.d).reshape(-1)
    assert abs(np.vdot(amp, psi)) ** 2 >= 1 - E - 1e-12
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


@pytest.mark.parametrize("seed,M,d,chi,n_sweeps", [(0, 6, 3, 9, 3), (1, 8, 4, 12, 3), (2, 7, 5, 20, 2)])
def test_sweep_trajectory_matches_oracle_dmrg(ctx, seed, M, d, chi, n_sweeps):
    """Same initial MPS (Philox), same Lanczos rule, same truncation rule: the energy after
    every sweep matches the oracle's two-site DMRG."""
    w = inputs.workload("split", seed, M=M, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, M, d)
    m, mps, rep, st = solve(ctx, w, chi, n_sweeps, seed + 7)
    cores = ompo.build_mpo(G, d)
    omps, orep = odmrg.dmrg(cores, d, chi, n_sweeps, seed=seed + 7,
                            lanczos=odmrg.LanczosParams(krylov_max=32, max_restarts=8, tol=1e-12))
    assert rep["sweeps_done"] == len(orep.energies)
    for a, b in zip(rep["energy"], orep.energies):
        assert abs(a - b) <= 1e-10 * Hn
    # transfer parity: each side's evaluator on the other's state
    sites = gpu_sites(ctx, mps)
    assert abs(odmrg.energy(sites, cores) - vtn.vtn_energy(ctx, m, mps)) <= 1e-12 * Hn
    # marginals of the GPU state vs the oracle's marginals of the same state
    marg = vtn.vtn_marginals_all(ctx, m, mps)
    for i in range(M):
        assert np.abs(marg[i] - oobs.marginal(sites, None, [i])).max() <= 1e-12
    # and of the two independently converged states
    for i in range(M):
        assert np.abs(marg[i] - oobs.marginal(omps, None, [i])).max() <= 1e-9
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_local_basis_workload_matches_oracle(ctx):
    """Optimal local basis (d < D): energies, Fock marginals after the inverse basis
    transformation, and the closed-form mean photon numbers."""
    w = inputs.workload("large", 3, M=5, D=24, d=5)
    S_list, nu, Grot = gbs.lbo_transform(w.r, w.U)
    Hn = gbs.norm_bound(Grot, w.M, w.d)
    m, mps, rep, st = solve(ctx, w, 25, 3, 9)
    cores = ompo.build_mpo(Grot, w.d)
    omps, orep = odmrg.dmrg(cores, w.d, 25, 3, seed=9,
                            lanczos=odmrg.LanczosParams(krylov_max=32, max_restarts=8, tol=1e-12))
    for a, b in zip(rep["energy"], orep.energies):
        assert abs(a - b) <= 1e-10 * Hn
    isos = [gbs.lbo_isometry(S, 24, 5) for S in S_list]
    sites = gpu_sites(ctx, mps)
    marg = vtn.vtn_marginals_all(ctx, m, mps)
    for i in range(w.M):
        assert np.abs(marg[i] - oobs.marginal(sites, isos, [i])).max() <= 1e-9
        assert marg[i].sum() <= 1 + 1e-12
    p2 = vtn.vtn_marginals(ctx, m, mps, [4, 1])
    assert np.abs(p2 - oobs.marginal(sites, isos, [4, 1])).max() <= 1e-9
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_samples_bit_identical_to_oracle(ctx):
    w = inputs.workload("plain", 4)
    m, mps, rep, st = solve(ctx, w, 16, 2, 3)
    got = vtn.vtn_sample(ctx, m, mps, seed=1234, n_samples=500)
    sites = gpu_sites(ctx, mps)
    expect = oobs.sample(sites, None, seed=1234, n_samples=500)
    assert np.array_equal(got, expect)
    # with a local basis too
    w2 = inputs.workload("large", 8, M=4, D=10, d=4)
    m2, mps2, _, _ = solve(ctx, w2, 16, 2, 5)
    S_list, _, _ = gbs.lbo_transform(w2.r, w2.U)
    isos = [gbs.lbo_isometry(S, 10, 4) for S in S_list]
    got2 = vtn.vtn_sample(ctx, m2, mps2, seed=99, n_samples=300)
    exp2 = oobs.sample(gpu_sites(ctx, mps2), isos, seed=99, n_samples=300)
    assert np.array_equal(got2, exp2)
    for h in (mps, mps2):
        vtn.vtn_mps_free(h)
    vtn.vtn_mpo_free(m)
    vtn.vtn_mpo_free(m2)


def test_product_state_identity_interferometer(ctx):
    """U = I: chi = 1 suffices and the energy is the sum of single-mode ground energies."""
    w = inputs.workload("plain", 12, M=5, identity_U=True, d=8, D=8)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    ops = gbs.local_ops(8)
    e_single = 0.0
    for i in range(5):
        h = G[i, i] * ops["X2"] + G[5 + i, 5 + i] * ops["P2"] + G[i, 5 + i] * ops["XPPX"] - 0.5 * ops["I"]
        e_single += np.linalg.eigvalsh(h)[0]
    m, mps, rep, st = solve(ctx, w, 1, 3, 4)
    assert abs(vtn.vtn_energy(ctx, m, mps) - e_single) <= 1e-10 * gbs.norm_bound(G, 5, 8)
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_save_load_roundtrip(ctx, tmp_path):
    w = inputs.workload("plain", 5)
    m, mps, rep, st = solve(ctx, w, 16, 2, 1)
    path = tmp_path / "state.vtn"
    vtn.vtn_mps_save(ctx, mps, path)
    mps2 = vtn.vtn_mps_load(ctx, m, path)
    assert vtn.vtn_energy(ctx, m, mps2) == vtn.vtn_energy(ctx, m, mps)
    for a, b in zip(gpu_sites(ctx, mps), gpu_sites(ctx, mps2)):
        assert np.array_equal(a, b)
    # resume: continue sweeping from the loaded state
    opts = vtn.vtn_sweep_opts_default(chi_max=16, n_sweeps=1, lanczos_tol=1e-12)
    st2, mps3, rep2 = vtn.vtn_sweep(ctx, m, mps2, opts)
    assert abs(rep2["energy"][0] - rep["energy"][-1]) <= 1e-9
    with open(path, "r+b") as f:
        f.write(b"XXXX")
    with pytest.raises(vtn.VtnError):
        vtn.vtn_mps_load(ctx, m, path)
    for h in (mps, mps2):
        vtn.vtn_mps_free(h)
    vtn.vtn_mpo_free(m)


def test_error_paths(ctx):
    w = inputs.workload("plain", 0)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, 4, 4)
    mps = vtn.vtn_mps_random(ctx, m, 4, 1)
    with pytest.raises(vtn.VtnError) as e:
        vtn.vtn_marginals(ctx, m, mps, [1, 1])
    assert e.value.status == vtn.VTN_EINVAL
    with pytest.raises(vtn.VtnError):
        vtn.vtn_marginals(ctx, m, mps, [4])
    with pytest.raises(vtn.VtnError):
        vtn.vtn_sweep(ctx, m, mps, vtn.vtn_sweep_opts_default(n_sweeps=65))
    with pytest.raises(vtn.VtnError) as e:
        vtn.vtn_sweep(ctx, m, mps, vtn.vtn_sweep_opts_default(prec=vtn.VTN_TF32X3))
    assert e.value.status == vtn.VTN_EUNSUPPORTED
    # Lanczos forced to miss its tolerance: VTN_ENOCONV, but the state is still valid
    st, mps2, rep = vtn.vtn_sweep(ctx, m, mps, vtn.vtn_sweep_opts_default(
        chi_max=16, n_sweeps=1, krylov_max=1, lanczos_max_restarts=0, lanczos_tol=1e-15))
    assert st == vtn.VTN_ENOCONV and rep["lanczos_not_converged"] > 0
    assert "Lanczos" in vtn.vtn_last_error(ctx)
    E = vtn.vtn_energy(ctx, m, mps2)
    assert np.isfinite(E) and E >= -1e-9
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_split_workload_full_size_properties(ctx):
    """Split workload at full size (M=24, d=8, chi=128), in the launch configuration of the
    benchmark but with a bounded number of H_eff products (one sweep, 4 Lanczos steps per
    bond): sampled checks the oracle can compute at this size -- the energy of the GPU
    state re-evaluated by the oracle's own MPO and contractions -- plus E >= 0 and
    normalised, non-negative marginals."""
    w = inputs.workload("split", 100)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, w.M, w.d)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, w.D, w.d)
    opts = vtn.vtn_sweep_opts_default(chi_max=128, n_sweeps=1, seed=1, lanczos_tol=1e-9, krylov_max=4,
                                      lanczos_max_restarts=0, chi_schedule=[128])
    st, mps, rep = vtn.vtn_sweep(ctx, m, None, opts)
    assert st in (vtn.VTN_OK, vtn.VTN_ENOCONV)
    _, _, dims = vtn.vtn_mps_info(mps)
    assert dims.max() == 128
    E = vtn.vtn_energy(ctx, m, mps)
    assert E >= -1e-10 * Hn
    sites = gpu_sites(ctx, mps)
    cores = ompo.build_mpo(G, w.d)
    assert abs(odmrg.energy(sites, cores) - E) <= 1e-10 * Hn
    marg = vtn.vtn_marginals_all(ctx, m, mps)
    assert np.all(marg >= -1e-12) and np.abs(marg.sum(axis=1) - 1).max() < 1e-10
    for i in (0, 11, 23):
        assert np.abs(marg[i] - oobs.marginal(sites, None, [i])).max() <= 1e-9
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_split_workload_full_size_bf16x3(ctx):
    """The benchmark's own mode at full size (M=24, d=8, chi=128, bf16x3 H_eff psi and
    environments, 8 Lanczos steps per bond, no restarts): the state it produces is checked by
    the oracle's FP64 energy of that state and by its marginals on sampled modes; the sweep's
    reported energy is the FP64 energy; the kept sites are isometries (right-canonical)."""
    w = inputs.workload("split", 100)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, w.M, w.d)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, w.D, w.d)
    opts = vtn.vtn_sweep_opts_default(chi_max=128, n_sweeps=1, seed=1, lanczos_tol=1e-12, krylov_max=8,
                                      lanczos_max_restarts=0, chi_schedule=[128], prec=vtn.VTN_BF16X3)
    st, mps, rep = vtn.vtn_sweep(ctx, m, None, opts)
    assert st in (vtn.VTN_OK, vtn.VTN_ENOCONV)
    E = vtn.vtn_energy(ctx, m, mps)
    assert abs(rep["energy"][-1] - E) <= 1e-12 * Hn
    assert E >= -1e-10 * Hn
    sites = gpu_sites(ctx, mps)
    assert abs(odmrg.energy(sites, ompo.build_mpo(G, w.d)) - E) <= 1e-10 * Hn
    for A in sites[1:]:
        Am = A.reshape(A.shape[0], -1)
        assert np.abs(Am @ Am.conj().T - np.eye(A.shape[0])).max() < 1e-10
    marg = vtn.vtn_marginals_all(ctx, m, mps)
    assert np.all(marg >= -1e-12) and np.abs(marg.sum(axis=1) - 1).max() < 1e-10
    for i in (0, 12, 23):
        assert np.abs(marg[i] - oobs.marginal(sites, None, [i])).max() <= 1e-9
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_converged_mean_photon_number(ctx):
    """Converged solve: Fock-basis <n_i> from the marginals agree with the covariance closed
    form (V_xx + V_pp)/2 - 1/2.  Rigorous bound: |d<n>| <= 2 (d-1) sqrt(1-F) with
    F >= 1 - <H> (trace distance, n < d inside the cutoff) plus the cutoff tail."""
    w = inputs.workload("split", 101, M=6, d=6, D=6, r_lo=0.2, r_hi=0.3)
    m, mps, rep, st = solve(ctx, w, 36, 4, 2, tol=1e-11)
    E = vtn.vtn_energy(ctx, m, mps)
    assert 0 <= E < 1e-3
    marg = vtn.vtn_marginals_all(ctx, m, mps)
    V = gbs.covariance(w.r, w.U)
    nfock = 0.5 * (np.diag(V)[:6] + np.diag(V)[6:]) - 0.5
    err = np.abs(marg @ np.arange(6) - nfock).max()
    assert err <= 2 * 5 * np.sqrt(E) + 1e-6
    assert err <= 5 * E          # observed: errors of observables scale like <H> (Fig. 4c)
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


@pytest.mark.parametrize("seed,M,d,chi", [(0, 4, 4, 6), (1, 6, 3, 5), (2, 5, 5, 8)])
def test_energy_variance_matches_oracle(ctx, seed, M, d, chi):
    """<H^2> and sigma_H of the same random, non-canonical MPS: GPU two-layer environments
    (centre-collapsed MPO) against the oracle's (w = 2N+2 MPO)."""
    w = inputs.workload("split", seed, M=M, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, M, d)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, w.D, w.d)
    rng = inputs.rng_for(950 + seed)
    dims = [1] + [min(chi, d ** s, d ** (M - s)) for s in range(1, M)] + [1]
    sites = [inputs.random_complex((dims[s], d, dims[s + 1]), rng) for s in range(M)]
    mps = vtn.vtn_mps_from_host(ctx, m, sites)
    e, h2, sg = vtn.vtn_energy_variance(ctx, m, mps)
    oe, oh2, osg = odmrg.energy_variance(sites, ompo.build_mpo(G, d))
    assert abs(e - oe) <= 1e-10 * Hn
    assert abs(h2 - oh2) <= 1e-10 * Hn * Hn
    assert abs(sg - osg) <= 1e-8 * Hn
    assert abs(e - vtn.vtn_energy(ctx, m, mps)) <= 1e-12 * Hn
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_energy_variance_of_the_converged_plain_state(ctx):
    """Plain workload (exact at chi = 16): the converged state is an eigenstate of P H P to the
    Lanczos tolerance, so sigma_H is tiny, while the seeded random start is far from one."""
    w = inputs.workload("plain", 0)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, w.M, w.d)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, w.D, w.d)
    start = vtn.vtn_mps_random(ctx, m, 16, 5)
    _, _, sg0 = vtn.vtn_energy_variance(ctx, m, start)
    vtn.vtn_mps_free(start)
    m2, mps, rep, st = solve(ctx, w, 16, 4, 100)
    e, h2, sg = vtn.vtn_energy_variance(ctx, m2, mps)
    assert sg <= 1e-5 * Hn
    assert sg0 >= 1e-2
    assert abs(e - rep["energy"][-1]) <= 1e-12 * Hn
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m2)
    vtn.vtn_mpo_free(m)


@pytest.mark.parametrize("seed,M,d,chi,kappa", [(0, 4, 4, 16, 0.3), (1, 5, 3, 9, 0.2), (2, 4, 3, 9, -0.4)])
def test_cz_workload_ground_state(ctx, seed, M, d, chi, kappa):
    """Non-Gaussian (global CZ) workload at sizes where the MPS is exact: the GPU sweep reaches
    the ground energy of the oracle's P H P built from its definition, the marginals of the
    dense ground state, and a vanishing energy variance."""
    w = inputs.workload("plain", seed, M=M, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Href = nongauss.hamiltonian_definition(G, d, kappa).toarray()
    evals, evecs = np.linalg.eigh(Href)
    Hn = np.abs(evals).max()
    m = vtn.vtn_build_mpo_cz(ctx, w.r, w.U, d, kappa)
    opts = vtn.vtn_sweep_opts_default(chi_max=chi, n_sweeps=4, seed=seed + 40, lanczos_tol=1e-12, krylov_max=32,
                                      lanczos_max_restarts=8)
    st, mps, rep = vtn.vtn_sweep(ctx, m, None, opts)
    assert st == vtn.VTN_OK
    E = vtn.vtn_energy(ctx, m, mps)
    assert abs(E - evals[0]) <= 1e-10 * Hn
    marg = vtn.vtn_marginals_all(ctx, m, mps)
    for i in range(M):
        assert np.abs(marg[i] - dense.marginals_from_vector(evecs[:, 0], M, d, [i])).max() <= 1e-8
    _, _, sg = vtn.vtn_energy_variance(ctx, m, mps)
    assert sg <= 1e-5 * Hn
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_cz_sweep_trajectory_matches_oracle(ctx):
    """Same initial MPS, Lanczos rule and truncation rule with the bond dimension below exact:
    energies after each sweep match the oracle's two-site DMRG on its own MPO of the same
    Hamiltonian."""
    M, d, chi, kappa = 6, 3, 8, 0.25
    w = inputs.workload("plain", 7, M=M, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    m = vtn.vtn_build_mpo_cz(ctx, w.r, w.U, d, kappa)
    Hn = np.abs(np.linalg.eigvalsh(nongauss.dense_hamiltonian(G, d, kappa).toarray())).max()
    opts = vtn.vtn_sweep_opts_default(chi_max=chi, n_sweeps=3, seed=11, lanczos_tol=1e-12, krylov_max=32,
                                      lanczos_max_restarts=8)
    st, mps, rep = vtn.vtn_sweep(ctx, m, None, opts)
    omps, orep = odmrg.dmrg(nongauss.build_mpo(G, d, kappa), d, chi, 3, seed=11,
                            lanczos=odmrg.LanczosParams(krylov_max=32, max_restarts=8, tol=1e-12))
    assert rep["sweeps_done"] == len(orep.energies)
    for a, b in zip(rep["energy"], orep.energies):
        assert abs(a - b) <= 1e-10 * Hn
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)
