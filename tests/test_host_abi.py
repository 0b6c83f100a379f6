"""CPU tests of the C-ABI library: it loads, exports every entry point include/vtn.h
declares, and its host-side problem set-up (coefficients, optimal local basis, MPO)
agrees with the oracle.  No kernel runs here."""
import os
import re

import numpy as np
import pytest

from oracle import dense, gbs, mpo as ompo, nongauss
from paper_2410_18740_gb300 import inputs, vtn
from tests.conftest import ROOT


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "vtn.h")).read()
    return sorted(set(re.findall(r"^\s*(?:vtn_status|const char\*)\s+(vtn_\w+)\s*\(", text, re.M)))


def test_library_exports_every_declared_symbol(libvtn):
    names = declared_symbols()
    assert len(names) >= 30
    for n in names:
        assert hasattr(libvtn, n), f"{n} not exported"
    assert set(names) == set(vtn.exported_symbols())


def _dense_from_abi(m):
    M, d, D, w = vtn.vtn_mpo_info(m)
    cores = []
    for s in range(M):
        wl, wr, rows, cols, ops = vtn.vtn_mpo_core(m, s)
        W = np.zeros((wl, wr, d, d), complex)
        for a, b, op in zip(rows, cols, ops):
            W[a, b] += op
        cores.append(W)
    return ompo.contract_dense(cores)


@pytest.mark.parametrize("seed,M,d", [(0, 1, 3), (1, 2, 3), (2, 3, 3), (3, 4, 4), (4, 5, 3)])
def test_centre_collapsed_mpo_equals_dense_hamiltonian(libvtn, seed, M, d):
    w = inputs.workload("plain", seed, M=M)
    m = vtn.vtn_build_mpo(None, w.r, w.U, d, d)
    try:
        G = gbs.hamiltonian_coefficients(w.r, w.U)
        assert np.abs(vtn.vtn_mpo_coefficients(m) - G).max() < 1e-12
        assert np.abs(vtn.vtn_mpo_covariance(m) - gbs.covariance(w.r, w.U)).max() < 1e-12
        H = _dense_from_abi(m)
        assert np.abs(H - dense.dense_hamiltonian(G, d).toarray()).max() < 1e-12
        _, _, _, wd = vtn.vtn_mpo_info(m)
        for s in range(1, M):
            assert wd[s] == 2 * min(s, M - s) + 2
        assert vtn.vtn_mpo_norm_bound(m) == pytest.approx(gbs.norm_bound(G, M, d), rel=1e-9)
    finally:
        vtn.vtn_mpo_free(m)


@pytest.mark.parametrize("seed", [5, 6])
def test_optimal_local_basis_against_oracle(libvtn, seed):
    w = inputs.workload("large", seed, M=5)
    m = vtn.vtn_build_mpo(None, w.r, w.U, 40, 6)
    try:
        S_list, nu, Grot = gbs.lbo_transform(w.r, w.U)
        assert np.abs(vtn.vtn_mpo_coefficients(m) - Grot).max() < 1e-12
        for i in range(5):
            V = vtn.vtn_mpo_isometry(m, i)
            Vo = gbs.lbo_isometry(S_list[i], 40, 6)
            ph = np.vdot(V.reshape(-1), Vo.reshape(-1))
            ph /= abs(ph)
            assert np.abs(V * ph - Vo).max() < 1e-12
        H = _dense_from_abi(vtn.vtn_build_mpo(None, w.r[:3], inputs.haar_unitary(3, inputs.rng_for(seed)), 3, 3))
        assert np.allclose(H, H.conj().T)
    finally:
        vtn.vtn_mpo_free(m)


def test_large_workload_mpo_against_oracle(libvtn):
    """The large workload at full size (M = 100, r ~ U(0.8, 1.2), Haar U, D = 24 -> d = 6 in the
    optimal local basis): coefficients G' = S^T G S, every mode's isometry (up to its global
    phase), the centre-collapsed bond dimensions 2 min(s, M - s) + 2 and the norm bound, against
    the oracle."""
    w = inputs.workload("large", 200)
    assert (w.M, w.D, w.d) == (100, 24, 6)
    m = vtn.vtn_build_mpo(None, w.r, w.U, w.D, w.d)
    try:
        S_list, nu, Grot = gbs.lbo_transform(w.r, w.U)
        assert np.abs(vtn.vtn_mpo_coefficients(m) - Grot).max() < 1e-11 * np.abs(Grot).max()
        for i in range(w.M):
            V = vtn.vtn_mpo_isometry(m, i)
            Vo = gbs.lbo_isometry(S_list[i], w.D, w.d)
            ph = np.vdot(V.reshape(-1), Vo.reshape(-1))
            ph /= abs(ph)
            assert np.abs(V * ph - Vo).max() < 1e-12
        M, d, D, wd = vtn.vtn_mpo_info(m)
        assert (M, d, D) == (100, 6, 24)
        expect = [1] + [2 * min(s, 100 - s) + 2 for s in range(1, 100)] + [1]
        assert list(wd) == expect
        G = gbs.hamiltonian_coefficients(w.r, w.U)
        assert abs(vtn.vtn_mpo_norm_bound(m) - gbs.norm_bound(Grot, 100, 6)) <= 1e-12 * gbs.norm_bound(Grot, 100, 6)
        assert np.abs(G - G.T).max() < 1e-12
    finally:
        vtn.vtn_mpo_free(m)


def test_fock_isometry_is_identity(libvtn):
    w = inputs.workload("plain", 0)
    m = vtn.vtn_build_mpo(None, w.r, w.U, 4, 4)
    for i in range(4):
        assert np.array_equal(vtn.vtn_mpo_isometry(m, i), np.eye(4))
    vtn.vtn_mpo_free(m)


def test_validation_errors(libvtn):
    w = inputs.workload("plain", 0)
    bad = w.U.copy()
    bad[0, 0] += 1e-6
    with pytest.raises(vtn.VtnError) as e:
        vtn.vtn_build_mpo(None, w.r, bad, 4, 4)
    assert e.value.status == vtn.VTN_EINVAL and "unitary" in e.value.msg
    with pytest.raises(vtn.VtnError):
        vtn.vtn_build_mpo(None, w.r, w.U, 4, 5)        # d > D
    with pytest.raises(vtn.VtnError):
        vtn.vtn_build_mpo(None, w.r, w.U, 1, 1)        # D < 2
    with pytest.raises(vtn.VtnError):
        vtn.vtn_build_mpo(None, w.r, w.U, 20, 17)      # d > 16
    r = w.r.copy()
    r[1] = np.nan
    with pytest.raises(vtn.VtnError):
        vtn.vtn_build_mpo(None, r, w.U, 4, 4)


def test_sweep_opts_defaults(libvtn):
    o = vtn.vtn_sweep_opts_default()
    assert o.chi_max == 16 and o.n_sweeps == 8 and o.krylov_max == 32 and o.prec == vtn.VTN_FP64
    assert o.lanczos_tol == 1e-10 and o.lanczos_max_restarts == 4


@pytest.mark.parametrize("seed,M,d,kappa", [(0, 3, 3, 0.3), (1, 4, 3, 0.2), (2, 3, 4, -0.5), (3, 2, 4, 0.7)])
def test_cz_mpo_equals_the_definition(libvtn, seed, M, d, kappa):
    """The non-Gaussian (global CZ) MPO built by the library, contracted to a matrix, equals the
    oracle's P H P of Eq. nonGBSHamiltonian built from its definition."""
    w = inputs.workload("plain", seed, M=M, d=d, D=d)
    m = vtn.vtn_build_mpo_cz(None, w.r, w.U, d, kappa)
    try:
        G = gbs.hamiltonian_coefficients(w.r, w.U)
        H = _dense_from_abi(m)
        Href = nongauss.hamiltonian_definition(G, d, kappa).toarray()
        assert np.abs(H - Href).max() <= 1e-13 * np.abs(Href).max()
        _, dd, D, wd = vtn.vtn_mpo_info(m)
        assert dd == d and D == d
        for s in range(1, M):
            assert wd[s] == 2 * min(s, M - s) + 2 + 4 + 4 * s
        assert vtn.vtn_mpo_norm_bound(m) >= np.abs(np.linalg.eigvalsh(Href)).max()
    finally:
        vtn.vtn_mpo_free(m)


def test_cz_mpo_kappa_zero_and_validation(libvtn):
    w = inputs.workload("plain", 0, M=3, d=3, D=3)
    m0 = vtn.vtn_build_mpo_cz(None, w.r, w.U, 3, 0.0)
    m1 = vtn.vtn_build_mpo(None, w.r, w.U, 3, 3)
    try:
        assert np.abs(_dense_from_abi(m0) - _dense_from_abi(m1)).max() == 0.0
    finally:
        vtn.vtn_mpo_free(m0)
        vtn.vtn_mpo_free(m1)
    with pytest.raises(vtn.VtnError):
        vtn.vtn_build_mpo_cz(None, w.r[:1], w.U[:1, :1], 3, 0.1)          # M = 1
    with pytest.raises(vtn.VtnError):
        vtn.vtn_build_mpo_cz(None, w.r, w.U, 3, float("nan"))


@pytest.mark.parametrize("seed,M,d", [(0, 1, 3), (1, 4, 3), (2, 3, 4)])
def test_mpo_from_cores_round_trip(libvtn, seed, M, d):
    """Cores handed over as dense arrays come back unchanged and contract to the same H."""
    w = inputs.workload("plain", seed, M=M, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    cores = ompo.build_mpo(G, d)
    m = vtn.vtn_mpo_from_cores(None, cores)
    try:
        Mo, do, Do, wd = vtn.vtn_mpo_info(m)
        assert (Mo, do, Do) == (M, d, d)
        assert list(wd) == [1] + [c.shape[1] for c in cores]
        assert np.abs(_dense_from_abi(m) - dense.dense_hamiltonian(G, d).toarray()).max() < 1e-12
        for s in range(M):
            assert np.abs(vtn.vtn_mpo_isometry(m, s) - np.eye(d)).max() == 0.0
        with pytest.raises(vtn.VtnError):
            vtn.vtn_mpo_coefficients(m)
        assert vtn.vtn_mpo_norm_bound(m) == 0.0
    finally:
        vtn.vtn_mpo_free(m)


def test_mpo_from_cores_validation(libvtn):
    w = inputs.workload("plain", 0, M=3, d=3, D=3)
    cores = ompo.build_mpo(gbs.hamiltonian_coefficients(w.r, w.U), 3)
    with pytest.raises(vtn.VtnError):
        vtn.vtn_mpo_from_cores(None, [cores[0], cores[1][:5], cores[2]])  # channels do not chain
    with pytest.raises(vtn.VtnError):
        vtn.vtn_mpo_from_cores(None, cores[1:])                          # first core has w_left > 1
    bad = [c.copy() for c in cores]
    bad[1] = np.zeros(bad[1].shape[:2] + (2, 2), complex)
    with pytest.raises(vtn.VtnError):
        vtn.vtn_mpo_from_cores(None, bad)                                # mixed d


@pytest.mark.parametrize("seed,M", [(0, 2), (1, 6), (2, 9)])
def test_gaussian_bond_spectrum_against_oracle(libvtn, seed, M):
    w = inputs.workload("split", seed, M=M)
    m = vtn.vtn_build_mpo(None, w.r, w.U, 4, 4)
    try:
        V = gbs.covariance(w.r, w.U)
        for cut in range(0, M + 1):
            got = vtn.vtn_gaussian_bond_spectrum(m, cut, 40)
            if cut in (0, M):
                assert got[0] == 1.0 and np.all(got[1:] == 0.0)
                continue
            ref = gbs.gaussian_schmidt_spectrum(V, cut, 40, n_max=60)
            ref = np.concatenate([ref, np.zeros(40 - ref.size)])
            assert np.abs(got - ref).max() <= 1e-11
        # bond dimensions for a discarded weight of at most eps, against the oracle's spectrum
        eps = 1e-3
        dims = vtn.vtn_gaussian_bond_dims(m, eps, 64)
        assert dims[0] == 1 and dims[M] == 1
        for s in range(1, M):
            mu = gbs.gaussian_schmidt_spectrum(V, s, 64, n_max=80)
            cap = min(64, 4 ** s, 4 ** (M - s))
            need = next((k + 1 for k in range(min(cap, mu.size)) if 1 - mu[: k + 1].sum() <= eps), cap)
            assert dims[s] == need
    finally:
        vtn.vtn_mpo_free(m)


def test_gaussian_bond_spectrum_special_cases(libvtn):
    w = inputs.workload("plain", 0, M=4, identity_U=True)
    m = vtn.vtn_build_mpo(None, w.r, w.U, 4, 4)
    try:
        for cut in range(5):
            s = vtn.vtn_gaussian_bond_spectrum(m, cut, 5)
            assert abs(s[0] - 1.0) < 1e-12 and np.abs(s[1:]).max() < 1e-12   # product state
        with pytest.raises(vtn.VtnError):
            vtn.vtn_gaussian_bond_spectrum(m, 5, 3)
    finally:
        vtn.vtn_mpo_free(m)
    w = inputs.workload("plain", 1, M=3, d=3, D=3)
    mcz = vtn.vtn_build_mpo_cz(None, w.r, w.U, 3, 0.2)
    mc = vtn.vtn_mpo_from_cores(None, ompo.build_mpo(gbs.hamiltonian_coefficients(w.r, w.U), 3))
    try:
        for mm in (mcz, mc):
            with pytest.raises(vtn.VtnError) as e:
                vtn.vtn_gaussian_bond_spectrum(mm, 1, 3)
            assert e.value.status == vtn.VTN_EUNSUPPORTED
    finally:
        vtn.vtn_mpo_free(mcz)
        vtn.vtn_mpo_free(mc)


def test_gaussian_bond_spectrum_large_blocks(libvtn):
    """M = 40: cuts whose blocks are 10-, 40- and 60-dimensional (the library works on the
    smaller side of each cut) against the oracle's direct block."""
    w = inputs.workload("large", 3, M=40)
    m = vtn.vtn_build_mpo(None, w.r, w.U, 6, 6)
    try:
        V = gbs.covariance(w.r, w.U)
        for cut in (5, 20, 30):
            got = vtn.vtn_gaussian_bond_spectrum(m, cut, 64)
            ref = gbs.gaussian_schmidt_spectrum(V, cut, 64, n_max=64)
            assert np.abs(got - ref).max() <= 1e-9 * ref[0]
    finally:
        vtn.vtn_mpo_free(m)


@pytest.mark.parametrize("seed,M", [(0, 5), (1, 24)])
def test_warm_features_against_oracle(libvtn, seed, M):
    from oracle import warm
    w = inputs.workload("split", seed, M=M)
    m = vtn.vtn_build_mpo(None, w.r, w.U, 4, 4)
    try:
        f = vtn.vtn_warm_features(m)
        fo = warm.features(gbs.covariance(w.r, w.U))
        assert f.shape == (M, 4) and np.abs(f - fo).max() < 1e-6 * max(1.0, np.abs(fo).max())
    finally:
        vtn.vtn_mpo_free(m)
