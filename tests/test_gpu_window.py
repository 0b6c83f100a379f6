"""GPU parity of windowed sweeps and orthogonality-centre handling against the oracle.

A windowed sweep optimises bonds lo .. hi-1 and back on a state centred at site lo, and
reports the Rayleigh quotient of its final centre; the oracle runs the same window on the
same state (``dmrg.dmrg(window=...)``).  Bars: the FP64 bar of the solver tests
(|dE| <= 1e-10 ||H||) and the split-precision bar of the tensor-core tests for BF16X3.
"""
import numpy as np
import pytest

from oracle import dmrg as odmrg, gbs, mpo as ompo
from paper_2410_18740_gb300 import inputs, vtn

pytestmark = pytest.mark.gpu


def gpu_sites(ctx, mps):
    M, _, _ = vtn.vtn_mps_info(mps)
    return [vtn.vtn_mps_get_site(ctx, mps, s) for s in range(M)]


def dense_vector(sites):
    v = sites[0]
    for A in sites[1:]:
        v = np.einsum("...a,asb->...sb", v, A)
    return v.reshape(-1)


@pytest.mark.parametrize("M,d,chi,center", [(5, 3, 7, 2), (8, 6, 512, 4), (6, 4, 16, 5)])
def test_random_center_matches_oracle(ctx, M, d, chi, center):
    w = inputs.workload("plain", 0, M=M, d=d, D=d)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, d, d)
    mps = vtn.vtn_mps_random_center(ctx, m, chi, 31, center)
    assert vtn.vtn_mps_get_center(mps) == center
    osites = odmrg.initial_mps(M, d, chi, seed=31, center=center)
    for a, b in zip(gpu_sites(ctx, mps), osites):
        assert a.shape == b.shape
        assert np.abs(a - b).max() < 1e-13
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_move_center_keeps_the_state(ctx):
    w = inputs.workload("plain", 0, M=6, d=3, D=3)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, 3, 3)
    mps = vtn.vtn_mps_random_center(ctx, m, 9, 5, 1)
    v0 = dense_vector(gpu_sites(ctx, mps))
    for dst in (4, 0, 3):
        vtn.vtn_mps_move_center(ctx, mps, dst)
        assert vtn.vtn_mps_get_center(mps) == dst
        sites = gpu_sites(ctx, mps)
        assert np.abs(dense_vector(sites) - v0).max() < 1e-12
        for s, A in enumerate(sites):
            if s < dst:
                Am = A.reshape(-1, A.shape[2])
                assert np.abs(Am.conj().T @ Am - np.eye(A.shape[2])).max() < 1e-12
            elif s > dst:
                Am = A.reshape(A.shape[0], -1)
                assert np.abs(Am @ Am.conj().T - np.eye(A.shape[0])).max() < 1e-12
    # unknown centre (host tensors): brought to the requested centre from scratch
    h = vtn.vtn_mps_from_host(ctx, m, odmrg.initial_mps(6, 3, 9, seed=5, center=1))
    assert vtn.vtn_mps_get_center(h) == -1
    vtn.vtn_mps_move_center(ctx, h, 2)
    assert vtn.vtn_mps_get_center(h) == 2
    assert np.abs(dense_vector(gpu_sites(ctx, h)) - v0).max() < 1e-12
    vtn.vtn_mps_free(h)
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


@pytest.mark.parametrize("window", [(2, 5), (0, 7), (3, 4)])
def test_windowed_sweep_matches_oracle(ctx, window):
    """FP64 windowed sweeps from the same centred state, energy by energy."""
    lo, hi = window
    M, d, chi = 8, 3, 20
    w = inputs.workload("split", 3, M=M, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, M, d)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, d, d)
    start = odmrg.initial_mps(M, d, chi, seed=8, center=lo)
    mps = vtn.vtn_mps_random_center(ctx, m, chi, 8, lo)
    opts = vtn.vtn_sweep_opts_default(chi_max=chi, n_sweeps=3, lanczos_tol=1e-12, krylov_max=32,
                                      lanczos_max_restarts=8, window_lo=lo, window_hi=hi)
    st, mps, rep = vtn.vtn_sweep(ctx, m, mps, opts)
    assert st == vtn.VTN_OK
    assert vtn.vtn_mps_get_center(mps) == lo
    cores = ompo.build_mpo(G, d)
    omps, orep = odmrg.dmrg(cores, d, chi, 3, seed=8, mps=start, window=window,
                            lanczos=odmrg.LanczosParams(krylov_max=32, max_restarts=8, tol=1e-12))
    assert rep["sweeps_done"] == 3
    for a, b in zip(rep["energy"], orep.energies):
        assert abs(a - b) <= 1e-10 * Hn
    # the reported centre energy is <psi|H|psi>/<psi|psi> of the returned state
    assert abs(vtn.vtn_energy(ctx, m, mps) - rep["energy"][-1]) <= 1e-10 * Hn
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_windowed_sweep_moves_the_centre_first(ctx):
    """A right-canonical start (centre 0) with a window at bond 3: the library moves the centre
    by exact splits, so the trajectory is the oracle's on the moved state (energies are
    gauge-invariant)."""
    M, d, chi, lo, hi = 7, 3, 12, 3, 5
    w = inputs.workload("split", 4, M=M, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, M, d)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, d, d)
    mps = vtn.vtn_mps_random(ctx, m, chi, 9)
    opts = vtn.vtn_sweep_opts_default(chi_max=chi, n_sweeps=2, lanczos_tol=1e-12, krylov_max=32,
                                      lanczos_max_restarts=8, window_lo=lo, window_hi=hi)
    st, mps, rep = vtn.vtn_sweep(ctx, m, mps, opts)
    assert st == vtn.VTN_OK
    start = odmrg.move_center(odmrg.initial_mps(M, d, chi, seed=9), 0, lo)
    cores = ompo.build_mpo(G, d)
    _, orep = odmrg.dmrg(cores, d, chi, 2, seed=9, mps=start, window=(lo, hi),
                         lanczos=odmrg.LanczosParams(krylov_max=32, max_restarts=8, tol=1e-12))
    for a, b in zip(rep["energy"], orep.energies):
        assert abs(a - b) <= 1e-10 * Hn
    # a full sweep afterwards starts from centre 0 again
    opts2 = vtn.vtn_sweep_opts_default(chi_max=chi, n_sweeps=1, lanczos_tol=1e-12, krylov_max=32,
                                       lanczos_max_restarts=8)
    st, mps, rep2 = vtn.vtn_sweep(ctx, m, mps, opts2)
    assert vtn.vtn_mps_get_center(mps) == 0
    assert rep2["energy"][0] <= rep["energy"][-1] + 1e-10 * Hn
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_windowed_sweep_bf16x3_against_fp64(ctx):
    """The split-precision window from the same state: the FP64 energy of the state it reaches
    agrees with the FP64 window's within the split-precision bar of the sweep tests; its own
    centre Rayleigh quotients (split-precision H_eff) agree with that FP64 energy to the
    per-product error of the split."""
    M, d, chi, lo, hi = 8, 4, 32, 3, 5
    w = inputs.workload("split", 5, M=M, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, M, d)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, d, d)
    out = {}
    for prec in (vtn.VTN_FP64, vtn.VTN_BF16X3):
        mps = vtn.vtn_mps_random_center(ctx, m, chi, 12, lo)
        opts = vtn.vtn_sweep_opts_default(chi_max=chi, n_sweeps=3, lanczos_tol=1e-10, krylov_max=32,
                                          lanczos_max_restarts=4, window_lo=lo, window_hi=hi, prec=prec)
        st, mps, rep = vtn.vtn_sweep(ctx, m, mps, opts)
        out[prec] = (rep["energy"][-1], vtn.vtn_energy(ctx, m, mps))
        vtn.vtn_mps_free(mps)
    e64 = out[vtn.VTN_FP64][1]
    assert abs(out[vtn.VTN_FP64][0] - e64) <= 1e-10 * Hn
    assert abs(out[vtn.VTN_BF16X3][1] - e64) <= 1e-6 * abs(e64) + 1e-8 * Hn
    assert abs(out[vtn.VTN_BF16X3][0] - out[vtn.VTN_BF16X3][1]) <= 1e-4 * abs(e64)
    vtn.vtn_mpo_free(m)


def test_window_validation(ctx):
    w = inputs.workload("plain", 0, M=4, d=3, D=3)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, 3, 3)
    mps = vtn.vtn_mps_random(ctx, m, 4, 1)
    for lo, hi in [(-1, 2), (1, 4), (2, 9)]:
        opts = vtn.vtn_sweep_opts_default(chi_max=4, n_sweeps=1, window_lo=lo, window_hi=hi)
        with pytest.raises(vtn.VtnError) as e:
            vtn.vtn_sweep(ctx, m, mps, opts)
        assert e.value.status == vtn.VTN_EINVAL
    with pytest.raises(vtn.VtnError):
        vtn.vtn_mps_set_center(mps, 4)
    vtn.vtn_mps_set_center(mps, -1)
    assert vtn.vtn_mps_get_center(mps) == -1
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_sweep_without_restarts_waits_for_the_gpu_once_per_sweep(ctx):
    """Lanczos without restarts and the exact truncation: the Krylov steps stop on a device flag
    and the truncation results are staged, so a sweep synchronises with the GPU once (its
    energy) plus the end-of-call checks -- none per bond -- and still follows the oracle's
    trajectory with the same Lanczos settings (12 Krylov vectors, no restart)."""
    lo, hi, M, d, chi = 2, 6, 9, 3, 20
    w = inputs.workload("split", 6, M=M, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, M, d)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, d, d)
    lp = dict(lanczos_tol=1e-12, krylov_max=12, lanczos_max_restarts=0)
    for window, n_sw in (((lo, hi), 3), ((0, M - 1), 2)):
        kw = dict(window_lo=window[0], window_hi=window[1]) if window != (0, M - 1) else {}
        start = vtn.vtn_mps_random_center(ctx, m, chi, 14, window[0])
        opts = vtn.vtn_sweep_opts_default(chi_max=chi, n_sweeps=n_sw, **lp, **kw)
        st, start, rep0 = vtn.vtn_sweep(ctx, m, start, opts)          # sizes every workspace
        vtn.vtn_mps_free(start)
        mps = vtn.vtn_mps_random_center(ctx, m, chi, 14, window[0])
        st, mps, rep = vtn.vtn_sweep(ctx, m, mps, opts)
        assert rep["energy"] == rep0["energy"]
        # a windowed sweep reads its centre energy once; the full contraction of a full sweep twice
        # (energy and norm); per-bond round trips would be (bonds) x (Krylov steps + 1)
        bound = n_sw + 3 if window != (0, M - 1) else 2 * n_sw + 4
        assert rep["host_syncs"] <= bound, rep["host_syncs"]
        cores = ompo.build_mpo(G, d)
        _, orep = odmrg.dmrg(cores, d, chi, n_sw, seed=14, mps=odmrg.initial_mps(M, d, chi, seed=14, center=window[0]),
                             window=None if window == (0, M - 1) else window,
                             lanczos=odmrg.LanczosParams(krylov_max=12, max_restarts=0, tol=1e-12))
        for a, b in zip(rep["energy"], orep.energies):
            assert abs(a - b) <= 1e-10 * Hn
        vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)
