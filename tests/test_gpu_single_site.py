"""GPU parity of single-site DMRG with subspace expansion against the CPU oracle.

Kernel level: the single-site H_eff product and both expansions on seeded random tensors
and random block-sparse cores (FP64, relative 1e-12 of the largest output).  Solver level:
the same initial MPS (Philox), the same Lanczos rule, expansion weights, truncation and
cutoff rules on the oracle's own MPO (handed to the library as cores, because the expansion
depends on the MPO representation), energies after every sweep within 1e-9 ||H||; and, on
the library's own MPO, convergence from a product state to the dense ground state.
"""
import numpy as np
import pytest
import torch

from oracle import dense, dmrg as odmrg, dmrg1 as odmrg1, gbs, mpo as ompo
from paper_2410_18740_gb300 import inputs, vtn

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def close(a, b, rel=1e-12):
    scale = max(np.abs(b).max(), 1e-300)
    err = np.abs(a - b).max() / scale
    assert err <= rel, f"relative error {err:.3e} > {rel:.1e}"


CASES = [
    # chi_l, chi_r, d, (w_l, w_r)
    (128, 128, 8, (26, 24)),   # middle bond of the split workload
    (1, 4, 2, (1, 4)),
    (4, 1, 3, (4, 1)),
    (5, 7, 3, (4, 5)),
    (37, 70, 4, (6, 9)),
    (130, 65, 2, (3, 7)),
    (16, 16, 16, (3, 3)),
]


@pytest.mark.parametrize("chi_l,chi_r,d,ws", CASES)
def test_heff1_apply_matches_oracle(ctx, chi_l, chi_r, d, ws):
    rng = inputs.rng_for(5000 + chi_l + 7 * chi_r + d)
    W = inputs.random_sparse_core(ws[0], ws[1], d, rng)
    L = inputs.random_complex((ws[0], chi_l, chi_l), rng)
    R = inputs.random_complex((ws[1], chi_r, chi_r), rng)
    A = inputs.random_complex((chi_l, d, chi_r), rng)
    y = torch.empty(A.shape, dtype=torch.complex128, device="cuda")
    vtn.vtn_heff1_apply(ctx, vtn.core_from_sparse(W), chi_l, chi_r, dev(L), dev(R), dev(A), y)
    close(host(y), odmrg1.heff1_apply(L, W.dense(), R, A))


@pytest.mark.parametrize("chi_l,chi_r,d,ws", CASES)
def test_expansion_matches_oracle(ctx, chi_l, chi_r, d, ws):
    rng = inputs.rng_for(6000 + chi_l + 7 * chi_r + d)
    wl, wr = ws
    W = inputs.random_sparse_core(wl, wr, d, rng)
    c = vtn.core_from_sparse(W)
    L = inputs.random_complex((wl, chi_l, chi_l), rng)
    R = inputs.random_complex((wr, chi_r, chi_r), rng)
    A = inputs.random_complex((chi_l, d, chi_r), rng)
    alpha = 0.0625 + rng.uniform()
    out = torch.empty((chi_l * d, chi_r * (1 + wr)), dtype=torch.complex128, device="cuda")
    vtn.vtn_expand(ctx, c, 0, chi_l, chi_r, dev(L), dev(A), alpha, out)
    close(host(out), odmrg1.expand_right(L, W.dense(), A, alpha))
    out = torch.empty((chi_l * (1 + wl), d * chi_r), dtype=torch.complex128, device="cuda")
    vtn.vtn_expand(ctx, c, 1, chi_l, chi_r, dev(R), dev(A), alpha, out)
    close(host(out), odmrg1.expand_left(R, W.dense(), A, alpha))


def _opts(chi, n_sweeps, seed):
    return vtn.vtn_sweep_opts_default(chi_max=chi, n_sweeps=n_sweeps, seed=seed, lanczos_tol=1e-12,
                                      krylov_max=32, lanczos_max_restarts=8)


@pytest.mark.parametrize("seed,M,d,chi,chi0,n_sweeps,alpha", [
    (0, 5, 3, 9, 1, 3, 0.1),
    (1, 6, 3, 6, 2, 3, 0.05),
    (2, 4, 4, 16, 1, 3, 0.2),
])
def test_single_site_trajectory_matches_oracle(ctx, seed, M, d, chi, chi0, n_sweeps, alpha):
    w = inputs.workload("split", seed, M=M, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, M, d)
    cores = ompo.build_mpo(G, d)
    m = vtn.vtn_mpo_from_cores(ctx, cores)
    mps0 = vtn.vtn_mps_random(ctx, m, chi0, seed=seed + 3)
    st, mps, rep = vtn.vtn_sweep_single_site(ctx, m, mps0, _opts(chi, n_sweeps, seed + 3), alpha=alpha,
                                             alpha_decay=0.5, cutoff=1e-12)
    omps, orep = odmrg1.dmrg1(cores, d, chi, n_sweeps, seed=seed + 3, chi0=chi0, alpha=alpha,
                              alpha_decay=0.5, cutoff=1e-12,
                              lanczos=odmrg.LanczosParams(krylov_max=32, max_restarts=8, tol=1e-12))
    assert rep["sweeps_done"] == n_sweeps
    for a, b in zip(rep["energy"], orep.energies):
        assert abs(a - b) <= 1e-9 * Hn
    _, _, dims = vtn.vtn_mps_info(mps)
    assert list(dims) == orep.dims[-1]
    # the GPU state evaluated by the oracle
    sites = [vtn.vtn_mps_get_site(ctx, mps, s) for s in range(M)]
    assert abs(odmrg.energy(sites, cores) - rep["energy"][-1]) <= 1e-12 * Hn
    # canonical form: sites 1.. right-canonical
    for B in sites[1:]:
        Bm = B.reshape(B.shape[0], -1)
        assert np.abs(Bm @ Bm.conj().T - np.eye(B.shape[0])).max() < 1e-10
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


@pytest.mark.parametrize("seed", [0, 1])
def test_single_site_reaches_dense_ground_state_from_product_state(ctx, seed):
    """Library MPO, plain workload (M = 4, d = 4, chi = 16 exact), start at bond dimension 1."""
    w = inputs.workload("plain", seed)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, w.M, w.d)
    e0 = dense.ground_state(G, w.d)[0][0]
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, w.D, w.d)
    mps0 = vtn.vtn_mps_random(ctx, m, 1, seed=seed + 40)
    st, mps, rep = vtn.vtn_sweep_single_site(ctx, m, mps0, _opts(16, 8, 0), alpha=0.1, alpha_decay=0.5)
    assert abs(rep["energy"][rep["sweeps_done"] - 1] - e0) <= 1e-9 * Hn
    assert min(rep["energy"][: rep["sweeps_done"]]) >= e0 - 1e-10 * Hn
    _, _, dims = vtn.vtn_mps_info(mps)
    assert list(dims) == [1, 4, 16, 4, 1]
    vtn.vtn_mps_free(mps)
    # without the expansion the bonds stay at 1
    mps0 = vtn.vtn_mps_random(ctx, m, 1, seed=seed + 40)
    st, mps, rep = vtn.vtn_sweep_single_site(ctx, m, mps0, _opts(16, 2, 0), alpha=0.0)
    _, _, dims = vtn.vtn_mps_info(mps)
    assert list(dims) == [1, 1, 1, 1, 1]
    assert rep["energy"][1] > e0 + 1e-6
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_single_site_single_mode_and_errors(ctx):
    w = inputs.workload("plain", 3, M=1, d=6, D=6)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    e0 = dense.ground_state(G, 6)[0][0]
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, 6, 6)
    st, mps, rep = vtn.vtn_sweep_single_site(ctx, m, None, vtn.vtn_sweep_opts_default(
        chi_max=4, n_sweeps=1, seed=1, lanczos_tol=1e-13))
    assert abs(rep["energy"][0] - e0) <= 1e-11
    vtn.vtn_mps_free(mps)
    opts = vtn.vtn_sweep_opts_default(chi_max=4, n_sweeps=1)
    opts.prec = vtn.VTN_BF16X3
    with pytest.raises(vtn.VtnError) as e:
        vtn.vtn_sweep_single_site(ctx, m, None, opts)
    assert e.value.status == vtn.VTN_EUNSUPPORTED
    for kw in ({"alpha": -1.0}, {"alpha_decay": float("nan")}, {"cutoff": 1.0}):
        with pytest.raises(vtn.VtnError) as e:
            vtn.vtn_sweep_single_site(ctx, m, None, vtn.vtn_sweep_opts_default(chi_max=4, n_sweeps=1), **kw)
        assert e.value.status == vtn.VTN_EINVAL
    vtn.vtn_mpo_free(m)
