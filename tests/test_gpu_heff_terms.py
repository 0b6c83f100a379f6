"""Split-precision H_eff psi in the term form (the MPO cores folded into the environments once per
bond) against the oracle, on the library's own GBS cores, and whole sweeps in the term form
against the channel-mixing form and FP64.

Bars: the split-precision bars of the tensor-core tests (2e-4 of the largest magnitude, 5e-5 in
norm) for single products; sweep energies from the same state agree between the two forms to the
precision of the split products (1e-6 relative), and with FP64 as in the mixed-precision tests.
"""
import numpy as np
import pytest
import torch

from oracle import dmrg as odmrg
from paper_2410_18740_gb300 import inputs, vtn

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def _cores(m, s):
    out = []
    for site in (s, s + 1):
        wl, wr, rows, cols, ops = vtn.vtn_mpo_core(m, site)
        sc = inputs.SparseCore(wl, wr, vtn.vtn_mpo_info(m)[1], rows, cols, ops)
        out.append((sc, vtn.core_from_sparse(sc)))
    return out


@pytest.mark.parametrize("bond,chi_l,chi_r", [
    (49, 37, 70),     # centre bond (the collapse core on the right), ragged tiles
    (50, 64, 64),     # the collapse core on the left
    (40, 1, 48),      # one left bond state
    (60, 40, 1),      # one right bond state
    (49, 96, 80),
])
def test_term_form_heff_matches_oracle(ctx, bond, chi_l, chi_r):
    """Bonds of the large workload (optimal local basis, d = 6, w ~ 80-102): the term form is used."""
    w = inputs.workload("large", 200)
    m = vtn.vtn_build_mpo(None, w.r, w.U, w.D, w.d)
    assert vtn.vtn_mpo_bond_terms(m, bond)["used"]
    (Wi_s, Wi), (Wj_s, Wj) = _cores(m, bond)
    d = Wi_s.d
    rng = inputs.rng_for(9100 + bond + chi_l)
    L = inputs.random_complex((Wi_s.w_left, chi_l, chi_l), rng)
    R = inputs.random_complex((Wj_s.w_right, chi_r, chi_r), rng)
    th = inputs.random_complex((chi_l, d, d, chi_r), rng)
    y = torch.full(th.shape, float("nan"), dtype=torch.complex128, device="cuda")
    vtn.vtn_heff_apply(ctx, Wi, Wj, chi_l, chi_r, dev(L), dev(R), dev(th), y, prec=vtn.VTN_BF16X3)
    got = y.cpu().numpy()
    ref = odmrg.heff_apply(L, Wi_s.dense(), Wj_s.dense(), R, th)
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() / np.abs(ref).max() < 2e-4
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 5e-5
    vtn.vtn_mpo_free(m)


def test_term_form_sweeps_match_mixing_form_and_fp64(ctx):
    """Four sweeps from the same seeded start in each H_eff form (split precision; heff_form 2
    forces the term form at every bond) and in FP64 (M = 8, d = 6 in the optimal local basis, chi
    to 36), Lanczos residual 1e-6 (the split products' resolution).  The trajectories differ by
    rounding: within 2e-5 relative at every sweep, 5e-6 at the last."""
    w = inputs.workload("split", 31, M=8, D=10, d=6)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, w.D, w.d)
    assert all(vtn.vtn_mpo_bond_terms(m, b) is not None for b in range(7))
    res = {}
    for key, prec, form in (("terms", vtn.VTN_BF16X3, 2), ("mixing", vtn.VTN_BF16X3, 1), ("fp64", vtn.VTN_FP64, 0)):
        opts = vtn.vtn_sweep_opts_default(chi_max=36, n_sweeps=4, seed=5, lanczos_tol=1e-6, krylov_max=24,
                                          lanczos_max_restarts=2, chi_schedule=[12, 36], prec=prec, heff_form=form)
        st, mps, rep = vtn.vtn_sweep(ctx, m, None, opts)
        assert st in (vtn.VTN_OK, vtn.VTN_ENOCONV)
        res[key] = np.array(rep["energy"])
        vtn.vtn_mps_free(mps)
    assert np.all(np.isfinite(res["terms"]))
    for other in ("mixing", "fp64"):
        rel = np.abs(res["terms"] - res[other]) / np.abs(res["fp64"])
        assert rel.max() <= 2e-5 and rel[-1] <= 5e-6, (other, rel)
    vtn.vtn_mpo_free(m)


def test_fp64_environments_in_split_precision(ctx):
    """env_fp64 = 1: split-precision H_eff psi with FP64 environment updates; four sweeps from the
    same start agree with FP64 sweeps as the all-split run does (M = 8, d = 6, chi to 36)."""
    w = inputs.workload("split", 31, M=8, D=10, d=6)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, w.D, w.d)
    res = {}
    for key, prec, env64 in (("env64", vtn.VTN_BF16X3, 1), ("fp64", vtn.VTN_FP64, 0)):
        opts = vtn.vtn_sweep_opts_default(chi_max=36, n_sweeps=4, seed=5, lanczos_tol=1e-6, krylov_max=24,
                                          lanczos_max_restarts=2, chi_schedule=[12, 36], prec=prec, env_fp64=env64)
        st, mps, rep = vtn.vtn_sweep(ctx, m, None, opts)
        assert st in (vtn.VTN_OK, vtn.VTN_ENOCONV)
        res[key] = np.array(rep["energy"])
        vtn.vtn_mps_free(mps)
    rel = np.abs(res["env64"] - res["fp64"]) / np.abs(res["fp64"])
    assert rel.max() <= 2e-5 and rel[-1] <= 5e-6, rel
    vtn.vtn_mpo_free(m)
