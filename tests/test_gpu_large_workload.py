"""GPU parity at the large workload's full shapes (M = 100, r ~ U(0.8, 1.2), Haar U, D = 24 ->
d = 6 in the optimal local basis, chi = 512).

At the middle bond one H_eff psi product is 7.7e12 flops and its GEMM intermediates hold about
2e9 elements, so these checks exercise the index ranges that the smaller shapes never reach.
The oracle cannot form the full product in seconds; it computes sampled outputs instead: a
few output columns l of Y (``heff_apply_columns``, the same sum restricted to those columns)
and a few output channels b of the environment updates (the oracle's ``env_left`` /
``env_right`` with the MPO core restricted to those channels).  The cores are the library's
own MPO cores at the middle of the chain; L, R and theta are seeded random tensors.
Bars: FP64 relative 1e-12 of the largest sampled magnitude (the kernel tests' bar); BF16X3
the split-precision bars of the tensor-core tests (2e-4 of the largest magnitude, 5e-5 in norm).
"""
import numpy as np
import pytest
import torch

from oracle import dmrg as odmrg
from paper_2410_18740_gb300 import inputs, vtn

pytestmark = pytest.mark.gpu

CHI, D_LOC, MID = 512, 6, 49


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


@pytest.fixture(scope="module")
def large_cores(ctx):
    w = inputs.workload("large", 200)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, w.D, w.d)
    out = {}
    for s in (MID - 1, MID, MID + 1):
        wl, wr, rows, cols, ops = vtn.vtn_mpo_core(m, s)
        sc = inputs.SparseCore(wl, wr, D_LOC, rows, cols, ops)
        out[s] = (sc, vtn.core_from_sparse(sc))
    vtn.vtn_mpo_free(m)
    return out


def _rel_max(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _rel_norm(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_heff_middle_bond_sampled_columns(ctx, large_cores, prec):
    Wi_s, Wi = large_cores[MID]
    Wj_s, Wj = large_cores[MID + 1]
    assert (Wi_s.w_left, Wj_s.w_right) == (100, 100)
    rng = inputs.rng_for(4242)
    L = inputs.random_complex((Wi_s.w_left, CHI, CHI), rng)
    R = inputs.random_complex((Wj_s.w_right, CHI, CHI), rng)
    th = inputs.random_complex((CHI, D_LOC, D_LOC, CHI), rng)
    y = torch.empty(th.shape, dtype=torch.complex128, device="cuda")
    p = vtn.VTN_FP64 if prec == "fp64" else vtn.VTN_BF16X3
    vtn.vtn_heff_apply(ctx, Wi, Wj, CHI, CHI, dev(L), dev(R), dev(th), y, prec=p)
    cols = [0, 257, 511]
    got = y[..., cols].cpu().numpy()
    ref = odmrg.heff_apply_columns(L, Wi_s.dense(), Wj_s.dense(), R, th, cols)
    assert np.isfinite(got).all()
    if prec == "fp64":
        assert _rel_max(got, ref) <= 1e-12
    else:
        assert _rel_max(got, ref) <= 2e-4
        assert _rel_norm(got, ref) <= 5e-5


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("side", [0, 1])
def test_env_update_middle_sampled_channels(ctx, large_cores, prec, side):
    W_s, W = large_cores[MID]
    rng = inputs.rng_for(4343 + side)
    A = inputs.random_complex((CHI, D_LOC, CHI), rng)
    p = vtn.VTN_FP64 if prec == "fp64" else vtn.VTN_BF16X3
    if side == 0:
        env = inputs.random_complex((W_s.w_left, CHI, CHI), rng)
        out = torch.empty((W_s.w_right, CHI, CHI), dtype=torch.complex128, device="cuda")
        chans = [0, 1, 37, W_s.w_right - 1]
        vtn.vtn_env_update(ctx, W, 0, CHI, CHI, dev(env), dev(A), out, prec=p)
        ref = odmrg.env_left(env, A, W_s.dense()[:, chans])
    else:
        env = inputs.random_complex((W_s.w_right, CHI, CHI), rng)
        out = torch.empty((W_s.w_left, CHI, CHI), dtype=torch.complex128, device="cuda")
        chans = [0, 1, 50, W_s.w_left - 1]
        vtn.vtn_env_update(ctx, W, 1, CHI, CHI, dev(env), dev(A), out, prec=p)
        ref = odmrg.env_right(env, A, W_s.dense()[chans, :])
    got = out[chans].cpu().numpy()
    assert np.isfinite(got).all()
    if prec == "fp64":
        assert _rel_max(got, ref) <= 1e-12
    else:
        assert _rel_max(got, ref) <= 2e-4
        assert _rel_norm(got, ref) <= 5e-5


def test_windowed_sweep_at_full_size(ctx):
    """One windowed sweep over the two middle bonds of the full large workload in split precision,
    from a seeded random state centred at site 49: it runs through the C ABI, keeps the bond
    dimension 512, returns isometries around the centre, and reports finite, non-negative
    centre Rayleigh quotients (P H P is positive semi-definite) that do not grow from the
    first sweep to the second beyond the truncation's effect."""
    w = inputs.workload("large", 200)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, w.D, w.d)
    mps = vtn.vtn_mps_random_center(ctx, m, CHI, 17, MID)
    opts = vtn.vtn_sweep_opts_default(chi_max=CHI, n_sweeps=2, prec=vtn.VTN_BF16X3, lanczos_tol=1e-12, krylov_max=8,
                                      lanczos_max_restarts=0, window_lo=MID, window_hi=MID + 2)
    st, mps, rep = vtn.vtn_sweep(ctx, m, mps, opts)
    assert st in (vtn.VTN_OK, vtn.VTN_ENOCONV)
    assert vtn.vtn_mps_get_center(mps) == MID
    _, _, dims = vtn.vtn_mps_info(mps)
    assert dims[MID] == dims[MID + 1] == dims[MID + 2] == CHI
    e = rep["energy"]
    assert np.isfinite(e).all() and min(e) >= -1e-6 * max(e)
    assert e[1] <= 1.01 * e[0]
    for s in (MID + 1, MID + 2):
        A = vtn.vtn_mps_get_site(ctx, mps, s).reshape(CHI, -1)
        assert np.abs(A @ A.conj().T - np.eye(CHI)).max() < 1e-12
    A = vtn.vtn_mps_get_site(ctx, mps, MID - 1).reshape(-1, CHI)
    assert np.abs(A.conj().T @ A - np.eye(CHI)).max() < 1e-12
    # read-out at this size: the Fock marginal of a middle mode (the optimal local basis rotated
    # back to D = 24 levels; the tail above D is lost, so the sum is at most one) and samples
    # (chi (D + 1) complex values of working set per sample: the largest the sampler takes)
    P = vtn.vtn_marginals(ctx, m, mps, [MID])
    assert np.isfinite(P).all() and P.min() >= -1e-12 and P.sum() <= 1 + 1e-9
    smp = vtn.vtn_sample(ctx, m, mps, 5, 16)
    assert smp.shape == (16, 100) and smp.min() >= 0 and smp.max() < 24
    vtn.vtn_mps_free(mps)
    vtn.vtn_mpo_free(m)


def test_shorter_accumulation_runs_are_more_accurate(ctx, large_cores):
    """The tensor cores' FP32 accumulation loses accuracy with the length of the sum: the left
    environment update at the middle of the large workload (K = 6 chi d = 18432 split terms per
    output) with 4 k-blocks per accumulator is closer to the oracle than with 256, and both meet
    the split-precision bars."""
    W_s, W = large_cores[MID]
    rng = inputs.rng_for(4545)
    A = inputs.random_complex((CHI, D_LOC, CHI), rng)
    env = inputs.random_complex((W_s.w_left, CHI, CHI), rng)
    chans = [0, 1, 37, W_s.w_right - 1]
    ref = odmrg.env_left(env, A, W_s.dense()[:, chans])
    errs = {}
    for kb in (256, 4):
        vtn.vtn_set_tc_accumulation(ctx, kb, 256)
        out = torch.empty((W_s.w_right, CHI, CHI), dtype=torch.complex128, device="cuda")
        vtn.vtn_env_update(ctx, W, 0, CHI, CHI, dev(env), dev(A), out, prec=vtn.VTN_BF16X3)
        got = out[chans].cpu().numpy()
        errs[kb] = _rel_norm(got, ref)
        assert _rel_max(got, ref) <= 2e-4 and errs[kb] <= 5e-5
    vtn.vtn_set_tc_accumulation(ctx)
    assert errs[4] < errs[256], errs
