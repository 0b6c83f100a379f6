"""Tensor-core (tcgen05) path: the bf16 GEMM kernel and the split-precision (VTN_BF16X3)
effective-Hamiltonian product and sweep, against the oracle / the FP64 path.

Tolerances are derived from the arithmetic: the GEMM accumulates exact bf16 products in
FP32 (relative error <= K * 2^-24 of sum |a||b|); the BF16X3 split drops lo*lo and rounds
each FP64 operand to 16 significant bits (relative error ~2^-16 per product, ~1.5e-5).
"""
import numpy as np
import pytest
import torch

from oracle import dense, dmrg as odmrg, gbs
from paper_2410_18740_gb300 import inputs, vtn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (200, 300, 128), (1000, 520, 640), (1, 1, 64), (129, 257, 192),
                                   (256, 256, 4096), (300, 130, 1024)])
@pytest.mark.parametrize("fp64_out", [False, True])
def test_bf16_gemm_matches_reference(ctx, M, N, K, fp64_out):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), device="cuda", dtype=torch.float64 if fp64_out else torch.float32)
    vtn.vtn_gemm_bf16(ctx, A, B, D)
    torch.cuda.synchronize()
    ref = A.double().cpu().numpy() @ B.double().cpu().numpy().T
    got = D.double().cpu().numpy()
    assert np.isfinite(got).all()
    bound = K * 2.0 ** -24 * (np.abs(A.double().cpu().numpy()) @ np.abs(B.double().cpu().numpy()).T)
    assert np.all(np.abs(got - ref) <= bound + 1e-30)


@pytest.mark.parametrize("chi_l,chi_r,d,ws", [(5, 7, 3, (4, 5, 3)), (37, 70, 4, (6, 8, 5)), (128, 128, 8, (26, 26, 24)),
                                              (1, 4, 2, (1, 3, 4))])
def test_heff_bf16x3_matches_oracle(ctx, chi_l, chi_r, d, ws):
    rng = inputs.rng_for(6000 + chi_l + d)
    wl, wm, wr = ws
    Wi = inputs.random_sparse_core(wl, wm, d, rng)
    Wj = inputs.random_sparse_core(wm, wr, d, rng)
    L = inputs.random_complex((wl, chi_l, chi_l), rng)
    R = inputs.random_complex((wr, chi_r, chi_r), rng)
    th = inputs.random_complex((chi_l, d, d, chi_r), rng)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()
    y = torch.empty(th.shape, dtype=torch.complex128, device="cuda")
    vtn.vtn_heff_apply(ctx, vtn.core_from_sparse(Wi), vtn.core_from_sparse(Wj), chi_l, chi_r, dev(L), dev(R), dev(th),
                       y, prec=vtn.VTN_BF16X3)
    torch.cuda.synchronize()
    expect = odmrg.heff_apply(L, Wi.dense(), Wj.dense(), R, th)
    got = y.cpu().numpy()
    err = np.abs(got - expect).max() / np.abs(expect).max()
    assert err < 2e-4, err
    # the split keeps ~16 significant bits: much better than a single bf16 rounding
    assert np.linalg.norm(got - expect) / np.linalg.norm(expect) < 5e-5


@pytest.mark.parametrize("chi_l,chi_r,d,w", [(5, 7, 3, (4, 5)), (37, 70, 4, (6, 8)), (128, 128, 8, (24, 26)),
                                            (1, 16, 4, (1, 4)), (16, 1, 4, (4, 1))])
def test_env_update_bf16x3_matches_oracle(ctx, chi_l, chi_r, d, w):
    """Split-precision environment updates (both sides) against the oracle's contraction."""
    rng = inputs.rng_for(7000 + chi_l + chi_r)
    wl, wr = w
    W = inputs.random_sparse_core(wl, wr, d, rng)
    A = inputs.random_complex((chi_l, d, chi_r), rng)
    L = inputs.random_complex((wl, chi_l, chi_l), rng)
    R = inputs.random_complex((wr, chi_r, chi_r), rng)
    c = vtn.core_from_sparse(W)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()
    outL = torch.full((wr, chi_r, chi_r), float("nan"), dtype=torch.complex128, device="cuda")
    vtn.vtn_env_update(ctx, c, 0, chi_l, chi_r, dev(L), dev(A), outL, prec=vtn.VTN_BF16X3)
    outR = torch.full((wl, chi_l, chi_l), float("nan"), dtype=torch.complex128, device="cuda")
    vtn.vtn_env_update(ctx, c, 1, chi_l, chi_r, dev(R), dev(A), outR, prec=vtn.VTN_BF16X3)
    torch.cuda.synchronize()
    for got, expect in ((outL.cpu().numpy(), odmrg.env_left(L, A, W.dense())),
                        (outR.cpu().numpy(), odmrg.env_right(R, A, W.dense()))):
        assert np.isfinite(got).all()
        assert np.abs(got - expect).max() / np.abs(expect).max() < 2e-4
        assert np.linalg.norm(got - expect) / np.linalg.norm(expect) < 5e-5


def test_bf16x3_sweep_energy_matches_fp64(ctx):
    """Mixed-precision sweeps reach the FP64 sweep's energy: the energy is evaluated in FP64
    and is quadratic in the state error, so it agrees far below the ~1e-5 product error."""
    w = inputs.workload("split", 3, M=8, d=5, D=5)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, 8, 5)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, 5, 5)
    res = {}
    for prec in (vtn.VTN_FP64, vtn.VTN_BF16X3):
        opts = vtn.vtn_sweep_opts_default(chi_max=24, n_sweeps=4, seed=3, lanczos_tol=1e-7, krylov_max=24,
                                          lanczos_max_restarts=4, prec=prec)
        st, mps, rep = vtn.vtn_sweep(ctx, m, None, opts)
        res[prec] = (rep["energy"], vtn.vtn_marginals_all(ctx, m, mps))
        vtn.vtn_mps_free(mps)
    e64, m64 = res[vtn.VTN_FP64]
    e16, m16 = res[vtn.VTN_BF16X3]
    assert abs(e16[-1] - e64[-1]) <= 1e-6 * max(1.0, abs(e64[-1]))
    assert abs(e16[-1] - e64[-1]) <= 1e-8 * Hn
    assert np.abs(m16 - m64).max() < 1e-4
    vtn.vtn_mpo_free(m)


@pytest.mark.parametrize("M,d,chi,seed", [(6, 3, 27, 11), (8, 3, 81, 12)])
def test_bf16x3_converges_to_the_fp64_energy(ctx, M, d, chi, seed):
    """Converged sweeps at a bond dimension that truncates nothing (chi = d^(M/2)): the FP64 and
    the split-precision solver both reach the ground energy of P H P, and agree with each other
    within 1e-8 relative -- the bar set for mixed against FP64.  The energy of each sweep is the
    full FP64 contraction; the split-precision state is only first-order wrong (~1e-5), so its
    energy is second-order close.  Also checked against the dense ground energy (oracle)."""
    w = inputs.workload("split", seed, M=M, d=d, D=d)
    G = gbs.hamiltonian_coefficients(w.r, w.U)
    Hn = gbs.norm_bound(G, M, d)
    e0 = dense.ground_state(G, d)[0][0]
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, d, d)
    res = {}
    for prec in (vtn.VTN_FP64, vtn.VTN_BF16X3):
        opts = vtn.vtn_sweep_opts_default(chi_max=chi, n_sweeps=10, seed=seed, lanczos_tol=1e-12, krylov_max=32,
                                          lanczos_max_restarts=4, prec=prec, e_tol=1e-13 * Hn)
        st, mps, rep = vtn.vtn_sweep(ctx, m, None, opts)
        res[prec] = rep["energy"][-1]
        vtn.vtn_mps_free(mps)
    e64, e16 = res[vtn.VTN_FP64], res[vtn.VTN_BF16X3]
    assert abs(e64 - e0) <= 1e-10 * Hn
    assert abs(e16 - e64) <= 1e-8 * abs(e64)
    assert abs(e16 - e0) <= 1e-8 * abs(e0)
    vtn.vtn_mpo_free(m)
