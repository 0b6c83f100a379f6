"""GPU parity of single solver steps against the CPU oracle, through the C ABI.

Inputs are seeded random tensors and random block-sparse MPO cores (same structure as
the GBS MPO: scaled identities plus dense blocks); the oracle evaluates the same
definitions with numpy einsum / eigh.  Sizes span several 64 x 64 GEMM tiles with
ragged tails, down to degenerate bond dimension 1.  FP64 tolerance: relative 1e-12 of
the largest output magnitude (rounding of sums of O(1e4) terms).
"""
import numpy as np
import pytest
import torch

from oracle import dmrg as odmrg
from paper_2410_18740_gb300 import inputs, vtn

pytestmark = pytest.mark.gpu

REL = 1e-12


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def close(a, b, rel=REL):
    scale = max(np.abs(b).max(), 1e-300)
    err = np.abs(a - b).max() / scale
    assert err <= rel, f"relative error {err:.3e} > {rel:.1e}"


HEFF_CASES = [
    # chi_l, chi_r, d, (w_l, w_m, w_r)
    (128, 128, 8, (26, 26, 24)),   # shape of the middle bond of the split workload
    (1, 4, 2, (1, 3, 4)),
    (4, 1, 3, (4, 3, 1)),
    (5, 7, 3, (4, 5, 3)),
    (37, 70, 4, (6, 8, 5)),
    (64, 64, 8, (10, 10, 10)),
    (130, 65, 2, (3, 7, 2)),
    (16, 16, 16, (3, 3, 3)),
]


@pytest.mark.parametrize("chi_l,chi_r,d,ws", HEFF_CASES)
def test_heff_apply_matches_oracle(ctx, chi_l, chi_r, d, ws):
    rng = inputs.rng_for(1000 + chi_l + 7 * chi_r + d)
    wl, wm, wr = ws
    Wi = inputs.random_sparse_core(wl, wm, d, rng)
    Wj = inputs.random_sparse_core(wm, wr, d, rng)
    L = inputs.random_complex((wl, chi_l, chi_l), rng)
    R = inputs.random_complex((wr, chi_r, chi_r), rng)
    th = inputs.random_complex((chi_l, d, d, chi_r), rng)
    y = torch.empty(th.shape, dtype=torch.complex128, device="cuda")
    vtn.vtn_heff_apply(ctx, vtn.core_from_sparse(Wi), vtn.core_from_sparse(Wj), chi_l, chi_r,
                       dev(L), dev(R), dev(th), y)
    expect = odmrg.heff_apply(L, Wi.dense(), Wj.dense(), R, th)
    close(host(y), expect)


@pytest.mark.parametrize("chi_l,chi_r,d,w", [(1, 3, 2, (1, 4)), (7, 5, 3, (5, 4)), (70, 33, 4, (6, 9)),
                                             (128, 128, 8, (12, 14))])
def test_env_updates_match_oracle(ctx, chi_l, chi_r, d, w):
    rng = inputs.rng_for(2000 + chi_l + chi_r)
    wl, wr = w
    W = inputs.random_sparse_core(wl, wr, d, rng)
    A = inputs.random_complex((chi_l, d, chi_r), rng)
    L = inputs.random_complex((wl, chi_l, chi_l), rng)
    R = inputs.random_complex((wr, chi_r, chi_r), rng)
    c = vtn.core_from_sparse(W)
    outL = torch.empty((wr, chi_r, chi_r), dtype=torch.complex128, device="cuda")
    vtn.vtn_env_update(ctx, c, 0, chi_l, chi_r, dev(L), dev(A), outL)
    close(host(outL), odmrg.env_left(L, A, W.dense()))
    outR = torch.empty((wl, chi_l, chi_l), dtype=torch.complex128, device="cuda")
    vtn.vtn_env_update(ctx, c, 1, chi_l, chi_r, dev(R), dev(A), outR)
    close(host(outR), odmrg.env_right(R, A, W.dense()))


def _random_theta(rng, cl, d1, d2, cr, decay=None):
    th = inputs.random_complex((cl, d1, d2, cr), rng)
    if decay is not None:
        # impose a decaying Schmidt spectrum so the kept subspace is well separated
        Tm = th.reshape(cl * d1, d2 * cr)
        U, s, Vh = np.linalg.svd(Tm, full_matrices=False)
        s = decay ** np.arange(s.size)
        th = ((U * s) @ Vh).reshape(th.shape)
    return th / np.linalg.norm(th)


TRUNC_CASES = [
    # chi_l, d1, d2, chi_r, direction, k_max
    (1, 4, 4, 16, 0, 16),
    (4, 4, 4, 1, 1, 16),
    (3, 3, 3, 5, 0, 6),
    (3, 3, 3, 5, 1, 6),
    (12, 4, 4, 9, 0, 20),
    (12, 4, 4, 9, 1, 20),
    (40, 8, 8, 40, 0, 64),
    (40, 8, 8, 40, 1, 64),
]


@pytest.mark.parametrize("tri_form", ["full", "lower"])
@pytest.mark.parametrize("cl,d1,d2,cr,direction,kmax", TRUNC_CASES + [(48, 6, 6, 50, 0, 64), (50, 6, 6, 48, 1, 64)])
def test_truncation_matches_oracle(ctx, cl, d1, d2, cr, direction, kmax, tri_form):
    """Both forms of the tridiagonalisation (the lower-triangle one normally runs from n = 1200);
    n = 288 and 300 take its two-column-per-lane chunks."""
    vtn.vtn_set_tridiag_lower(ctx, 0 if tri_form == "lower" else 1 << 30)
    rng = inputs.rng_for(3000 + cl * 31 + cr + direction)
    # Schmidt values decaying slowly enough that every kept weight is resolved in FP64
    # (rho = T T^dag carries sigma^2, so weights below ~1e-16 are numerical noise)
    th = _random_theta(rng, cl, d1, d2, cr, decay=0.9)
    k = min(kmax, cl * d1, d2 * cr)
    left = torch.empty((cl, d1, k), dtype=torch.complex128, device="cuda")
    right = torch.empty((k, d2, cr), dtype=torch.complex128, device="cuda")
    kk, lam, disc = vtn.vtn_truncate(ctx, cl, d1, d2, cr, direction, kmax, dev(th), left, right)
    assert kk == k
    oleft, oright, olam, odisc = odmrg.truncate(th, "right" if direction == 0 else "left", kmax)
    assert np.abs(lam - olam).max() <= 1e-13
    assert abs(disc - odisc) <= 1e-13
    L, R = host(left), host(right)
    # canonical factor is an isometry
    if direction == 0:
        Lm = L.reshape(cl * d1, k)
        assert np.abs(Lm.conj().T @ Lm - np.eye(k)).max() < 1e-12
    else:
        Rm = R.reshape(k, d2 * cr)
        assert np.abs(Rm @ Rm.conj().T - np.eye(k)).max() < 1e-12
    # the product (projected theta) is gauge invariant
    prod = np.einsum("asb,btc->astc", L, R)
    oprod = np.einsum("asb,btc->astc", oleft, oright)
    assert np.abs(prod - oprod).max() < 1e-11
    vtn.vtn_set_tridiag_lower(ctx)


@pytest.mark.parametrize("tri_form", ["full", "lower"])
def test_truncation_rank_deficient(ctx, tri_form):
    """Product state: rho has one non-zero eigenvalue and a degenerate null space (reflectors
    with tau = 0 once the trailing block vanishes); the kept factor must still be an isometry
    and reproduce theta."""
    vtn.vtn_set_tridiag_lower(ctx, 0 if tri_form == "lower" else 1 << 30)
    rng = inputs.rng_for(77)
    a = inputs.random_complex((2, 3), rng)
    b = inputs.random_complex((3, 4), rng)
    th = np.einsum("as,tb->astb", a, b)[:, :, :, :] / np.linalg.norm(a) / np.linalg.norm(b)
    th = th.reshape(2, 3, 3, 4)
    for direction in (0, 1):
        k = 6
        left = torch.empty((2, 3, k), dtype=torch.complex128, device="cuda")
        right = torch.empty((k, 3, 4), dtype=torch.complex128, device="cuda")
        kk, lam, disc = vtn.vtn_truncate(ctx, 2, 3, 3, 4, direction, k, dev(th), left, right)
        assert kk == 6
        assert abs(lam[0] - 1.0) < 1e-13 and np.all(np.abs(lam[1:]) < 1e-13)
        L, R = host(left), host(right)
        if direction == 0:
            Lm = L.reshape(6, 6)
            assert np.abs(Lm.conj().T @ Lm - np.eye(6)).max() < 1e-10
        else:
            Rm = R.reshape(6, 12)
            assert np.abs(Rm @ Rm.conj().T - np.eye(6)).max() < 1e-10
        assert np.abs(np.einsum("asb,btc->astc", L, R) - th).max() < 1e-12
    vtn.vtn_set_tridiag_lower(ctx)


@pytest.mark.parametrize("chi_l,chi_r,d,ws", [(3, 4, 3, (2, 3, 2)), (8, 8, 4, (4, 5, 4))])
def test_lanczos_ground_matches_dense(ctx, chi_l, chi_r, d, ws):
    """Lowest eigenpair of a Hermitian H_eff: environments made Hermitian per channel pair
    so that the operator is Hermitian; compared with dense eigh of the oracle operator."""
    rng = inputs.rng_for(4000 + chi_l)
    wl, wm, wr = ws
    # Hermitian construction: every term L_a (x) W1[a,b] (x) W2[b,c] (x) R_c is a tensor
    # product of Hermitian factors (Hermitian operators with real weights)
    Wi = inputs.random_sparse_core(wl, wm, d, rng, identity_frac=0.0)
    Wj = inputs.random_sparse_core(wm, wr, d, rng, identity_frac=0.0)
    Wi.ops = np.array([o + o.conj().T for o in Wi.ops])
    Wj.ops = np.array([o + o.conj().T for o in Wj.ops])
    L = inputs.random_complex((wl, chi_l, chi_l), rng)
    L = L + np.conj(np.transpose(L, (0, 2, 1)))
    R = inputs.random_complex((wr, chi_r, chi_r), rng)
    R = R + np.conj(np.transpose(R, (0, 2, 1)))
    n = chi_l * d * d * chi_r
    Hd = np.zeros((n, n), complex)
    eye = np.eye(n)
    for j in range(n):
        Hd[:, j] = odmrg.heff_apply(L, Wi.dense(), Wj.dense(), R, eye[:, j].reshape(chi_l, d, d, chi_r)).reshape(-1)
    assert np.abs(Hd - Hd.conj().T).max() < 1e-12
    lam, vec = np.linalg.eigh(Hd)
    x0 = inputs.random_complex(n, rng)
    th = dev(x0.reshape(chi_l, d, d, chi_r))
    st, E, nmv = vtn.vtn_heff_ground(ctx, vtn.core_from_sparse(Wi), vtn.core_from_sparse(Wj), chi_l, chi_r,
                                     dev(L), dev(R), th, tol=1e-11, krylov_max=40, max_restarts=20)
    assert st == vtn.VTN_OK
    assert abs(E - lam[0]) <= 1e-10 * max(1.0, abs(lam).max())
    x = host(th).reshape(-1)
    assert abs(abs(np.vdot(vec[:, 0], x)) - 1.0) < 1e-8
    # the oracle's Lanczos on the same operator agrees
    th_o, xo, _, conv = odmrg.lanczos_lowest(lambda v: Hd @ v, x0, odmrg.LanczosParams(40, 20, 1e-11))
    assert conv and abs(th_o - E) <= 1e-10 * max(1.0, abs(lam).max())


def test_lbo_rotate_matches_oracle(ctx):
    rng = inputs.rng_for(5000)
    cl, d, D, cr = 7, 6, 24, 5
    V = inputs.random_complex((D, d), rng)
    A = inputs.random_complex((cl, d, cr), rng)
    out = torch.empty((cl, D, cr), dtype=torch.complex128, device="cuda")
    vtn.vtn_lbo_rotate(ctx, cl, d, D, cr, dev(V), dev(A), out)
    close(host(out), np.einsum("nm,amb->anb", V, A))


def test_kernel_calls_reject_bad_arguments(ctx):
    rng = inputs.rng_for(1)
    W = inputs.random_sparse_core(2, 2, 2, rng)
    c = vtn.core_from_sparse(W)
    x = torch.zeros(8, dtype=torch.complex128, device="cuda")
    with pytest.raises(vtn.VtnError) as e:
        vtn.vtn_heff_apply(ctx, c, c, 1, 1, x, x, x, x)   # y aliases theta
    assert e.value.status == vtn.VTN_EINVAL
    with pytest.raises(vtn.VtnError) as e:
        vtn.vtn_env_update(ctx, c, 2, 1, 1, x, x, x)       # bad side
    assert e.value.status == vtn.VTN_EINVAL
    bad = vtn.make_core(2, 2, 2, [0, 5], [0, 1], np.ones((2, 2, 2)))
    with pytest.raises(vtn.VtnError):
        vtn.vtn_env_update(ctx, bad, 0, 1, 1, x, x, x)    # channel out of range
    with pytest.raises(vtn.VtnError) as e:
        vtn.vtn_heff_apply(ctx, c, c, 1, 1, x, x, x, torch.zeros_like(x), prec=vtn.VTN_TF32X3)
    assert e.value.status == vtn.VTN_EUNSUPPORTED


@pytest.mark.parametrize("tri_form", ["lower", "full"])
def test_truncation_at_the_large_workload_shape(ctx, tri_form):
    """Maximum size used by the solver: theta (512, 6, 6, 512) as at the middle bond of the
    large workload (chi = 512, d = 6), n = 3072, k = 512.  Theta = U diag(s) V^dag is built with
    a known SVD (Haar U, V; s_i = exp(-i / 300)), so the kept weights, the discarded weight and
    the projected product are known without a CPU eigensolver."""
    vtn.vtn_set_tridiag_lower(ctx, 0 if tri_form == "lower" else 1 << 30)
    rng = inputs.rng_for(4242)
    chi, d, k = 512, 6, 512
    n = chi * d
    U = inputs.haar_unitary(n, rng)
    V = inputs.haar_unitary(n, rng)
    s = np.exp(-np.arange(n) / 300.0)
    s /= np.linalg.norm(s)
    th = ((U * s) @ V.conj().T).reshape(chi, d, d, chi)
    left = torch.empty((chi, d, k), dtype=torch.complex128, device="cuda")
    right = torch.empty((k, d, chi), dtype=torch.complex128, device="cuda")
    kk, lam, disc = vtn.vtn_truncate(ctx, chi, d, d, chi, 0, k, dev(th), left, right)
    assert kk == k
    assert np.abs(np.asarray(lam) - s[:k] ** 2).max() <= 1e-13
    assert abs(disc - (s[k:] ** 2).sum()) <= 1e-12
    Lm = host(left).reshape(n, k)
    assert np.abs(Lm.conj().T @ Lm - np.eye(k)).max() < 1e-11
    prod = Lm @ host(right).reshape(k, n)
    expect = (U[:, :k] * s[:k]) @ V[:, :k].conj().T
    assert np.abs(prod - expect).max() < 1e-11
    vtn.vtn_set_tridiag_lower(ctx)
