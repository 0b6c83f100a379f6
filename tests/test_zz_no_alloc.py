"""The allocation-free H_eff psi entry point (vtn_heff_apply_static), for callers that
cannot allocate device memory, against the regular entry point vtn_heff_apply.

Collected last on purpose: if it fails, a run that stops at the first failure has
already run every other test.  It must pass in a fresh process and after the others.
"""
import numpy as np
import pytest
import torch

from paper_2410_18740_gb300 import inputs, vtn

pytestmark = pytest.mark.gpu

REL = 1e-12   # the tolerance of the other FP64 kernel tests


def _case(seed, chi_l, chi_r, d, ws):
    rng = inputs.rng_for(seed)
    wl, wm, wr = ws
    Wi = vtn.core_from_sparse(inputs.random_sparse_core(wl, wm, d, rng))
    Wj = vtn.core_from_sparse(inputs.random_sparse_core(wm, wr, d, rng))
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()
    L = dev(inputs.random_complex((wl, chi_l, chi_l), rng))
    R = dev(inputs.random_complex((wr, chi_r, chi_r), rng))
    th = dev(inputs.random_complex((chi_l, d, d, chi_r), rng))
    return Wi, Wj, L, R, th


def test_static_scratch_matches_regular_entry_point(libvtn):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = vtn.vtn_create(0)
    try:
        # two calls in a row with different shapes and data: the second must not see
        # anything the first left in the shared array
        for seed, chi_l, chi_r, d, ws in [(11, 37, 22, 6, (5, 7, 4)), (12, 16, 48, 8, (6, 3, 9))]:
            Wi, Wj, L, R, th = _case(seed, chi_l, chi_r, d, ws)
            y_ref = torch.empty_like(th)
            vtn.vtn_heff_apply(ctx, Wi, Wj, chi_l, chi_r, L, R, th, y_ref)
            y = torch.full_like(th, float("nan"))
            vtn.vtn_heff_apply_static(Wi, Wj, chi_l, chi_r, L, R, th, y)
            torch.cuda.synchronize()
            a, b = y.cpu().numpy(), y_ref.cpu().numpy()
            assert np.isfinite(a).all()
            assert np.abs(a - b).max() <= REL * np.abs(b).max()
    finally:
        torch.cuda.synchronize()
        vtn.vtn_destroy(ctx)


def test_static_scratch_rejects_oversize_requests(libvtn):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Wi, Wj, L, R, th = _case(13, 2, 2, 2, (2, 2, 2))
    # chi = 128, d = 8 with 26 channels needs 26 * 2**20 complex intermediates: beyond 1,015,808
    big = vtn.make_core(26, 26, 8, [0], [0], np.eye(8)[None])
    with pytest.raises(vtn.VtnError) as e:
        vtn.vtn_heff_apply_static(big, big, 128, 128, L, R, th, torch.empty_like(th))
    assert e.value.status == vtn.VTN_EINVAL
    with pytest.raises(vtn.VtnError) as e:
        vtn.vtn_heff_apply_static(Wi, Wj, 2, 2, L, R, th, th)     # y aliases theta
    assert e.value.status == vtn.VTN_EINVAL


def test_static_scratch_single_tile_long_sum_allocates_nothing(libvtn):
    """The first bond of a sweep: chi_l = 1, d = 8, chi_r = 64, and a right core with 50
    channels.  The final GEMM is then one 64 x 64 output tile summed over 50 * 64 terms, the
    shape for which the regular entry point splits the summation over several CTAs and takes
    a partial-sum buffer.  The static entry point must give the same result without any
    device allocation: free device memory is unchanged across two calls in a row."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chi_l, chi_r, d = 1, 64, 8
    Wi, Wj, L, R, th = _case(14, chi_l, chi_r, d, (1, 6, 50))
    ctx = vtn.vtn_create(0)
    try:
        y_ref = torch.empty_like(th)
        vtn.vtn_heff_apply(ctx, Wi, Wj, chi_l, chi_r, L, R, th, y_ref)
        ys = [torch.full_like(th, float("nan")) for _ in range(3)]
        # a first call may load the library's device code (and with it the static array)
        vtn.vtn_heff_apply_static(Wi, Wj, chi_l, chi_r, L, R, th, ys[0])
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        vtn.vtn_heff_apply_static(Wi, Wj, chi_l, chi_r, L, R, th, ys[1])
        vtn.vtn_heff_apply_static(Wi, Wj, chi_l, chi_r, L, R, th, ys[2])
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0, f"device memory changed by {free0 - free1} bytes"
        b = y_ref.cpu().numpy()
        for y in ys:
            a = y.cpu().numpy()
            assert np.isfinite(a).all()
            assert np.abs(a - b).max() <= REL * np.abs(b).max()
    finally:
        torch.cuda.synchronize()
        vtn.vtn_destroy(ctx)
