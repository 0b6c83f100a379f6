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
