"""GPU parity of the warm start's MLP kernels (FP32) against the float64 oracle.

The parameters and inputs are float32 values, so both sides start from the same numbers;
tolerances are FP32-level relative to the largest magnitude (sums of up to 256 products per
layer, three layers).
"""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2410_18740_gb300 import inputs, vtn

pytestmark = pytest.mark.gpu

DIMS = (5, 256, 3, 7)   # n_in, width, depth, n_out


def _f32(rng, shape, scale=1.0):
    return (rng.standard_normal(shape) * scale).astype(np.float32)


def _params(rng, dims):
    n_in, width, depth, n_out = dims
    out = []
    for a, b in omlp.layer_sizes(*dims):
        out.append(rng.uniform(-1, 1, a * b) * np.sqrt(6.0 / a))
        out.append(rng.uniform(-0.1, 0.1, b))
    return np.concatenate(out).astype(np.float32)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("B", [1, 63, 300])
def test_forward_matches_oracle(ctx, B):
    rng = inputs.rng_for(7000 + B)
    m = vtn.vtn_mlp_create(ctx, *DIMS, seed=1)
    p = _params(rng, DIMS)
    vtn.vtn_mlp_set_params(ctx, m, p)
    x = _f32(rng, (B, DIMS[0]))
    y = torch.empty((B, DIMS[3]), dtype=torch.float32, device="cuda")
    vtn.vtn_mlp_forward(ctx, m, B, _dev(x), y)
    torch.cuda.synchronize()
    ref, _ = omlp.forward(p.astype(np.float64), x.astype(np.float64), *DIMS)
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-4 * np.abs(ref).max()
    vtn.vtn_mlp_free(m)


@pytest.mark.parametrize("dims,B", [(DIMS, 130), ((3, 17, 2, 2), 9), ((4, 33, 0, 3), 70)])
def test_loss_and_gradient_match_oracle(ctx, dims, B):
    rng = inputs.rng_for(7100 + B)
    m = vtn.vtn_mlp_create(ctx, *dims, seed=2)
    p = _params(rng, dims)
    vtn.vtn_mlp_set_params(ctx, m, p)
    x = _f32(rng, (B, dims[0]))
    t = _f32(rng, (B, dims[3]))
    loss, g = vtn.vtn_mlp_loss_grad(ctx, m, B, _dev(x), _dev(t))
    rl, rg = omlp.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), *dims)
    assert abs(loss - rl) <= 1e-5 * rl
    assert np.abs(g - rg).max() <= 1e-4 * np.abs(rg).max()
    vtn.vtn_mlp_free(m)


def test_adam_step_matches_oracle_and_training_converges(ctx):
    dims = (2, 64, 2, 1)
    rng = inputs.rng_for(7200)
    m = vtn.vtn_mlp_create(ctx, *dims, seed=3)
    p = _params(rng, dims)
    vtn.vtn_mlp_set_params(ctx, m, p)
    B = 256
    x = rng.uniform(-1, 1, (B, 2)).astype(np.float32)
    t = (np.sin(2 * x[:, 0]) + x[:, 1] ** 2).astype(np.float32)[:, None]
    xd, td = _dev(x), _dev(t)
    lr = 1e-3
    l0 = vtn.vtn_mlp_train_step(ctx, m, B, xd, td, lr)
    p1 = vtn.vtn_mlp_get_params(ctx, m)
    rl, rg = omlp.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), *dims)
    rp1, _, _ = omlp.adam_step(p.astype(np.float64), 0.0, 0.0, rg, 1, lr)
    assert abs(l0 - rl) <= 1e-5 * rl
    # the first Adam step is lr * g / (|g| + eps): compare where the gradient's sign is well
    # determined at FP32, and bound the step elsewhere
    big = np.abs(rg) > 1e-3 * np.abs(rg).max()
    assert big.sum() > 0.3 * big.size
    assert np.abs((p1 - p)[big] - (rp1 - p)[big]).max() <= 1e-3 * lr
    assert np.abs(p1 - p).max() <= lr * (1 + 1e-3)
    assert vtn.vtn_mlp_info(m)[5] == 1
    for _ in range(399):
        last = vtn.vtn_mlp_train_step(ctx, m, B, xd, td, 1e-2)
    assert last < 1e-2 * l0
    vtn.vtn_mlp_free(m)


def test_initialisation_and_errors(ctx):
    dims = (6, 40, 3, 4)
    a = vtn.vtn_mlp_create(ctx, *dims, seed=11)
    b = vtn.vtn_mlp_create(ctx, *dims, seed=11)
    c = vtn.vtn_mlp_create(ctx, *dims, seed=12)
    pa, pb, pc = (vtn.vtn_mlp_get_params(ctx, z) for z in (a, b, c))
    assert np.array_equal(pa, pb) and not np.array_equal(pa, pc)
    assert pa.size == omlp.param_count(*dims) == vtn.vtn_mlp_info(a)[4]
    layers = omlp.unpack(pa.astype(np.float64), *dims)
    for (W, bias), (n_in, _) in zip(layers, omlp.layer_sizes(*dims)):
        lim = np.sqrt(6.0 / n_in)
        assert np.abs(W).max() <= lim * (1 + 1e-6) and np.abs(W).max() > 0.8 * lim
        assert np.all(bias == 0.0)
    for z in (a, b, c):
        vtn.vtn_mlp_free(z)
    for bad in ((0, 8, 1, 1), (3, 8, 17, 1), (3, 5000, 1, 1)):
        with pytest.raises(vtn.VtnError):
            vtn.vtn_mlp_create(ctx, *bad)
    m = vtn.vtn_mlp_create(ctx, 2, 4, 1, 1)
    x = torch.zeros((3, 2), dtype=torch.float32, device="cuda")
    t = torch.zeros((3, 1), dtype=torch.float32, device="cuda")
    with pytest.raises(vtn.VtnError):
        vtn.vtn_mlp_train_step(ctx, m, 3, x, t, 0.0)
    with pytest.raises(vtn.VtnError):
        vtn.vtn_mlp_forward(ctx, m, 0, x, t)
    vtn.vtn_mlp_free(m)
