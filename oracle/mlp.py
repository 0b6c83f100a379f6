"""Multilayer perceptron of the learned warm start -- oracle (test infrastructure only).

The paper has no learned component; the warm start maps features of a GBS instance
(per-mode reduced covariances) to solver inputs and is assessed by the variational energy
<H> it leads to (Eq. MagOfSimError).  This module is the plain reference for the network
itself: fully connected layers with ReLU between them, mean-squared-error loss, gradients
by the chain rule written out layer by layer, and the Adam update (Kingma and Ba, ICLR
2015, Algorithm 1).  It runs in float64 so that it can be pinned against central finite
differences; the GPU kernels (FP32) are compared with it at FP32 tolerances.

Parameters (the library's layout): for layer l = 0..L-1, W_l (n_out_l x n_in_l, row-major)
followed by b_l (n_out_l), concatenated.  Layer sizes: n_in -> width (x depth) -> n_out, ReLU
after every layer but the last.

Parity: backward pinned by central differences of the loss; a single linear layer against
the closed-form least-squares gradient; Adam's first step against its closed form
lr * g / (|g| + eps).
"""
import numpy as np


def layer_sizes(n_in, width, depth, n_out):
    sizes = [n_in] + [width] * depth + [n_out]
    return list(zip(sizes[:-1], sizes[1:]))           # (n_in_l, n_out_l)


def unpack(params, n_in, width, depth, n_out):
    """List of (W_l, b_l) views into the flat parameter vector."""
    out, off = [], 0
    for a, b in layer_sizes(n_in, width, depth, n_out):
        W = params[off:off + a * b].reshape(b, a)
        off += a * b
        bias = params[off:off + b]
        off += b
        out.append((W, bias))
    assert off == params.size
    return out


def param_count(n_in, width, depth, n_out):
    return sum(a * b + b for a, b in layer_sizes(n_in, width, depth, n_out))


def forward(params, x, n_in, width, depth, n_out):
    """Returns (y, activations) with activations[0] = x and activations[l] the ReLU output of
    hidden layer l."""
    layers = unpack(params, n_in, width, depth, n_out)
    acts = [x]
    h = x
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        h = np.maximum(z, 0.0) if l + 1 < len(layers) else z
        acts.append(h)
    return h, acts[:-1]


def loss_and_grad(params, x, t, n_in, width, depth, n_out):
    """MSE loss = mean over all B * n_out entries of (y - t)^2 and its gradient (flat)."""
    layers = unpack(params, n_in, width, depth, n_out)
    y, acts = forward(params, x, n_in, width, depth, n_out)
    B = x.shape[0]
    loss = float(np.mean((y - t) ** 2))
    g = 2.0 * (y - t) / (B * n_out)                    # dloss / dy
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        h = acts[l]
        gW = g.T @ h
        gb = g.sum(axis=0)
        grads.append((gW, gb))
        if l > 0:
            g = (g @ W) * (acts[l] > 0)                # ReLU of the layer below (derivative 0 at 0)
    flat = []
    for gW, gb in reversed(grads):
        flat.append(gW.reshape(-1))
        flat.append(gb)
    return loss, np.concatenate(flat)


def adam_step(params, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v
