"""Matrix product operator of the Gaussian parent Hamiltonian -- oracle (test
infrastructure only).

H = R^T G R - N/2 (Eq. GBSHamiltonian) expanded into
    sum_i h_i + sum_{j < i} sum_{a in mode j, b in mode i} 2 G_ab R_a R_b,
    h_i = G_{x_i x_i} X_i^2 + G_{p_i p_i} P_i^2 + G_{x_i p_i} (X_i P_i + P_i X_i) - 1/2,
with every same-mode product exactly projected (``gbs.local_ops``).  SM Sec. 8 builds
the MPO with centre-collapsed cores; the oracle deliberately uses the plainest finite
state machine instead, so that it shares no construction with the CUDA path:

    channel 0           "nothing yet"  (identity so far)
    channel 1 + a       "R_a seen"     for every quadrature a = x_0..x_{N-1}, p_0..p_{N-1}
    channel 2N + 1      "complete"

giving bond dimension w = 2N + 2 in the bulk, 1 at the two ends.  Pinned by contracting
it to a dense matrix and comparing with ``dense.dense_hamiltonian`` built term by term.
"""
import numpy as np

from . import gbs


def build_mpo(G, d):
    """List of dense cores W[s] with shape (w_left, w_right, d, d), W[a, b, s', s]."""
    G = np.asarray(G, dtype=np.float64)
    N = G.shape[0] // 2
    ops = gbs.local_ops(d)
    I, X, P = ops["I"], ops["X"], ops["P"]
    w = 2 * N + 2
    DONE = 2 * N + 1
    cores = []
    for s in range(N):
        W = np.zeros((w, w, d, d), dtype=np.complex128)
        xs, ps = s, N + s
        W[0, 0] = I
        W[0, 1 + xs] = X
        W[0, 1 + ps] = P
        W[0, DONE] = (G[xs, xs] * ops["X2"] + G[ps, ps] * ops["P2"]
                      + G[xs, ps] * ops["XPPX"] - 0.5 * I)
        for a in range(2 * N):
            W[1 + a, 1 + a] = I
            mode_a = a % N
            if mode_a < s:
                W[1 + a, DONE] = 2.0 * G[a, xs] * X + 2.0 * G[a, ps] * P
        W[DONE, DONE] = I
        if s == 0:
            W = W[0:1]
        if s == N - 1:
            W = W[:, DONE:DONE + 1]
        cores.append(np.ascontiguousarray(W))
    return cores


def contract_dense(cores):
    """Dense operator sum_{b} W_1 ... W_N (for tiny N only)."""
    d = cores[0].shape[2]
    acc = cores[0][0]                      # (w1, d, d)
    for W in cores[1:]:
        # acc[b, S', S] with S multi-index; new[c, S' s', S s]
        acc = np.einsum("bXY,bcuv->cXuYv", acc, W)
        c = acc.shape[0]
        n = acc.shape[1] * acc.shape[2]
        acc = acc.reshape(c, n, n)
    return acc[0]
