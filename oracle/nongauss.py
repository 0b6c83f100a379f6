"""Non-Gaussian workload: the fully connected phase gate -- oracle (test infrastructure only).

Sec. "Beyond GBS: fully connected CZ-gate": |psi> = exp(-i kappa prod_k X_k)|psi_G>
(Eq. GlobalCZgate) leaves every X invariant and shifts P_i by xi_i = kappa prod_{n != i} X_n,
so its parent Hamiltonian (Eq. nonGBSHamiltonian, zero means) is

    H = R'^T G R' - N/2,   R' = (X_1..X_N, P_1 + xi_1, .., P_N + xi_N),   G = V^{-1}/4.

Three independent constructions of P H P on the truncated space d^N:

* ``hamiltonian_definition``: R' built as operators on a padded per-mode space d + pad
  (Kronecker products of the padded X, P), H formed by matrix products exactly as written,
  then restricted to n_i < d on every mode (the exact projection: every mode carries at most
  a product of two quadratures, so one padding level already holds the intermediate state).
* ``dense_hamiltonian``: the expansion used by the MPOs, term by term from projected local
  operators.  With Xi_i = prod_{n != i} X_n and G symmetric,
      H = H_G + kappa sum_{a,i} G_{a p_i} (R_a Xi_i + Xi_i R_a) + kappa^2 sum_{ij} G_{p_i p_j} Xi_i Xi_j
  where, per mode: X_m Xi_i -> X^2 at m (m != i), identity at i; P_m Xi_i + Xi_i P_m ->
  XP + PX at m (m != i), identity at i; P_i Xi_i -> P at i; X_i Xi_i -> X on every mode;
  Xi_i Xi_j -> X at i and j, X^2 elsewhere (i != j); Xi_i^2 -> identity at i, X^2 elsewhere.
* ``build_mpo``: a finite-state-machine MPO of the same expansion (cores W[a, b, s', s]).
"""
import numpy as np
import scipy.sparse as sp

from . import dense, gbs


def _kron_list(mats):
    out = None
    for A in mats:
        A = sp.csr_matrix(A)
        out = A if out is None else sp.kron(out, A, format="csr")
    return out


def hamiltonian_definition(G, d, kappa, pad=2):
    """P H P of Eq. nonGBSHamiltonian from its definition (see the module docstring)."""
    G = np.asarray(G, dtype=np.float64)
    N = G.shape[0] // 2
    b = d + pad
    a = gbs.ladder(b)
    X = (a + a.conj().T) / np.sqrt(2.0)
    P = -1j * (a - a.conj().T) / np.sqrt(2.0)
    Ib = np.eye(b, dtype=np.complex128)

    def on(i, A):
        return _kron_list([A if n == i else Ib for n in range(N)])

    Xs = [on(i, X) for i in range(N)]
    Ps = [on(i, P) for i in range(N)]
    R = list(Xs)
    for i in range(N):
        xi = _kron_list([X if n != i else Ib for n in range(N)])
        R.append(Ps[i] + kappa * xi)
    dim = b ** N
    H = sp.csr_matrix((dim, dim), dtype=np.complex128)
    for p in range(2 * N):
        for q in range(2 * N):
            if G[p, q] != 0.0:
                H = H + G[p, q] * (R[p] @ R[q])
    H = H - 0.5 * N * sp.identity(dim, dtype=np.complex128, format="csr")
    # restrict to n_i < d on every mode
    keep = np.array([all(((idx // b ** (N - 1 - n)) % b) < d for n in range(N)) for idx in range(dim)])
    sel = np.nonzero(keep)[0]
    return H[sel][:, sel]


def _terms(G, d, kappa):
    """List of (coefficient, {mode: op}, bulk op) of the non-Gaussian part (kappa > 0 terms);
    modes absent from the dict carry the bulk operator."""
    G = np.asarray(G, dtype=np.float64)
    N = G.shape[0] // 2
    o = gbs.local_ops(d)
    x = lambda i: i
    p = lambda i: N + i
    out = []
    # linear in kappa, bulk X
    out.append((kappa * sum(2.0 * G[x(i), p(i)] for i in range(N)), {}, o["X"]))
    for i in range(N):
        out.append((kappa * 2.0 * G[p(i), p(i)], {i: o["P"]}, o["X"]))
        for m in range(N):
            if m == i:
                continue
            out.append((kappa * 2.0 * G[x(m), p(i)], {m: o["X2"], i: o["I"]}, o["X"]))
            out.append((kappa * G[p(m), p(i)], {m: o["XPPX"], i: o["I"]}, o["X"]))
    # quadratic in kappa, bulk X^2
    for i in range(N):
        out.append((kappa ** 2 * G[p(i), p(i)], {i: o["I"]}, o["X2"]))
        for j in range(N):
            if j != i:
                out.append((kappa ** 2 * G[p(i), p(j)], {i: o["X"], j: o["X"]}, o["X2"]))
    return out


def dense_hamiltonian(G, d, kappa):
    """P H P assembled from the expansion (projected local operators, Kronecker products)."""
    G = np.asarray(G, dtype=np.float64)
    N = G.shape[0] // 2
    H = dense.dense_hamiltonian(G, d)
    for c, special, bulk in _terms(G, d, kappa):
        if c == 0.0:
            continue
        H = H + c * _kron_list([special.get(n, bulk) for n in range(N)])
    return H


def build_mpo(G, d, kappa):
    """Cores W[s] (w_l, w_r, d, d) of H: the Gaussian part as in ``mpo.build_mpo`` (carry the
    raw quadratures of the left block) plus, for each bulk operator B (X for the kappa terms,
    X^2 for the kappa^2 terms), the states "bulk so far", "first special of type T at site f"
    and "term complete, bulk continues"; the coefficient of a pair is applied at the second
    special site.  All complete terms end in the common final state."""
    G = np.asarray(G, dtype=np.float64)
    N = G.shape[0] // 2
    o = gbs.local_ops(d)
    I, X, P, X2, XP = o["I"], o["X"], o["P"], o["X2"], o["XPPX"]
    xq = lambda i: i
    pq = lambda i: N + i
    T1 = ["I", "X2", "XPPX"]
    Top = {"I": I, "X2": X2, "XPPX": XP}

    def states(s):
        """Ordered state labels at cut s (0..N)."""
        if s == 0:
            return [("start",)]
        if s == N:
            return [("done",)]
        st = [("start",), ("done",)]
        st += [("gopen", j, k) for j in range(s) for k in range(2)]
        st += [("sx",), ("dx",)] + [("mx", f, t) for f in range(s) for t in T1]
        st += [("sx2",), ("dx2",)] + [("mx2", f) for f in range(s)]
        return st

    def pair1(f, t, g):
        """Operator at the second special site g after first special t at site f (bulk X)."""
        if t == "I":
            return kappa * (2.0 * G[xq(g), pq(f)] * X2 + G[pq(g), pq(f)] * XP)
        if t == "X2":
            return kappa * 2.0 * G[xq(f), pq(g)] * I
        return kappa * G[pq(f), pq(g)] * I

    cores = []
    for k in range(N):
        L, R = states(k), states(k + 1)
        li = {s: n for n, s in enumerate(L)}
        ri = {s: n for n, s in enumerate(R)}
        W = np.zeros((len(L), len(R), d, d), dtype=np.complex128)
        last = k == N - 1

        def add(sl, sr, op):
            if sl not in li:
                return
            if last:
                if sr[0] in ("done", "dx", "dx2"):
                    W[li[sl], ri[("done",)]] += op
                return
            if sr in ri:
                W[li[sl], ri[sr]] += op

        h = G[xq(k), xq(k)] * X2 + G[pq(k), pq(k)] * o["P2"] + G[xq(k), pq(k)] * XP - 0.5 * I
        # Gaussian part
        add(("start",), ("start",), I)
        add(("start",), ("done",), h)
        add(("done",), ("done",), I)
        add(("start",), ("gopen", k, 0), X)
        add(("start",), ("gopen", k, 1), P)
        for j in range(k):
            for kind in range(2):
                bq = j + kind * N
                add(("gopen", j, kind), ("gopen", j, kind), I)
                add(("gopen", j, kind), ("done",), 2.0 * G[bq, xq(k)] * X + 2.0 * G[bq, pq(k)] * P)
        # kappa terms, bulk X
        sx = ("start",) if k == 0 else ("sx",)
        add(sx, ("sx",), X)
        for t in T1:
            add(sx, ("mx", k, t), Top[t])
        single = kappa * 2.0 * G[pq(k), pq(k)] * P
        if k == 0:
            single = single + kappa * sum(2.0 * G[xq(i), pq(i)] for i in range(N)) * X
        add(sx, ("dx",), single)
        for f in range(k):
            for t in T1:
                add(("mx", f, t), ("mx", f, t), X)
                add(("mx", f, t), ("dx",), pair1(f, t, k))
        add(("dx",), ("dx",), X)
        # kappa^2 terms, bulk X^2
        sx2 = ("start",) if k == 0 else ("sx2",)
        add(sx2, ("sx2",), X2)
        add(sx2, ("mx2", k), X)
        add(sx2, ("dx2",), kappa ** 2 * G[pq(k), pq(k)] * I)
        for f in range(k):
            add(("mx2", f), ("mx2", f), X2)
            add(("mx2", f), ("dx2",), kappa ** 2 * 2.0 * G[pq(f), pq(k)] * X)
        add(("dx2",), ("dx2",), X2)
        cores.append(W)
    return cores


def ground_state(G, d, kappa, k=1):
    """Lowest k eigenpairs of P H P (dense eigh of the definition-based matrix)."""
    H = hamiltonian_definition(G, d, kappa).toarray()
    w, v = np.linalg.eigh(H)
    return w[:k], v[:, :k]


def norm(G, d, kappa):
    """Spectral norm of P H P (dense, tiny N only)."""
    H = hamiltonian_definition(G, d, kappa).toarray()
    return float(np.abs(np.linalg.eigvalsh(H)).max())
