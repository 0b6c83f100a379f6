"""Host logic of the split-precision H_eff's term form (no GPU).

For a bond (i, i+1) the library writes the two-site operator content of the MPO,
sum_b W_i[a,b] (x) W_{i+1}[b,c] for every pair of outer channels (a, c), as
sum_t U[t][a] V[t][c] Bi[o_t] (x) Bj[p_t] with small operator bases Bi, Bj.  These tests rebuild
that sum from the exported terms and compare it with the cores' own product (the cores are pinned
against the oracle's MPO in test_host_abi): for random channel weights x, y the contraction
sum_{a,c} x_a y_c (.) must agree to rounding, and so must individual channel pairs.
"""
import numpy as np
import pytest

from paper_2410_18740_gb300 import inputs, vtn


def _dense_core(m, s, d):
    wl, wr, rows, cols, ops = vtn.vtn_mpo_core(m, s)
    W = np.zeros((wl, wr, d, d), np.complex128)
    for a, b, op in zip(rows, cols, ops):
        W[a, b] += op
    return W


def _check_bond(m, bond, rng):
    _, d, _, w = vtn.vtn_mpo_info(m)
    Wi, Wj = _dense_core(m, bond, d), _dense_core(m, bond + 1, d)
    t = vtn.vtn_mpo_bond_terms(m, bond)
    assert t is not None
    n_t = len(t["ops"])
    wl, wr = Wi.shape[0], Wj.shape[1]
    assert t["used"] == (n_t <= 1.15 * max(wl, wr) + 4)
    assert np.allclose(t["Bi"][0], np.eye(d)) and np.allclose(t["Bj"][0], np.eye(d))
    assert (t["ops"][: t["n_id"]] == 0).all() and (t["ops"][t["n_id"]:] != 0).any(axis=1).all()
    kr = [np.kron(t["Bi"][o], t["Bj"][p]) for o, p in t["ops"]]
    scale = max(np.abs(np.einsum("abst,bcuv->acsutv", Wi[:1], Wj[:, :1])).max(), 1.0)
    for _ in range(3):
        x = rng.standard_normal(wl) + 1j * rng.standard_normal(wl)
        y = rng.standard_normal(wr) + 1j * rng.standard_normal(wr)
        # reference: sum_{a,b,c} x_a y_c W_i[a,b] (x) W_j[b,c]
        A = np.einsum("a,abst->bst", x, Wi)
        Bm = np.einsum("c,bcuv->buv", y, Wj)
        ref = np.einsum("bst,buv->sutv", A, Bm).reshape(d * d, d * d)
        got = sum((x @ t["U"][k]) * (y @ t["V"][k]) * kr[k] for k in range(n_t))
        assert np.abs(got - ref).max() <= 1e-11 * max(np.abs(ref).max(), 1.0)
    # single channel pairs, including the edges of the channel ranges
    for a, c in [(0, 0), (wl - 1, wr - 1), (0, wr - 1), (wl - 1, 0), (wl // 2, wr // 3)]:
        ref = np.einsum("bst,buv->sutv", Wi[a], Wj[:, c]).reshape(d * d, d * d)
        got = sum(t["U"][k][a] * t["V"][k][c] * kr[k] for k in range(n_t))
        assert np.abs(got - ref).max() <= 1e-11 * max(scale, np.abs(ref).max())
    return n_t, wl, wr


@pytest.mark.parametrize("bond", [0, 1, 11, 22])
def test_bond_terms_split_workload(bond):
    """w <= 26 here: the term form exists (up to 14 terms beyond the identity block); at the
    middle bonds the channel-mixing form is the cheaper one, so the sweeps do not use it there."""
    w = inputs.workload("split", 100)
    m = vtn.vtn_build_mpo(None, w.r, w.U, w.D, w.d)
    _check_bond(m, bond, inputs.rng_for(7 + bond))
    if bond == 11:
        assert not vtn.vtn_mpo_bond_terms(m, bond)["used"]
    vtn.vtn_mpo_free(m)


@pytest.mark.parametrize("bond", [48, 49, 50])
def test_bond_terms_large_workload_centre(bond):
    """The collapse core at the centre (a near-dense block of scaled identities): the term count
    stays at w + O(1), so the term form's two GEMMs cost about what the mixing form's do."""
    w = inputs.workload("large", 200)
    m = vtn.vtn_build_mpo(None, w.r, w.U, w.D, w.d)
    n_t, wl, wr = _check_bond(m, bond, inputs.rng_for(11 + bond))
    assert n_t <= max(wl, wr) + 16
    assert vtn.vtn_mpo_bond_terms(m, bond)["used"]
    vtn.vtn_mpo_free(m)


def test_bond_terms_plain_fock_basis():
    w = inputs.workload("plain", 3)
    m = vtn.vtn_build_mpo(None, w.r, w.U, w.D, w.d)
    M = vtn.vtn_mpo_info(m)[0]
    for bond in range(M - 1):
        _check_bond(m, bond, inputs.rng_for(100 + bond))
    vtn.vtn_mpo_free(m)


def test_bond_terms_random_dense_cores():
    """Random dense entries: with d = 4 the basis is the whole 16-dimensional operator space, the
    factorisation is still exact but far longer than the channel count (not used); with d = 6 the
    entries span more than 16 operators and there is no compact term form."""
    rng = inputs.rng_for(5)
    for d, w in ((4, 6), (6, 6)):
        cores = [rng.standard_normal((1 if s == 0 else w, 1 if s == 2 else w, d, d))
                 + 1j * rng.standard_normal((1 if s == 0 else w, 1 if s == 2 else w, d, d)) for s in range(3)]
        m = vtn.vtn_mpo_from_cores(None, cores)
        for bond in (0, 1):
            t = vtn.vtn_mpo_bond_terms(m, bond)
            if d == 4:
                _check_bond(m, bond, inputs.rng_for(40 + bond))
                assert not t["used"]
            else:
                assert t is None
        vtn.vtn_mpo_free(m)
