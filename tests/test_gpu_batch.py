"""Batched sweeps of many instances of uneven size (vtn_sweep_batch) against one-by-one sweeps
and the oracle.  The instances run concurrently on worker streams, but every kernel's launch
shape and summation order depend only on its own instance, so the energies must equal the
one-by-one vtn_sweep results bit for bit; a few instances are also checked against the
oracle's two-site DMRG (the FP64 bar |dE| <= 1e-10 ||H||)."""
import numpy as np
import pytest

from oracle import dmrg as odmrg, gbs, mpo as ompo
from paper_2410_18740_gb300 import inputs, vtn

pytestmark = pytest.mark.gpu

CASES = [  # (M, d, chi, seed)
    (4, 3, 9, 300), (7, 3, 12, 301), (5, 4, 16, 302), (9, 3, 9, 303), (6, 3, 16, 304), (8, 4, 12, 305),
]


def _opts(chi, seed, prec=vtn.VTN_FP64):
    return vtn.vtn_sweep_opts_default(chi_max=chi, n_sweeps=3, seed=seed, lanczos_tol=1e-12, krylov_max=24,
                                      lanczos_max_restarts=4, prec=prec, chi_schedule=[max(2, chi // 3), chi])


@pytest.mark.parametrize("prec", [vtn.VTN_FP64, vtn.VTN_BF16X3])
def test_batch_equals_one_by_one(ctx, prec):
    ws = [inputs.workload("split", s, M=M, d=d, D=d, r_lo=0.3, r_hi=1.0) for M, d, chi, s in CASES]
    mpos = [vtn.vtn_build_mpo(ctx, w.r, w.U, w.D, w.d) for w in ws]
    one = []
    for m, (M, d, chi, s) in zip(mpos, CASES):
        st, mps, rep = vtn.vtn_sweep(ctx, m, None, _opts(chi, s, prec))
        one.append(rep["energy"])
        vtn.vtn_mps_free(mps)
    st, sts, states, reps = vtn.vtn_sweep_batch(ctx, mpos, [None] * len(CASES),
                                                [_opts(chi, s, prec) for M, d, chi, s in CASES], n_streams=3)
    assert all(x in (vtn.VTN_OK, vtn.VTN_ENOCONV) for x in sts)
    for a, b in zip(reps, one):
        assert a["energy"] == b
    for (M, d, chi, s), w, m, mps, rep in zip(CASES, ws, mpos, states, reps):
        _, _, dims = vtn.vtn_mps_info(mps)
        assert len(dims) == M + 1 and max(dims) <= chi
        if prec == vtn.VTN_FP64 and M <= 7:
            G = gbs.hamiltonian_coefficients(w.r, w.U)
            _, orep = odmrg.dmrg(ompo.build_mpo(G, d), d, chi, 3, seed=s, chi_schedule=[max(2, chi // 3), chi],
                                 lanczos=odmrg.LanczosParams(krylov_max=24, max_restarts=4, tol=1e-12))
            for a, b in zip(rep["energy"], orep.energies):
                assert abs(a - b) <= 1e-10 * gbs.norm_bound(G, M, d)
        vtn.vtn_mps_free(mps)
    for m in mpos:
        vtn.vtn_mpo_free(m)


def test_batch_validation(ctx):
    w = inputs.workload("plain", 0)
    m = vtn.vtn_build_mpo(ctx, w.r, w.U, 4, 4)
    with pytest.raises(vtn.VtnError) as e:
        vtn.vtn_sweep_batch(ctx, [m], [None], [_opts(4, 1)], n_streams=0)
    assert e.value.status == vtn.VTN_EINVAL
    vtn.vtn_mpo_free(m)
