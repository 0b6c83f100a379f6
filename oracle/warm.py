"""Inputs and targets of the learned warm start -- oracle (test infrastructure only).

The paper has no learned component.  The warm start learns, for one mode at a time, the map
from the mode's reduced covariance to the state that mode takes in a solved MPS, and begins the
sweeps from the product of its predictions instead of a random MPS.  This module states the two
ends of that map plainly:

* ``features``: for mode i with reduced covariance V_i = [[V_xx, V_xp], [V_xp, V_pp]] (the 2 x 2
  block of the covariance matrix of Eq. GBSHamiltonian's V, xxpp order):
  [log V_xx, log V_pp, V_xp / sqrt(V_xx V_pp), log det V_i / 2].
* ``targets``: for mode i the dominant eigenvector u_i of the single-mode reduced density
  matrix of the solved MPS (``observables.reduced_density``; the best single-mode state of that
  mode), phase fixed so that u_i[0] is real and non-negative (or, when |u_i[0]| < 1e-8, the
  largest component), as (Re, Im) interleaved.
"""
import numpy as np

from . import gbs, observables


def features(V):
    M = V.shape[0] // 2
    out = np.zeros((M, 4))
    for i in range(M):
        Vi = gbs.reduced_covariance(V, i)
        vxx, vpp, vxp = Vi[0, 0], Vi[1, 1], Vi[0, 1]
        out[i] = [np.log(vxx), np.log(vpp), vxp / np.sqrt(vxx * vpp), 0.5 * np.log(np.linalg.det(Vi))]
    return out


def fix_phase(u):
    ref = 0 if abs(u[0]) >= 1e-8 else int(np.argmax(np.abs(u)))
    return u * (np.conj(u[ref]) / abs(u[ref]))


def targets(mps):
    M = len(mps)
    d = mps[0].shape[1]
    out = np.zeros((M, 2 * d))
    for i in range(M):
        w, vecs = np.linalg.eigh(observables.reduced_density(mps, i))
        u = fix_phase(vecs[:, -1])
        out[i, 0::2], out[i, 1::2] = u.real, u.imag
    return out
