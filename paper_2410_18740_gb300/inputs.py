"""Seeded synthetic inputs shared by the CUDA path, its tests, the benchmark and the oracle.

This module holds no arithmetic of the method itself: it only draws random problem
instances (squeezing parameters, Haar interferometers, random tensors for kernel-level
tests).  Both the CUDA library and the CPU oracle consume what it produces, so neither
depends on the other.

Workloads (the paper measures on no public dataset; its Borealis covariances are not
available, so seeded Haar-random GBS instances stand in for every workload):

* ``plain``  -- M=4 modes, r_k ~ U(0.3, 0.8), Fock cutoff d=D=4, chi=16 (the exactly
  representable case, Fig. 4c scale: D=8, chi=16 in Sec. "Results").
* ``split``  -- M=24, r_k ~ U(0.5, 1.0), d=D=8, chi=128.
* ``large``  -- M=100, r_k ~ U(0.8, 1.2), physical cutoff D=24 rotated to d=6 by the
  Gaussian optimal local basis (Sec. "Optimal Local Basis for Gaussian States"), chi=512.

The Haar unitary follows Mezzadri (2007): QR of a complex Ginibre matrix with the phases
of R's diagonal moved into Q.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def haar_unitary(M: int, rng: np.random.Generator) -> np.ndarray:
    """M x M Haar-random unitary (complex128)."""
    Z = (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    ph = np.diag(R) / np.abs(np.diag(R))
    return Q * ph[None, :]


@dataclass
class Workload:
    name: str
    M: int
    r: np.ndarray          # [M] squeezing parameters
    U: np.ndarray          # [M, M] complex interferometer, a_out = U a_in
    D: int                 # physical Fock cutoff
    d: int                 # local dimension used by the solver (d == D: Fock basis)
    chi: int               # maximum bond dimension
    n_sweeps: int = 8
    chi_schedule: list = field(default_factory=list)
    seed: int = 0

    @property
    def U_interleaved(self) -> np.ndarray:
        """U as row-major (re, im) interleaved float64, the C-ABI layout."""
        out = np.empty((self.M, self.M, 2), dtype=np.float64)
        out[..., 0] = self.U.real
        out[..., 1] = self.U.imag
        return out


_SPECS = {
    # name: (M, r_lo, r_hi, D, d, chi, n_sweeps, chi_schedule)
    "plain": (4, 0.3, 0.8, 4, 4, 16, 6, []),
    "split": (24, 0.5, 1.0, 8, 8, 128, 8, [16, 32, 64, 128]),
    "large": (100, 0.8, 1.2, 24, 6, 512, 6, [16, 64, 256, 512]),
}


def workload(name: str, seed: int, **override) -> Workload:
    """Seeded GBS instance.  ``override`` may replace M, D, d, chi, r range etc. for
    reduced test sizes (keys: M, r_lo, r_hi, D, d, chi, n_sweeps, chi_schedule)."""
    M, lo, hi, D, d, chi, ns, sched = _SPECS[name]
    M = override.get("M", M)
    lo = override.get("r_lo", lo)
    hi = override.get("r_hi", hi)
    D = override.get("D", D)
    d = override.get("d", d)
    chi = override.get("chi", chi)
    ns = override.get("n_sweeps", ns)
    sched = list(override.get("chi_schedule", sched))
    rng = rng_for(seed)
    U = haar_unitary(M, rng)
    r = rng.uniform(lo, hi, size=M)
    if override.get("identity_U", False):
        U = np.eye(M, dtype=np.complex128)
    return Workload(name=name, M=M, r=r, U=U, D=D, d=d, chi=chi, n_sweeps=ns,
                    chi_schedule=sched, seed=seed)


def random_complex(shape, rng: np.random.Generator) -> np.ndarray:
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def to_interleaved(z: np.ndarray) -> np.ndarray:
    """complex128 array -> float64 array with a trailing (re, im) axis, C-contiguous."""
    z = np.ascontiguousarray(z, dtype=np.complex128)
    return np.ascontiguousarray(z.view(np.float64).reshape(z.shape + (2,)))


def from_interleaved(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return x.view(np.complex128).reshape(x.shape[:-1])


@dataclass
class SparseCore:
    """A block-sparse MPO core: entries (row a, column b, d x d complex operator)."""
    w_left: int
    w_right: int
    d: int
    rows: np.ndarray       # int32 [nnz]
    cols: np.ndarray       # int32 [nnz]
    ops: np.ndarray        # complex128 [nnz, d, d]; ops[k][s', s] = <s'|op|s>

    def dense(self) -> np.ndarray:
        W = np.zeros((self.w_left, self.w_right, self.d, self.d), dtype=np.complex128)
        for a, b, op in zip(self.rows, self.cols, self.ops):
            W[a, b] += op
        return W


def random_sparse_core(w_left: int, w_right: int, d: int, rng: np.random.Generator,
                       density: float = 0.3, identity_frac: float = 0.5) -> SparseCore:
    """Random block-sparse core with the structure of the GBS MPO: a share of entries
    are scalar multiples of the identity (pass-through channels), the rest dense d x d
    complex blocks.  Every row and column receives at least one entry."""
    pairs = set()
    for a in range(w_left):
        pairs.add((a, int(rng.integers(w_right))))
    for b in range(w_right):
        pairs.add((int(rng.integers(w_left)), b))
    n_extra = int(density * w_left * w_right)
    for _ in range(n_extra):
        pairs.add((int(rng.integers(w_left)), int(rng.integers(w_right))))
    pairs = sorted(pairs)
    ops = []
    for _ in pairs:
        if rng.random() < identity_frac:
            ops.append(complex(rng.standard_normal(), rng.standard_normal()) * np.eye(d))
        else:
            ops.append(random_complex((d, d), rng))
    rows = np.array([p[0] for p in pairs], dtype=np.int32)
    cols = np.array([p[1] for p in pairs], dtype=np.int32)
    return SparseCore(w_left, w_right, d, rows, cols, np.array(ops, dtype=np.complex128))
