"""Thin Python binding of libvtn (include/vtn.h): one function per C entry point, same
names, argument marshalling only.  Every computation happens in the CUDA library; if the
library is missing this module raises instead of falling back to anything else.

Device buffers are passed as torch CUDA tensors (complex128, contiguous); host arrays as
numpy arrays.  By default the library draws device memory from PyTorch's caching
allocator through the vtn_allocator callbacks, on the stream given to vtn_create.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libvtn.so")

VTN_OK, VTN_EINVAL, VTN_ENOMEM, VTN_ECUDA, VTN_ENOCONV, VTN_ETIMEOUT, VTN_EUNSUPPORTED = range(7)
VTN_FP64, VTN_TF32X3, VTN_BF16X3 = 0, 1, 2
VTN_FLAG_LBO = 1
TIMING_CLASSES = {"gemm": 0, "heff": 1, "eig": 2, "lanczos": 3, "mix": 4, "tc": 5, "tridiag": 6}
STATUS_NAMES = {0: "VTN_OK", 1: "VTN_EINVAL", 2: "VTN_ENOMEM", 3: "VTN_ECUDA", 4: "VTN_ENOCONV",
                5: "VTN_ETIMEOUT", 6: "VTN_EUNSUPPORTED"}


class VtnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
        self.msg = msg


class vtn_allocator(C.Structure):
    _fields_ = [("alloc", C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)),
                ("free", C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)),
                ("user", C.c_void_p)]


class vtn_sweep_opts(C.Structure):
    _fields_ = [("chi_max", C.c_int), ("chi_schedule", C.POINTER(C.c_int)), ("n_schedule", C.c_int),
                ("n_sweeps", C.c_int), ("prec", C.c_int), ("lanczos_tol", C.c_double),
                ("krylov_max", C.c_int), ("lanczos_max_restarts", C.c_int), ("e_tol", C.c_double),
                ("e_target", C.c_double), ("use_e_target", C.c_int), ("seed", C.c_uint64),
                ("trunc_mode", C.c_int), ("trunc_q", C.c_int), ("window_lo", C.c_int), ("window_hi", C.c_int),
                ("energy_mode", C.c_int), ("heff_form", C.c_int), ("env_fp64", C.c_int)]


class vtn_sweep_report(C.Structure):
    _fields_ = [("sweeps_done", C.c_int), ("energy", C.c_double * 64), ("max_discarded", C.c_double * 64),
                ("seconds", C.c_double * 64), ("matvecs", C.c_longlong), ("lanczos_not_converged", C.c_longlong),
                ("heff_flops", C.c_double), ("heff_seconds", C.c_double), ("gemm_flops", C.c_double),
                ("gemm_seconds", C.c_double), ("eig_seconds", C.c_double), ("host_syncs", C.c_longlong)]


class vtn_core(C.Structure):
    _fields_ = [("w_left", C.c_int), ("w_right", C.c_int), ("d", C.c_int), ("nnz", C.c_int),
                ("rows", C.POINTER(C.c_int)), ("cols", C.POINTER(C.c_int)), ("ops", C.POINTER(C.c_double))]


_lib = None
_keep = []   # callbacks and buffers that must outlive the calls using them

_P = C.c_void_p
_I = C.c_int
_D = C.c_double
_PD = C.POINTER(C.c_double)
_PI = C.POINTER(C.c_int)

_SIGS = {
    "vtn_create": [C.POINTER(_P), _I, _P, C.POINTER(vtn_allocator)],
    "vtn_destroy": [_P],
    "vtn_last_error": [_P],
    "vtn_launch_count": [_P, C.POINTER(C.c_longlong)],
    "vtn_build_mpo": [_P, _I, _PD, _PD, _I, _I, C.c_uint, C.POINTER(_P)],
    "vtn_mpo_free": [_P],
    "vtn_mpo_info": [_P, _PI, _PI, _PI, _PI],
    "vtn_mpo_coefficients": [_P, _PD],
    "vtn_mpo_covariance": [_P, _PD],
    "vtn_mpo_isometry": [_P, _I, _PD],
    "vtn_mpo_core": [_P, _I, _PI, _PI, _PI, _PD],
    "vtn_mpo_bond_terms": [_P, _I, _PI, _PI, _PI, _PI, _PI, _PI, _PD, _PD, _PD, _PD],
    "vtn_mpo_norm_bound": [_P, _PD],
    "vtn_mps_random": [_P, _P, _I, C.c_uint64, C.POINTER(_P)],
    "vtn_mps_from_host": [_P, _P, _PI, C.POINTER(_PD), C.POINTER(_P)],
    "vtn_mps_random_center": [_P, _P, _I, C.c_uint64, _I, C.POINTER(_P)],
    "vtn_mps_product": [_P, _P, _PD, C.POINTER(_P)],
    "vtn_reduced_density": [_P, _P, _P, _I, _PD],
    "vtn_warm_features": [_P, C.POINTER(C.c_float)],
    "vtn_warm_targets": [_P, _P, _P, C.POINTER(C.c_float)],
    "vtn_mlp_train": [_P, _P, _I, _P, _P, C.c_float, _I, C.POINTER(C.c_float)],
    "vtn_sweep_batch": [_P, _I, C.POINTER(_P), C.POINTER(_P), C.POINTER(vtn_sweep_opts), C.POINTER(vtn_sweep_report),
                        C.POINTER(C.c_int), _I],
    "vtn_mps_warm_start": [_P, _P, _P, C.POINTER(_P)],
    "vtn_mps_get_center": [_P, _PI],
    "vtn_mps_set_center": [_P, _I],
    "vtn_mps_move_center": [_P, _P, _I],
    "vtn_mps_free": [_P],
    "vtn_mps_info": [_P, _PI, _PI, _PI],
    "vtn_mps_get_site": [_P, _P, _I, _PD],
    "vtn_mps_save": [_P, _P, C.c_char_p],
    "vtn_mps_load": [_P, _P, C.c_char_p, C.POINTER(_P)],
    "vtn_sweep_opts_default": [C.POINTER(vtn_sweep_opts)],
    "vtn_sweep": [_P, _P, C.POINTER(_P), C.POINTER(vtn_sweep_opts), C.POINTER(vtn_sweep_report)],
    "vtn_build_mpo_cz": [_P, _I, _PD, _PD, _I, _D, C.POINTER(C.c_void_p)],
    "vtn_mpo_from_cores": [_P, _I, C.POINTER(vtn_core), C.POINTER(_P)],
    "vtn_gaussian_bond_spectrum": [_P, _I, _I, _PD],
    "vtn_gaussian_bond_dims": [_P, _D, _I, _PI],
    "vtn_sweep_single_site": [_P, _P, C.POINTER(_P), C.POINTER(vtn_sweep_opts), _D, _D, _D,
                              C.POINTER(vtn_sweep_report)],
    "vtn_heff1_apply": [_P, C.POINTER(vtn_core), _I, _I, _P, _P, _P, _P],
    "vtn_mlp_create": [_P, _I, _I, _I, _I, C.c_uint64, C.POINTER(_P)],
    "vtn_mlp_free": [_P],
    "vtn_mlp_info": [_P, _PI, _PI, _PI, _PI, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)],
    "vtn_mlp_get_params": [_P, _P, C.POINTER(C.c_float)],
    "vtn_mlp_set_params": [_P, _P, C.POINTER(C.c_float)],
    "vtn_mlp_forward": [_P, _P, _I, _P, _P],
    "vtn_mlp_loss_grad": [_P, _P, _I, _P, _P, C.POINTER(C.c_float), C.POINTER(C.c_float)],
    "vtn_mlp_train_step": [_P, _P, _I, _P, _P, C.c_float, C.POINTER(C.c_float)],
    "vtn_expand": [_P, C.POINTER(vtn_core), _I, _I, _I, _P, _P, _D, _P],
    "vtn_energy": [_P, _P, _P, _PD],
    "vtn_energy_variance": [_P, _P, _P, _PD, _PD, _PD],
    "vtn_marginals": [_P, _P, _P, _PI, _I, _PD],
    "vtn_marginals_all": [_P, _P, _P, _PD],
    "vtn_sample": [_P, _P, _P, C.c_uint64, _I, _PI],
    "vtn_heff_apply": [_P, C.POINTER(vtn_core), C.POINTER(vtn_core), _I, _I, _P, _P, _P, _P, _I],
    "vtn_env_update": [_P, C.POINTER(vtn_core), _I, _I, _I, _P, _P, _P, _I],
    "vtn_heff_ground": [_P, C.POINTER(vtn_core), C.POINTER(vtn_core), _I, _I, _P, _P, _P, _D, _I, _I, _PD, _PI],
    "vtn_truncate": [_P, _I, _I, _I, _I, _I, _I, _P, _P, _P, _PD, _PD, _PI],
    "vtn_truncate_warm": [_P, _I, _I, _I, _I, _I, _I, _P, _P, _I, _I, _I, C.c_uint64, _I, _P, _P, _PD, _PD, _PI],
    "vtn_lbo_rotate": [_P, _I, _I, _I, _I, _P, _P, _P],
    "vtn_heff_apply_static": [C.POINTER(vtn_core), C.POINTER(vtn_core), _I, _I, _P, _P, _P, _P, _P],
    "vtn_gemm_bf16": [_P, _I, _I, _I, _P, C.c_longlong, _P, C.c_longlong, _P, C.c_longlong, _I],
    "vtn_timing": [_P, _I],
    "vtn_set_tc_accumulation": [_P, _I, _I],
    "vtn_set_tridiag_lower": [_P, _I],
    "vtn_timing_read": [_P, _I, C.POINTER(C.c_longlong), _PD, _PD],
    "vtn_timing_reset": [_P],
}


def lib():
    """Load libvtn.so (built by ``paper_2410_18740_gb300.build``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2410_18740_gb300.build.build() "
                               "(there is no fallback implementation)")
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_char_p if name == "vtn_last_error" else C.c_int
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(ctx, st, ok=(VTN_OK,)):
    if st not in ok:
        raise VtnError(st, vtn_last_error(ctx))
    return st


def _dptr(x):
    """Device pointer of a torch CUDA tensor (must be contiguous)."""
    if x is None:
        return None
    if not x.is_contiguous():
        raise ValueError("device tensor must be contiguous")
    return C.c_void_p(x.data_ptr())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _cplx_interleaved(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.view(np.float64)


# ----------------------------------------------------------------------- context
def _torch_allocator(device):
    import torch

    def _alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, torch.cuda.current_stream(device))
        except Exception:
            return None

    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    a = vtn_allocator(vtn_allocator._fields_[0][1](_alloc), vtn_allocator._fields_[1][1](_free), None)
    _keep.append(a)
    return a


def vtn_create(device=0, stream=None, torch_allocator=True):
    """Context on CUDA device `device`.  stream: torch.cuda.Stream, raw cudaStream_t int,
    or None for torch's current stream."""
    L = lib()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(device)
    raw = getattr(stream, "cuda_stream", stream)
    alloc = _torch_allocator(device) if torch_allocator else None
    out = C.c_void_p()
    st = L.vtn_create(C.byref(out), int(device), C.c_void_p(int(raw) if raw else 0),
                      C.byref(alloc) if alloc is not None else None)
    _check(None, st)
    return out


def vtn_destroy(ctx):
    return lib().vtn_destroy(ctx)


def vtn_last_error(ctx):
    r = lib().vtn_last_error(ctx)
    return r.decode() if r else ""


def vtn_launch_count(ctx):
    v = C.c_longlong()
    _check(ctx, lib().vtn_launch_count(ctx, C.byref(v)))
    return v.value


# ----------------------------------------------------------------------- MPO
def vtn_build_mpo(ctx, r, U, D, d, flags=0):
    """ctx may be None: host-only MPO (queries only; uploaded on first use by a context)."""
    r = _f64(r)
    Ui = _cplx_interleaved(U)
    M = r.shape[0]
    assert Ui.size == 2 * M * M
    out = C.c_void_p()
    st = lib().vtn_build_mpo(ctx, M, r.ctypes.data_as(_PD), Ui.ctypes.data_as(_PD), int(D), int(d),
                             int(flags), C.byref(out))
    _check(ctx, st)
    return out


def vtn_mpo_free(mpo):
    return lib().vtn_mpo_free(mpo)


def vtn_mpo_info(mpo):
    M, d, D = C.c_int(), C.c_int(), C.c_int()
    lib().vtn_mpo_info(mpo, C.byref(M), C.byref(d), C.byref(D), None)
    w = np.zeros(M.value + 1, dtype=np.int32)
    _check(None, lib().vtn_mpo_info(mpo, None, None, None, w.ctypes.data_as(_PI)))
    return M.value, d.value, D.value, w


def vtn_mpo_coefficients(mpo):
    M = vtn_mpo_info(mpo)[0]
    G = np.zeros((2 * M, 2 * M))
    _check(None, lib().vtn_mpo_coefficients(mpo, G.ctypes.data_as(_PD)))
    return G


def vtn_mpo_covariance(mpo):
    M = vtn_mpo_info(mpo)[0]
    V = np.zeros((2 * M, 2 * M))
    _check(None, lib().vtn_mpo_covariance(mpo, V.ctypes.data_as(_PD)))
    return V


def vtn_mpo_isometry(mpo, site):
    _, d, D, _ = vtn_mpo_info(mpo)
    V = np.zeros((D, d, 2))
    _check(None, lib().vtn_mpo_isometry(mpo, int(site), V.ctypes.data_as(_PD)))
    return V.view(np.complex128)[..., 0]


def vtn_build_mpo_cz(ctx, r, U, D, kappa):
    """Non-Gaussian (global CZ) workload MPO, Fock basis; ctx may be None (host-only)."""
    r = _f64(r)
    Ui = _cplx_interleaved(U)
    M = r.shape[0]
    assert Ui.size == 2 * M * M
    out = C.c_void_p()
    st = lib().vtn_build_mpo_cz(ctx, M, r.ctypes.data_as(_PD), Ui.ctypes.data_as(_PD), int(D), float(kappa),
                                C.byref(out))
    _check(ctx, st)
    return out


def vtn_mpo_core(mpo, site):
    _, d, _, w = vtn_mpo_info(mpo)
    n = C.c_int(0)
    _check(None, lib().vtn_mpo_core(mpo, int(site), C.byref(n), None, None, None))
    rows = np.zeros(n.value, np.int32)
    cols = np.zeros(n.value, np.int32)
    ops = np.zeros((max(n.value, 1), d, d, 2))
    _check(None, lib().vtn_mpo_core(mpo, int(site), C.byref(n), rows.ctypes.data_as(_PI),
                                    cols.ctypes.data_as(_PI), ops.ctypes.data_as(_PD)))
    return int(w[site]), int(w[site + 1]), rows, cols, ops.view(np.complex128)[..., 0][: n.value]


def vtn_mpo_bond_terms(mpo, bond):
    """Term form of bond (bond, bond+1): None when the bond has no compact one, else a dict with
    used (the split-precision sweeps use it), n_id, ops (n_terms x 2), U (n_terms x w_l),
    V (n_terms x w_r), Bi (ri x d x d), Bj."""
    _, d, _, w = vtn_mpo_info(mpo)
    usable, nt, nid, ri, rj = C.c_int(0), C.c_int(0), C.c_int(0), C.c_int(0), C.c_int(0)
    _check(None, lib().vtn_mpo_bond_terms(mpo, int(bond), C.byref(usable), C.byref(nt), C.byref(nid), C.byref(ri),
                                          C.byref(rj), None, None, None, None, None))
    if not usable.value:
        return None
    n, wl, wr = nt.value, int(w[bond]), int(w[bond + 2])
    ops = np.zeros((max(n, 1), 2), np.int32)
    U = np.zeros((max(n, 1), wl, 2))
    V = np.zeros((max(n, 1), wr, 2))
    Bi = np.zeros((ri.value, d, d, 2))
    Bj = np.zeros((rj.value, d, d, 2))
    _check(None, lib().vtn_mpo_bond_terms(mpo, int(bond), C.byref(usable), C.byref(nt), C.byref(nid), C.byref(ri),
                                          C.byref(rj), ops.ctypes.data_as(_PI), U.ctypes.data_as(_PD),
                                          V.ctypes.data_as(_PD), Bi.ctypes.data_as(_PD), Bj.ctypes.data_as(_PD)))
    cv = lambda x: x.view(np.complex128)[..., 0]
    return {"used": usable.value == 1, "n_id": nid.value, "ops": ops[:n], "U": cv(U)[:n], "V": cv(V)[:n],
            "Bi": cv(Bi), "Bj": cv(Bj)}


def vtn_gaussian_bond_spectrum(mpo, cut, k):
    out = np.zeros(int(k))
    _check(None, lib().vtn_gaussian_bond_spectrum(mpo, int(cut), int(k), out.ctypes.data_as(_PD)))
    return out


def vtn_gaussian_bond_dims(mpo, eps, chi_max):
    M = vtn_mpo_info(mpo)[0]
    out = np.zeros(M + 1, np.int32)
    _check(None, lib().vtn_gaussian_bond_dims(mpo, float(eps), int(chi_max), out.ctypes.data_as(_PI)))
    return out


def vtn_mpo_norm_bound(mpo):
    v = C.c_double()
    _check(None, lib().vtn_mpo_norm_bound(mpo, C.byref(v)))
    return v.value


# ----------------------------------------------------------------------- MPS
def vtn_mps_random(ctx, mpo, chi, seed):
    out = C.c_void_p()
    _check(ctx, lib().vtn_mps_random(ctx, mpo, int(chi), C.c_uint64(int(seed)), C.byref(out)))
    return out


def vtn_mps_random_center(ctx, mpo, chi, seed, center):
    out = C.c_void_p()
    _check(ctx, lib().vtn_mps_random_center(ctx, mpo, int(chi), C.c_uint64(int(seed)), int(center), C.byref(out)))
    return out


def vtn_mps_product(ctx, mpo, amps):
    """amps: complex array (M, d) of site vectors (normalised by the library)."""
    a = _cplx_interleaved(amps)
    out = C.c_void_p()
    _check(ctx, lib().vtn_mps_product(ctx, mpo, a.ctypes.data_as(_PD), C.byref(out)))
    return out


def vtn_reduced_density(ctx, mpo, mps, site):
    _, d, _, _ = vtn_mpo_info(mpo)
    out = np.zeros((d, d, 2))
    _check(ctx, lib().vtn_reduced_density(ctx, mpo, mps, int(site), out.ctypes.data_as(_PD)))
    return out.view(np.complex128)[..., 0]


def vtn_warm_features(mpo):
    M = vtn_mpo_info(mpo)[0]
    out = np.zeros((M, 4), np.float32)
    _check(None, lib().vtn_warm_features(mpo, out.ctypes.data_as(C.POINTER(C.c_float))))
    return out


def vtn_warm_targets(ctx, mpo, mps):
    M, d, _, _ = vtn_mpo_info(mpo)
    out = np.zeros((M, 2 * d), np.float32)
    _check(ctx, lib().vtn_warm_targets(ctx, mpo, mps, out.ctypes.data_as(C.POINTER(C.c_float))))
    return out


def vtn_mps_get_center(mps):
    c = C.c_int()
    _check(None, lib().vtn_mps_get_center(mps, C.byref(c)))
    return c.value


def vtn_mps_set_center(mps, center):
    _check(None, lib().vtn_mps_set_center(mps, int(center)))


def vtn_mps_move_center(ctx, mps, center):
    _check(ctx, lib().vtn_mps_move_center(ctx, mps, int(center)))


def vtn_mps_from_host(ctx, mpo, sites):
    dims = np.array([1] + [s.shape[2] for s in sites], dtype=np.int32)
    bufs = [_cplx_interleaved(s) for s in sites]
    arr = (_PD * len(bufs))(*[b.ctypes.data_as(_PD) for b in bufs])
    out = C.c_void_p()
    _check(ctx, lib().vtn_mps_from_host(ctx, mpo, dims.ctypes.data_as(_PI), arr, C.byref(out)))
    return out


def vtn_mps_free(mps):
    return lib().vtn_mps_free(mps)


def vtn_mps_info(mps):
    M, d = C.c_int(), C.c_int()
    lib().vtn_mps_info(mps, C.byref(M), C.byref(d), None)
    dims = np.zeros(M.value + 1, np.int32)
    _check(None, lib().vtn_mps_info(mps, None, None, dims.ctypes.data_as(_PI)))
    return M.value, d.value, dims


def vtn_mps_get_site(ctx, mps, site, out=None):
    """Site tensor (chi_l, d, chi_r) on the host; out: optional C-contiguous complex128 array of that
    shape to write into (e.g. a view of pinned memory)."""
    _, d, dims = vtn_mps_info(mps)
    shape = (int(dims[site]), d, int(dims[site + 1]))
    if out is None:
        buf = np.zeros(shape + (2,))
        _check(ctx, lib().vtn_mps_get_site(ctx, mps, int(site), buf.ctypes.data_as(_PD)))
        return buf.view(np.complex128)[..., 0]
    if out.shape != shape or out.dtype != np.complex128 or not out.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous complex128 array of the site's shape")
    _check(ctx, lib().vtn_mps_get_site(ctx, mps, int(site), out.view(np.float64).ctypes.data_as(_PD)))
    return out


def vtn_mps_save(ctx, mps, path):
    _check(ctx, lib().vtn_mps_save(ctx, mps, str(path).encode()))


def vtn_mps_load(ctx, mpo, path):
    out = C.c_void_p()
    _check(ctx, lib().vtn_mps_load(ctx, mpo, str(path).encode(), C.byref(out)))
    return out


# ----------------------------------------------------------------------- solver
def vtn_sweep_opts_default(**kw):
    o = vtn_sweep_opts()
    lib().vtn_sweep_opts_default(C.byref(o))
    sched = kw.pop("chi_schedule", None)
    for k, v in kw.items():
        setattr(o, k, v)
    if sched:
        arr = (C.c_int * len(sched))(*sched)
        _keep.append(arr)
        o.chi_schedule = C.cast(arr, C.POINTER(C.c_int))
        o.n_schedule = len(sched)
    return o


def _report_dict(rep):
    n = rep.sweeps_done
    return {"sweeps_done": n, "energy": list(rep.energy[:n]), "max_discarded": list(rep.max_discarded[:n]),
            "seconds": list(rep.seconds[:n]), "matvecs": rep.matvecs,
            "lanczos_not_converged": rep.lanczos_not_converged, "heff_flops": rep.heff_flops,
            "heff_seconds": rep.heff_seconds, "gemm_flops": rep.gemm_flops, "gemm_seconds": rep.gemm_seconds,
            "eig_seconds": rep.eig_seconds, "host_syncs": rep.host_syncs}


def vtn_sweep(ctx, mpo, state=None, opts=None, **kw):
    """Returns (status, mps, report).  VTN_ENOCONV is returned, not raised."""
    if opts is None:
        opts = vtn_sweep_opts_default(**kw)
    st_ptr = C.c_void_p(state.value if state is not None else None)
    rep = vtn_sweep_report()
    st = lib().vtn_sweep(ctx, mpo, C.byref(st_ptr), C.byref(opts), C.byref(rep))
    _check(ctx, st, ok=(VTN_OK, VTN_ENOCONV))
    return st, st_ptr, _report_dict(rep)


def vtn_sweep_batch(ctx, mpos, states, opts, n_streams=8):
    """Sweeps of many instances at once.  mpos: list of MPO handles; states: list of MPS handles or
    None; opts: list of vtn_sweep_opts.  Returns (status, [per-instance status], [mps], [report])."""
    n = len(mpos)
    M_arr = (C.c_void_p * n)(*[m.value if isinstance(m, C.c_void_p) else m for m in mpos])
    S_arr = (C.c_void_p * n)(*[(s.value if isinstance(s, C.c_void_p) else s) if s is not None else None
                               for s in states])
    O_arr = (vtn_sweep_opts * n)(*opts)
    R_arr = (vtn_sweep_report * n)()
    st_arr = (C.c_int * n)()
    st = lib().vtn_sweep_batch(ctx, n, C.cast(M_arr, C.POINTER(_P)), C.cast(S_arr, C.POINTER(_P)), O_arr, R_arr,
                               st_arr, int(n_streams))
    _check(ctx, st, ok=(VTN_OK, VTN_ENOCONV))
    return st, list(st_arr), [C.c_void_p(S_arr[j]) for j in range(n)], [_report_dict(R_arr[j]) for j in range(n)]


def vtn_sweep_single_site(ctx, mpo, state=None, opts=None, alpha=1e-2, alpha_decay=0.5, cutoff=1e-12, **kw):
    """Single-site DMRG with subspace expansion.  Returns (status, mps, report);
    VTN_ENOCONV is returned, not raised."""
    if opts is None:
        opts = vtn_sweep_opts_default(**kw)
    st_ptr = C.c_void_p(state.value if state is not None else None)
    rep = vtn_sweep_report()
    st = lib().vtn_sweep_single_site(ctx, mpo, C.byref(st_ptr), C.byref(opts), float(alpha), float(alpha_decay),
                                     float(cutoff), C.byref(rep))
    _check(ctx, st, ok=(VTN_OK, VTN_ENOCONV))
    return st, st_ptr, _report_dict(rep)


def vtn_energy(ctx, mpo, mps):
    v = C.c_double()
    _check(ctx, lib().vtn_energy(ctx, mpo, mps, C.byref(v)))
    return v.value


def vtn_energy_variance(ctx, mpo, mps):
    """(E, <H^2>, sigma_H) of the MPS, FP64."""
    e, h2, sg = C.c_double(), C.c_double(), C.c_double()
    _check(ctx, lib().vtn_energy_variance(ctx, mpo, mps, C.byref(e), C.byref(h2), C.byref(sg)))
    return e.value, h2.value, sg.value


def vtn_marginals(ctx, mpo, mps, modes):
    _, _, D, _ = vtn_mpo_info(mpo)
    modes = np.ascontiguousarray(modes, dtype=np.int32)
    k = modes.size
    out = np.zeros(D ** k)
    _check(ctx, lib().vtn_marginals(ctx, mpo, mps, modes.ctypes.data_as(_PI), int(k), out.ctypes.data_as(_PD)))
    return out.reshape((D,) * k)


def vtn_marginals_all(ctx, mpo, mps):
    M, _, D, _ = vtn_mpo_info(mpo)
    out = np.zeros((M, D))
    _check(ctx, lib().vtn_marginals_all(ctx, mpo, mps, out.ctypes.data_as(_PD)))
    return out


def vtn_sample(ctx, mpo, mps, seed, n_samples):
    M = vtn_mpo_info(mpo)[0]
    out = np.zeros((n_samples, M), np.int32)
    _check(ctx, lib().vtn_sample(ctx, mpo, mps, C.c_uint64(int(seed)), int(n_samples), out.ctypes.data_as(_PI)))
    return out


# ----------------------------------------------------------------------- kernel-level
def make_core(w_left, w_right, d, rows, cols, ops):
    rows = np.ascontiguousarray(rows, np.int32)
    cols = np.ascontiguousarray(cols, np.int32)
    opsf = _cplx_interleaved(ops)
    c = vtn_core(int(w_left), int(w_right), int(d), int(rows.size), rows.ctypes.data_as(_PI),
                 cols.ctypes.data_as(_PI), opsf.ctypes.data_as(_PD))
    c._bufs = (rows, cols, opsf)
    return c


def core_from_sparse(sc):
    """vtn_core from a paper_2410_18740_gb300.inputs.SparseCore."""
    return make_core(sc.w_left, sc.w_right, sc.d, sc.rows, sc.cols, sc.ops)


def core_from_dense(W):
    """vtn_core from a dense core W[a, b, s', s]: one entry per (a, b) block that is not zero."""
    W = np.asarray(W, dtype=np.complex128)
    wl, wr, d, _ = W.shape
    pairs = [(a, b) for a in range(wl) for b in range(wr) if np.any(W[a, b] != 0)]
    ops = np.array([W[a, b] for a, b in pairs]) if pairs else np.zeros((0, d, d), np.complex128)
    return make_core(wl, wr, d, [a for a, _ in pairs], [b for _, b in pairs], ops)


def vtn_mpo_from_cores(ctx, cores):
    """MPO from its cores (dense W[a, b, s', s] arrays or vtn_core); ctx may be None."""
    cs = [c if isinstance(c, vtn_core) else core_from_dense(c) for c in cores]
    arr = (vtn_core * len(cs))(*cs)
    out = C.c_void_p()
    _check(ctx, lib().vtn_mpo_from_cores(ctx, len(cs), arr, C.byref(out)))
    return out


def vtn_heff1_apply(ctx, W, chi_l, chi_r, L, R, A, y):
    _check(ctx, lib().vtn_heff1_apply(ctx, C.byref(W), int(chi_l), int(chi_r), _dptr(L), _dptr(R), _dptr(A),
                                      _dptr(y)))


def vtn_expand(ctx, W, side, chi_l, chi_r, env, A, alpha, out):
    _check(ctx, lib().vtn_expand(ctx, C.byref(W), int(side), int(chi_l), int(chi_r), _dptr(env), _dptr(A),
                                 float(alpha), _dptr(out)))


# ----------------------------------------------------------------------- learned warm start (MLP)
_PF = C.POINTER(C.c_float)


def vtn_mlp_create(ctx, n_in, width, depth, n_out, seed=0):
    out = C.c_void_p()
    _check(ctx, lib().vtn_mlp_create(ctx, int(n_in), int(width), int(depth), int(n_out), C.c_uint64(int(seed)),
                                     C.byref(out)))
    return out


def vtn_mlp_free(mlp):
    return lib().vtn_mlp_free(mlp)


def vtn_mlp_info(mlp):
    """(n_in, width, depth, n_out, n_params, steps)."""
    v = [C.c_int() for _ in range(4)]
    n, st = C.c_longlong(), C.c_longlong()
    _check(None, lib().vtn_mlp_info(mlp, *[C.byref(x) for x in v], C.byref(n), C.byref(st)))
    return tuple(x.value for x in v) + (n.value, st.value)


def vtn_mlp_get_params(ctx, mlp):
    out = np.zeros(vtn_mlp_info(mlp)[4], np.float32)
    _check(ctx, lib().vtn_mlp_get_params(ctx, mlp, out.ctypes.data_as(_PF)))
    return out


def vtn_mlp_set_params(ctx, mlp, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == vtn_mlp_info(mlp)[4]
    _check(ctx, lib().vtn_mlp_set_params(ctx, mlp, p.ctypes.data_as(_PF)))


def vtn_mlp_forward(ctx, mlp, batch, x, y):
    _check(ctx, lib().vtn_mlp_forward(ctx, mlp, int(batch), _dptr(x), _dptr(y)))


def vtn_mlp_loss_grad(ctx, mlp, batch, x, t, with_grad=True):
    """(loss, grad or None) on the batch (x, t device float32 tensors)."""
    loss = C.c_float()
    g = np.zeros(vtn_mlp_info(mlp)[4], np.float32) if with_grad else None
    _check(ctx, lib().vtn_mlp_loss_grad(ctx, mlp, int(batch), _dptr(x), _dptr(t), C.byref(loss),
                                        g.ctypes.data_as(_PF) if with_grad else None))
    return loss.value, g


def vtn_mlp_train_step(ctx, mlp, batch, x, t, lr):
    """One Adam step; returns the loss before it."""
    loss = C.c_float()
    _check(ctx, lib().vtn_mlp_train_step(ctx, mlp, int(batch), _dptr(x), _dptr(t), float(lr), C.byref(loss)))
    return loss.value


def vtn_mlp_train(ctx, mlp, batch, x, t, lr, steps):
    """`steps` Adam steps on the batch; returns the loss before the last one."""
    loss = C.c_float()
    _check(ctx, lib().vtn_mlp_train(ctx, mlp, int(batch), _dptr(x), _dptr(t), float(lr), int(steps), C.byref(loss)))
    return loss.value


def vtn_mps_warm_start(ctx, mpo, mlp):
    out = C.c_void_p()
    _check(ctx, lib().vtn_mps_warm_start(ctx, mpo, mlp, C.byref(out)))
    return out


def vtn_heff_apply(ctx, Wi, Wj, chi_l, chi_r, L, R, theta, y, prec=VTN_FP64):
    _check(ctx, lib().vtn_heff_apply(ctx, C.byref(Wi), C.byref(Wj), int(chi_l), int(chi_r), _dptr(L), _dptr(R),
                                     _dptr(theta), _dptr(y), int(prec)))


def vtn_env_update(ctx, W, side, chi_l, chi_r, env, A, out, prec=VTN_FP64):
    _check(ctx, lib().vtn_env_update(ctx, C.byref(W), int(side), int(chi_l), int(chi_r), _dptr(env), _dptr(A),
                                     _dptr(out), int(prec)))


def vtn_heff_ground(ctx, Wi, Wj, chi_l, chi_r, L, R, theta, tol=1e-10, krylov_max=32, max_restarts=4):
    E = C.c_double()
    nmv = C.c_int()
    st = lib().vtn_heff_ground(ctx, C.byref(Wi), C.byref(Wj), int(chi_l), int(chi_r), _dptr(L), _dptr(R),
                               _dptr(theta), float(tol), int(krylov_max), int(max_restarts), C.byref(E),
                               C.byref(nmv))
    _check(ctx, st, ok=(VTN_OK, VTN_ENOCONV))
    return st, E.value, nmv.value


def vtn_truncate_warm(ctx, chi_l, d1, d2, chi_r, direction, k_max, theta, Q0, q, p, seed, bond, left, right):
    """Q0: device complex tensor (n x k0) or None.  Returns (k, ritz values, discarded)."""
    kmax_eff = min(k_max, chi_l * d1, d2 * chi_r)
    lam = np.zeros(kmax_eff)
    disc = C.c_double()
    k = C.c_int()
    k0 = 0 if Q0 is None else int(Q0.shape[1])
    _check(ctx, lib().vtn_truncate_warm(ctx, int(chi_l), int(d1), int(d2), int(chi_r), int(direction), int(k_max),
                                        _dptr(theta), _dptr(Q0), k0, int(q), int(p), C.c_uint64(int(seed)), int(bond),
                                        _dptr(left), _dptr(right), lam.ctypes.data_as(_PD), C.byref(disc),
                                        C.byref(k)))
    return k.value, lam[: k.value], disc.value


def vtn_truncate(ctx, chi_l, d1, d2, chi_r, direction, k_max, theta, left, right):
    kmax_eff = min(k_max, chi_l * d1, d2 * chi_r)
    lam = np.zeros(kmax_eff)
    disc = C.c_double()
    k = C.c_int()
    _check(ctx, lib().vtn_truncate(ctx, int(chi_l), int(d1), int(d2), int(chi_r), int(direction), int(k_max),
                                   _dptr(theta), _dptr(left), _dptr(right), lam.ctypes.data_as(_PD),
                                   C.byref(disc), C.byref(k)))
    return k.value, lam[: k.value], disc.value


def vtn_lbo_rotate(ctx, chi_l, d, D, chi_r, V, A, out):
    _check(ctx, lib().vtn_lbo_rotate(ctx, int(chi_l), int(d), int(D), int(chi_r), _dptr(V), _dptr(A), _dptr(out)))


def vtn_heff_apply_static(Wi, Wj, chi_l, chi_r, L, R, theta, y, stream=None):
    """H_eff psi with the library's static device scratch: no context, no allocation.
    stream: torch.cuda.Stream, raw cudaStream_t int, or None for torch's current stream."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    raw = getattr(stream, "cuda_stream", stream)
    st = lib().vtn_heff_apply_static(C.byref(Wi), C.byref(Wj), int(chi_l), int(chi_r), _dptr(L), _dptr(R),
                                     _dptr(theta), _dptr(y), C.c_void_p(int(raw) if raw else 0))
    if st != VTN_OK:
        raise VtnError(st, "vtn_heff_apply_static: request beyond the static scratch limits, bad arguments, "
                           "or a CUDA failure (see include/vtn.h)")


def vtn_gemm_bf16(ctx, A, B, D):
    """D = A B^T on the tensor cores: A (M, K) and B (N, K) torch bf16 CUDA tensors, K a
    multiple of 64; D (M, N) float32 or float64 CUDA tensor."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    _check(ctx, lib().vtn_gemm_bf16(ctx, int(M), int(N), int(K), _dptr(A), int(A.stride(0)), _dptr(B),
                                    int(B.stride(0)), _dptr(D), int(D.stride(0)),
                                    1 if D.dtype == torch.float64 else 0))


def vtn_set_tc_accumulation(ctx, env_kblocks=64, heff_kblocks=256):
    _check(ctx, lib().vtn_set_tc_accumulation(ctx, int(env_kblocks), int(heff_kblocks)))


def vtn_set_tridiag_lower(ctx, min_n=1200):
    _check(ctx, lib().vtn_set_tridiag_lower(ctx, int(min_n)))


def vtn_timing(ctx, enable):
    _check(ctx, lib().vtn_timing(ctx, int(bool(enable))))


def vtn_timing_read(ctx, cls):
    cls = TIMING_CLASSES.get(cls, cls)
    n, fl, s = C.c_longlong(), C.c_double(), C.c_double()
    _check(ctx, lib().vtn_timing_read(ctx, int(cls), C.byref(n), C.byref(fl), C.byref(s)))
    return n.value, fl.value, s.value


def vtn_timing_reset(ctx):
    _check(ctx, lib().vtn_timing_reset(ctx))
