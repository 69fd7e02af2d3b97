"""ctypes binding of libvv10 (include/vv10.h), one Python function per C entry point.

Argument marshalling only: tensors are checked for device, dtype, shape and contiguity
and passed as raw device pointers together with the current torch CUDA stream; every
step of the computation runs in the library's CUDA kernels.  There is no CPU fallback:
if the library is missing or the device is not a CUDA GPU the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

from . import build as _build

VV10_OK = 0
VV10_ERR_INVALID_ARG = 1
VV10_ERR_CUDA = 2
VV10_ERR_OOM = 3
VV10_ERR_TIMEOUT = 4
VV10_ERR_NONFINITE = 5
VV10_ERR_UNSUPPORTED = 6

VV10_FP64 = 0
VV10_MIXED_TF32X3 = 1
VV10_MIXED_BF16X3 = 2
VV10_MIXED_F16X3 = 3
VV10_FP64_TC = 4
PRECISIONS = {"fp64": VV10_FP64, "tf32x3": VV10_MIXED_TF32X3, "bf16x3": VV10_MIXED_BF16X3,
              "f16x3": VV10_MIXED_F16X3, "fp64tc": VV10_FP64_TC, "mixed": VV10_MIXED_TF32X3}

VV10_OPT_FUSE_HESSIAN_SUMS = 1
VV10_TUNE_PAIRSUMS = 1
VV10_TUNE_BATCH = 2
VV10_TUNE_CONTRACTION = 4
TILES_BATCH = 6        # vv10_set_tiles / vv10_get_tiles: 6 + fp64 = batched pair sums
TILES_CONTRACTION = 8  # the widest trial group of the tensor-core contraction

VV10_DEBUG_FAIL_ALLOC = 1
VV10_DEBUG_STALL_COPY = 2

# Function names declared in include/vv10.h (checked against the header by the tests).
EXPORTS = ("vv10_create", "vv10_destroy", "vv10_status_string", "vv10_last_error",
           "vv10_prepare_points", "vv10_energy_potential", "vv10_hessian_contract",
           "vv10_coord_grad", "vv10_weight_grad", "vv10_sync", "vv10_set_tiles",
           "vv10_debug_inject", "vv10_profile_enable", "vv10_profile_read",
           "vv10_profile_phase_name", "vv10_energy_potential_noalloc",
           "vv10_batch_prepare", "vv10_batch_energy_potential", "vv10_batch_hessian_contract",
           "vv10_batch_run", "vv10_get_tiles", "vv10_autotune", "vv10_set_autotune",
           "vv10_set_options", "vv10_evaluate", "vv10_coord_hessian",
           "vv10_weight_response", "vv10_energy", "vv10_fock_matrix",
           "vv10_orbital_hessian", "vv10_nuclear_gradient", "vv10_fock_derivative",
           "vv10_nuclear_hessian", "vv10_hessian_vector_product")
VV10_NOALLOC_MAX_POINTS = 32768
VV10_MAX_TRIALS = 4096  # include/vv10.h: VV10_MAX_TRIALS (also the most weight directions)
VV10_N_PHASES = 16


class VV10Params(ctypes.Structure):
    _fields_ = [("b", ctypes.c_double), ("C", ctypes.c_double), ("rho_cut", ctypes.c_double)]


class VV10Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libvv10 (optionally compiling it first).  Raises if it is not available."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libvv10 is not built ({_build.LIB} missing); run "
                           "paper_2208_14639_gb300.build.build() or __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.c_void_p
    I32, I64, D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    st = ctypes.c_int
    sig = {
        "vv10_create": (st, [ctypes.POINTER(P), ctypes.c_int]),
        "vv10_destroy": (st, [P]),
        "vv10_status_string": (ctypes.c_char_p, [st]),
        "vv10_last_error": (ctypes.c_char_p, [P]),
        "vv10_prepare_points": (st, [P, I64, P, P, P, P, P, I32, VV10Params,
                                     ctypes.POINTER(I64), P]),
        "vv10_energy_potential": (st, [P, st, ctypes.POINTER(D), P, P, P]),
        "vv10_hessian_contract": (st, [P, st, I32, P, P, P, P, P]),
        "vv10_hessian_vector_product": (st, [P, st, I32, P, P, P, P, P]),
        "vv10_coord_grad": (st, [P, st, P, P, P, P]),
        "vv10_coord_hessian": (st, [P, st, P, P, P]),
        "vv10_weight_response": (st, [P, st, ctypes.c_int32, P, P, P, P, P]),
        "vv10_energy": (st, [P, st, ctypes.POINTER(D), P]),
        "vv10_fock_matrix": (st, [P, I32, P, P, P, P, P, P]),
        "vv10_nuclear_gradient": (st, [P, I32, P, P, P, P, P]),
        "vv10_nuclear_hessian": (st, [P, st, P, P, P, P, P, P, P, P]),
        "vv10_orbital_hessian": (st, [P, I32, P, P, I32, P, P, P, P, P, P]),
        "vv10_fock_derivative": (st, [P, I32] + [P] * 16),
        "vv10_weight_grad": (st, [P, P, P]),
        "vv10_sync": (st, [P, P]),
        "vv10_set_tiles": (st, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "vv10_debug_inject": (st, [P, ctypes.c_int, I64]),
        "vv10_profile_enable": (st, [P, ctypes.c_int]),
        "vv10_profile_read": (st, [P, ctypes.c_int, P, P]),
        "vv10_profile_phase_name": (ctypes.c_char_p, [ctypes.c_int]),
        "vv10_energy_potential_noalloc": (st, [I64, P, P, P, P, VV10Params, st, P, P, P, P]),
        "vv10_batch_prepare": (st, [P, I32, P, P, P, P, P, P, P, VV10Params, P, P]),
        "vv10_batch_energy_potential": (st, [P, st, P, P, P, P]),
        "vv10_batch_hessian_contract": (st, [P, st, P, P, P, P, P, P]),
        "vv10_batch_run": (st, [P, st, P, P, P, P, P, P, P, P, P]),
        "vv10_get_tiles": (st, [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int)]),
        "vv10_autotune": (st, [P, st, ctypes.c_int, P]),
        "vv10_set_autotune": (st, [P, ctypes.c_int]),
        "vv10_set_options": (st, [P, ctypes.c_int]),
        "vv10_evaluate": (st, [P, st, I32, P, P, ctypes.POINTER(D), P, P, P, P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(h, status: int, what: str):
    if status != VV10_OK:
        lib = load()
        msg = lib.vv10_status_string(status).decode()
        detail = lib.vv10_last_error(h).decode() if h else ""
        raise VV10Error(status, f"{what}: {msg}" + (f" ({detail})" if detail else ""))


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dptr(t: Optional[torch.Tensor], name: str, dtype=torch.float64, shape=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- one wrapper per entry point

def vv10_create(device: int = 0) -> ctypes.c_void_p:
    lib = load()
    h = ctypes.c_void_p()
    _check(None, lib.vv10_create(ctypes.byref(h), int(device)), "vv10_create")
    return h


def vv10_destroy(h) -> None:
    _check(None, load().vv10_destroy(h), "vv10_destroy")


def vv10_status_string(status: int) -> str:
    return load().vv10_status_string(int(status)).decode()


def vv10_last_error(h) -> str:
    return load().vv10_last_error(h).decode()


def vv10_prepare_points(h, xyz, w, rho, grad_rho, atom_of_point=None, n_atom: int = 0,
                        b: float = 6.0, C: float = 0.01, rho_cut: float = 1e-10,
                        stream=None) -> int:
    n = int(w.shape[0])
    nk = ctypes.c_int64()
    st = load().vv10_prepare_points(
        h, n, _dptr(xyz, "xyz", shape=(n, 3)), _dptr(w, "w", shape=(n,)),
        _dptr(rho, "rho", shape=(n,)), _dptr(grad_rho, "grad_rho", shape=(n, 3)),
        _dptr(atom_of_point, "atom_of_point", torch.int32, (n,)), int(n_atom),
        VV10Params(b, C, rho_cut), ctypes.byref(nk), _stream(stream))
    _check(h, st, "vv10_prepare_points")
    return int(nk.value)


def vv10_energy_potential(h, prec: int, vrho=None, vgamma=None, stream=None,
                          want_energy: bool = True) -> Optional[float]:
    e = ctypes.c_double()
    st = load().vv10_energy_potential(h, int(prec), ctypes.byref(e) if want_energy else None,
                                      _dptr(vrho, "vrho"), _dptr(vgamma, "vgamma"),
                                      _stream(stream))
    _check(h, st, "vv10_energy_potential")
    return float(e.value) if want_energy else None


def vv10_hessian_contract(h, prec: int, rho_t, grad_rho_t, f_rho_t, f_gamma_t,
                          stream=None) -> None:
    P, n = int(rho_t.shape[0]), int(rho_t.shape[1])
    st = load().vv10_hessian_contract(
        h, int(prec), P, _dptr(rho_t, "rho_t", shape=(P, n)),
        _dptr(grad_rho_t, "grad_rho_t", shape=(P, n, 3)),
        _dptr(f_rho_t, "f_rho_t", shape=(P, n)), _dptr(f_gamma_t, "f_gamma_t", shape=(P, n)),
        _stream(stream))
    _check(h, st, "vv10_hessian_contract")


def vv10_hessian_vector_product(h, prec: int, rho_t, grad_rho_t, hv_rho, hv_grad,
                                stream=None) -> None:
    """hv_rho = w f^{rho,t}, hv_grad = 2 w (f^{gamma,t} grad rho + f^gamma grad rho^t)."""
    P, n = int(rho_t.shape[0]), int(rho_t.shape[1])
    st = load().vv10_hessian_vector_product(
        h, int(prec), P, _dptr(rho_t, "rho_t", shape=(P, n)),
        _dptr(grad_rho_t, "grad_rho_t", shape=(P, n, 3)),
        _dptr(hv_rho, "hv_rho", shape=(P, n)), _dptr(hv_grad, "hv_grad", shape=(P, n, 3)),
        _stream(stream))
    _check(h, st, "vv10_hessian_vector_product")


def vv10_coord_grad(h, prec: int, grad_points=None, grad_atoms=None, EUW_Bgr=None,
                    stream=None) -> None:
    st = load().vv10_coord_grad(h, int(prec), _dptr(grad_points, "grad_points"),
                                _dptr(grad_atoms, "grad_atoms"), _dptr(EUW_Bgr, "EUW_Bgr"),
                                _stream(stream))
    _check(h, st, "vv10_coord_grad")


def vv10_coord_hessian(h, prec: int, E_grgr=None, D_points=None, stream=None) -> None:
    st = load().vv10_coord_hessian(h, int(prec), _dptr(E_grgr, "E_grgr"),
                                   _dptr(D_points, "D_points"), _stream(stream))
    _check(h, st, "vv10_coord_hessian")


def vv10_weight_response(h, prec: int, w_t, E_t=None, U_t=None, W_t=None, stream=None) -> None:
    P, n = w_t.shape
    st = load().vv10_weight_response(h, int(prec), int(P), _dptr(w_t, "w_t", shape=(P, n)),
                                     _dptr(E_t, "E_t", shape=(P, n)), _dptr(U_t, "U_t", shape=(P, n)),
                                     _dptr(W_t, "W_t", shape=(P, n)), _stream(stream))
    _check(h, st, "vv10_weight_response")


def vv10_energy(h, prec: int, stream=None) -> float:
    e = ctypes.c_double()
    _check(h, load().vv10_energy(h, int(prec), ctypes.byref(e), _stream(stream)), "vv10_energy")
    return e.value


def vv10_fock_matrix(h, phi, grad_phi, vrho, vgamma, F, stream=None) -> None:
    n, nbf = phi.shape
    st = load().vv10_fock_matrix(h, int(nbf), _dptr(phi, "phi", shape=(n, nbf)),
                                 _dptr(grad_phi, "grad_phi", shape=(n, nbf, 3)),
                                 _dptr(vrho, "vrho", shape=(n,)), _dptr(vgamma, "vgamma", shape=(n,)),
                                 _dptr(F, "F", shape=(nbf, nbf)), _stream(stream))
    _check(h, st, "vv10_fock_matrix")


def vv10_orbital_hessian(h, phi, grad_phi, f_rho_t, f_gamma_t, grad_rho_t, vgamma, G,
                         stream=None) -> None:
    n, nbf = phi.shape
    P = int(f_rho_t.shape[0])
    st = load().vv10_orbital_hessian(
        h, int(nbf), _dptr(phi, "phi", shape=(n, nbf)), _dptr(grad_phi, "grad_phi", shape=(n, nbf, 3)),
        P, _dptr(f_rho_t, "f_rho_t", shape=(P, n)), _dptr(f_gamma_t, "f_gamma_t", shape=(P, n)),
        _dptr(grad_rho_t, "grad_rho_t", shape=(P, n, 3)), _dptr(vgamma, "vgamma", shape=(n,)),
        _dptr(G, "G", shape=(P, nbf, nbf)), _stream(stream))
    _check(h, st, "vv10_orbital_hessian")


def vv10_fock_derivative(h, phi, grad_phi, hess_phi, bf_atom, vrho, vgamma, f_rho_a, f_gamma_a,
                         grad_rho_a, w_a, E_w, U_w, W_w, EUW_gr, FA, stream=None) -> None:
    n, nbf = phi.shape
    P = int(FA.shape[0])
    na = P // 3
    dirs = dict(shape=(P, n))
    st = load().vv10_fock_derivative(
        h, int(nbf), _dptr(phi, "phi", shape=(n, nbf)), _dptr(grad_phi, "grad_phi", shape=(n, nbf, 3)),
        _dptr(hess_phi, "hess_phi", shape=(n, nbf, 3, 3)),
        _dptr(bf_atom, "bf_atom", torch.int32, shape=(nbf,)),
        _dptr(vrho, "vrho", shape=(n,)), _dptr(vgamma, "vgamma", shape=(n,)),
        _dptr(f_rho_a, "f_rho_a", **dirs), _dptr(f_gamma_a, "f_gamma_a", **dirs),
        _dptr(grad_rho_a, "grad_rho_a", shape=(P, n, 3)), _dptr(w_a, "w_a", **dirs),
        _dptr(E_w, "E_w", **dirs), _dptr(U_w, "U_w", **dirs), _dptr(W_w, "W_w", **dirs),
        _dptr(EUW_gr, "EUW_gr", shape=(3, n, na, 3)), _dptr(FA, "FA", shape=(P, nbf, nbf)),
        _stream(stream))
    _check(h, st, "vv10_fock_derivative")


def vv10_nuclear_gradient(h, out, rho_t=None, grad_rho_t=None, w_t=None, stream=None) -> None:
    P = int(out.shape[0])
    n = int((rho_t if rho_t is not None else w_t).shape[1])
    st = load().vv10_nuclear_gradient(
        h, P, _dptr(rho_t, "rho_t", shape=(P, n)), _dptr(grad_rho_t, "grad_rho_t", shape=(P, n, 3)),
        _dptr(w_t, "w_t", shape=(P, n)), _dptr(out, "out", shape=(P,)), _stream(stream))
    _check(h, st, "vv10_nuclear_gradient")


def vv10_nuclear_hessian(h, prec: int, rho_a, grad_rho_a, rho_ab, grad_rho_ab, w_a, w_ab, H,
                         stream=None) -> None:
    """The nine-term nuclear Hessian (P x P, P = 3 n_atom) from the prepared points."""
    P, n = int(rho_a.shape[0]), int(rho_a.shape[1])
    st = load().vv10_nuclear_hessian(
        h, int(prec), _dptr(rho_a, "rho_a", shape=(P, n)),
        _dptr(grad_rho_a, "grad_rho_a", shape=(P, n, 3)), _dptr(rho_ab, "rho_ab", shape=(P, P, n)),
        _dptr(grad_rho_ab, "grad_rho_ab", shape=(P, P, n, 3)), _dptr(w_a, "w_a", shape=(P, n)),
        _dptr(w_ab, "w_ab", shape=(P, P, n)), _dptr(H, "H", shape=(P, P)), _stream(stream))
    _check(h, st, "vv10_nuclear_hessian")


def vv10_weight_grad(h, dEdw, stream=None) -> None:
    _check(h, load().vv10_weight_grad(h, _dptr(dEdw, "dEdw"), _stream(stream)),
           "vv10_weight_grad")


def vv10_sync(h, stream=None) -> None:
    _check(h, load().vv10_sync(h, _stream(stream)), "vv10_sync")


def vv10_set_tiles(h, what: int, rows_per_thread: int, n_split: int) -> None:
    _check(h, load().vv10_set_tiles(h, int(what), int(rows_per_thread), int(n_split)),
           "vv10_set_tiles")


def vv10_get_tiles(h, what: int) -> tuple:
    """(rows_per_thread, n_split) in effect for `what` (see vv10_set_tiles)."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(h, load().vv10_get_tiles(h, int(what), ctypes.byref(a), ctypes.byref(b)),
           "vv10_get_tiles")
    return int(a.value), int(b.value)


def vv10_autotune(h, prec: int, what: int, stream=None) -> None:
    _check(h, load().vv10_autotune(h, int(prec), int(what), _stream(stream)), "vv10_autotune")


def vv10_evaluate(h, prec: int, rho_t=None, grad_rho_t=None, f_rho_t=None, f_gamma_t=None,
                  vrho=None, vgamma=None, grad_points=None, grad_atoms=None, EUW_Bgr=None,
                  stream=None, want_energy: bool = True) -> Optional[float]:
    """Energy, potential, Hessian contraction (when trials are given) and coordinate terms
    in one call; returns the energy (synchronising) when want_energy."""
    P = 0 if rho_t is None else int(rho_t.shape[0])
    e = ctypes.c_double()
    if P:
        n = int(rho_t.shape[1])
        args = (_dptr(rho_t, "rho_t", shape=(P, n)), _dptr(grad_rho_t, "grad_rho_t", shape=(P, n, 3)),
                _dptr(f_rho_t, "f_rho_t", shape=(P, n)), _dptr(f_gamma_t, "f_gamma_t", shape=(P, n)))
    else:
        args = (None, None, None, None)
    st = load().vv10_evaluate(h, int(prec), P, args[0], args[1],
                              ctypes.byref(e) if want_energy else None, _dptr(vrho, "vrho"),
                              _dptr(vgamma, "vgamma"), args[2], args[3],
                              _dptr(grad_points, "grad_points"), _dptr(grad_atoms, "grad_atoms"),
                              _dptr(EUW_Bgr, "EUW_Bgr"), _stream(stream))
    _check(h, st, "vv10_evaluate")
    return float(e.value) if want_energy else None


def vv10_set_options(h, flags: int) -> None:
    _check(h, load().vv10_set_options(h, int(flags)), "vv10_set_options")


def vv10_set_autotune(h, flags: int) -> None:
    _check(h, load().vv10_set_autotune(h, int(flags)), "vv10_set_autotune")


def vv10_profile_enable(h, on: bool) -> None:
    _check(h, load().vv10_profile_enable(h, 1 if on else 0), "vv10_profile_enable")


def vv10_profile_phase_name(phase: int) -> str:
    return load().vv10_profile_phase_name(int(phase)).decode()


def vv10_profile_read(h) -> dict:
    """{phase name: (milliseconds, launches)}; synchronises and resets the counters."""
    import numpy as np
    ms = np.zeros(VV10_N_PHASES)
    n = np.zeros(VV10_N_PHASES, dtype=np.int64)
    _check(h, load().vv10_profile_read(h, VV10_N_PHASES, ms.ctypes.data_as(ctypes.c_void_p),
                                       n.ctypes.data_as(ctypes.c_void_p)), "vv10_profile_read")
    return {vv10_profile_phase_name(k): (float(ms[k]), int(n[k])) for k in range(VV10_N_PHASES)}


def vv10_energy_potential_noalloc(xyz, w, rho, grad_rho, prec: int, energy, vrho=None,
                                  vgamma=None, b: float = 6.0, C: float = 0.01,
                                  rho_cut: float = 1e-10, stream=None) -> None:
    """Energy (into the 1-element device tensor `energy`) and potential without any device
    allocation; for callers that may not allocate (see include/vv10.h)."""
    n = int(w.shape[0])
    st = load().vv10_energy_potential_noalloc(
        n, _dptr(xyz, "xyz", shape=(n, 3)), _dptr(w, "w", shape=(n,)),
        _dptr(rho, "rho", shape=(n,)), _dptr(grad_rho, "grad_rho", shape=(n, 3)),
        VV10Params(b, C, rho_cut), int(prec), _dptr(energy, "energy", shape=(1,)),
        _dptr(vrho, "vrho", shape=(n,)), _dptr(vgamma, "vgamma", shape=(n,)), _stream(stream))
    _check(None, st, "vv10_energy_potential_noalloc")


def _host(a, dtype):
    """Contiguous host copy (numpy) of a sequence of integers, and its address."""
    import numpy as np
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    return arr, ctypes.c_void_p(arr.ctypes.data)


def vv10_batch_prepare(h, offsets, xyz, w, rho, grad_rho, atom_of_point=None, n_atom=None,
                       b: float = 6.0, C: float = 0.01, rho_cut: float = 1e-10,
                       stream=None) -> list:
    """Prepare n_mol molecules; molecule m owns rows offsets[m]:offsets[m+1] of the
    concatenated arrays.  Returns the kept points per molecule."""
    import numpy as np
    off, off_p = _host(offsets, np.int64)
    n_mol = int(off.shape[0]) - 1
    n = int(w.shape[0])
    if n_mol < 1 or int(off[-1]) != n:
        raise ValueError("offsets must have n_mol + 1 entries ending at the number of points")
    na, na_p = _host(n_atom, np.int32) if n_atom is not None else (None, None)
    nk = np.zeros(n_mol, dtype=np.int64)
    st = load().vv10_batch_prepare(
        h, n_mol, off_p, _dptr(xyz, "xyz", shape=(n, 3)), _dptr(w, "w", shape=(n,)),
        _dptr(rho, "rho", shape=(n,)), _dptr(grad_rho, "grad_rho", shape=(n, 3)),
        _dptr(atom_of_point, "atom_of_point", torch.int32, (n,)), na_p,
        VV10Params(b, C, rho_cut), ctypes.c_void_p(nk.ctypes.data), _stream(stream))
    _check(h, st, "vv10_batch_prepare")
    return [int(x) for x in nk]


def vv10_batch_energy_potential(h, prec: int, energies, vrho=None, vgamma=None,
                                stream=None) -> None:
    """Energies (device tensor, one per molecule) and the concatenated potential."""
    st = load().vv10_batch_energy_potential(h, int(prec), _dptr(energies, "energies"),
                                            _dptr(vrho, "vrho"), _dptr(vgamma, "vgamma"),
                                            _stream(stream))
    _check(h, st, "vv10_batch_energy_potential")


def vv10_batch_hessian_contract(h, prec: int, P, rho_t, grad_rho_t, f_rho_t, f_gamma_t,
                                stream=None) -> None:
    """P[m] trials per molecule; rho_t, f_rho_t, f_gamma_t: 1-D concatenations of the
    molecules' [P[m], n_m] blocks, grad_rho_t of their [P[m], n_m, 3] blocks."""
    import numpy as np
    Pa, P_p = _host(P, np.int32)
    tot = int(rho_t.numel())
    st = load().vv10_batch_hessian_contract(
        h, int(prec), P_p, _dptr(rho_t, "rho_t", shape=(tot,)),
        _dptr(grad_rho_t, "grad_rho_t", shape=(tot, 3)), _dptr(f_rho_t, "f_rho_t", shape=(tot,)),
        _dptr(f_gamma_t, "f_gamma_t", shape=(tot,)), _stream(stream))
    _check(h, st, "vv10_batch_hessian_contract")


def vv10_batch_run(h, prec: int, P, rho_t, grad_rho_t, energies, vrho, vgamma, f_rho_t,
                   f_gamma_t, stream=None) -> None:
    """Energy, potential and Hessian contraction of the prepared batch; repeated calls with
    the same tensors replay one recorded CUDA graph."""
    import numpy as np
    Pa, P_p = _host(P, np.int32)
    tot = int(rho_t.numel())
    st = load().vv10_batch_run(
        h, int(prec), P_p, _dptr(rho_t, "rho_t", shape=(tot,)),
        _dptr(grad_rho_t, "grad_rho_t", shape=(tot, 3)), _dptr(energies, "energies"),
        _dptr(vrho, "vrho"), _dptr(vgamma, "vgamma"), _dptr(f_rho_t, "f_rho_t", shape=(tot,)),
        _dptr(f_gamma_t, "f_gamma_t", shape=(tot,)), _stream(stream))
    _check(h, st, "vv10_batch_run")


def vv10_debug_inject(h, what: int, value: int) -> None:
    _check(h, load().vv10_debug_inject(h, int(what), int(value)), "vv10_debug_inject")


# ---------------------------------------------------------------- convenience owner

class VV10:
    """Owns a handle and allocates outputs; every computation is a library call."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        self.h = vv10_create(self.device)
        self.n = 0
        self.n_atom = 0
        self.n_kept = 0

    def close(self):
        if self.h is not None:
            vv10_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def prepare(self, xyz, w, rho, grad_rho, atom_of_point=None, n_atom=0, b=6.0, C=0.01,
                rho_cut=1e-10, stream=None) -> int:
        self.n = int(w.shape[0])
        self.n_atom = int(n_atom)
        self.n_kept = vv10_prepare_points(self.h, xyz, w, rho, grad_rho, atom_of_point, n_atom,
                                          b, C, rho_cut, stream)
        return self.n_kept

    def energy_potential(self, prec=VV10_FP64, stream=None, want_energy=True):
        dev = torch.device("cuda", self.device)
        vrho = torch.empty(self.n, dtype=torch.float64, device=dev)
        vgamma = torch.empty(self.n, dtype=torch.float64, device=dev)
        e = vv10_energy_potential(self.h, prec, vrho, vgamma, stream, want_energy)
        return e, vrho, vgamma

    def hessian_contract(self, rho_t, grad_rho_t, prec=VV10_FP64, stream=None):
        fr = torch.empty_like(rho_t)
        fg = torch.empty_like(rho_t)
        vv10_hessian_contract(self.h, prec, rho_t, grad_rho_t, fr, fg, stream)
        return fr, fg

    def hessian_vector_product(self, rho_t, grad_rho_t, prec=VV10_FP64, stream=None):
        hr = torch.empty_like(rho_t)
        hg = torch.empty_like(grad_rho_t)
        vv10_hessian_vector_product(self.h, prec, rho_t, grad_rho_t, hr, hg, stream)
        return hr, hg

    def coord_grad(self, prec=VV10_FP64, atoms=True, resolved=False, stream=None):
        dev = torch.device("cuda", self.device)
        gp = torch.empty(self.n, 3, dtype=torch.float64, device=dev)
        ga = torch.empty(self.n_atom, 3, dtype=torch.float64, device=dev) if atoms and self.n_atom else None
        euw = (torch.empty(3, self.n, self.n_atom, 3, dtype=torch.float64, device=dev)
               if resolved and self.n_atom else None)
        vv10_coord_grad(self.h, prec, gp, ga, euw, stream)
        return gp, ga, euw

    def coord_hessian(self, prec=VV10_FP64, points=False, stream=None):
        """Grid-grid nuclear Hessian blocks E^{AB}_{gr,gr} as (n_atom, n_atom, 3, 3) and, when
        points is set, D_i^B as (n, n_atom, 3, 3); needs atom labels at prepare time."""
        dev = torch.device("cuda", self.device)
        f64 = dict(dtype=torch.float64, device=dev)
        E = torch.empty(self.n_atom, self.n_atom, 3, 3, **f64)
        D = torch.empty(self.n, self.n_atom, 3, 3, **f64) if points else None
        vv10_coord_hessian(self.h, prec, E, D, stream)
        return E, D

    def nuclear_gradient(self, rho_t=None, grad_rho_t=None, w_t=None, stream=None):
        """E^A_G + E^A_w along the P directions (P,), after an energy call."""
        ref = rho_t if rho_t is not None else w_t
        out = torch.empty(ref.shape[0], dtype=torch.float64, device=ref.device)
        vv10_nuclear_gradient(self.h, out, rho_t, grad_rho_t, w_t, stream)
        return out

    def nuclear_hessian(self, rho_a, grad_rho_a, rho_ab, grad_rho_ab, w_a, w_ab, prec=VV10_FP64,
                        stream=None):
        """The nine-term VV10 nuclear Hessian (3 n_atom x 3 n_atom)."""
        P = rho_a.shape[0]
        H = torch.empty(P, P, dtype=torch.float64, device=rho_a.device)
        vv10_nuclear_hessian(self.h, prec, rho_a, grad_rho_a, rho_ab, grad_rho_ab, w_a, w_ab, H,
                             stream)
        return H

    def fock_matrix(self, phi, grad_phi, vrho, vgamma, stream=None):
        """The VV10 Fock matrix (nbf x nbf) from f^rho, f^gamma and the basis on the grid."""
        F = torch.empty(phi.shape[1], phi.shape[1], dtype=torch.float64, device=phi.device)
        vv10_fock_matrix(self.h, phi, grad_phi, vrho, vgamma, F, stream)
        return F

    def orbital_hessian(self, phi, grad_phi, f_rho_t, f_gamma_t, grad_rho_t, vgamma, stream=None):
        """G^t (P x nbf x nbf) from the Hessian contraction and the basis on the grid."""
        G = torch.empty(f_rho_t.shape[0], phi.shape[1], phi.shape[1], dtype=torch.float64,
                        device=phi.device)
        vv10_orbital_hessian(self.h, phi, grad_phi, f_rho_t, f_gamma_t, grad_rho_t, vgamma, G, stream)
        return G

    def fock_derivative(self, phi, grad_phi, hess_phi, bf_atom, vrho, vgamma, f_rho_a, f_gamma_a,
                        grad_rho_a, w_a, E_w, U_w, W_w, EUW_gr, stream=None):
        """F^A (3 n_atom x nbf x nbf), the nuclear derivative of the Fock matrix, from the
        potential, the Hessian contraction with the nuclear trials, the weight-derivative and
        the atom-resolved sums and the basis (values, gradients, Hessians) on the grid."""
        FA = torch.empty(3 * self.n_atom, phi.shape[1], phi.shape[1], dtype=torch.float64,
                         device=phi.device)
        vv10_fock_derivative(self.h, phi, grad_phi, hess_phi, bf_atom, vrho, vgamma, f_rho_a,
                             f_gamma_a, grad_rho_a, w_a, E_w, U_w, W_w, EUW_gr, FA, stream)
        return FA

    def energy(self, prec=VV10_FP64, stream=None) -> float:
        """E alone, from the unordered pairs (half the pair evaluations)."""
        return vv10_energy(self.h, prec, stream)

    def weight_response(self, w_t, prec=VV10_FP64, stream=None):
        """E_i^{Bw}, U_i^{Bw}, W_i^{Bw} for the weight directions w_t (P x n): three P x n."""
        E, U, W = (torch.empty_like(w_t) for _ in range(3))
        vv10_weight_response(self.h, prec, w_t, E, U, W, stream)
        return E, U, W

    def evaluate(self, prec=VV10_FP64, rho_t=None, grad_rho_t=None, resolved=False, stream=None):
        """Energy, potential, Hessian contraction (when trials are given) and coordinate terms
        in one vv10_evaluate call: (energy, vrho, vgamma, f_rho_t, f_gamma_t, grad_points,
        grad_atoms, EUW_Bgr); atom outputs need atom labels at prepare time."""
        dev = torch.device("cuda", self.device)
        f64 = dict(dtype=torch.float64, device=dev)
        vrho, vgamma = torch.empty(self.n, **f64), torch.empty(self.n, **f64)
        fr = torch.empty_like(rho_t) if rho_t is not None else None
        fg = torch.empty_like(rho_t) if rho_t is not None else None
        gp = torch.empty(self.n, 3, **f64)
        ga = torch.empty(self.n_atom, 3, **f64) if self.n_atom else None
        euw = torch.empty(3, self.n, self.n_atom, 3, **f64) if resolved and self.n_atom else None
        e = vv10_evaluate(self.h, prec, rho_t, grad_rho_t, fr, fg, vrho, vgamma, gp, ga, euw, stream)
        return e, vrho, vgamma, fr, fg, gp, ga, euw

    def weight_grad(self, stream=None):
        out = torch.empty(self.n, dtype=torch.float64, device=torch.device("cuda", self.device))
        vv10_weight_grad(self.h, out, stream)
        return out
