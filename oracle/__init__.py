"""FP64 CPU oracle for the VV10 quadrature sums (arXiv 2208.14639, Sec. II).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` and by the
benchmark's CPU-baseline leg, never by the library.  It shares no code with the CUDA
path; both sides only share the seeded input generator.

The arithmetic lives in ``vv10_oracle.c`` (plain C, FP64, Neumaier-compensated sums,
OpenMP over rows); this module compiles it with gcc (``-O2 -fopenmp``, no fast-math,
no FMA contraction) and wraps it with ctypes.  Every wrapper takes FP64 numpy arrays in
original point indexing; ``rows`` selects a subset of output rows (full j sums), which
is how large grids are checked on sampled outputs.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import platform
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vv10_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, f"liborc_vv10_{platform.machine()}.so")
_lock = threading.Lock()
_lib = None

B_DEFAULT = 6.0
C_DEFAULT = 0.01
RHO_CUT_DEFAULT = 1e-10


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    _lib = _configure(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def planted(old: str, new: str, tag: str):
    """Test infrastructure for checking the pins themselves: inside the block every wrapper of
    this module runs a copy of vv10_oracle.c in which the text ``old`` (which must occur exactly
    once) is replaced by ``new``, i.e. with one planted mistake.  The copy is compiled with the
    same flags under _build/."""
    global _lib
    with open(_SRC) as f:
        src = f.read()
    if src.count(old) != 1:
        raise ValueError(f"planted mistake {tag!r}: the text to replace occurs {src.count(old)} times")
    keep = _load()
    os.makedirs(_BUILD, exist_ok=True)
    csrc = os.path.join(_BUILD, f"planted_{tag}.c")
    so = os.path.join(_BUILD, f"liborc_planted_{tag}_{platform.machine()}.so")
    with open(csrc, "w") as f:
        f.write(src.replace(old, new))
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-ffp-contract=off",
                    "-o", so, csrc, "-lm"], check=True)
    with _lock:
        _lib = _configure(ctypes.CDLL(so))
    try:
        yield
    finally:
        with _lock:
            _lib = keep


def _configure(lib):
    D = ctypes.c_double
    I64 = ctypes.c_int64
    I32 = ctypes.c_int32
    P = ctypes.c_void_p
    lib.orc_beta.restype = D
    lib.orc_beta.argtypes = [D]
    lib.orc_phi.restype = D
    lib.orc_phi.argtypes = [D, D, D, D, D]
    lib.orc_point_props.restype = None
    lib.orc_point_props.argtypes = [I64, P, P, D, D, P]
    lib.orc_energy.argtypes = [I64, P, P, P, P, D, D, D, P]
    lib.orc_pair_sums.argtypes = [I64, P, P, P, P, D, D, D, I64, P, P]
    lib.orc_potential.argtypes = [I64, P, P, P, P, D, D, D, I64, P, P, P, P]
    lib.orc_hessian_contract.argtypes = [I64, P, P, P, P, D, D, D, I32, P, P, I64, P, P, P]
    lib.orc_point_grad.argtypes = [I64, P, P, P, P, D, D, D, I64, P, P]
    lib.orc_atom_grad.argtypes = [I64, P, P, P, P, P, I32, D, D, D, P]
    lib.orc_atom_resolved.argtypes = [I64, P, P, P, P, P, I32, D, D, D, I64, P, P, P, P]
    lib.orc_point_coord_hessian.argtypes = [I64, P, P, P, P, P, I32, D, D, D, I64, P, P]
    lib.orc_coord_hessian.argtypes = [I64, P, P, P, P, P, I32, D, D, D, P]
    lib.orc_weight_response.argtypes = [I64, P, P, P, P, D, D, D, I32, P, I64, P, P, P, P]
    lib.orc_num_threads.restype = ctypes.c_int
    lib.orc_set_num_threads.argtypes = [ctypes.c_int]
    for name in ("orc_energy", "orc_pair_sums", "orc_potential", "orc_hessian_contract",
                 "orc_point_grad", "orc_atom_grad", "orc_atom_resolved", "orc_point_coord_hessian",
                 "orc_coord_hessian", "orc_weight_response"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _rows(rows, n):
    if rows is None:
        return None, n
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    if r.size and (r.min() < 0 or r.max() >= n):
        raise IndexError("row index out of range")
    return r, int(r.size)


def _check(rc: int, what: str):
    if rc != 0:
        raise MemoryError(f"oracle {what} failed (rc={rc})")


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(k: int) -> None:
    _load().orc_set_num_threads(int(k))


def beta(b: float = B_DEFAULT) -> float:
    return float(_load().orc_beta(b))


def phi(om_i, ka_i, om_j, ka_j, R2) -> float:
    return float(_load().orc_phi(om_i, ka_i, om_j, ka_j, R2))


POINT_FIELDS = ("gamma", "omega", "kappa", "omega_rho", "omega_gamma", "kappa_rho",
                "omega_rhorho", "omega_rhogamma", "omega_gammagamma", "kappa_rhorho")


def point_props(rho, grad_rho, b=B_DEFAULT, C=C_DEFAULT) -> dict:
    rho = _f64(rho)
    grad = _f64(grad_rho).reshape(-1, 3)
    out = np.zeros((rho.size, 11))
    _load().orc_point_props(rho.size, _ptr(rho), _ptr(grad), b, C, _ptr(out))
    return {k: out[:, q].copy() for q, k in enumerate(POINT_FIELDS)}


def _sys(coords, weights, rho, grad_rho):
    xyz = _f64(coords).reshape(-1, 3)
    w = _f64(weights)
    r = _f64(rho)
    g = _f64(grad_rho).reshape(-1, 3)
    n = w.size
    if not (xyz.shape[0] == n and r.size == n and g.shape[0] == n):
        raise ValueError("inconsistent point arrays")
    return n, xyz, w, r, g


def energy(coords, weights, rho, grad_rho, b=B_DEFAULT, C=C_DEFAULT,
           rho_cut=RHO_CUT_DEFAULT) -> float:
    """E^VV10 from the quadrature definition (double loop)."""
    n, xyz, w, r, g = _sys(coords, weights, rho, grad_rho)
    e = np.zeros(1)
    _check(_load().orc_energy(n, _ptr(xyz), _ptr(w), _ptr(r), _ptr(g), b, C, rho_cut,
                              _ptr(e)), "energy")
    return float(e[0])


def pair_sums(coords, weights, rho, grad_rho, rows=None, b=B_DEFAULT, C=C_DEFAULT,
              rho_cut=RHO_CUT_DEFAULT) -> dict:
    """Row sums E_i, U_i, W_i, A_i, B_i, C_i (j = i included)."""
    n, xyz, w, r, g = _sys(coords, weights, rho, grad_rho)
    rr, nr = _rows(rows, n)
    out = np.zeros((nr, 6))
    _check(_load().orc_pair_sums(n, _ptr(xyz), _ptr(w), _ptr(r), _ptr(g), b, C, rho_cut, nr,
                                 _ptr(rr), _ptr(out)), "pair_sums")
    return {k: out[:, q].copy() for q, k in enumerate("EUWABC")}


def potential(coords, weights, rho, grad_rho, rows=None, b=B_DEFAULT, C=C_DEFAULT,
              rho_cut=RHO_CUT_DEFAULT):
    """(energy or None, vrho = f^rho, vgamma = f^gamma).  Energy only when rows is None."""
    n, xyz, w, r, g = _sys(coords, weights, rho, grad_rho)
    rr, nr = _rows(rows, n)
    vr = np.zeros(nr)
    vg = np.zeros(nr)
    e = np.zeros(1)
    _check(_load().orc_potential(n, _ptr(xyz), _ptr(w), _ptr(r), _ptr(g), b, C, rho_cut, nr,
                                 _ptr(rr), _ptr(vr), _ptr(vg),
                                 _ptr(e) if rr is None else None), "potential")
    return (float(e[0]) if rr is None else None), vr, vg


def hessian_contract(coords, weights, rho, grad_rho, rho_t, grad_rho_t, rows=None,
                     b=B_DEFAULT, C=C_DEFAULT, rho_cut=RHO_CUT_DEFAULT):
    """(f^{rho,t}, f^{gamma,t}), each P x n_rows, from the printed pair coefficients."""
    n, xyz, w, r, g = _sys(coords, weights, rho, grad_rho)
    rt = _f64(rho_t).reshape(-1, n)
    P = rt.shape[0]
    gt = _f64(grad_rho_t).reshape(P, n, 3)
    rr, nr = _rows(rows, n)
    fr = np.zeros((P, nr))
    fg = np.zeros((P, nr))
    _check(_load().orc_hessian_contract(n, _ptr(xyz), _ptr(w), _ptr(r), _ptr(g), b, C, rho_cut,
                                        P, _ptr(rt), _ptr(gt), nr, _ptr(rr), _ptr(fr), _ptr(fg)),
           "hessian_contract")
    return fr, fg


def point_grad(coords, weights, rho, grad_rho, rows=None, b=B_DEFAULT, C=C_DEFAULT,
               rho_cut=RHO_CUT_DEFAULT) -> np.ndarray:
    """dE/dr_i for every (selected) grid point, n_rows x 3."""
    n, xyz, w, r, g = _sys(coords, weights, rho, grad_rho)
    rr, nr = _rows(rows, n)
    out = np.zeros((nr, 3))
    _check(_load().orc_point_grad(n, _ptr(xyz), _ptr(w), _ptr(r), _ptr(g), b, C, rho_cut, nr,
                                  _ptr(rr), _ptr(out)), "point_grad")
    return out


def atom_grad(coords, weights, rho, grad_rho, atom_of_point, n_atom, b=B_DEFAULT,
              C=C_DEFAULT, rho_cut=RHO_CUT_DEFAULT) -> np.ndarray:
    """E^A_gr (first form of Eq. grad_gr), n_atom x 3."""
    n, xyz, w, r, g = _sys(coords, weights, rho, grad_rho)
    aop = np.ascontiguousarray(np.asarray(atom_of_point, dtype=np.int32))
    out = np.zeros((n_atom, 3))
    _check(_load().orc_atom_grad(n, _ptr(xyz), _ptr(w), _ptr(r), _ptr(g), _ptr(aop), n_atom, b,
                                 C, rho_cut, _ptr(out)), "atom_grad")
    return out


def atom_resolved(coords, weights, rho, grad_rho, atom_of_point, n_atom, rows=None,
                  b=B_DEFAULT, C=C_DEFAULT, rho_cut=RHO_CUT_DEFAULT):
    """(E^{Bgr}, U^{Bgr}, W^{Bgr}), each n_rows x n_atom x 3 (Eq. EiBgr and after)."""
    n, xyz, w, r, g = _sys(coords, weights, rho, grad_rho)
    aop = np.ascontiguousarray(np.asarray(atom_of_point, dtype=np.int32))
    rr, nr = _rows(rows, n)
    oE = np.zeros((nr, n_atom, 3))
    oU = np.zeros((nr, n_atom, 3))
    oW = np.zeros((nr, n_atom, 3))
    _check(_load().orc_atom_resolved(n, _ptr(xyz), _ptr(w), _ptr(r), _ptr(g), _ptr(aop), n_atom,
                                     b, C, rho_cut, nr, _ptr(rr), _ptr(oE), _ptr(oU), _ptr(oW)),
           "atom_resolved")
    return oE, oU, oW


def point_coord_hessian(coords, weights, rho, grad_rho, atom_of_point, n_atom, rows=None,
                        b=B_DEFAULT, C=C_DEFAULT, rho_cut=RHO_CUT_DEFAULT) -> np.ndarray:
    """D_i^B (Sec. II.B), n_rows x n_atom x 3 x 3, zero for B = atom(i)."""
    n, xyz, w, r, g = _sys(coords, weights, rho, grad_rho)
    aop = np.ascontiguousarray(np.asarray(atom_of_point, dtype=np.int32))
    rr, nr = _rows(rows, n)
    out = np.zeros((nr, n_atom, 3, 3))
    _check(_load().orc_point_coord_hessian(n, _ptr(xyz), _ptr(w), _ptr(r), _ptr(g), _ptr(aop),
                                           n_atom, b, C, rho_cut, nr, _ptr(rr), _ptr(out)),
           "point_coord_hessian")
    return out


def coord_hessian(coords, weights, rho, grad_rho, atom_of_point, n_atom, b=B_DEFAULT,
                  C=C_DEFAULT, rho_cut=RHO_CUT_DEFAULT) -> np.ndarray:
    """E^{AB}_{gr,gr} (Sec. II.B), n_atom x n_atom x 3 x 3: the grid-grid block of the
    nuclear Hessian (points move with their atoms; rho, grad rho and w held fixed)."""
    n, xyz, w, r, g = _sys(coords, weights, rho, grad_rho)
    aop = np.ascontiguousarray(np.asarray(atom_of_point, dtype=np.int32))
    out = np.zeros((n_atom, n_atom, 3, 3))
    _check(_load().orc_coord_hessian(n, _ptr(xyz), _ptr(w), _ptr(r), _ptr(g), _ptr(aop), n_atom,
                                     b, C, rho_cut, _ptr(out)), "coord_hessian")
    return out


def weight_response(coords, weights, rho, grad_rho, w_t, rows=None, b=B_DEFAULT, C=C_DEFAULT,
                    rho_cut=RHO_CUT_DEFAULT):
    """E_i^{Bw}, U_i^{Bw}, W_i^{Bw} (Sec. II.B) for P weight directions w_t (P x n, e.g. the
    components of w^B): three arrays P x n_rows."""
    n, xyz, w, r, g = _sys(coords, weights, rho, grad_rho)
    wt = _f64(w_t).reshape(-1, n)
    P = wt.shape[0]
    rr, nr = _rows(rows, n)
    out = [np.zeros((P, nr)) for _ in range(3)]
    _check(_load().orc_weight_response(n, _ptr(xyz), _ptr(w), _ptr(r), _ptr(g), b, C, rho_cut, P,
                                       _ptr(wt), nr, _ptr(rr), *[_ptr(o) for o in out]),
           "weight_response")
    return tuple(out)


# ---------------------------------------------------------------- AO-side assembly (numpy)

def fock_matrix(weights, grad_rho, vrho, vgamma, phi, grad_phi) -> np.ndarray:
    """The VV10 contribution to the Fock matrix (Sec. II.A):
    F_mu_nu = sum_i w_i [f^rho_i phi_mu,i phi_nu,i
                         + 2 f^gamma_i grad rho_i . (phi_nu,i grad phi_mu,i + phi_mu,i grad phi_nu,i)]
    with f^rho = vrho, f^gamma = vgamma (per unit weight, zero at dropped points).
    phi: n x nbf, grad_phi: n x nbf x 3.  Returns nbf x nbf."""
    w = _f64(weights)
    s = w * _f64(vrho)
    v = 2.0 * (w * _f64(vgamma))[:, None] * _f64(grad_rho).reshape(-1, 3)
    phi = _f64(phi)
    vdphi = np.einsum("nk,nmk->nm", v, _f64(grad_phi))  # v_i . grad phi_mu,i
    return phi.T @ (s[:, None] * phi) + vdphi.T @ phi + phi.T @ vdphi


def orbital_hessian(weights, grad_rho, vgamma, f_rho_t, f_gamma_t, grad_rho_t, phi,
                    grad_phi) -> np.ndarray:
    """The contracted orbital Hessian (Sec. II.B):
    G^t_mu_nu = sum_i w_i [f^{rho,t}_i phi_mu phi_nu
                           + 2 (f^{gamma,t}_i grad rho_i + f^gamma_i grad rho^t_i)
                             . (phi_nu grad phi_mu + phi_mu grad phi_nu)]
    for each trial t (f_rho_t, f_gamma_t: P x n; grad_rho_t: P x n x 3).  Returns P x nbf x nbf."""
    w = _f64(weights)
    g = _f64(grad_rho).reshape(-1, 3)
    fr, fg = _f64(f_rho_t), _f64(f_gamma_t)
    gt = _f64(grad_rho_t).reshape(fr.shape[0], -1, 3)
    phi, dphi = _f64(phi), _f64(grad_phi)
    vg = _f64(vgamma)
    out = np.zeros((fr.shape[0], phi.shape[1], phi.shape[1]))
    for t in range(fr.shape[0]):
        s = w * fr[t]
        v = 2.0 * w[:, None] * (fg[t][:, None] * g + vg[:, None] * gt[t])
        vdphi = np.einsum("nk,nmk->nm", v, dphi)
        out[t] = phi.T @ (s[:, None] * phi) + vdphi.T @ phi + phi.T @ vdphi
    return out


# ---------------------------------------------------------------- nuclear Hessian (numpy)

def nuclear_hessian(weights, rho, grad_rho, kept, kappa_rho, omega_rho, omega_gamma, vrho, vgamma,
                    E, rho_a, grad_rho_a, rho_ab, grad_rho_ab, w_a, w_ab, E_w, U_w, W_w,
                    E_gr, U_gr, W_gr, f_rho_a, f_gamma_a, H_grgr) -> np.ndarray:
    """The nine terms of the VV10 nuclear Hessian (Sec. II.B, Eq. E_hess):
      E^{ab} = E_GG + E_ww + E_grgr + E_Gw + E_Gw^T + E_Ggr + E_Ggr^T + E_wgr + E_wgr^T
    with, over the kept points i (a, b = 3 A + c):
      E_GG  = sum w [f^rho rho^{ab} + f^gamma gamma^{ab} + rho^a f^{rho,b} + gamma^a f^{gamma,b}]
      E_ww  = sum w^{ab} rho (beta + E) + sum w^a rho E^{bw}
      E_wgr = sum w^a rho E^{b,gr}
      E_Gw  = sum w^b (f^rho rho^a + f^gamma gamma^a)
              + sum w rho^a [E^{bw} + rho (kappa' U^{bw} + omega_rho W^{bw})]
              + sum w gamma^a rho omega_gamma W^{bw}
      E_Ggr = sum w rho^a [E^{b,gr} + rho (kappa' U^{b,gr} + omega_rho W^{b,gr})]
              + sum w gamma^a rho omega_gamma W^{b,gr}
    gamma^a = 2 grad rho . grad rho^a and gamma^{ab} = 2 (grad rho^a . grad rho^b + grad rho .
    grad rho^{ab}) are full derivatives of gamma; f^{rho,b}, f^{gamma,b} are the Hessian
    contraction with the trial (rho^b, grad rho^b); E = the row sums E_i (beta not included);
    H_grgr = E^{AB}_{gr,gr} flattened to (3 N_atom, 3 N_atom).  Per-point arrays are over all
    n points (caller order), direction arrays (P, n), second-derivative arrays (P, P, n).
    Returns (P, P)."""
    m = np.asarray(kept, dtype=float)
    w = _f64(weights) * m
    rho, g = _f64(rho), _f64(grad_rho).reshape(-1, 3)
    mask = lambda a: np.where(m > 0, np.nan_to_num(_f64(a)), 0.0)
    kr, omr, omg = mask(kappa_rho), mask(omega_rho), mask(omega_gamma)
    vr, vg, E = mask(vrho), mask(vgamma), mask(E)
    ra, ga = _f64(rho_a), _f64(grad_rho_a)
    gam_a = 2.0 * np.einsum("nd,pnd->pn", g, ga)
    gam_ab = 2.0 * (np.einsum("and,bnd->abn", ga, ga) + np.einsum("nd,abnd->abn", g, _f64(grad_rho_ab)))
    wa, wab = _f64(w_a), _f64(w_ab)
    rb = beta()
    EGG = (np.einsum("n,abn->ab", w * vr, _f64(rho_ab)) + np.einsum("n,abn->ab", w * vg, gam_ab)
           + np.einsum("n,an,bn->ab", w, ra, _f64(f_rho_a))
           + np.einsum("n,an,bn->ab", w, gam_a, _f64(f_gamma_a)))
    Eww = (np.einsum("abn,n->ab", wab, m * rho * (rb + E))
           + np.einsum("an,n,bn->ab", wa, m * rho, _f64(E_w)))
    Ewgr = np.einsum("an,n,bn->ab", wa, m * rho, _f64(E_gr))
    EGw = (np.einsum("bn,an->ab", wa * m, vr * ra + vg * gam_a)
           + np.einsum("n,an,bn->ab", w, ra, _f64(E_w) + rho * (kr * _f64(U_w) + omr * _f64(W_w)))
           + np.einsum("n,an,bn->ab", w, gam_a, rho * omg * _f64(W_w)))
    EGgr = (np.einsum("n,an,bn->ab", w, ra, _f64(E_gr) + rho * (kr * _f64(U_gr) + omr * _f64(W_gr)))
            + np.einsum("n,an,bn->ab", w, gam_a, rho * omg * _f64(W_gr)))
    return EGG + Eww + _f64(H_grgr) + EGw + EGw.T + EGgr + EGgr.T + Ewgr + Ewgr.T


# ------------------------------------------------------- nuclear derivative of F (numpy)

def fock_derivative(weights, rho, grad_rho, kept, kappa_rho, omega_rho, omega_gamma, vrho, vgamma,
                    phi, grad_phi, hess_phi, bf_atom, atom_of_point, grad_rho_a, w_a, E_w, U_w,
                    W_w, E_gr, U_gr, W_gr, f_rho_a, f_gamma_a) -> np.ndarray:
    """The nuclear derivative of the VV10 Fock matrix (Sec. II.B), F^a = F^a_G + F^a_gr + F^a_w,
    over the kept points i (a = 3 A + c), with B_mu_nu = grad(phi_mu phi_nu):
      F_G  = sum w [f^rho d_a(phi_mu phi_nu) + 2 f^gamma d_a(grad rho . B_mu_nu)]
             + sum w [phi_mu phi_nu f^{rho,a} + 2 grad rho . B_mu_nu f^{gamma,a}]
      F_gr = sum w phi_mu phi_nu [E^{a,gr} + rho (kappa' U^{a,gr} + omega_rho W^{a,gr})]
             + 2 sum w grad rho . B_mu_nu rho omega_gamma W^{a,gr}
      F_w  = sum w^a [f^rho phi_mu phi_nu + 2 f^gamma grad rho . B_mu_nu]
             + sum w phi_mu phi_nu [E^{aw} + rho (kappa' U^{aw} + omega_rho W^{aw})]
             + 2 sum w grad rho . B_mu_nu rho omega_gamma W^{aw}
    The basis functions and the grid points move with their atoms: phi^a_mu(i) = (delta(A, owner
    of i) - delta(A, atom of mu)) d phi_mu / d x_c, and d_a(grad rho . B) = grad rho^a . B +
    grad rho . d_a B.  f^{rho,a}, f^{gamma,a}: the Hessian contraction with the trial (rho^a,
    grad rho^a); E/U/W^{aw} the weight-derivative sums along w^a; E/U/W^{a,gr} the atom-resolved
    sums.  phi (n, nbf), grad_phi (n, nbf, 3), hess_phi (n, nbf, 3, 3), bf_atom (nbf,),
    direction arrays (P, n) or (P, n, 3).  Returns (P, nbf, nbf)."""
    m = np.asarray(kept, dtype=float)
    w = _f64(weights) * m
    rho, g = _f64(rho), _f64(grad_rho).reshape(-1, 3)
    mask = lambda a: np.where(m > 0, np.nan_to_num(_f64(a)), 0.0)
    kr, omr, omg = mask(kappa_rho), mask(omega_rho), mask(omega_gamma)
    vr, vg = mask(vrho), mask(vgamma)
    phi, dphi, d2phi = _f64(phi), _f64(grad_phi), _f64(hess_phi)
    own = np.asarray(atom_of_point)
    bfa = np.asarray(bf_atom)
    ga, wa = _f64(grad_rho_a), _f64(w_a)
    Ew, Uw, Ww = mask(E_w), mask(U_w), mask(W_w)
    Eg, Ug, Wg = mask(E_gr), mask(U_gr), mask(W_gr)
    fra, fga = mask(f_rho_a), mask(f_gamma_a)

    def S(c):  # sum_i c_i phi_mu phi_nu
        return (phi * c[:, None]).T @ phi

    def D(v):  # sum_i v_i . B_mu_nu
        X = np.einsum("nd,nmd->nm", v, dphi)
        return X.T @ phi + phi.T @ X

    P = fra.shape[0]
    out = np.zeros((P, phi.shape[1], phi.shape[1]))
    b = 2.0 * (w * vg)[:, None] * g                       # 2 w f^gamma grad rho
    bdphi = np.einsum("nd,nmd->nm", b, dphi)
    for a in range(P):
        A, c = divmod(a, 3)
        sig = (own == A).astype(float)[:, None] - (bfa == A).astype(float)[None, :]
        pa = sig * dphi[:, :, c]                           # phi^a
        gpa = sig[..., None] * d2phi[:, :, c, :]           # grad phi^a
        wfp = (w * vr)[:, None] * phi
        bga = np.einsum("nd,nmd->nm", b, gpa)
        FG = (pa.T @ wfp + wfp.T @ pa
              + D(2.0 * (w * vg)[:, None] * ga[a])
              + bga.T @ phi + pa.T @ bdphi + bdphi.T @ pa + phi.T @ bga
              + S(w * fra[a]) + D(2.0 * (w * fga[a])[:, None] * g))
        Fgr = (S(w * (Eg[a] + rho * (kr * Ug[a] + omr * Wg[a])))
               + D(2.0 * (w * rho * omg * Wg[a])[:, None] * g))
        Fw = (S(wa[a] * m * vr) + D(2.0 * (wa[a] * m * vg)[:, None] * g)
              + S(w * (Ew[a] + rho * (kr * Uw[a] + omr * Ww[a])))
              + D(2.0 * (w * rho * omg * Ww[a])[:, None] * g))
        out[a] = FG + Fgr + Fw
    return out
