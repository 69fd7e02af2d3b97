"""torch.autograd wrapper of the VV10 energy, with first and second derivatives.

    E = vv10_energy(rho, grad_rho, coords, weights, precision="fp64")

is differentiable: the backward gives (Sec. II.A)
    dE/d rho_i      = w_i f^rho_i
    dE/d grad rho_i = 2 w_i f^gamma_i grad rho_i
    dE/d r_i        = -2 w_i rho_i sum_j w_j rho_j Phi_ij D_ij (r_i - r_j)   (Eq. grad_gr, per point)
    dE/d w_i        = rho_i (beta + E_i)
and differentiating the first two again (double backward, e.g. a Hessian-vector product)
gives, for a direction (d rho, d grad rho) (Sec. II.B, Eq. frhot):
    d(dE/d rho_i)      = w_i f^{rho,t}_i
    d(dE/d grad rho_i) = 2 w_i (f^{gamma,t}_i grad rho_i + f^gamma_i d grad rho_i)
with rho^t = d rho, grad rho^t = d grad rho; by symmetry of the Hessian this is also the
vector-Jacobian product of the first derivatives.  For many directions at once, vv10_hvp
contracts a (P, n) batch in one call (batched autograd cotangents are rejected).
Second derivatives that involve the coordinates or the weights are not provided (they raise).

Every number comes from the CUDA library through the C ABI; this module only routes tensors.
"""
from __future__ import annotations

import threading
from typing import Optional

import torch

from . import vv10 as _vv

_PREC = {"fp64": _vv.VV10_FP64, "mixed": _vv.VV10_MIXED_TF32X3, "tf32x3": _vv.VV10_MIXED_TF32X3,
         "f16x3": _vv.VV10_MIXED_F16X3, "fp64tc": _vv.VV10_FP64_TC}


class _DeviceHandle:
    """One library handle per device, shared by all energies evaluated on it; the handle's
    prepared point set belongs to the most recent _State that (re)prepared it.  Each slot
    carries a re-entrant lock: re-preparing the handle and the library calls that read the
    prepared points happen under it, so energies and Hessian-vector products taken from
    several threads on one device do not interleave (their work is queued in that order on
    the calling threads' streams)."""

    _lock = threading.Lock()
    _handles = {}

    @classmethod
    def get(cls, device: int):
        with cls._lock:
            h = cls._handles.get(device)
            if h is None:
                _vv.load(build_if_missing=True)
                h = cls._handles[device] = {"h": _vv.vv10_create(device), "owner": None,
                                            "lock": threading.RLock()}
            return h


class _State:
    """Inputs of one energy evaluation and the potential it produced."""

    def __init__(self, rho, grad_rho, coords, weights, atom_of_point, n_atom, prec, b, C, rho_cut):
        self.rho, self.grad_rho, self.coords, self.weights = rho, grad_rho, coords, weights
        self.atom_of_point, self.n_atom = atom_of_point, n_atom
        self.prec, self.b, self.C, self.rho_cut = prec, b, C, rho_cut
        self.device = rho.device.index if rho.device.index is not None else torch.cuda.current_device()
        self.slot = _DeviceHandle.get(self.device)
        self.energy = None
        self.vrho = None
        self.vgamma = None

    @property
    def h(self):
        return self.slot["h"]

    def ensure(self):
        """(Re)prepare the handle for these inputs and compute E, f^rho, f^gamma."""
        if self.slot["owner"] is self and self.vrho is not None:
            return
        n = self.rho.shape[0]
        _vv.vv10_prepare_points(self.h, self.coords, self.weights, self.rho, self.grad_rho,
                                self.atom_of_point, self.n_atom, self.b, self.C, self.rho_cut)
        vrho = torch.empty(n, dtype=torch.float64, device=self.rho.device)
        vgamma = torch.empty(n, dtype=torch.float64, device=self.rho.device)
        self.energy = _vv.vv10_energy_potential(self.h, self.prec, vrho, vgamma)
        self.vrho, self.vgamma = vrho, vgamma
        self.slot["owner"] = self

    @property
    def lock(self):
        return self.slot["lock"]

    def hessian(self, a_rho, a_grad):
        """(w f^{rho,t}, 2 w (f^{gamma,t} grad rho + f^gamma d grad rho)) for trials (P, n),
        both formed by the library (vv10_hessian_vector_product)."""
        d_rho = torch.empty_like(a_rho)
        d_grad = torch.empty_like(a_grad)
        with self.lock:
            self.ensure()
            _vv.vv10_hessian_vector_product(self.h, self.prec, a_rho.contiguous(),
                                            a_grad.contiguous(), d_rho, d_grad)
        return d_rho, d_grad


def _c64(t: torch.Tensor) -> torch.Tensor:
    if t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError("vv10_energy expects float64 CUDA tensors")
    return t.detach().contiguous()


def _is_batched(t: Optional[torch.Tensor]) -> bool:
    """True for tensors that carry a hidden vmap batch (these cannot be handed to the C ABI)."""
    if t is None:
        return False
    from torch._C import _functorch as ft
    return bool(ft.is_batchedtensor(t) or ft.is_legacy_batchedtensor(t))


class _FirstDerivs(torch.autograd.Function):
    """dE/d(rho, grad rho, coords, weights); differentiable in rho and grad rho."""

    @staticmethod
    def forward(ctx, state, want_coords, want_w, rho, grad_rho, coords, weights):
        n = state.weights.shape[0]
        g_coords = torch.zeros(n, 3, dtype=torch.float64, device=state.weights.device)
        g_w = torch.zeros(n, dtype=torch.float64, device=state.weights.device)
        with state.lock:
            state.ensure()
            if want_coords:
                _vv.vv10_coord_grad(state.h, state.prec, g_coords)
            if want_w:
                _vv.vv10_weight_grad(state.h, g_w)
        w = state.weights
        g_rho = w * state.vrho
        g_grad = 2.0 * (w * state.vgamma)[:, None] * state.grad_rho
        ctx.state = state
        ctx.set_materialize_grads(False)
        return g_rho, g_grad, g_coords, g_w

    @staticmethod
    def backward(ctx, a_rho, a_grad, a_coords, a_w):
        if a_coords is not None or a_w is not None:
            raise NotImplementedError("second derivatives involving coordinates or weights "
                                      "of the VV10 energy are not provided")
        if ctx.needs_input_grad[5] or ctx.needs_input_grad[6]:
            raise NotImplementedError("second derivatives with respect to coordinates or "
                                      "weights of the VV10 energy are not provided")
        if a_rho is None and a_grad is None:
            return None, None, None, None, None, None, None
        if _is_batched(a_rho) or _is_batched(a_grad):
            raise NotImplementedError("batched directions through autograd (vmap / "
                                      "is_grads_batched) are not supported; use vv10_hvp, which "
                                      "contracts all directions in one call")
        st = ctx.state
        u_rho = (a_rho if a_rho is not None else torch.zeros_like(st.rho))[None]
        u_grad = (a_grad if a_grad is not None else torch.zeros_like(st.grad_rho))[None]
        d_rho, d_grad = st.hessian(u_rho.contiguous(), u_grad.contiguous())
        return None, None, None, d_rho[0], d_grad[0], None, None


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, grad_rho, coords, weights, state):
        with state.lock:
            state.ensure()
        ctx.state = state
        ctx.save_for_backward(rho, grad_rho, coords, weights)
        return torch.tensor(state.energy, dtype=torch.float64, device=rho.device)

    @staticmethod
    def backward(ctx, gE):
        rho, grad_rho, coords, weights = ctx.saved_tensors
        want = ctx.needs_input_grad
        g_rho, g_grad, g_coords, g_w = _FirstDerivs.apply(ctx.state, bool(want[2]), bool(want[3]),
                                                          rho, grad_rho, coords, weights)
        return (gE * g_rho if want[0] else None, gE * g_grad if want[1] else None,
                gE * g_coords if want[2] else None, gE * g_w if want[3] else None, None)


def vv10_energy(rho: torch.Tensor, grad_rho: torch.Tensor, coords: torch.Tensor,
                weights: torch.Tensor, atom_of_point: Optional[torch.Tensor] = None,
                n_atom: int = 0, precision: str = "fp64", b: float = 6.0, C: float = 0.01,
                rho_cut: float = 1e-10) -> torch.Tensor:
    """Differentiable VV10 energy (0-dim float64 tensor on the inputs' CUDA device)."""
    state = _State(_c64(rho), _c64(grad_rho), _c64(coords), _c64(weights),
                   None if atom_of_point is None else atom_of_point.detach().contiguous(),
                   int(n_atom), _PREC[precision], b, C, rho_cut)
    return _Energy.apply(rho, grad_rho, coords, weights, state)


def vv10_hvp(rho: torch.Tensor, grad_rho: torch.Tensor, coords: torch.Tensor,
             weights: torch.Tensor, d_rho: torch.Tensor, d_grad_rho: torch.Tensor,
             precision: str = "fp64", b: float = 6.0, C: float = 0.01, rho_cut: float = 1e-10):
    """Second derivatives of E along P directions at once (Sec. II.B, Eq. frhot):
    returns (P, n) d(dE/d rho) and (P, n, 3) d(dE/d grad rho) for directions
    d_rho (P, n), d_grad_rho (P, n, 3).  Not differentiable."""
    state = _State(_c64(rho), _c64(grad_rho), _c64(coords), _c64(weights), None, 0,
                   _PREC[precision], b, C, rho_cut)
    return state.hessian(_c64(d_rho), _c64(d_grad_rho))
