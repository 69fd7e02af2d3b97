"""The torch.autograd wrapper: first derivatives against the oracle and central finite
differences, double backward (Hessian-vector products) against the oracle contraction,
batched directions, and the 24-atom / 100,080-point cluster with P = 72 directions."""
import numpy as np
import pytest
import torch

from paper_2208_14639_gb300 import synth
from paper_2208_14639_gb300.autograd import vv10_energy, vv10_hvp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch.device("cuda", 0)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def leaves(g, dev, grad=(True, True, True, True)):
    T = lambda a, r: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev,
                                  requires_grad=r)
    return (T(g.rho, grad[0]), T(g.grad_rho, grad[1]), T(g.coords, grad[2]), T(g.weights, grad[3]))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_first_derivatives(dev, oracle_mod, precision, tol):
    g = synth.random_points(300, seed=41, n_atom=3)
    rho, grad, xyz, w = leaves(g, dev)
    E = vv10_energy(rho, grad, xyz, w, precision=precision)
    E.backward()
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    e_ref, vr, vg = oracle_mod.potential(*args)
    assert abs(E.item() - e_ref) <= (1e-11 * abs(e_ref) if precision == "fp64" else 1e-7)
    assert rel(rho.grad.cpu(), g.weights * vr) <= tol
    assert rel(grad.grad.cpu(), 2 * (g.weights * vg)[:, None] * g.grad_rho) <= tol
    assert rel(xyz.grad.cpu(), oracle_mod.point_grad(*args)) <= tol
    Ei = oracle_mod.pair_sums(*args)["E"]
    assert rel(w.grad.cpu(), g.rho * (oracle_mod.beta() + Ei)) <= tol


def test_gradient_by_central_differences(dev):
    """Directional central differences of the FP64 GPU energy, h = 1e-4 (relative)."""
    g = synth.random_points(400, seed=43, n_atom=3)
    rho, grad, xyz, w = leaves(g, dev)
    E = vv10_energy(rho, grad, xyz, w)
    gr = torch.autograd.grad(E, (rho, grad, xyz, w))
    rng = np.random.default_rng(0)
    for k, base in enumerate((g.rho, g.grad_rho, g.coords, g.weights)):
        d = rng.normal(size=base.shape) * (np.abs(base) if k != 2 else 1.0)
        h = 1e-4
        vals = []
        for sgn in (1, -1):
            pert = [g.rho, g.grad_rho, g.coords, g.weights]
            pert[k] = base + sgn * h * d
            r2, g2, x2, w2 = leaves(synth.GridDensity(pert[2], pert[3], pert[0], pert[1],
                                                      g.atom_of_point, g.molecule), dev,
                                    (False,) * 4)
            vals.append(vv10_energy(r2, g2, x2, w2).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        an = float((gr[k].cpu().numpy() * d).sum())
        assert fd == pytest.approx(an, rel=1e-6, abs=1e-12)


def _hvp_ref(oracle_mod, g, d_rho, d_grad):
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    _, _, vg = oracle_mod.potential(*args)
    fr, fg = oracle_mod.hessian_contract(*args, d_rho[None], d_grad[None])
    return (g.weights * fr[0], 2 * g.weights[:, None] * (fg[0][:, None] * g.grad_rho
                                                           + vg[:, None] * d_grad))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_double_backward_is_hessian_vector_product(dev, oracle_mod, precision, tol):
    g = synth.random_points(300, seed=45, n_atom=3)
    rho, grad, xyz, w = leaves(g, dev, (True, True, False, False))
    E = vv10_energy(rho, grad, xyz, w, precision=precision)
    g_rho, g_grad = torch.autograd.grad(E, (rho, grad), create_graph=True)
    rng = np.random.default_rng(1)
    d_rho = rng.normal(size=g.n) * g.rho
    d_grad = rng.normal(size=(g.n, 3)) * np.abs(g.grad_rho)
    v_rho = torch.tensor(d_rho, device=dev)
    v_grad = torch.tensor(d_grad, device=dev)
    h_rho, h_grad = torch.autograd.grad((g_rho * v_rho).sum() + (g_grad * v_grad).sum(), (rho, grad))
    ref_rho, ref_grad = _hvp_ref(oracle_mod, g, d_rho, d_grad)
    assert rel(h_rho.cpu(), ref_rho) <= tol
    assert rel(h_grad.cpu(), ref_grad) <= tol


def test_batched_directions_match_single(dev):
    """vv10_hvp on P directions equals P single double-backward products."""
    g = synth.random_points(256, seed=47, n_atom=2)
    rho, grad, xyz, w = leaves(g, dev, (True, True, False, False))
    E = vv10_energy(rho, grad, xyz, w)
    g_rho, g_grad = torch.autograd.grad(E, (rho, grad), create_graph=True)
    B = 6
    rng = np.random.default_rng(2)
    V_rho = torch.tensor(rng.normal(size=(B, g.n)) * g.rho, device=dev)
    V_grad = torch.tensor(rng.normal(size=(B, g.n, 3)) * np.abs(g.grad_rho), device=dev)
    e_rho, e_grad = vv10_hvp(rho, grad, xyz, w, V_rho, V_grad)
    for k in range(B):
        h_rho, h_grad = torch.autograd.grad((g_rho, g_grad), (rho, grad), (V_rho[k], V_grad[k]),
                                            retain_graph=True)
        assert rel(e_rho[k].cpu(), h_rho.cpu()) <= 1e-12
        assert rel(e_grad[k].cpu(), h_grad.cpu()) <= 1e-12
    with pytest.raises(NotImplementedError):
        torch.autograd.grad((g_rho, g_grad), (rho, grad), (V_rho, V_grad), retain_graph=True,
                            is_grads_batched=True)


def test_second_derivatives_with_coordinates_raise(dev):
    g = synth.random_points(64, seed=49, n_atom=2)
    rho, grad, xyz, w = leaves(g, dev, (True, False, True, False))
    E = vv10_energy(rho, grad, xyz, w)
    g_rho, = torch.autograd.grad(E, (rho,), create_graph=True)
    with pytest.raises(NotImplementedError):
        torch.autograd.grad(g_rho.sum(), (xyz,))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_cluster24_gradient_and_batched_hvp(dev, oracle_mod, precision, tol):
    """24-atom cluster, 100,080 points; gradient and P = 72 nuclear-displacement directions
    in one contraction against the oracle on sampled rows."""
    g = synth.config_cluster24()
    rt, gt = synth.trial_densities(g.molecule, g.coords)
    rho, grad, xyz, w = leaves(g, dev, (True, True, False, False))
    E = vv10_energy(rho, grad, xyz, w, precision=precision)
    g_rho, g_grad = torch.autograd.grad(E, (rho, grad), create_graph=True)
    rows = np.linspace(0, g.n - 1, 64).astype(np.int64)
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    _, vr, vg = oracle_mod.potential(*args, rows=rows)
    assert rel(g_rho.detach().cpu().numpy()[rows], g.weights[rows] * vr) <= tol
    hb_rho, hb_grad = vv10_hvp(rho, grad, xyz, w, torch.tensor(rt, device=dev),
                               torch.tensor(gt, device=dev), precision=precision)
    assert hb_rho.shape == (72, g.n)
    fr, fg = oracle_mod.hessian_contract(*args, rt, gt, rows=rows)
    assert rel(hb_rho.cpu().numpy()[:, rows], g.weights[rows] * fr) <= tol
    _, _, vg_rows = oracle_mod.potential(*args, rows=rows)
    ref_grad = 2 * g.weights[rows][None, :, None] * (fg[:, :, None] * g.grad_rho[rows][None]
                                                      + vg_rows[None, :, None] * gt[:, rows, :])
    assert rel(hb_grad.cpu().numpy()[:, rows, :], ref_grad) <= tol
