"""Parity of the AO-side assembly (Sec. II.A Fock matrix, Sec. II.B contracted orbital Hessian)
with the FP64 oracle, through the C ABI.

The GPU path is checked two ways: end to end (the GPU's own f^rho, f^gamma, f^{rho,t},
f^{gamma,t} assembled on the GPU, against the oracle's potential and contraction assembled by
the oracle: FP64 <= 1e-10, mixed <= 1e-6 relative Frobenius), and the assembly alone (the same
per-point inputs on both sides: <= 1e-12).  Water with its AO basis in full; the full-size
water-hexamer grid (174,600 points, 78 basis functions) for the assembly alone.
"""
import numpy as np
import pytest
import torch

from paper_2208_14639_gb300 import synth, vv10

pytestmark = pytest.mark.gpu

FP64 = vv10.VV10_FP64
MIXED = vv10.VV10_MIXED_TF32X3


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    vv10.load(build_if_missing=True)
    return torch.device("cuda", 0)


def T(a, dev, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)


@pytest.fixture(scope="module")
def water_ao(oracle_mod):
    g, phi, dphi, P, Pt, rt, gt = synth.ao_system(synth.water(), 30, 110, 11, n_trials=3)
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    _, vr, vg = oracle_mod.potential(*args)
    fr, fg = oracle_mod.hessian_contract(*args, rt, gt)
    F = oracle_mod.fock_matrix(g.weights, g.grad_rho, vr, vg, phi, dphi)
    G = oracle_mod.orbital_hessian(g.weights, g.grad_rho, vg, fr, fg, gt, phi, dphi)
    return dict(g=g, phi=phi, dphi=dphi, rt=rt, gt=gt, vr=vr, vg=vg, fr=fr, fg=fg, F=F, G=G)


def make_engine(g, dev):
    eng = vv10.VV10(0)
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                T(g.atom_of_point, dev, torch.int32), g.molecule.n_atom)
    return eng


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-6)], ids=["fp64", "mixed"])
def test_fock_and_orbital_hessian_end_to_end(dev, water_ao, prec, tol):
    c = water_ao
    eng = make_engine(c["g"], dev)
    phi, dphi = T(c["phi"], dev), T(c["dphi"], dev)
    _, vr, vg = eng.energy_potential(prec)
    F = eng.fock_matrix(phi, dphi, vr, vg).cpu().numpy()
    assert rel(F, c["F"]) <= tol
    assert np.array_equal(F, F.T)
    gt = T(c["gt"], dev)
    fr, fg = eng.hessian_contract(T(c["rt"], dev), gt, prec)
    G = eng.orbital_hessian(phi, dphi, fr, fg, gt, vg).cpu().numpy()
    for t in range(G.shape[0]):
        assert rel(G[t], c["G"][t]) <= tol
        assert np.array_equal(G[t], G[t].T)
    eng.close()


def test_assembly_alone_and_repeatable(dev, water_ao):
    """The oracle's per-point inputs assembled on the GPU give the oracle's matrices to FP64
    rounding; repeated calls agree bit for bit."""
    c = water_ao
    eng = make_engine(c["g"], dev)
    phi, dphi = T(c["phi"], dev), T(c["dphi"], dev)
    F1 = eng.fock_matrix(phi, dphi, T(c["vr"], dev), T(c["vg"], dev))
    F2 = eng.fock_matrix(phi, dphi, T(c["vr"], dev), T(c["vg"], dev))
    assert torch.equal(F1, F2)
    assert rel(F1.cpu().numpy(), c["F"]) <= 1e-12
    G = eng.orbital_hessian(phi, dphi, T(c["fr"], dev), T(c["fg"], dev), T(c["gt"], dev),
                            T(c["vg"], dev)).cpu().numpy()
    assert rel(G, c["G"]) <= 1e-12
    eng.close()


def test_argument_errors(dev, water_ao):
    c = water_ao
    eng = make_engine(c["g"], dev)
    phi, dphi = T(c["phi"], dev), T(c["dphi"], dev)
    n, nbf = c["phi"].shape
    vr, vg = T(c["vr"], dev), T(c["vg"], dev)
    F = torch.empty(nbf, nbf, dtype=torch.float64, device=dev)
    with pytest.raises(ValueError):  # shape mismatch caught by the binding
        vv10.vv10_fock_matrix(eng.h, phi, dphi[:, :, :2].contiguous(), vr, vg, F)
    lib = vv10.load()
    import ctypes
    null = ctypes.c_void_p(0)
    st = lib.vv10_fock_matrix(eng.h, 0, ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(dphi.data_ptr()),
                              ctypes.c_void_p(vr.data_ptr()), ctypes.c_void_p(vg.data_ptr()),
                              ctypes.c_void_p(F.data_ptr()), null)
    assert st == vv10.VV10_ERR_INVALID_ARG
    st = lib.vv10_orbital_hessian(eng.h, nbf, ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(dphi.data_ptr()),
                                  1, ctypes.c_void_p(vr.data_ptr()), ctypes.c_void_p(vg.data_ptr()),
                                  null, null, ctypes.c_void_p(F.data_ptr()), null)
    assert st == vv10.VV10_ERR_INVALID_ARG
    eng.close()


def test_full_size_hexamer_assembly(dev, oracle_mod):
    """The water-hexamer grid with its 78-function basis: the GPU assembly of the GPU's own
    potential against the oracle's assembly of the same potential, and the symmetry."""
    oracle = oracle_mod
    mol = synth.config_water_hexamer().molecule
    g, phi, dphi, P, Pt, rt, gt = synth.ao_system(mol, 50, 194, 12, n_trials=2)
    eng = make_engine(g, dev)
    phid, dphid = T(phi, dev), T(dphi, dev)
    _, vr, vg = eng.energy_potential(MIXED)
    F = eng.fock_matrix(phid, dphid, vr, vg).cpu().numpy()
    vr, vg = vr.cpu().numpy(), vg.cpu().numpy()
    ref = oracle.fock_matrix(g.weights * (g.rho >= 1e-10), g.grad_rho, vr, vg, phi, dphi)
    assert rel(F, ref) <= 1e-12 and np.array_equal(F, F.T)
    gtd = T(gt, dev)
    fr, fg = eng.hessian_contract(T(rt, dev), gtd, MIXED)
    G = eng.orbital_hessian(phid, dphid, fr, fg, gtd, T(vg, dev)).cpu().numpy()
    refG = oracle.orbital_hessian(g.weights * (g.rho >= 1e-10), g.grad_rho, vg, fr.cpu().numpy(),
                                  fg.cpu().numpy(), gt, phi, dphi)
    assert rel(G, refG) <= 1e-12
    eng.close()
