"""The VV10 nuclear gradient assembled on the GPU (Sec. II.A: E^A_G + E^A_w from
vv10_nuclear_gradient, E^A_gr from vv10_coord_grad) against the oracle's terms and against
central differences of the energy of the whole synthetic pipeline (grid points, Becke weights
and density moving with the atoms), through the C ABI.

Tolerances: against the oracle's terms FP64 <= 1e-10 and mixed <= 1e-6 relative (max norm over
the 3 N_atom components); against the finite differences 1e-6 relative.  The full-size
water-hexamer grid checks translational invariance of the total gradient and the agreement of
the FP64 and mixed paths.
"""
import numpy as np
import pytest
import torch

from paper_2208_14639_gb300 import synth, vv10

pytestmark = pytest.mark.gpu

FP64 = vv10.VV10_FP64
MIXED = vv10.VV10_MIXED_TF32X3


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    vv10.load(build_if_missing=True)
    return torch.device("cuda", 0)


def T(a, dev, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)


def gpu_gradient(g, rt, gt, W, prec, dev):
    eng = vv10.VV10(0)
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                T(g.atom_of_point, dev, torch.int32), g.molecule.n_atom)
    eng.energy_potential(prec)
    terms = eng.nuclear_gradient(T(rt, dev), T(gt, dev), T(W, dev)).cpu().numpy()
    _, ga, _ = eng.coord_grad(prec, atoms=True)
    eng.close()
    return terms + ga.cpu().numpy().reshape(-1)


def oracle_gradient(oracle_mod, g, rt, gt, W):
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    kept = g.rho >= 1e-10
    _, vr, vg = oracle_mod.potential(*args)
    E = oracle_mod.pair_sums(*args)["E"]
    ga = oracle_mod.atom_grad(*args, g.atom_of_point, g.molecule.n_atom).reshape(-1)
    out = np.zeros(rt.shape[0])
    for p in range(out.size):
        out[p] = (np.sum(g.weights * (vr * rt[p] + 2 * vg * np.einsum("nd,nd->n", g.grad_rho, gt[p])))
                  + np.sum((W[p] * g.rho * (oracle_mod.beta() + E))[kept]) + ga[p])
    return out


def rel_max(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def system(mol, nr, na):
    g = synth.make_system(mol, nr, na)
    rt, gt = synth.nuclear_density_derivatives(mol, g.coords, g.atom_of_point)
    return g, rt, gt, synth.weight_directions(mol, nr, na)


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-6)], ids=["fp64", "mixed"])
def test_water_against_oracle_terms_and_finite_differences(dev, oracle_mod, prec, tol):
    mol, nr, na = synth.water(), 10, 26
    g, rt, gt, W = system(mol, nr, na)
    ref = oracle_gradient(oracle_mod, g, rt, gt, W)
    got = gpu_gradient(g, rt, gt, W, prec, dev)
    assert rel_max(got, ref) <= tol
    if prec == FP64:
        h, kept = 1e-4, g.rho >= 1e-10
        fd = np.zeros_like(ref)
        for p in range(ref.size):
            es = []
            for sg in (1, -1):
                c = mol.coords.copy()
                c[p // 3, p % 3] += sg * h
                g2 = synth.make_system(synth.Molecule(mol.symbols, c), nr, na)
                assert np.array_equal(g2.rho >= 1e-10, kept)
                es.append(oracle_mod.energy(g2.coords, g2.weights, g2.rho, g2.grad_rho))
            fd[p] = (es[0] - es[1]) / (2 * h)
        assert rel_max(got, fd) <= 1e-6


def test_larger_grid_and_single_terms(dev, oracle_mod):
    """The 9,900-point water grid; each of the two terms alone."""
    g, rt, gt, W = system(synth.water(), 30, 110)
    ref = oracle_gradient(oracle_mod, g, rt, gt, W)
    assert rel_max(gpu_gradient(g, rt, gt, W, FP64, dev), ref) <= 1e-10
    eng = vv10.VV10(0)
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                T(g.atom_of_point, dev, torch.int32), g.molecule.n_atom)
    with pytest.raises(vv10.VV10Error):  # no energy call yet
        eng.nuclear_gradient(w_t=T(W, dev))
    eng.energy_potential(FP64)
    both = eng.nuclear_gradient(T(rt, dev), T(gt, dev), T(W, dev))
    only_g = eng.nuclear_gradient(T(rt, dev), T(gt, dev))
    only_w = eng.nuclear_gradient(w_t=T(W, dev))
    assert torch.allclose(both, only_g + only_w, rtol=1e-12, atol=1e-15)
    assert torch.equal(both, eng.nuclear_gradient(T(rt, dev), T(gt, dev), T(W, dev)))
    eng.close()


def test_full_size_hexamer_invariance(dev):
    mol = synth.config_water_hexamer().molecule
    g, rt, gt, W = system(mol, 50, 194)
    g64 = gpu_gradient(g, rt, gt, W, FP64, dev)
    gmx = gpu_gradient(g, rt, gt, W, MIXED, dev)
    scale = np.abs(g64).max()
    assert np.abs(g64.reshape(-1, 3).sum(axis=0)).max() <= 1e-6 * scale
    assert rel_max(gmx, g64) <= 1e-6
