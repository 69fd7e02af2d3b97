"""Parity of vv10_energy (the energy from the unordered pairs, Sec. II.A) with the FP64 oracle,
through the C ABI.

Tolerances as for the energy of vv10_energy_potential: FP64 |dE|/|E| <= 1e-11, mixed
|dE| <= 1e-7 Eh.  Point counts around the 128-point blocks (the diagonal blocks carry the
j >= i half and the halved self term), the full-size water-hexamer grid, all points below
the cutoff, repeatability, and the row sums cached by vv10_energy_potential left intact.
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


def make_engine(g, dev):
    eng = vv10.VV10(0)
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                T(g.atom_of_point, dev, torch.int32), g.molecule.n_atom)
    return eng


def check_energy(e, e_ref, prec):
    if prec == FP64:
        assert abs(e - e_ref) <= 1e-11 * abs(e_ref)
    else:
        assert abs(e - e_ref) <= 1e-7


SIZES = [1, 2, 37, 127, 128, 129, 255, 256, 257, 700, 2000]


@pytest.mark.parametrize("prec", [FP64, MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("n", SIZES)
def test_random_systems(dev, oracle_mod, n, prec):
    g = synth.random_points(n, seed=200 + n, n_atom=2)
    e_ref = oracle_mod.energy(g.coords, g.weights, g.rho, g.grad_rho)
    eng = make_engine(g, dev)
    e = eng.energy(prec)
    check_energy(e, e_ref, prec)
    assert eng.energy(prec) == e  # fixed summation order
    eng.close()


def test_water_and_cached_sums(dev, oracle_mod):
    g = synth.config_water()
    e_ref = oracle_mod.energy(g.coords, g.weights, g.rho, g.grad_rho)
    E_ref = oracle_mod.pair_sums(g.coords, g.weights, g.rho, g.grad_rho)["E"]
    eng = make_engine(g, dev)
    e_ep, _, _ = eng.energy_potential(FP64)
    for prec in (FP64, MIXED):
        check_energy(eng.energy(prec), e_ref, prec)
    # the row sums of the energy call are still there for vv10_weight_grad
    dw = eng.weight_grad().cpu().numpy()
    ref = g.rho * (oracle_mod.beta() + E_ref)
    assert np.linalg.norm(dw - ref) <= 1e-10 * np.linalg.norm(ref)
    assert abs(eng.energy(FP64) - e_ep) <= 1e-12 * abs(e_ep)
    eng.close()


def test_all_points_below_cutoff(dev):
    g = synth.random_points(300, seed=210, n_atom=2)
    h = synth.GridDensity(g.coords, g.weights, np.zeros_like(g.rho), g.grad_rho,
                          g.atom_of_point, g.molecule)
    eng = make_engine(h, dev)
    assert eng.energy(FP64) == 0.0 and eng.energy(MIXED) == 0.0
    eng.close()


def test_full_size_hexamer(dev, oracle_mod):
    g = synth.config_water_hexamer()
    e_ref = oracle_mod.energy(g.coords, g.weights, g.rho, g.grad_rho)
    eng = make_engine(g, dev)
    for prec in (FP64, MIXED):
        check_energy(eng.energy(prec), e_ref, prec)
    eng.close()
