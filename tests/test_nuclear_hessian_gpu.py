"""The VV10 nuclear Hessian (Sec. II.B, Eq. E_hess) on the GPU, through the C ABI:
vv10_nuclear_hessian forms every pair sum with the library's own entry points (energy and
potential, the Hessian contraction with the nuclear trials, the weight-derivative sums, the
atom-resolved sums, the grid-grid blocks), takes the local derivatives (kappa', omega_rho,
omega_gamma) from its prepared points, and assembles the nine terms on the device.

Against the oracle (its own pair sums through its numpy nine-term assembly): FP64 <= 1e-10,
mixed <= 1e-6 relative (max norm); against central differences of the nuclear gradient of
the whole synthetic pipeline: 1e-6.
"""
import numpy as np
import pytest
import torch

from paper_2208_14639_gb300 import synth, vv10

pytestmark = pytest.mark.gpu

FP64 = vv10.VV10_FP64
MIXED = vv10.VV10_MIXED_TF32X3
F16 = vv10.VV10_MIXED_F16X3
F64TC = vv10.VV10_FP64_TC


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    vv10.load(build_if_missing=True)
    return torch.device("cuda", 0)


def T(a, dev, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)


def case(mol, nr, na):
    g = synth.make_system(mol, nr, na)
    rt, gt = synth.nuclear_density_derivatives(mol, g.coords, g.atom_of_point)
    r2, g2 = synth.nuclear_density_second_derivatives(mol, g.coords, g.atom_of_point)
    return dict(g=g, rt=rt, gt=gt, r2=r2, g2=g2, W=synth.weight_directions(mol, nr, na),
                Wab=synth.weight_second_derivatives(mol, nr, na))


def assemble(oracle_mod, c, vr, vg, E, Ew, Uw, Ww, Egr, Ugr, Wgr, fr, fg, Hgg):
    g = c["g"]
    pp = oracle_mod.point_props(g.rho, g.grad_rho)
    return oracle_mod.nuclear_hessian(g.weights, g.rho, g.grad_rho, g.rho >= 1e-10, pp["kappa_rho"],
                                      pp["omega_rho"], pp["omega_gamma"], vr, vg, E, c["rt"], c["gt"],
                                      c["r2"], c["g2"], c["W"], c["Wab"], Ew, Uw, Ww, Egr, Ugr, Wgr,
                                      fr, fg, Hgg)


def oracle_hessian(oracle_mod, c):
    g = c["g"]
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    NA = g.molecule.n_atom
    P = 3 * NA
    _, vr, vg = oracle_mod.potential(*args)
    E = oracle_mod.pair_sums(*args)["E"]
    Ew, Uw, Ww = oracle_mod.weight_response(*args, c["W"])
    Egr, Ugr, Wgr = (x.reshape(g.n, P).T for x in oracle_mod.atom_resolved(*args, g.atom_of_point, NA))
    fr, fg = oracle_mod.hessian_contract(*args, c["rt"], c["gt"])
    Hgg = oracle_mod.coord_hessian(*args, g.atom_of_point, NA).transpose(0, 2, 1, 3).reshape(P, P)
    return assemble(oracle_mod, c, vr, vg, E, Ew, Uw, Ww, Egr, Ugr, Wgr, fr, fg, Hgg)


def gpu_hessian(oracle_mod, c, prec, dev):
    g = c["g"]
    NA = g.molecule.n_atom
    eng = vv10.VV10(0)
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                T(g.atom_of_point, dev, torch.int32), NA)
    H = eng.nuclear_hessian(T(c["rt"], dev), T(c["gt"], dev), T(c["r2"], dev), T(c["g2"], dev),
                            T(c["W"], dev), T(c["Wab"], dev), prec)
    out = H.cpu().numpy()
    eng.close()
    return out


def rel_max(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.fixture(scope="module")
def water_small():
    return case(synth.water(), 10, 26)


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-6), (F16, 1e-6), (F64TC, 1e-10)],
                         ids=["fp64", "tf32x3", "f16x3", "fp64tc"])
def test_water_against_oracle_terms(dev, oracle_mod, water_small, prec, tol):
    ref = oracle_hessian(oracle_mod, water_small)
    got = gpu_hessian(oracle_mod, water_small, prec, dev)
    assert rel_max(got, ref) <= tol


def test_water_against_finite_differences(dev, oracle_mod, water_small):
    mol, nr, na = synth.water(), 10, 26
    got = gpu_hessian(oracle_mod, water_small, FP64, dev)
    g0 = water_small["g"]
    kept = g0.rho >= 1e-10
    P = 3 * mol.n_atom
    h = 1e-4
    fd = np.zeros((P, P))
    for b in range(P):
        gs = []
        for sg in (1, -1):
            c = mol.coords.copy()
            c[b // 3, b % 3] += sg * h
            m2 = synth.Molecule(mol.symbols, c)
            g = synth.make_system(m2, nr, na)
            assert np.array_equal(g.rho >= 1e-10, kept)
            rt, gt = synth.nuclear_density_derivatives(m2, g.coords, g.atom_of_point)
            W = synth.weight_directions(m2, nr, na)
            args = (g.coords, g.weights, g.rho, g.grad_rho)
            _, vr, vg = oracle_mod.potential(*args)
            E = oracle_mod.pair_sums(*args)["E"]
            ga = oracle_mod.atom_grad(*args, g.atom_of_point, mol.n_atom).reshape(-1)
            gs.append(np.array([np.sum(g.weights * (vr * rt[p] + 2 * vg * np.einsum("nd,nd->n", g.grad_rho, gt[p])))
                                + np.sum((W[p] * g.rho * (oracle_mod.beta() + E))[kept]) + ga[p]
                                for p in range(P)]))
        fd[:, b] = (gs[0] - gs[1]) / (2 * h)
    assert rel_max(got, fd) <= 1e-6


def test_larger_water_grid(dev, oracle_mod):
    """The 9,900-point water grid, FP64 and mixed against the oracle's terms."""
    c = case(synth.water(), 30, 110)
    ref = oracle_hessian(oracle_mod, c)
    assert rel_max(gpu_hessian(oracle_mod, c, FP64, dev), ref) <= 1e-10
    assert rel_max(gpu_hessian(oracle_mod, c, MIXED, dev), ref) <= 1e-6


def test_symmetric_and_translation_invariant(dev, oracle_mod):
    """A 4-atom CHON molecule: H = H^T, and every row sums to zero over the three
    translations (a rigid shift of the whole system leaves the gradient unchanged)."""
    c = case(synth.random_chon(np.random.default_rng(41), 4), 10, 26)
    H = gpu_hessian(oracle_mod, c, FP64, dev)
    scale = np.abs(H).max()
    assert np.abs(H - H.T).max() <= 1e-7 * scale  # w^{ab} comes from central differences
    na = c["g"].molecule.n_atom
    shift = H.reshape(3 * na, na, 3).sum(axis=1)
    assert np.abs(shift).max() <= 1e-6 * scale
    ref = oracle_hessian(oracle_mod, c)
    assert rel_max(H, ref) <= 1e-10


def test_requires_atom_labels(dev):
    g = synth.random_points(64, seed=3, n_atom=2)
    eng = vv10.VV10(0)
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev))
    z = lambda *shape: torch.zeros(*shape, dtype=torch.float64, device=dev)
    with pytest.raises(vv10.VV10Error) as ei:
        eng.nuclear_hessian(z(6, g.n), z(6, g.n, 3), z(6, 6, g.n), z(6, 6, g.n, 3), z(6, g.n),
                            z(6, 6, g.n))
    assert ei.value.status == vv10.VV10_ERR_INVALID_ARG
    eng.close()
