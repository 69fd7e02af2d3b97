"""Parity of the nuclear derivative of the Fock matrix (Sec. II.B, F^A = F^A_G + F^A_gr + F^A_w)
with the FP64 oracle, through the C ABI.

Two ways: the assembly alone (the same per-point inputs on both sides, seeded random pair-sum
results on a shuffled caller order with dropped points and an atom without kept points:
<= 1e-12 relative Frobenius), and end to end (the GPU's potential, Hessian contraction with the
nuclear trials, weight-derivative and atom-resolved sums assembled on the GPU, against the
oracle's assembled by the oracle: FP64 <= 1e-10, mixed <= 1e-6; and against central
differences of the Fock matrix of the moving pipeline: 1e-6 of the largest element).
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


def make_engine(g, dev):
    eng = vv10.VV10(0)
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                T(g.atom_of_point, dev, torch.int32), g.molecule.n_atom)
    return eng


def oracle_assembly(oracle_mod, g, phi, dphi, d2phi, basis, inp):
    pp = oracle_mod.point_props(g.rho, g.grad_rho)
    Pd = 3 * g.molecule.n_atom
    Egr, Ugr, Wgr = (x.reshape(g.n, Pd).T for x in inp["euw"])
    return oracle_mod.fock_derivative(g.weights, g.rho, g.grad_rho, g.rho >= 1e-10, pp["kappa_rho"],
                                      pp["omega_rho"], pp["omega_gamma"], inp["vr"], inp["vg"], phi,
                                      dphi, d2phi, basis.atom, g.atom_of_point, inp["gt"], inp["W"],
                                      inp["Ew"], inp["Uw"], inp["Ww"], Egr, Ugr, Wgr, inp["fr"],
                                      inp["fg"])


def gpu_assembly(eng, dev, phi, dphi, d2phi, basis, inp):
    return eng.fock_derivative(T(phi, dev), T(dphi, dev), T(d2phi, dev),
                               T(basis.atom, dev, torch.int32), T(inp["vr"], dev), T(inp["vg"], dev),
                               T(inp["fr"], dev), T(inp["fg"], dev), T(inp["gt"], dev),
                               T(inp["W"], dev), T(inp["Ew"], dev), T(inp["Uw"], dev),
                               T(inp["Ww"], dev), T(inp["euw"], dev)).cpu().numpy()


def oracle_inputs(oracle_mod, g, rt, gt, W):
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    NA = g.molecule.n_atom
    _, vr, vg = oracle_mod.potential(*args)
    Ew, Uw, Ww = oracle_mod.weight_response(*args, W)
    euw = np.stack(oracle_mod.atom_resolved(*args, g.atom_of_point, NA))
    fr, fg = oracle_mod.hessian_contract(*args, rt, gt)
    return dict(vr=vr, vg=vg, Ew=Ew, Uw=Uw, Ww=Ww, euw=euw, fr=fr, fg=fg, gt=gt, W=W)


def gpu_inputs(eng, dev, rt, gt, W, prec):
    _, vr, vg = eng.energy_potential(prec)
    Ew, Uw, Ww = eng.weight_response(T(W, dev), prec)
    _, _, euw = eng.coord_grad(prec, atoms=False, resolved=True)
    fr, fg = eng.hessian_contract(T(rt, dev), T(gt, dev), prec)
    return dict(vr=vr, vg=vg, Ew=Ew, Uw=Uw, Ww=Ww, euw=euw, fr=fr, fg=fg, gt=T(gt, dev), W=T(W, dev))


CASES = [("water", lambda: synth.water(), 10, 26, 5),
         ("chon4", lambda: synth.random_chon(np.random.default_rng(2), 4), 8, 14, 6)]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def moving(request, oracle_mod):
    name, make, nr, na, seed = request.param
    mol = make()
    g, phi, dphi, d2phi, basis, Pm, sel, rt, gt, W = synth.ao_moving_system(mol, nr, na, seed=seed)
    inp = oracle_inputs(oracle_mod, g, rt, gt, W)
    ref = oracle_assembly(oracle_mod, g, phi, dphi, d2phi, basis, inp)
    return dict(mol=mol, nr=nr, na=na, g=g, phi=phi, dphi=dphi, d2phi=d2phi, basis=basis, Pm=Pm,
                sel=sel, rt=rt, gt=gt, W=W, ref=ref)


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-6)], ids=["fp64", "mixed"])
def test_end_to_end_against_oracle(dev, moving, prec, tol):
    c = moving
    eng = make_engine(c["g"], dev)
    try:
        inp = gpu_inputs(eng, dev, c["rt"], c["gt"], c["W"], prec)
        FA = eng.fock_derivative(T(c["phi"], dev), T(c["dphi"], dev), T(c["d2phi"], dev),
                                 T(c["basis"].atom, dev, torch.int32), inp["vr"], inp["vg"],
                                 inp["fr"], inp["fg"], inp["gt"], inp["W"], inp["Ew"], inp["Uw"],
                                 inp["Ww"], inp["euw"]).cpu().numpy()
    finally:
        eng.close()
    assert rel(FA, c["ref"]) <= tol
    assert np.abs(FA - FA.transpose(0, 2, 1)).max() <= 1e-14 * np.abs(FA).max()


def test_end_to_end_against_finite_differences(dev, oracle_mod, moving):
    c = moving
    mol = c["mol"]
    eng = make_engine(c["g"], dev)
    try:
        inp = gpu_inputs(eng, dev, c["rt"], c["gt"], c["W"], FP64)
        FA = eng.fock_derivative(T(c["phi"], dev), T(c["dphi"], dev), T(c["d2phi"], dev),
                                 T(c["basis"].atom, dev, torch.int32), inp["vr"], inp["vg"],
                                 inp["fr"], inp["fg"], inp["gt"], inp["W"], inp["Ew"], inp["Uw"],
                                 inp["Ww"], inp["euw"]).cpu().numpy()
    finally:
        eng.close()
    h = 1e-4
    scale = np.abs(FA).max()
    for a in range(3 * mol.n_atom):
        Fs = []
        for sg in (1, -1):
            x = mol.coords.copy()
            x[a // 3, a % 3] += sg * h
            g2, f2, df2 = synth.ao_moving_system(synth.Molecule(mol.symbols, x), c["nr"], c["na"],
                                                 P=c["Pm"], sel=c["sel"])[:3]
            _, vr2, vg2 = oracle_mod.potential(g2.coords, g2.weights, g2.rho, g2.grad_rho)
            Fs.append(oracle_mod.fock_matrix(g2.weights, g2.grad_rho, vr2, vg2, f2, df2))
        assert np.abs(FA[a] - (Fs[0] - Fs[1]) / (2 * h)).max() <= 1e-6 * scale


def random_inputs(rng, n, Pd, NA):
    return dict(vr=rng.normal(size=n), vg=rng.normal(size=n), fr=rng.normal(size=(Pd, n)),
                fg=rng.normal(size=(Pd, n)), gt=rng.normal(size=(Pd, n, 3)),
                W=rng.normal(size=(Pd, n)), Ew=rng.normal(size=(Pd, n)),
                Uw=rng.normal(size=(Pd, n)), Ww=rng.normal(size=(Pd, n)),
                euw=rng.normal(size=(3, n, NA, 3)))


@pytest.mark.parametrize("nr,na", [(8, 14), (30, 110)], ids=["336pts", "9900pts"])
def test_assembly_alone(dev, oracle_mod, nr, na):
    """Same per-point inputs on both sides; the caller order shuffled, the points of the first
    atom and a few more below the cutoff (an atom with no kept point)."""
    mol = synth.water()
    g, phi, dphi, d2phi, basis = synth.ao_moving_system(mol, nr, na, seed=3, rho_min=-1.0)[:5]
    rng = np.random.default_rng(nr)
    perm = rng.permutation(g.n)
    rho = g.rho[perm].copy()
    own = g.atom_of_point[perm]
    rho[own == 0] = 1e-12
    rho[rng.choice(g.n, size=g.n // 10, replace=False)] = 0.0
    gs = synth.GridDensity(g.coords[perm], g.weights[perm], rho, g.grad_rho[perm], own, mol)
    phi, dphi, d2phi = phi[perm], dphi[perm], d2phi[perm]
    Pd = 3 * mol.n_atom
    inp = random_inputs(rng, g.n, Pd, mol.n_atom)
    ref = oracle_assembly(oracle_mod, gs, phi, dphi, d2phi, basis, inp)
    eng = make_engine(gs, dev)
    try:
        got = gpu_assembly(eng, dev, phi, dphi, d2phi, basis, inp)
        again = gpu_assembly(eng, dev, phi, dphi, d2phi, basis, inp)
    finally:
        eng.close()
    assert rel(got, ref) <= 1e-12
    assert np.array_equal(got, again)


def test_all_points_below_cutoff(dev, oracle_mod):
    mol = synth.water()
    g, phi, dphi, d2phi, basis = synth.ao_moving_system(mol, 6, 14, seed=3, rho_min=-1.0)[:5]
    gs = synth.GridDensity(g.coords, g.weights, np.zeros(g.n), g.grad_rho, g.atom_of_point, mol)
    inp = random_inputs(np.random.default_rng(1), g.n, 3 * mol.n_atom, mol.n_atom)
    eng = make_engine(gs, dev)
    try:
        got = gpu_assembly(eng, dev, phi, dphi, d2phi, basis, inp)
    finally:
        eng.close()
    assert got.shape == (9, basis.nbf, basis.nbf) and not got.any()


def test_needs_atom_labels(dev):
    mol = synth.water()
    g, phi, dphi, d2phi, basis = synth.ao_moving_system(mol, 6, 14, seed=3)[:5]
    eng = vv10.VV10(0)
    try:
        eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev))
        inp = random_inputs(np.random.default_rng(1), g.n, 9, 3)
        FA = torch.empty(9, basis.nbf, basis.nbf, dtype=torch.float64, device=dev)
        with pytest.raises(vv10.VV10Error) as ei:
            vv10.vv10_fock_derivative(eng.h, T(phi, dev), T(dphi, dev), T(d2phi, dev),
                                      T(basis.atom, dev, torch.int32), T(inp["vr"], dev),
                                      T(inp["vg"], dev), T(inp["fr"], dev), T(inp["fg"], dev),
                                      T(inp["gt"], dev), T(inp["W"], dev), T(inp["Ew"], dev),
                                      T(inp["Uw"], dev), T(inp["Ww"], dev), T(inp["euw"], dev), FA)
        assert ei.value.status == vv10.VV10_ERR_INVALID_ARG
    finally:
        eng.close()
