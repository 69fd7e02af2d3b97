"""Parity of the grid-grid block of the nuclear Hessian (Sec. II.B: D_i^B and E^{AB}_{gr,gr})
with the FP64 oracle, through the C ABI.

Tolerances against the FP64 oracle (relative Frobenius norm over the whole output):
  FP64 path:  blocks and per-point D_i^B <= 1e-10;
  mixed path: blocks <= 1e-6, per-point D_i^B <= 1e-5 (as for the other per-point,
              per-atom coordinate terms: single rows of far atoms are small sums of FP32
              terms).
Small systems compare every element; the full-size water-hexamer grid compares sampled
D_i^B rows with the oracle's full j sums, and the blocks through properties that hold at
any size: symmetry, the per-point sums, and finite differences of the atom gradient.
Without the per-point output the library evaluates only the atom pairs A < B (the pair
term is symmetric in i and j); both ways are checked.
"""
import numpy as np
import pytest
import torch

from paper_2208_14639_gb300 import synth, vv10

pytestmark = pytest.mark.gpu

FP64 = vv10.VV10_FP64
MIXED = vv10.VV10_MIXED_TF32X3
TOL_BLOCKS = {FP64: 1e-10, MIXED: 1e-6}
TOL_POINTS = {FP64: 1e-10, MIXED: 1e-5}


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


def make_engine(g, dev, coords=None):
    eng = vv10.VV10(0)
    eng.prepare(T(g.coords if coords is None else coords, dev), T(g.weights, dev), T(g.rho, dev),
                T(g.grad_rho, dev), T(g.atom_of_point, dev, torch.int32), g.molecule.n_atom)
    return eng


def oracle_refs(oracle_mod, g):
    args = (g.coords, g.weights, g.rho, g.grad_rho, g.atom_of_point, g.molecule.n_atom)
    return oracle_mod.coord_hessian(*args), oracle_mod.point_coord_hessian(*args)


def small_systems():
    out = [("water", synth.config_water())]
    # one atom (no off-diagonal blocks), segments shorter than, equal to and just above one
    # CTA's 128 rows, several CTAs per atom with ragged tails
    for n, seed, na in ((1, 1, 1), (2, 2, 2), (37, 3, 2), (255, 4, 3), (256, 5, 2), (257, 6, 2),
                        (700, 7, 4), (1500, 9, 5)):
        out.append((f"rand{n}", synth.random_points(n, seed=seed, n_atom=na)))
    return out


SMALL = small_systems()


@pytest.mark.parametrize("prec", [FP64, MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name,g", SMALL, ids=[s[0] for s in SMALL])
def test_small_systems(dev, oracle_mod, name, g, prec):
    E_ref, D_ref = oracle_refs(oracle_mod, g)
    eng = make_engine(g, dev)
    E, D = eng.coord_hessian(prec, points=True)
    E, D = E.cpu().numpy(), D.cpu().numpy()
    assert rel(E, E_ref) <= TOL_BLOCKS[prec]
    assert rel(D, D_ref) <= TOL_POINTS[prec]
    Eh, _ = eng.coord_hessian(prec, points=False)
    assert rel(Eh.cpu().numpy(), E_ref) <= TOL_BLOCKS[prec]
    # D_i^B is zero for the own atom
    na = g.molecule.n_atom
    assert not D[np.arange(g.n), g.atom_of_point].any()
    # translational invariance of the blocks (the diagonal is minus the row sum)
    scale = max(np.abs(E).max(), 1e-300)
    assert np.abs(E.sum(axis=1)).max() <= 1e-12 * scale * na
    eng.close()


def test_outputs_optional_and_repeatable(dev):
    g = synth.random_points(900, seed=41, n_atom=3)
    eng = make_engine(g, dev)
    for prec in (FP64, MIXED):
        E1, D1 = eng.coord_hessian(prec, points=True)
        E2, _ = eng.coord_hessian(prec, points=False)  # the atom pairs A < B only
        E3, D3 = eng.coord_hessian(prec, points=True)
        E4, _ = eng.coord_hessian(prec, points=False)
        assert torch.equal(E1, E3) and torch.equal(D1, D3) and torch.equal(E2, E4)
        # the half evaluation is exactly symmetric and agrees with the full one
        assert torch.equal(E2, E2.transpose(0, 1).transpose(2, 3))
        assert rel(E2.cpu().numpy(), E1.cpu().numpy()) <= (1e-13 if prec == FP64 else 1e-6)
        # D_i^B alone (the blocks go to scratch)
        D4 = torch.full_like(D1, 7.0)
        vv10.vv10_coord_hessian(eng.h, prec, None, D4)
        assert torch.equal(D1, D4)
    vv10.vv10_coord_hessian(eng.h, FP64, None, None)  # nothing asked: no-op
    eng.close()


def test_interleaved_atoms_and_empty_atoms(dev, oracle_mod):
    """Points in a random order (atoms interleaved) are grouped by the library; an atom all of
    whose points lie below the density cutoff, and an atom with no points, give zero blocks."""
    g = synth.random_points(600, seed=43, n_atom=4)
    rho = g.rho.copy()
    rho[g.atom_of_point == 1] = 0.0          # atom 1: every point below the cutoff
    aop = g.atom_of_point.copy()
    aop[aop == 3] = 2                        # atom 3: no points at all
    perm = np.random.default_rng(2).permutation(g.n)
    h = synth.GridDensity(g.coords[perm], g.weights[perm], rho[perm], g.grad_rho[perm],
                          aop[perm], g.molecule)
    E_ref, D_ref = oracle_refs(oracle_mod, h)
    eng = make_engine(h, dev)
    E, D = eng.coord_hessian(FP64, points=True)
    E, D = E.cpu().numpy(), D.cpu().numpy()
    assert rel(E, E_ref) <= 1e-10 and rel(D, D_ref) <= 1e-10
    Eh, _ = eng.coord_hessian(FP64, points=False)
    assert rel(Eh.cpu().numpy(), E_ref) <= 1e-10
    for a in (1, 3):
        assert not E[a].any() and not E[:, a].any()
    assert not D[h.atom_of_point == 1].any()
    eng.close()


def test_needs_atom_labels(dev):
    g = synth.random_points(64, seed=44, n_atom=2)
    eng = vv10.VV10(0)
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev))
    E = torch.empty(2, 2, 3, 3, dtype=torch.float64, device=dev)
    with pytest.raises(vv10.VV10Error):
        vv10.vv10_coord_hessian(eng.h, FP64, E, None)
    eng.close()
    eng = make_engine(g, dev)
    with pytest.raises(vv10.VV10Error):
        vv10.vv10_coord_hessian(eng.h, 7, E, None)
    eng.close()


# ----------------------------------------------------------------- full-size grid

@pytest.fixture(scope="module")
def hexamer():
    return synth.config_water_hexamer()


def test_full_size_hexamer(dev, oracle_mod, hexamer):
    g = hexamer
    na = g.molecule.n_atom
    rows = np.linspace(0, g.n - 1, 48).astype(np.int64)
    D_ref = oracle_mod.point_coord_hessian(g.coords, g.weights, g.rho, g.grad_rho,
                                           g.atom_of_point, na, rows=rows)
    eng = make_engine(g, dev)
    out = {}
    for prec in (FP64, MIXED):
        E, D = eng.coord_hessian(prec, points=True)
        E, D = E.cpu().numpy(), D.cpu().numpy()
        out[prec] = E
        assert rel(D[rows], D_ref) <= TOL_POINTS[prec]
        scale = np.abs(E).max()
        # a symmetric Hessian: E^{AB} = (E^{BA})^T and each block symmetric
        assert np.abs(E - E.transpose(1, 0, 3, 2)).max() <= (1e-10 if prec == FP64 else 1e-6) * scale
        assert np.abs(E - E.transpose(0, 1, 3, 2)).max() == 0.0
        # the blocks are the weighted per-point sums
        c = g.weights * g.rho
        for A in range(na):
            m = g.atom_of_point == A
            blk = np.einsum("i,ibuv->buv", c[m], D[m])
            off = [B for B in range(na) if B != A]
            assert rel(E[A, off], blk[off]) <= 1e-12
    assert rel(out[MIXED], out[FP64]) <= TOL_BLOCKS[MIXED]
    # the blocks alone: the atom pairs A < B only, exactly symmetric
    for prec in (FP64, MIXED):
        Eh, _ = eng.coord_hessian(prec)
        Eh = Eh.cpu().numpy()
        assert np.array_equal(Eh, Eh.transpose(1, 0, 3, 2))
        assert rel(Eh, out[FP64]) <= TOL_BLOCKS[prec]
    eng.close()
    # finite differences of the FP64 atom gradient when the points of one atom move rigidly
    B, hstep = 4, 1e-4
    fd = np.zeros((na, 3, 3))
    for d in range(3):
        ga = []
        for sgn in (1, -1):
            c = g.coords.copy()
            c[g.atom_of_point == B, d] += sgn * hstep
            e2 = make_engine(g, dev, coords=c)
            _, gat, _ = e2.coord_grad(FP64, atoms=True)
            ga.append(gat.cpu().numpy())
            e2.close()
        fd[:, :, d] = (ga[0] - ga[1]) / (2 * hstep)
    assert rel(out[FP64][:, B], fd) <= 1e-6
