"""Parity of the weight-derivative sums (Sec. II.B: E_i^{Bw}, U_i^{Bw}, W_i^{Bw} for given weight
directions) with the FP64 oracle, through the C ABI.

Tolerances against the FP64 oracle (relative Frobenius norm over each output, E, U and W
separately): FP64 path <= 1e-10, mixed path <= 1e-6.  The mixed path runs on tensor cores
(split TF32) from 5 directions up and as FP32 SIMT arithmetic below.  Small systems compare
every element; the full-size water-hexamer grid with its 54 Becke weight directions compares
sampled rows (full j sums) and checks properties that hold at any size: the symmetry of the
weight-weight second derivative sum_i a_i rho_i E_i^b, and, with w itself as the direction,
the row sums E_i that vv10_weight_grad reports.
"""
import numpy as np
import pytest
import torch

from paper_2208_14639_gb300 import synth, vv10

pytestmark = pytest.mark.gpu

FP64 = vv10.VV10_FP64
MIXED = vv10.VV10_MIXED_TF32X3
TOL = {FP64: 1e-10, MIXED: 1e-6}


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


def random_dirs(g, P, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(P, g.n)) * g.weights[None, :]


def check(eng, g, V, prec, oracle_mod, rows=None):
    ref = oracle_mod.weight_response(g.coords, g.weights, g.rho, g.grad_rho, V, rows=rows)
    got = eng.weight_response(T(V, eng_dev(eng)), prec)
    for x, r in zip(got, ref):
        x = x.cpu().numpy()
        if rows is not None:
            x = x[:, rows]
        assert rel(x, r) <= TOL[prec]
    return got


def eng_dev(eng):
    return torch.device("cuda", eng.device)


CASES = [("rand1", 1, 1, 1), ("rand2", 2, 2, 3), ("rand37", 37, 3, 5), ("rand255", 255, 4, 8),
         ("rand256", 256, 5, 9), ("rand257", 257, 6, 16), ("rand700", 700, 7, 17),
         ("rand1500", 1500, 8, 33)]


@pytest.mark.parametrize("prec", [FP64, MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name,n,seed,P", CASES, ids=[c[0] for c in CASES])
def test_random_systems(dev, oracle_mod, name, n, seed, P, prec):
    """Ragged point counts around the 128-row and 128-j tiles, direction counts around the
    8- and 16-direction groups."""
    g = synth.random_points(n, seed=seed, n_atom=3)
    eng = make_engine(g, dev)
    check(eng, g, random_dirs(g, P, seed + 100), prec, oracle_mod)
    eng.close()


@pytest.mark.parametrize("P", [4, 5, 32, 33, 63, 64, 65, 130])
def test_direction_groups(dev, oracle_mod, P):
    """Direction counts around the tensor-core path's limits: below 5 directions the mixed
    path uses the SIMT kernel, up to 32 one 32-wide group, up to 64 one 64-wide group, then
    several groups."""
    g = synth.random_points(900, seed=70 + P, n_atom=3)
    eng = make_engine(g, dev)
    check(eng, g, random_dirs(g, P, P), MIXED, oracle_mod)
    eng.close()


@pytest.mark.parametrize("prec", [FP64, MIXED], ids=["fp64", "mixed"])
def test_water_becke_directions(dev, oracle_mod, prec):
    """The water grid with the nuclear derivatives of its Becke weights (P = 9)."""
    g = synth.config_water()
    V = synth.weight_directions(g.molecule, 30, 110)
    eng = make_engine(g, dev)
    check(eng, g, V, prec, oracle_mod)
    eng.close()


def test_cutoff_optional_outputs_and_repeatability(dev, oracle_mod):
    g = synth.random_points(500, seed=61, n_atom=2)
    rho = g.rho.copy()
    rho[::7] = 0.0  # below the cutoff: zero outputs, no contribution
    h = synth.GridDensity(g.coords, g.weights, rho, g.grad_rho, g.atom_of_point, g.molecule)
    V = random_dirs(h, 11, 5)
    eng = make_engine(h, dev)
    for prec in (FP64, MIXED):
        E, U, W = check(eng, h, V, prec, oracle_mod)
        assert not E[:, ::7].any() and not U[:, ::7].any() and not W[:, ::7].any()
        E2, U2, W2 = eng.weight_response(T(V, dev), prec)
        assert torch.equal(E, E2) and torch.equal(U, U2) and torch.equal(W, W2)
        Wonly = torch.full_like(W, 3.0)
        vv10.vv10_weight_response(eng.h, prec, T(V, dev), None, None, Wonly)
        assert torch.equal(Wonly, W)
    eng.close()


def test_argument_errors(dev):
    g = synth.random_points(64, seed=62, n_atom=2)
    eng = make_engine(g, dev)
    V = T(random_dirs(g, 2, 1), dev)
    out = torch.empty_like(V)
    with pytest.raises(vv10.VV10Error):
        vv10.vv10_weight_response(eng.h, 7, V, out)
    with pytest.raises(ValueError):
        vv10.vv10_weight_response(eng.h, FP64, V, torch.empty(3, g.n, dtype=torch.float64, device=dev))
    with pytest.raises(TypeError):
        vv10.vv10_weight_response(eng.h, FP64, V.cpu(), out)
    big = torch.zeros(vv10.VV10_MAX_TRIALS + 1, g.n, dtype=torch.float64, device=dev)
    with pytest.raises(vv10.VV10Error):
        vv10.vv10_weight_response(eng.h, FP64, big, torch.empty_like(big))
    eng.close()


# ----------------------------------------------------------------- full-size grid

@pytest.fixture(scope="module")
def hexamer():
    return synth.config_water_hexamer()


def test_full_size_hexamer(dev, oracle_mod, hexamer):
    g = hexamer
    V = synth.weight_directions(g.molecule, 50, 194)  # P = 54
    rows = np.linspace(0, g.n - 1, 24).astype(np.int64)
    eng = make_engine(g, dev)
    Vd = T(V, dev)
    res = {}
    for prec in (FP64, MIXED):
        res[prec] = check(eng, g, V, prec, oracle_mod, rows=rows)
    # the weight-weight second derivative sum_i a_i rho_i E_i^b is symmetric in (a, b)
    E = res[FP64][0].cpu().numpy()
    M = (V * g.rho[None, :]) @ E.T
    assert np.abs(M - M.T).max() <= 1e-9 * np.abs(M).max()
    assert rel(res[MIXED][0].cpu().numpy(), E) <= TOL[MIXED]
    # with w as the direction: E_i, as vv10_weight_grad reports it (dE/dw_i = rho_i (beta + E_i))
    Ew, _, _ = eng.weight_response(T(g.weights[None, :], dev), FP64)
    eng.energy_potential(FP64)
    kept = g.rho >= 1e-10
    Ei = eng.weight_grad().cpu().numpy()[kept] / g.rho[kept] - oracle_mod.beta()
    assert rel(Ew.cpu().numpy()[0][kept], Ei) <= 1e-10
    del Vd
    eng.close()
