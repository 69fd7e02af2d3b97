"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (each error against the FP64 oracle):
  FP64 path:  |dE|/|E| <= 1e-11; potential, Hessian contraction and coordinate terms
              <= 1e-10 relative (L2 / Frobenius over the whole output);
  mixed path: |dE| <= 1e-7 Eh; potential <= 1e-6 relative L2 (vrho and vgamma separately);
              coordinate gradient <= 1e-6 relative.
Every output check also bounds each element, |d_i| <= el_tol (|ref_i| + rms(ref)) with
el_tol = tol (FP64) or 10 tol (mixed; see parity_util), and reports
the largest absolute error (parity_util.check).
Small cases compare every output element; the full-size water-hexamer grid (174,600
points) compares the energy in full and sampled output rows (full j sums) otherwise.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2208_14639_gb300 import synth, vv10
from parity_util import check, rel

pytestmark = pytest.mark.gpu

FP64 = vv10.VV10_FP64
MIXED = vv10.VV10_MIXED_TF32X3
F16 = vv10.VV10_MIXED_F16X3
F64TC = vv10.VV10_FP64_TC
# the two FP64 contractions: FP64 SIMT and five-slice integer products on the tensor cores
F64_PRECS = pytest.mark.parametrize("fp", [FP64, F64TC], ids=["fp64", "fp64tc"])
# the two tensor-core contractions of the mixed path: split TF32 and scaled split FP16
TC_PRECS = pytest.mark.parametrize("tcp", [MIXED, F16], ids=["tf32x3", "f16x3"])




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


def small_systems():
    out = [("water", synth.config_water())]
    for n, seed, na in ((1, 1, 1), (2, 2, 2), (37, 3, 2), (255, 4, 3), (256, 5, 3), (257, 6, 3),
                        (700, 7, 4)):
        out.append((f"rand{n}", synth.random_points(n, seed=seed, n_atom=na)))
    return out


SMALL = small_systems()


@pytest.mark.parametrize("name,g", SMALL, ids=[s[0] for s in SMALL])
@pytest.mark.parametrize("prec", [FP64, MIXED], ids=["fp64", "mixed"])
def test_energy_potential(dev, oracle_mod, name, g, prec):
    e_ref, vr_ref, vg_ref = oracle_mod.potential(g.coords, g.weights, g.rho, g.grad_rho)
    eng = make_engine(g, dev)
    e, vr, vg = eng.energy_potential(prec)
    vr, vg = vr.cpu().numpy(), vg.cpu().numpy()
    if prec == FP64:
        assert abs(e - e_ref) <= 1e-11 * abs(e_ref)
        check(vr, vr_ref, 1e-10)
        check(vg, vg_ref, 1e-10)
    else:
        assert abs(e - e_ref) <= 1e-7
        check(vr, vr_ref, 1e-6)
        check(vg, vg_ref, 1e-6)
    kept = g.rho >= 1e-10
    assert np.all(vr[~kept] == 0.0) and np.all(vg[~kept] == 0.0)
    eng.close()


@F64_PRECS
@pytest.mark.parametrize("name,g", SMALL[:1] + SMALL[3:], ids=[s[0] for s in SMALL[:1] + SMALL[3:]])
def test_hessian_contraction_fp64(dev, oracle_mod, name, g, fp):
    rt, gt = synth.trial_densities(g.molecule, g.coords)
    fr_ref, fg_ref = oracle_mod.hessian_contract(g.coords, g.weights, g.rho, g.grad_rho, rt, gt)
    eng = make_engine(g, dev)
    eng.energy_potential(FP64)
    fr, fg = eng.hessian_contract(T(rt, dev), T(gt, dev), fp)
    check(fr.cpu().numpy(), fr_ref, 1e-10)
    check(fg.cpu().numpy(), fg_ref, 1e-10)
    eng.close()


@F64_PRECS
def test_hessian_single_trial_and_odd_P(dev, oracle_mod, fp):
    g = synth.random_points(300, seed=11, n_atom=3)
    rng = np.random.default_rng(1)
    for P in (1, 5, 33, 65, 130):
        rt = rng.normal(size=(P, g.n)) * g.rho
        gt = rng.normal(size=(P, g.n, 3)) * np.abs(g.grad_rho)[None]
        fr_ref, fg_ref = oracle_mod.hessian_contract(g.coords, g.weights, g.rho, g.grad_rho, rt, gt)
        eng = make_engine(g, dev)
        eng.energy_potential(FP64)
        fr, fg = eng.hessian_contract(T(rt, dev), T(gt, dev), fp)
        check(fr.cpu().numpy(), fr_ref, 1e-10)
        check(fg.cpu().numpy(), fg_ref, 1e-10)
        eng.close()


MIXED_HESS = [("water", synth.config_water()), ("rand255", synth.random_points(255, seed=4, n_atom=3)),
              ("rand700", synth.random_points(700, seed=7, n_atom=4))]


@TC_PRECS
@pytest.mark.parametrize("name,g", MIXED_HESS, ids=[s[0] for s in MIXED_HESS])
def test_hessian_contraction_mixed(dev, oracle_mod, name, g, tcp):
    """Split-TF32 and split-FP16 tensor-core contractions: <= 1e-6 relative Frobenius per
    output, every element within 1e-6 (|ref| + rms)."""
    rt, gt = synth.trial_densities(g.molecule, g.coords)
    fr_ref, fg_ref = oracle_mod.hessian_contract(g.coords, g.weights, g.rho, g.grad_rho, rt, gt)
    eng = make_engine(g, dev)
    eng.energy_potential(MIXED)
    fr, fg = eng.hessian_contract(T(rt, dev), T(gt, dev), tcp)
    vv10.vv10_sync(eng.h)
    check(fr.cpu().numpy(), fr_ref, 1e-6)
    check(fg.cpu().numpy(), fg_ref, 1e-6)
    eng.close()


@TC_PRECS
@pytest.mark.parametrize("P", [1, 33, 65, 97, 200])
def test_hessian_mixed_trial_counts(dev, oracle_mod, P, tcp):
    """Trial counts below one MMA tile, ragged, across the widths where both output kinds share
    a tile (<= 64) or not, and above one launch's 192 (two groups)."""
    g = synth.random_points(300, seed=17, n_atom=3)
    rng = np.random.default_rng(P)
    rt = rng.normal(size=(P, g.n)) * g.rho
    gt = rng.normal(size=(P, g.n, 3)) * np.abs(g.grad_rho)[None]
    fr_ref, fg_ref = oracle_mod.hessian_contract(g.coords, g.weights, g.rho, g.grad_rho, rt, gt)
    eng = make_engine(g, dev)
    eng.energy_potential(MIXED)
    fr, fg = eng.hessian_contract(T(rt, dev), T(gt, dev), tcp)
    vv10.vv10_sync(eng.h)
    check(fr.cpu().numpy(), fr_ref, 1e-6)
    check(fg.cpu().numpy(), fg_ref, 1e-6)
    eng.close()


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-6), (F64TC, 1e-10)],
                         ids=["fp64", "mixed", "fp64tc"])
def test_hessian_vector_product(dev, oracle_mod, prec, tol):
    """vv10_hessian_vector_product: w f^{rho,t} and 2 w (f^{gamma,t} grad rho + f^gamma grad
    rho^t) against the same quantities from the oracle's contraction and potential; dropped
    points zero."""
    g = synth.config_water(n_rad=16, n_ang=38)
    rt, gt = synth.trial_densities(g.molecule, g.coords)
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    fr, fg = oracle_mod.hessian_contract(*args, rt, gt)
    _, _, vg = oracle_mod.potential(*args)
    w = g.weights
    ref_r = w[None] * fr
    ref_g = 2.0 * w[None, :, None] * (fg[..., None] * g.grad_rho[None] + vg[None, :, None] * gt)
    eng = make_engine(g, dev)
    eng.energy_potential(prec)
    hr, hg = eng.hessian_vector_product(T(rt, dev), T(gt, dev), prec)
    vv10.vv10_sync(eng.h)
    hr, hg = hr.cpu().numpy(), hg.cpu().numpy()
    check(hr, ref_r, tol, what="hv_rho")
    check(hg, ref_g, tol, what="hv_grad")
    kept = g.rho >= 1e-10
    assert not hr[:, ~kept].any() and not hg[:, ~kept].any()
    eng.close()


def test_fp64tc_trial_scales(dev, oracle_mod):
    """Trials 20 orders of magnitude apart, one zero trial and one with zero u or y part:
    each column has its own power-of-two factor, so every trial keeps FP64 accuracy relative
    to itself (checked trial by trial, not over the whole output)."""
    g = synth.random_points(400, seed=31, n_atom=3)
    rng = np.random.default_rng(9)
    P = 6
    rt = rng.normal(size=(P, g.n)) * g.rho
    gt = rng.normal(size=(P, g.n, 3)) * np.abs(g.grad_rho)[None]
    rt[1] *= 1e-12
    gt[1] *= 1e-12
    rt[2] *= 1e8
    gt[2] *= 1e8
    rt[3] = 0.0
    gt[3] = 0.0
    gt[4] = 0.0          # no gradient part: y' = 0 in this column
    rt[5] = 0.0          # no density part: u' = 0 in this column
    fr_ref, fg_ref = oracle_mod.hessian_contract(g.coords, g.weights, g.rho, g.grad_rho, rt, gt)
    eng = make_engine(g, dev)
    eng.energy_potential(FP64)
    fr, fg = eng.hessian_contract(T(rt, dev), T(gt, dev), F64TC)
    vv10.vv10_sync(eng.h)
    fr, fg = fr.cpu().numpy(), fg.cpu().numpy()
    for t in range(P):
        if t == 3:
            assert not fr[t].any() and not fg[t].any()
            continue
        check(fr[t], fr_ref[t], 1e-10, what=f"f_rho_t trial {t}")
        check(fg[t], fg_ref[t], 1e-10, what=f"f_gamma_t trial {t}")
    eng.close()


def test_fp64tc_matches_fp64_simt(dev):
    """The two FP64 contractions on the same GPU inputs (a 4-atom CHON system of 26,400
    points, 54 random trials as for the water hexamer): agreement to 1e-11 relative, element
    by element against |ref_i| + rms."""
    g = synth.make_system(synth.random_chon(np.random.default_rng(3), 4), 60, 110)
    rng = np.random.default_rng(54)
    rt = rng.normal(size=(54, g.n)) * g.rho
    gt = rng.normal(size=(54, g.n, 3)) * np.abs(g.grad_rho)[None]
    eng = make_engine(g, dev)
    eng.energy_potential(FP64)
    rtd, gtd = T(rt, dev), T(gt, dev)
    fr0, fg0 = eng.hessian_contract(rtd, gtd, FP64)
    fr0, fg0 = fr0.cpu().numpy(), fg0.cpu().numpy()
    fr1, fg1 = eng.hessian_contract(rtd, gtd, F64TC)
    vv10.vv10_sync(eng.h)
    check(fr1.cpu().numpy(), fr0, 1e-11, what="f_rho_t")
    check(fg1.cpu().numpy(), fg0, 1e-11, what="f_gamma_t")
    eng.close()


@pytest.mark.parametrize("prec", [FP64, MIXED], ids=["fp64", "mixed"])
def test_coordinate_terms(dev, oracle_mod, prec):
    g = synth.config_water()
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    pg_ref = oracle_mod.point_grad(*args)
    rows = np.arange(0, g.n, 97)
    oE, oU, oW = oracle_mod.atom_resolved(*args, g.atom_of_point, 3, rows=rows)
    eng = make_engine(g, dev)
    gp, ga, euw = eng.coord_grad(prec, atoms=True, resolved=True)
    gp, ga, euw = gp.cpu().numpy(), ga.cpu().numpy(), euw.cpu().numpy()
    tol = 1e-10 if prec == FP64 else 1e-6
    check(gp, pg_ref, tol)
    seg = np.array([pg_ref[g.atom_of_point == a].sum(axis=0) for a in range(3)])
    check(ga, seg, 1e-9 if prec == FP64 else 1e-5)
    # translational invariance: the atom terms sum to zero up to rounding
    assert np.abs(ga.sum(axis=0)).max() <= (1e-9 if prec == FP64 else 1e-6) * np.abs(ga).max()
    for q, ref in enumerate((oE, oU, oW)):
        check(euw[q][rows], ref, 1e-10 if prec == FP64 else 1e-5)
    eng.close()


def test_atom_resolved_and_gradient_with_interleaved_atoms(dev, oracle_mod):
    """Points given in a random order (atoms interleaved) are grouped by the library."""
    g = synth.random_points(400, seed=13, n_atom=4)
    perm = np.random.default_rng(0).permutation(g.n)
    h = synth.GridDensity(g.coords[perm], g.weights[perm], g.rho[perm], g.grad_rho[perm],
                          g.atom_of_point[perm], g.molecule)
    args = (h.coords, h.weights, h.rho, h.grad_rho)
    pg_ref = oracle_mod.point_grad(*args)
    ag_ref = oracle_mod.atom_grad(*args, h.atom_of_point, 4)
    oE, oU, oW = oracle_mod.atom_resolved(*args, h.atom_of_point, 4)
    eng = make_engine(h, dev)
    gp, ga, euw = eng.coord_grad(FP64, atoms=True, resolved=True)
    check(gp.cpu().numpy(), pg_ref, 1e-10)
    check(ga.cpu().numpy(), ag_ref, 1e-10)
    euw = euw.cpu().numpy()
    for q, ref in enumerate((oE, oU, oW)):
        check(euw[q], ref, 1e-10)
    eng.close()


def test_permutation_and_determinism(dev):
    g = synth.random_points(333, seed=21, n_atom=3)
    perm = np.random.default_rng(5).permutation(g.n)
    eng = make_engine(g, dev)
    e1, vr1, _ = eng.energy_potential(MIXED)
    e1b, vr1b, _ = eng.energy_potential(MIXED)
    assert e1 == e1b and torch.equal(vr1, vr1b)  # bitwise repeatable
    h = synth.GridDensity(g.coords[perm], g.weights[perm], g.rho[perm], g.grad_rho[perm],
                          g.atom_of_point[perm], g.molecule)
    eng2 = make_engine(h, dev)
    e2, vr2, _ = eng2.energy_potential(FP64)
    e3, vr3, _ = eng.energy_potential(FP64)
    assert abs(e2 - e3) <= 1e-13 * abs(e3)
    check(vr2.cpu().numpy(), vr3.cpu().numpy()[perm], 1e-12)
    eng.close()
    eng2.close()


def test_weight_gradient(dev, oracle_mod):
    g = synth.random_points(500, seed=8, n_atom=3)
    E = oracle_mod.pair_sums(g.coords, g.weights, g.rho, g.grad_rho)["E"]
    ref = g.rho * (oracle_mod.beta() + E)
    eng = make_engine(g, dev)
    eng.energy_potential(FP64)
    check(eng.weight_grad().cpu().numpy(), ref, 1e-10)
    eng.close()


# ----------------------------------------------------------------- full-size grid

@pytest.fixture(scope="module")
def hexamer():
    return synth.config_water_hexamer()


def test_full_size_hexamer_energy_potential(dev, oracle_mod, hexamer):
    g = hexamer
    e_ref = oracle_mod.energy(g.coords, g.weights, g.rho, g.grad_rho)
    rows = np.linspace(0, g.n - 1, 400).astype(np.int64)
    _, vr_ref, vg_ref = oracle_mod.potential(g.coords, g.weights, g.rho, g.grad_rho, rows=rows)
    eng = make_engine(g, dev)
    for prec in (FP64, MIXED):
        e, vr, vg = eng.energy_potential(prec)
        vr, vg = vr.cpu().numpy()[rows], vg.cpu().numpy()[rows]
        if prec == FP64:
            assert abs(e - e_ref) <= 1e-11 * abs(e_ref)
            check(vr, vr_ref, 1e-10)
            check(vg, vg_ref, 1e-10)
        else:
            assert abs(e - e_ref) <= 1e-7
            check(vr, vr_ref, 1e-6)
            check(vg, vg_ref, 1e-6)
    eng.close()


def test_full_size_hexamer_hessian_sampled(dev, oracle_mod, hexamer):
    g = hexamer
    rt, gt = synth.trial_densities(g.molecule, g.coords)
    rows = np.linspace(0, g.n - 1, 96).astype(np.int64)
    fr_ref, fg_ref = oracle_mod.hessian_contract(g.coords, g.weights, g.rho, g.grad_rho, rt, gt,
                                                 rows=rows)
    eng = make_engine(g, dev)
    rtd, gtd = T(rt, dev), T(gt, dev)
    eng.energy_potential(MIXED)
    for tcp in (MIXED, F16):
        fr, fg = eng.hessian_contract(rtd, gtd, tcp)
        vv10.vv10_sync(eng.h)
        check(fr.cpu().numpy()[:, rows], fr_ref, 1e-6, what=f"f_rho_t prec {tcp}")
        check(fg.cpu().numpy()[:, rows], fg_ref, 1e-6, what=f"f_gamma_t prec {tcp}")
    eng.energy_potential(FP64)
    for fp in (FP64, F64TC):
        fr, fg = eng.hessian_contract(rtd, gtd, fp)
        vv10.vv10_sync(eng.h)
        check(fr.cpu().numpy()[:, rows], fr_ref, 1e-10, what=f"f_rho_t prec {fp}")
        check(fg.cpu().numpy()[:, rows], fg_ref, 1e-10, what=f"f_gamma_t prec {fp}")
    eng.close()


# ----------------------------------------------------------------- error paths

def test_error_paths(dev):
    g = synth.random_points(64, seed=3)
    eng = vv10.VV10(0)
    lib = vv10.load()
    # call order: nothing prepared
    assert lib.vv10_energy_potential(eng.h, FP64, None, None, None, None) == vv10.VV10_ERR_INVALID_ARG
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                T(g.atom_of_point, dev, torch.int32), 2)
    rt = T(np.ones((2, g.n)), dev)
    gt = T(np.ones((2, g.n, 3)), dev)
    fr = torch.empty_like(rt)
    with pytest.raises(vv10.VV10Error) as ei:  # Hessian before energy/potential
        vv10.vv10_hessian_contract(eng.h, FP64, rt, gt, fr, fr.clone())
    assert ei.value.status == vv10.VV10_ERR_INVALID_ARG
    # a host pointer where a device pointer is required
    host = np.zeros(g.n)
    st = lib.vv10_energy_potential(eng.h, FP64, None, ctypes.c_void_p(host.ctypes.data), None, None)
    assert st == vv10.VV10_ERR_INVALID_ARG
    # bad precision, P out of range
    assert lib.vv10_energy_potential(eng.h, 7, None, None, None, None) == vv10.VV10_ERR_INVALID_ARG
    # injected allocation failure, then recovery
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev))
    vv10.vv10_debug_inject(eng.h, vv10.VV10_DEBUG_FAIL_ALLOC, 1)
    with pytest.raises(vv10.VV10Error) as ei:
        eng.energy_potential(FP64)
    assert ei.value.status == vv10.VV10_ERR_OOM
    e_ok, _, _ = eng.energy_potential(FP64)
    # bounded wait that runs out: TIMEOUT reported, the context stays usable
    vv10.vv10_debug_inject(eng.h, vv10.VV10_DEBUG_STALL_COPY, 1)
    with pytest.raises(vv10.VV10Error) as ei:
        eng.energy_potential(FP64)
    assert ei.value.status == vv10.VV10_ERR_TIMEOUT
    e_again, _, _ = eng.energy_potential(FP64)
    assert e_again == e_ok
    # non-finite input is rejected
    bad = g.weights.copy()
    bad[5] = np.nan
    with pytest.raises(vv10.VV10Error) as ei:
        eng.prepare(T(g.coords, dev), T(bad, dev), T(g.rho, dev), T(g.grad_rho, dev))
    assert ei.value.status == vv10.VV10_ERR_INVALID_ARG
    # atom index out of range is rejected
    atoms = g.atom_of_point.copy()
    atoms[3] = 9
    with pytest.raises(vv10.VV10Error) as ei:
        eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                    T(atoms, dev, torch.int32), 2)
    assert ei.value.status == vv10.VV10_ERR_INVALID_ARG
    eng.close()


# ----------------------------------------------------------------- 60-atom CHON, 1.36 M points

def chon60_rows(g, oracle_mod, n_spread=128, n_tail=64, n_omg=64):
    """Rows of the 60-atom grid checked against the oracle: n_spread kept points spread over
    the grid, the n_tail kept points of lowest density and the n_omg kept points of largest
    |omega_gamma| not already chosen (where the FP32 pair arithmetic is most fragile: rho^4
    small, omega_gamma up to ~1e10; the two sets overlap, so the second takes the next
    largest)."""
    kept = np.flatnonzero(g.rho >= 1e-10)
    spread = kept[np.linspace(0, kept.size - 1, n_spread).astype(np.int64)]
    tail = kept[np.argsort(g.rho[kept], kind="stable")[:n_tail]]
    om_g = np.abs(oracle_mod.point_props(g.rho[kept], g.grad_rho[kept])["omega_gamma"])
    chosen = set(spread.tolist()) | set(tail.tolist())
    big = [int(i) for i in kept[np.argsort(-om_g, kind="stable")] if int(i) not in chosen][:n_omg]
    rows = np.unique(np.concatenate([spread, tail, np.array(big, dtype=np.int64)]))
    return rows, tail, np.array(big, dtype=np.int64)


def test_full_size_chon60_mixed(dev, oracle_mod):
    """60-atom CHON molecule, 75 x 302 points per atom (1,359,000 points), P = 180, mixed
    precision, against the oracle on >= 256 rows (full j sums): spread rows, the 64 kept
    points of lowest density and the 64 of largest |omega_gamma|.  Potential, Hessian
    contraction, point gradient and the per-row energy terms dE/dw_i = rho_i (beta + E_i)
    (their weighted sum over the rows is the rows' share of the energy) each per element;
    the energy against the FP64 GPU path (|dE| <= 1e-7 Eh)."""
    g = synth.config_chon60()
    eng = make_engine(g, dev)
    xyz = T(g.coords, dev)
    rt, gt = synth.trial_densities_torch(g.molecule, xyz)
    assert rt.shape == (180, g.n)
    e_mixed, vr, vg = eng.energy_potential(MIXED)
    dedw = eng.weight_grad()
    fr, fg = eng.hessian_contract(rt, gt, MIXED)
    gp, _, _ = eng.coord_grad(MIXED, atoms=False)
    vv10.vv10_sync(eng.h)
    rows, tail, big = chon60_rows(g, oracle_mod)
    assert rows.size >= 250 and tail.size == 64 and big.size == 64  # overlap of spread and tail only
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    _, vr_ref, vg_ref = oracle_mod.potential(*args, rows=rows)
    check(vr.cpu().numpy()[rows], vr_ref, 1e-6, what="vrho")
    check(vg.cpu().numpy()[rows], vg_ref, 1e-6, what="vgamma")
    E_ref = oracle_mod.pair_sums(*args, rows=rows)["E"]
    dedw_ref = g.rho[rows] * (oracle_mod.beta() + E_ref)
    dedw = dedw.cpu().numpy()[rows]
    check(dedw, dedw_ref, 1e-6, what="dE/dw")
    # the rows' share of E = sum_i w_i rho_i (beta + E_i / 2)
    share = lambda d: float(np.sum(g.weights[rows] * (0.5 * d + 0.5 * g.rho[rows] * oracle_mod.beta())))
    assert abs(share(dedw) - share(dedw_ref)) <= 1e-8
    fr_ref, fg_ref = oracle_mod.hessian_contract(*args, rt.cpu().numpy(), gt.cpu().numpy(), rows=rows)
    check(fr.cpu().numpy()[:, rows], fr_ref, 1e-6, what="f_rho_t")
    check(fg.cpu().numpy()[:, rows], fg_ref, 1e-6, what="f_gamma_t")
    fr, fg = eng.hessian_contract(rt, gt, F16)  # the split-FP16 contraction, same rows
    vv10.vv10_sync(eng.h)
    check(fr.cpu().numpy()[:, rows], fr_ref, 1e-6, what="f_rho_t (f16x3)")
    check(fg.cpu().numpy()[:, rows], fg_ref, 1e-6, what="f_gamma_t (f16x3)")
    check(gp.cpu().numpy()[rows], oracle_mod.point_grad(*args, rows=rows), 1e-6, what="grad")
    e_fp64, _, _ = eng.energy_potential(FP64, want_energy=True)
    assert abs(e_mixed - e_fp64) <= 1e-7
    eng.close()


# ----------------------------------------------------------------- limits and degenerate inputs

@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-6), (F16, 1e-6), (F64TC, 1e-10)],
                         ids=["fp64", "tf32x3", "f16x3", "fp64tc"])
def test_hessian_maximum_trial_count(dev, oracle_mod, prec, tol):
    """P = VV10_MAX_TRIALS (4096): 22 tensor-core groups of 187 trials, 64 groups of 64 on the
    FP64 tensor-core path, or 128 FP64 chunks."""
    g = synth.random_points(96, seed=23, n_atom=2)
    P = 4096
    rng = np.random.default_rng(5)
    rt = rng.normal(size=(P, g.n)) * g.rho
    gt = rng.normal(size=(P, g.n, 3)) * np.abs(g.grad_rho)[None]
    fr_ref, fg_ref = oracle_mod.hessian_contract(g.coords, g.weights, g.rho, g.grad_rho, rt, gt)
    eng = make_engine(g, dev)
    eng.energy_potential(prec)
    fr, fg = eng.hessian_contract(T(rt, dev), T(gt, dev), prec)
    vv10.vv10_sync(eng.h)
    check(fr.cpu().numpy(), fr_ref, tol)
    check(fg.cpu().numpy(), fg_ref, tol)
    with pytest.raises(vv10.VV10Error):  # one more is refused
        eng.hessian_contract(T(np.zeros((P + 1, g.n)), dev), T(np.zeros((P + 1, g.n, 3)), dev), prec)
    eng.close()


@pytest.mark.parametrize("prec", [FP64, MIXED, F64TC], ids=["fp64", "mixed", "fp64tc"])
def test_all_points_below_cutoff(dev, prec):
    """Every point below rho_cut: no kept point, zero energy and zero outputs everywhere."""
    g0 = synth.random_points(50, seed=29, n_atom=2)
    g = synth.GridDensity(g0.coords, g0.weights, np.full(g0.n, 1e-12), g0.grad_rho * 1e-12,
                          g0.atom_of_point, g0.molecule)
    eng = vv10.VV10(0)
    nk = eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                     T(g.atom_of_point, dev, torch.int32), g.molecule.n_atom)
    assert nk == 0
    e, vr, vg = eng.energy_potential(prec)
    assert e == 0.0 and not vr.any() and not vg.any()
    rt = torch.ones(3, g.n, dtype=torch.float64, device=dev)
    gt = torch.ones(3, g.n, 3, dtype=torch.float64, device=dev)
    fr, fg = eng.hessian_contract(rt, gt, prec)
    gp, ga, euw = eng.coord_grad(prec, atoms=True, resolved=True)
    vv10.vv10_sync(eng.h)
    for t in (fr, fg, gp, ga, euw):
        assert not t.any()
    # the one-call evaluation (both of its pass layouts), the energy alone and the calls beyond
    # the step: zero results, outputs given non-zero beforehand are overwritten
    na = g.molecule.n_atom
    full = lambda *shape: torch.full(shape, 5.0, dtype=torch.float64, device=dev)
    for resolved in (True, False):
        out = dict(vrho=full(g.n), vgamma=full(g.n), f_rho_t=full(3, g.n), f_gamma_t=full(3, g.n),
                   grad_points=full(g.n, 3), grad_atoms=full(na, 3),
                   EUW_Bgr=full(3, g.n, na, 3) if resolved else None)
        assert vv10.vv10_evaluate(eng.h, prec, rt, gt, **out) == 0.0
        assert not any(t.any() for t in out.values() if t is not None)
    assert eng.energy(prec) == 0.0
    E, D = eng.coord_hessian(prec, points=True)
    Ew, Uw, Ww = eng.weight_response(torch.ones(2, g.n, dtype=torch.float64, device=dev), prec)
    ng = eng.nuclear_gradient(w_t=torch.ones(2, g.n, dtype=torch.float64, device=dev))
    vv10.vv10_sync(eng.h)
    for t in (E, D, Ew, Uw, Ww, ng):
        assert not t.any()
    eng.close()
