"""Fused passes: the A/B/C sums formed in the energy pass (VV10_OPT_FUSE_HESSIAN_SUMS) and the
point gradient taken from the atom-resolved pass give the oracle's results, and the calls
that follow run no pair pass of their own."""
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
def case(oracle_mod):
    g = synth.random_points(1500, seed=101, n_atom=4)
    rng = np.random.default_rng(7)
    P = 20
    rt = rng.normal(size=(P, g.n)) * g.rho
    gt = rng.normal(size=(P, g.n, 3)) * (np.abs(g.grad_rho) + 1e-3 * g.rho[:, None])
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    e, vr, vg = oracle_mod.potential(*args)
    fr, fg = oracle_mod.hessian_contract(*args, rt, gt)
    gp = oracle_mod.point_grad(*args)
    ga = oracle_mod.atom_grad(*args, g.atom_of_point, g.molecule.n_atom)
    euw = np.stack(oracle_mod.atom_resolved(*args, g.atom_of_point, g.molecule.n_atom))
    return g, rt, gt, dict(e=e, vr=vr, vg=vg, fr=fr, fg=fg, gp=gp, ga=ga, euw=euw)


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-6)], ids=["fp64", "mixed"])
def test_fused_hessian_sums(dev, case, prec, tol):
    g, rt, gt, ref = case
    eng = vv10.VV10(0)
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                T(g.atom_of_point, dev, torch.int32), g.molecule.n_atom)
    vv10.vv10_set_options(eng.h, vv10.VV10_OPT_FUSE_HESSIAN_SUMS)
    vv10.vv10_profile_enable(eng.h, True)
    vv10.vv10_profile_read(eng.h)
    e, vr, vg = eng.energy_potential(prec)
    p_energy = vv10.vv10_profile_read(eng.h)
    fr, fg = eng.hessian_contract(T(rt, dev), T(gt, dev), prec)
    vv10.vv10_sync(eng.h)
    p_hess = vv10.vv10_profile_read(eng.h)
    assert p_energy["pair_sums_EUW"][1] == 1 and p_energy["pair_sums_ABC"][1] == 1  # 1 pass + A/B/C epilogue
    assert p_hess["pair_sums_ABC"][1] == 0 and p_hess["pair_sums_EUW"][1] == 0      # no pair pass
    if prec == FP64:
        assert abs(e - ref["e"]) <= 1e-11 * abs(ref["e"])
    else:
        assert abs(e - ref["e"]) <= 1e-7
    for x, y in ((vr, ref["vr"]), (vg, ref["vg"]), (fr, ref["fr"]), (fg, ref["fg"])):
        assert rel(x.cpu().numpy(), y) <= tol
    # after an unfused energy call of the other precision the Hessian recomputes what it needs
    vv10.vv10_set_options(eng.h, 0)
    eng.energy_potential(MIXED if prec == FP64 else FP64)
    fr2, fg2 = eng.hessian_contract(T(rt, dev), T(gt, dev), prec)
    assert rel(fr2.cpu().numpy(), ref["fr"]) <= tol and rel(fg2.cpu().numpy(), ref["fg"]) <= tol
    with pytest.raises(vv10.VV10Error):
        vv10.vv10_set_options(eng.h, 2)
    eng.close()


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-6)], ids=["fp64", "mixed"])
def test_gradient_from_atom_resolved_pass(dev, case, prec, tol):
    g, _, _, ref = case
    eng = vv10.VV10(0)
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                T(g.atom_of_point, dev, torch.int32), g.molecule.n_atom)
    eng.energy_potential(prec)
    vv10.vv10_profile_enable(eng.h, True)
    vv10.vv10_profile_read(eng.h)
    gp, ga, euw = eng.coord_grad(prec, atoms=True, resolved=True)
    vv10.vv10_sync(eng.h)
    prof = vv10.vv10_profile_read(eng.h)
    assert prof["pair_sums_grad"][1] == 0 and prof["atom_resolved"][1] == 1
    assert rel(gp.cpu().numpy(), ref["gp"]) <= tol
    assert rel(ga.cpu().numpy(), ref["ga"]) <= tol
    assert rel(euw.cpu().numpy(), ref["euw"]) <= tol
    # the same gradient as the separate gradient pass
    gp2, ga2, _ = eng.coord_grad(prec, atoms=True, resolved=False)
    assert rel(gp.cpu().numpy(), gp2.cpu().numpy()) <= (1e-13 if prec == FP64 else 1e-6)
    assert rel(ga.cpu().numpy(), ga2.cpu().numpy()) <= (1e-13 if prec == FP64 else 1e-6)
    eng.close()


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (MIXED, 1e-6)], ids=["fp64", "mixed"])
@pytest.mark.parametrize("resolved", [True, False], ids=["atom-resolved-pass", "sums-and-gradient-pass"])
def test_evaluate_everything_in_one_call(dev, case, prec, tol, resolved):
    g, rt, gt, ref = case
    eng = vv10.VV10(0)
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                T(g.atom_of_point, dev, torch.int32), g.molecule.n_atom)
    f64 = dict(dtype=torch.float64, device=dev)
    n, na, P = g.n, g.molecule.n_atom, rt.shape[0]
    out = dict(vrho=torch.empty(n, **f64), vgamma=torch.empty(n, **f64),
               f_rho_t=torch.empty(P, n, **f64), f_gamma_t=torch.empty(P, n, **f64),
               grad_points=torch.empty(n, 3, **f64), grad_atoms=torch.empty(na, 3, **f64),
               EUW_Bgr=torch.empty(3, n, na, 3, **f64) if resolved else None)
    vv10.vv10_profile_enable(eng.h, True)
    vv10.vv10_profile_read(eng.h)
    e = vv10.vv10_evaluate(eng.h, prec, T(rt, dev), T(gt, dev), **out)
    prof = vv10.vv10_profile_read(eng.h)
    if resolved:  # a single pass over the pairs
        assert prof["atom_resolved"][1] == 1 and prof["pair_sums_EUW"][1] == 0
        assert prof["pair_sums_grad"][1] == 0
    else:  # one pass for the six row sums and the gradient (MODE_EUWABCG)
        assert prof["pair_sums_EUW"][1] == 1 and prof["pair_sums_grad"][1] == 0
    if prec == FP64:
        assert abs(e - ref["e"]) <= 1e-11 * abs(ref["e"])
    else:
        assert abs(e - ref["e"]) <= 1e-7
    for name, key in (("vrho", "vr"), ("vgamma", "vg"), ("f_rho_t", "fr"), ("f_gamma_t", "fg"),
                      ("grad_points", "gp"), ("grad_atoms", "ga")):
        assert rel(out[name].cpu().numpy(), ref[key]) <= tol, name
    if resolved:
        assert rel(out["EUW_Bgr"].cpu().numpy(), ref["euw"]) <= tol
    # the cached sums serve a later Hessian call
    fr, fg = eng.hessian_contract(T(rt, dev), T(gt, dev), prec)
    assert rel(fr.cpu().numpy(), ref["fr"]) <= tol
    # no trials: energy and coordinate terms only
    e0 = vv10.vv10_evaluate(eng.h, prec, vrho=out["vrho"], grad_points=out["grad_points"])
    # (the one-pass and the pair-sum kernels sum their FP32 tiles in different orders)
    assert abs(e0 - e) <= (1e-12 * abs(e) if prec == FP64 else 1e-7)
    eng.close()


def test_engine_evaluate_convenience(dev, case):
    g, rt, gt, ref = case
    eng = vv10.VV10(0)
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                T(g.atom_of_point, dev, torch.int32), g.molecule.n_atom)
    e, vr, vg, fr, fg, gp, ga, euw = eng.evaluate(MIXED, T(rt, dev), T(gt, dev), resolved=True)
    assert abs(e - ref["e"]) <= 1e-7
    assert rel(fr.cpu().numpy(), ref["fr"]) <= 1e-6 and rel(euw.cpu().numpy(), ref["euw"]) <= 1e-6
    e2, *_ = eng.evaluate(MIXED)  # no trials, no atom-resolved terms
    assert abs(e2 - ref["e"]) <= 1e-7
    eng.close()
