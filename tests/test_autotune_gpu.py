"""Autotuner and tile-shape controls: every tuned or fixed shape gives the oracle's results
within the stated tolerances, tuned choices are cached across handles, fixed shapes are
never replaced, and tuning runs do not show in the launch counters."""
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
def system():
    return synth.random_points(3000, seed=81, n_atom=5)


@pytest.fixture(scope="module")
def refs(oracle_mod, system):
    g = system
    rng = np.random.default_rng(4)
    P = 100
    rt = rng.normal(size=(P, g.n)) * g.rho
    gt = rng.normal(size=(P, g.n, 3)) * (np.abs(g.grad_rho) + 1e-3 * g.rho[:, None])
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    e, vr, vg = oracle_mod.potential(*args)
    fr, fg = oracle_mod.hessian_contract(*args, rt, gt)
    gp = oracle_mod.point_grad(*args)
    return dict(rt=rt, gt=gt, e=e, vr=vr, vg=vg, fr=fr, fg=fg, gp=gp)


def run_all(eng, g, refs, dev, prec):
    e, vr, vg = eng.energy_potential(prec)
    fr, fg = eng.hessian_contract(T(refs["rt"], dev), T(refs["gt"], dev), prec)
    gp = torch.zeros(g.n, 3, dtype=torch.float64, device=dev)
    vv10.vv10_coord_grad(eng.h, prec, gp)
    vv10.vv10_sync(eng.h)
    return e, vr.cpu().numpy(), vg.cpu().numpy(), fr.cpu().numpy(), fg.cpu().numpy(), gp.cpu().numpy()


def check(out, refs, prec):
    e, vr, vg, fr, fg, gp = out
    if prec == FP64:
        assert abs(e - refs["e"]) <= 1e-11 * abs(refs["e"])
        tol = 1e-10
    else:
        assert abs(e - refs["e"]) <= 1e-7
        tol = 1e-6
    for x, y in ((vr, refs["vr"]), (vg, refs["vg"]), (fr, refs["fr"]), (fg, refs["fg"]), (gp, refs["gp"])):
        assert rel(x, y) <= tol


def engine(g, dev):
    eng = vv10.VV10(0)
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                T(g.atom_of_point, dev, torch.int32), g.molecule.n_atom)
    return eng


@pytest.mark.parametrize("prec", [FP64, MIXED], ids=["fp64", "mixed"])
def test_tuned_pairsums_match_oracle_and_are_cached(dev, system, refs, prec):
    g = system
    eng = engine(g, dev)
    vv10.vv10_profile_enable(eng.h, True)
    vv10.vv10_profile_read(eng.h)
    vv10.vv10_autotune(eng.h, prec, vv10.VV10_TUNE_PAIRSUMS)
    counted = vv10.vv10_profile_read(eng.h)
    assert sum(n for _, n in counted.values()) == 0  # tuning runs are not counted
    fp64 = 1 if prec == FP64 else 0
    chosen = [vv10.vv10_get_tiles(eng.h, mode + 3 * fp64) for mode in range(3)]
    for rpt, ns in chosen:
        assert rpt in ((1, 2) if fp64 else (1, 2, 4)) and ns >= 1
    check(run_all(eng, g, refs, dev, prec), refs, prec)
    # a second handle tuning on first use finds the cached choices
    eng2 = engine(g, dev)
    vv10.vv10_set_autotune(eng2.h, vv10.VV10_TUNE_PAIRSUMS)
    out = run_all(eng2, g, refs, dev, prec)
    assert [vv10.vv10_get_tiles(eng2.h, mode + 3 * fp64) for mode in range(3)] == chosen
    check(out, refs, prec)
    eng2.close()
    eng.close()


@pytest.mark.parametrize("width", [32, 64, 96, 128, 192])
def test_contraction_widths_match_oracle(dev, system, refs, width):
    g = system
    eng = engine(g, dev)
    vv10.vv10_set_tiles(eng.h, vv10.TILES_CONTRACTION, width, 0)
    assert vv10.vv10_get_tiles(eng.h, vv10.TILES_CONTRACTION)[0] == width
    check(run_all(eng, g, refs, dev, MIXED), refs, MIXED)
    eng.close()


def test_contraction_width_tuned_on_first_use(dev, system, refs):
    g = system
    eng = engine(g, dev)
    vv10.vv10_set_autotune(eng.h, vv10.VV10_TUNE_CONTRACTION | vv10.VV10_TUNE_PAIRSUMS)
    assert vv10.vv10_get_tiles(eng.h, vv10.TILES_CONTRACTION)[0] == 0
    check(run_all(eng, g, refs, dev, MIXED), refs, MIXED)
    w = vv10.vv10_get_tiles(eng.h, vv10.TILES_CONTRACTION)[0]
    assert w in (64, 96, 128, 192)
    check(run_all(eng, g, refs, dev, MIXED), refs, MIXED)  # cached: same width, same results
    assert vv10.vv10_get_tiles(eng.h, vv10.TILES_CONTRACTION)[0] == w
    eng.close()


def test_fixed_shapes_are_not_replaced(dev, system, refs):
    g = system
    eng = engine(g, dev)
    vv10.vv10_set_tiles(eng.h, 0, 1, 3)  # energy sums, FP32: 1 row per thread, 3 splits
    vv10.vv10_set_autotune(eng.h, vv10.VV10_TUNE_PAIRSUMS)
    vv10.vv10_autotune(eng.h, MIXED, vv10.VV10_TUNE_PAIRSUMS)
    assert vv10.vv10_get_tiles(eng.h, 0) == (1, 3)
    check(run_all(eng, g, refs, dev, MIXED), refs, MIXED)
    vv10.vv10_set_tiles(eng.h, 0, 0, 0)  # back to automatic
    vv10.vv10_autotune(eng.h, MIXED, vv10.VV10_TUNE_PAIRSUMS)
    assert vv10.vv10_get_tiles(eng.h, 0)[0] in (1, 2, 4)
    for bad in ((9, 1, 0), (0, 3, 0), (3, 4, 0), (8, 16, 0), (8, 256, 0), (-1, 1, 0)):
        with pytest.raises(vv10.VV10Error):
            vv10.vv10_set_tiles(eng.h, *bad)
    with pytest.raises(vv10.VV10Error):  # the contraction is tuned on first use only
        vv10.vv10_autotune(eng.h, MIXED, vv10.VV10_TUNE_CONTRACTION)
    with pytest.raises(vv10.VV10Error):  # no batch prepared
        vv10.vv10_autotune(eng.h, MIXED, vv10.VV10_TUNE_BATCH)
    with pytest.raises(vv10.VV10Error):
        vv10.vv10_set_autotune(eng.h, 8)
    eng.close()


def test_tuned_batch_matches_untuned(dev):
    systems = [synth.random_points(n, seed=90 + k, n_atom=2 + k % 3) for k, n in
               enumerate((2000, 300, 1200, 50, 900))]
    Ps = [6, 3, 12, 1, 9]
    rng = np.random.default_rng(9)
    off = np.concatenate([[0], np.cumsum([g.n for g in systems])]).astype(np.int64)
    cat = lambda f: T(np.concatenate([getattr(g, f) for g in systems]), dev)
    xyz, w, rho, grad = cat("coords"), cat("weights"), cat("rho"), cat("grad_rho")
    rt = T(np.concatenate([(rng.normal(size=(P, g.n)) * g.rho).ravel() for g, P in zip(systems, Ps)]), dev)
    gt = T(np.concatenate([(rng.normal(size=(P, g.n, 3)) * np.abs(g.grad_rho)).reshape(-1, 3)
                           for g, P in zip(systems, Ps)]), dev)
    outs = []
    for tuned in (False, True):
        h = vv10.vv10_create(0)
        vv10.vv10_batch_prepare(h, off, xyz, w, rho, grad)
        if tuned:
            vv10.vv10_autotune(h, FP64, vv10.VV10_TUNE_BATCH)
            rpt, tiles = vv10.vv10_get_tiles(h, vv10.TILES_BATCH + 1)
            assert rpt in (1, 2) and tiles in (16, 32, 64)
        E = torch.empty(len(systems), dtype=torch.float64, device=dev)
        vr = torch.empty(int(off[-1]), dtype=torch.float64, device=dev)
        vg = torch.empty_like(vr)
        fr = torch.empty_like(rt)
        fg = torch.empty_like(rt)
        vv10.vv10_batch_run(h, FP64, Ps, rt, gt, E, vr, vg, fr, fg)
        vv10.vv10_sync(h)
        outs.append([t.cpu().numpy() for t in (E, vr, vg, fr, fg)])
        vv10.vv10_destroy(h)
    for a, b in zip(*outs):
        assert rel(a, b) <= 1e-12


def test_contraction_j_chunks(dev):
    """The split-FP16 contraction's j chunk (MB of trial tiles kept in L2): 4, 24 and 96 MB
    walk the same sums in different chunks (and so flush the FP32 register sums at different
    stages), agreeing to the mixed tolerance; sizes outside [4, 96] are refused."""
    g = synth.make_system(synth.random_chon(np.random.default_rng(11), 4), 40, 110)
    rng = np.random.default_rng(180)
    P = 180  # one 192-wide group: 50 KB per 32-j stage, so 4 MB chunks are 82 stages
    rt = torch.from_numpy(rng.normal(size=(P, g.n)) * g.rho).to(dev)
    gt = torch.from_numpy(rng.normal(size=(P, g.n, 3)) * np.abs(g.grad_rho)[None]).to(dev)
    eng = engine(g, dev)
    eng.energy_potential(vv10.VV10_MIXED_F16X3)
    out = {}
    for mb in (4, 24, 96):
        vv10.vv10_set_tiles(eng.h, vv10.TILES_CONTRACTION, 0, mb)
        assert vv10.vv10_get_tiles(eng.h, vv10.TILES_CONTRACTION)[1] == mb
        fr, fg = eng.hessian_contract(rt, gt, vv10.VV10_MIXED_F16X3)
        vv10.vv10_sync(eng.h)
        out[mb] = (fr.cpu().numpy(), fg.cpu().numpy())
    for mb in (4, 96):
        for k in range(2):
            ref = out[24][k]
            assert np.linalg.norm(out[mb][k] - ref) <= 1e-6 * np.linalg.norm(ref)
    for bad in (2, 100):
        with pytest.raises(vv10.VV10Error):
            vv10.vv10_set_tiles(eng.h, vv10.TILES_CONTRACTION, 0, bad)
    vv10.vv10_set_tiles(eng.h, vv10.TILES_CONTRACTION, 0, 0)
    assert vv10.vv10_get_tiles(eng.h, vv10.TILES_CONTRACTION)[1] == 24
    eng.close()
