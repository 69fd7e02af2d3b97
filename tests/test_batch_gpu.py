"""Batched molecules (vv10_batch_*): each molecule of a batch against the FP64 oracle,
against the single-system entry points, through a recorded CUDA graph, and the batch of
64 molecules (3-30 atoms, 50 x 194 points per atom, P = 3 N_atom) on sampled rows.

Tolerances as for one system (each error against the FP64 oracle):
  FP64 path:  |dE|/|E| <= 1e-11; potential and Hessian contraction <= 1e-10 relative;
  mixed path: |dE| <= 1e-7 Eh; potential and Hessian contraction <= 1e-6 relative
              (L2 / Frobenius per molecule and per output).
"""
import numpy as np
import pytest
import torch

from paper_2208_14639_gb300 import synth, vv10

pytestmark = pytest.mark.gpu

FP64 = vv10.VV10_FP64
MIXED = vv10.VV10_MIXED_TF32X3
F16 = vv10.VV10_MIXED_F16X3
TOL = {FP64: (1e-11, 1e-10), MIXED: (1e-7, 1e-6), F16: (1e-7, 1e-6)}  # (energy, arrays)
PRECS = pytest.mark.parametrize("prec", [FP64, MIXED, F16], ids=["fp64", "tf32x3", "f16x3"])


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def e_ok(prec, e, ref):
    tol = TOL[prec][0]
    return abs(e - ref) <= (tol * abs(ref) if prec == FP64 else tol)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    vv10.load(build_if_missing=True)
    return torch.device("cuda", 0)


def T(a, dev, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)


class Batch:
    """Concatenated inputs of several molecules, with random trial densities."""

    def __init__(self, systems, Ps, dev, seed=0):
        rng = np.random.default_rng(seed)
        self.sys = systems
        self.P = list(Ps)
        self.n = [g.n for g in systems]
        self.off = np.concatenate([[0], np.cumsum(self.n)]).astype(np.int64)
        cat = lambda f: np.concatenate([getattr(g, f) for g in systems])
        self.d = {"xyz": T(cat("coords"), dev), "w": T(cat("weights"), dev),
                  "rho": T(cat("rho"), dev), "grad": T(cat("grad_rho"), dev),
                  "atom": T(cat("atom_of_point"), dev, torch.int32)}
        self.n_atom = [g.molecule.n_atom for g in systems]
        self.rt, self.gt = [], []
        for g, P in zip(systems, Ps):
            self.rt.append(rng.normal(size=(P, g.n)) * g.rho)
            self.gt.append(rng.normal(size=(P, g.n, 3)) * (np.abs(g.grad_rho) + 1e-3 * g.rho[:, None]))
        self.toff = np.concatenate([[0], np.cumsum([P * n for P, n in zip(Ps, self.n)])])
        self.d_rt = T(np.concatenate([r.ravel() for r in self.rt]), dev)
        self.d_gt = T(np.concatenate([g.reshape(-1, 3) for g in self.gt]), dev)
        tot = int(self.toff[-1])
        N = int(self.off[-1])
        f64 = dict(dtype=torch.float64, device=dev)
        self.E = torch.empty(len(systems), **f64)
        self.vr = torch.empty(N, **f64)
        self.vg = torch.empty(N, **f64)
        self.fr = torch.empty(tot, **f64)
        self.fg = torch.empty(tot, **f64)

    def prepare(self, h, with_atoms=True):
        d = self.d
        return vv10.vv10_batch_prepare(h, self.off, d["xyz"], d["w"], d["rho"], d["grad"],
                                       d["atom"] if with_atoms else None,
                                       self.n_atom if with_atoms else None)

    def mol_out(self, m):
        a, b = int(self.off[m]), int(self.off[m + 1])
        s, e = int(self.toff[m]), int(self.toff[m + 1])
        P, n = self.P[m], self.n[m]
        return (self.E[m].item(), self.vr[a:b].cpu().numpy(), self.vg[a:b].cpu().numpy(),
                self.fr[s:e].view(P, n).cpu().numpy(), self.fg[s:e].view(P, n).cpu().numpy())


def dead_molecule():
    """A molecule whose points all fall below rho_cut (no kept point)."""
    g = synth.random_points(40, seed=68, n_atom=1)
    return synth.GridDensity(g.coords, g.weights, np.full(g.n, 1e-13), g.grad_rho * 1e-13,
                             g.atom_of_point, g.molecule)


def small_batch():
    systems = [synth.random_points(300, seed=61, n_atom=3), synth.random_points(1, seed=62, n_atom=1),
               synth.random_points(257, seed=63, n_atom=2), dead_molecule(),
               synth.random_points(700, seed=64, n_atom=4), synth.random_points(520, seed=65, n_atom=3)]
    # trial counts cover every padded width class (32, 64, 96) and more than one group of 192
    return systems, [9, 1, 33, 4, 200, 70]


@pytest.fixture(scope="module")
def oracle_refs(oracle_mod):
    systems, Ps = small_batch()
    b = Batch(systems, Ps, torch.device("cpu"))
    refs = []
    for m, g in enumerate(systems):
        args = (g.coords, g.weights, g.rho, g.grad_rho)
        e, vr, vg = oracle_mod.potential(*args)
        fr, fg = oracle_mod.hessian_contract(*args, b.rt[m], b.gt[m])
        refs.append((e, vr, vg, fr, fg))
    return refs


@PRECS
def test_batch_matches_oracle(dev, oracle_refs, prec):
    systems, Ps = small_batch()
    b = Batch(systems, Ps, dev)
    h = vv10.vv10_create(0)
    try:
        nk = b.prepare(h)
        assert nk[3] == 0 and nk[1] == 1
        vv10.vv10_batch_energy_potential(h, prec, b.E, b.vr, b.vg)
        vv10.vv10_batch_hessian_contract(h, prec, b.P, b.d_rt, b.d_gt, b.fr, b.fg)
        vv10.vv10_sync(h)
        tol = TOL[prec][1]
        for m, ref in enumerate(oracle_refs):
            e, vr, vg, fr, fg = b.mol_out(m)
            assert e_ok(prec, e, ref[0]), (m, e, ref[0])
            for name, x, y in (("vrho", vr, ref[1]), ("vgamma", vg, ref[2]),
                               ("f_rho_t", fr, ref[3]), ("f_gamma_t", fg, ref[4])):
                assert rel(x, y) <= tol, (m, name, rel(x, y))
        # the molecule without kept points contributes exact zeros
        e, vr, vg, fr, fg = b.mol_out(3)
        assert e == 0.0 and not vr.any() and not vg.any() and not fr.any() and not fg.any()
    finally:
        vv10.vv10_destroy(h)


@PRECS
def test_batch_matches_single_system_path(dev, prec):
    systems, Ps = small_batch()
    b = Batch(systems, Ps, dev, seed=3)
    h = vv10.vv10_create(0)
    hs = vv10.vv10_create(0)
    try:
        b.prepare(h)
        vv10.vv10_batch_energy_potential(h, prec, b.E, b.vr, b.vg)
        vv10.vv10_batch_hessian_contract(h, prec, b.P, b.d_rt, b.d_gt, b.fr, b.fg)
        vv10.vv10_sync(h)
        for m, g in enumerate(systems):
            a, e_ = int(b.off[m]), int(b.off[m + 1])
            vv10.vv10_prepare_points(hs, b.d["xyz"][a:e_], b.d["w"][a:e_], b.d["rho"][a:e_],
                                     b.d["grad"][a:e_], b.d["atom"][a:e_], g.molecule.n_atom)
            vr = torch.empty(g.n, dtype=torch.float64, device=dev)
            vg = torch.empty_like(vr)
            e = vv10.vv10_energy_potential(hs, prec, vr, vg)
            rt = T(b.rt[m], dev)
            gt = T(b.gt[m], dev)
            fr = torch.empty_like(rt)
            fg = torch.empty_like(rt)
            vv10.vv10_hessian_contract(hs, prec, rt, gt, fr, fg)
            eb, vrb, vgb, frb, fgb = b.mol_out(m)
            # same kernels, different j-splits: agreement to summation-order rounding
            assert eb == pytest.approx(e, rel=1e-12, abs=1e-300)
            tol = 1e-12 if prec == FP64 else 1e-7
            for x, y in ((vrb, vr), (vgb, vg), (frb, fr), (fgb, fg)):
                assert rel(x, y.cpu().numpy()) <= tol
    finally:
        vv10.vv10_destroy(hs)
        vv10.vv10_destroy(h)


@PRECS
def test_batch_run_graph_replay(dev, prec):
    """vv10_batch_run: the first call runs eagerly and records a graph; replays read the
    current contents of the same buffers (the contraction is linear in the trials)."""
    systems, Ps = small_batch()
    b = Batch(systems, Ps, dev, seed=5)
    h = vv10.vv10_create(0)
    try:
        b.prepare(h)
        vv10.vv10_profile_enable(h, True)
        vv10.vv10_profile_read(h)
        args = (b.P, b.d_rt, b.d_gt, b.E, b.vr, b.vg, b.fr, b.fg)
        vv10.vv10_batch_run(h, prec, *args)
        vv10.vv10_sync(h)
        first = [t.clone() for t in (b.E, b.vr, b.vg, b.fr, b.fg)]
        eager = sum(n for _, n in vv10.vv10_profile_read(h).values())
        b.d_rt.mul_(2.0)
        b.d_gt.mul_(2.0)
        for t in (b.E, b.vr, b.vg, b.fr, b.fg):
            t.fill_(float("nan"))
        vv10.vv10_batch_run(h, prec, *args)  # replay
        vv10.vv10_sync(h)
        replay = sum(n for _, n in vv10.vv10_profile_read(h).values())
        assert replay == eager > 0  # a replay runs (and counts) the same kernels
        assert torch.equal(b.E, first[0]) and torch.equal(b.vr, first[1]) and torch.equal(b.vg, first[2])
        assert torch.equal(b.fr, 2.0 * first[3]) and torch.equal(b.fg, 2.0 * first[4])
        # other output buffers record a new graph with the same results
        fr2 = torch.empty_like(b.fr)
        fg2 = torch.empty_like(b.fg)
        vv10.vv10_batch_run(h, prec, b.P, b.d_rt, b.d_gt, b.E, b.vr, b.vg, fr2, fg2)
        vv10.vv10_sync(h)
        assert torch.equal(fr2, b.fr) and torch.equal(fg2, b.fg)
    finally:
        vv10.vv10_destroy(h)


def test_batch_errors(dev):
    systems, Ps = small_batch()
    b = Batch(systems, Ps, dev)
    h = vv10.vv10_create(0)
    try:
        with pytest.raises(vv10.VV10Error) as ei:  # energy before any prepare
            vv10.vv10_batch_energy_potential(h, FP64, b.E)
        assert ei.value.status == vv10.VV10_ERR_INVALID_ARG
        bad = b.off.copy()
        bad[2] = bad[1]  # an empty molecule
        with pytest.raises(vv10.VV10Error):
            vv10.vv10_batch_prepare(h, bad, b.d["xyz"], b.d["w"], b.d["rho"], b.d["grad"])
        with pytest.raises(vv10.VV10Error):  # n_atom out of range
            vv10.vv10_batch_prepare(h, b.off, b.d["xyz"], b.d["w"], b.d["rho"], b.d["grad"],
                                    b.d["atom"], [0] * len(systems))
        b.prepare(h)
        with pytest.raises(vv10.VV10Error):  # Hessian before the energy
            vv10.vv10_batch_hessian_contract(h, MIXED, b.P, b.d_rt, b.d_gt, b.fr, b.fg)
        with pytest.raises((vv10.VV10Error, TypeError)):  # energies on the host
            vv10.vv10_batch_energy_potential(h, MIXED, b.E.cpu())
        vv10.vv10_batch_energy_potential(h, MIXED, b.E)
        with pytest.raises(vv10.VV10Error) as ei:
            vv10.vv10_batch_hessian_contract(h, vv10.VV10_MIXED_BF16X3, b.P, b.d_rt, b.d_gt,
                                             b.fr, b.fg)
        assert ei.value.status == vv10.VV10_ERR_UNSUPPORTED
        with pytest.raises(vv10.VV10Error) as ei:  # the FP64 tensor-core path: single systems only
            vv10.vv10_batch_hessian_contract(h, vv10.VV10_FP64_TC, b.P, b.d_rt, b.d_gt, b.fr, b.fg)
        assert ei.value.status == vv10.VV10_ERR_UNSUPPORTED
        with pytest.raises(vv10.VV10Error) as ei:  # an unknown precision
            vv10.vv10_batch_hessian_contract(h, 7, b.P, b.d_rt, b.d_gt, b.fr, b.fg)
        assert ei.value.status == vv10.VV10_ERR_INVALID_ARG
        with pytest.raises(vv10.VV10Error):  # P = 0
            vv10.vv10_batch_hessian_contract(h, MIXED, [0] + b.P[1:], b.d_rt, b.d_gt, b.fr, b.fg)
        vv10.vv10_sync(h)
    finally:
        vv10.vv10_destroy(h)


def test_batch_without_atom_labels(dev, oracle_refs):
    systems, Ps = small_batch()
    b = Batch(systems, Ps, dev)
    h = vv10.vv10_create(0)
    try:
        b.prepare(h, with_atoms=False)
        vv10.vv10_batch_energy_potential(h, FP64, b.E, b.vr, b.vg)
        vv10.vv10_sync(h)
        for m, ref in enumerate(oracle_refs):
            e, vr, vg, _, _ = b.mol_out(m)
            assert e_ok(FP64, e, ref[0])
            assert rel(vr, ref[1]) <= 1e-10
    finally:
        vv10.vv10_destroy(h)


def test_batch_64_molecules_sampled_rows(dev, oracle_mod):
    """The batch of 64 molecules (3-30 atoms, 50 x 194 points per atom, 9.7k-291k points,
    P = 3 N_atom), mixed precision (split TF32 and split FP16) through recorded graphs, as
    timed by the benchmark;
    energies of the four smallest molecules in full and 16 sampled rows of the potential
    and of the Hessian contraction of the smallest, a middle and the largest molecule
    against the oracle."""
    import os
    systems = synth.config_batch(workers=os.cpu_count() or 1)
    Ps = [3 * g.molecule.n_atom for g in systems]
    n = [g.n for g in systems]
    off = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
    toff = np.concatenate([[0], np.cumsum([P * k for P, k in zip(Ps, n)])]).astype(np.int64)
    cat = lambda f: np.concatenate([getattr(g, f) for g in systems])
    d = {"xyz": T(cat("coords"), dev), "w": T(cat("weights"), dev), "rho": T(cat("rho"), dev),
         "grad": T(cat("grad_rho"), dev), "atom": T(cat("atom_of_point"), dev, torch.int32)}
    tot = int(toff[-1])
    f64 = dict(dtype=torch.float64, device=dev)
    rt = torch.empty(tot, **f64)
    gt = torch.empty(tot, 3, **f64)
    for m, g in enumerate(systems):
        s, e = int(toff[m]), int(toff[m + 1])
        synth.trial_densities_torch(g.molecule, d["xyz"][int(off[m]):int(off[m + 1])],
                                    out_rho=rt[s:e].view(Ps[m], n[m]),
                                    out_grad=gt[s:e].view(Ps[m], n[m], 3))
    E = torch.empty(len(systems), **f64)
    vr = torch.empty(int(off[-1]), **f64)
    vg = torch.empty_like(vr)
    fr = torch.empty(tot, **f64)
    fg = torch.empty(tot, **f64)
    h = vv10.vv10_create(0)
    try:
        vv10.vv10_batch_prepare(h, off, d["xyz"], d["w"], d["rho"], d["grad"], d["atom"],
                                [g.molecule.n_atom for g in systems])
        for _ in range(2):  # record, then replay
            vv10.vv10_batch_run(h, MIXED, Ps, rt, gt, E, vr, vg, fr, fg)
        vv10.vv10_sync(h)
        # the split-FP16 contraction of the same batch (its own recorded graph) against the
        # split-TF32 one, every molecule and element (both within 1e-6 of the oracle)
        fr16 = torch.empty_like(fr)
        fg16 = torch.empty_like(fg)
        for _ in range(2):
            vv10.vv10_batch_run(h, F16, Ps, rt, gt, E, vr, vg, fr16, fg16)
        vv10.vv10_sync(h)
        assert rel(fr16.cpu().numpy(), fr.cpu().numpy()) <= 1e-6
        assert rel(fg16.cpu().numpy(), fg.cpu().numpy()) <= 1e-6
        order = np.argsort(n, kind="stable")
        for m in order[:4]:
            g = systems[m]
            ref = oracle_mod.energy(g.coords, g.weights, g.rho, g.grad_rho)
            assert abs(E[m].item() - ref) <= 1e-7, (m, E[m].item(), ref)
        for m in (order[0], order[len(order) // 2], order[-1]):
            g = systems[m]
            rows = np.linspace(0, g.n - 1, 16).astype(np.int64)
            args = (g.coords, g.weights, g.rho, g.grad_rho)
            _, r_vr, r_vg = oracle_mod.potential(*args, rows=rows)
            a = int(off[m])
            assert rel(vr[a + rows].cpu().numpy(), r_vr) <= 1e-6
            assert rel(vg[a + rows].cpu().numpy(), r_vg) <= 1e-6
            s, e = int(toff[m]), int(toff[m + 1])
            rt_m = rt[s:e].view(Ps[m], n[m]).cpu().numpy()
            gt_m = gt[s:e].view(Ps[m], n[m], 3).cpu().numpy()
            r_fr, r_fg = oracle_mod.hessian_contract(*args, rt_m, gt_m, rows=rows)
            for f_r, f_g in ((fr, fg), (fr16, fg16)):
                assert rel(f_r[s:e].view(Ps[m], n[m])[:, rows].cpu().numpy(), r_fr) <= 1e-6
                assert rel(f_g[s:e].view(Ps[m], n[m])[:, rows].cpu().numpy(), r_fg) <= 1e-6
    finally:
        vv10.vv10_destroy(h)
