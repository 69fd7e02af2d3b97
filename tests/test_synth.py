"""Self-checks of the seeded synthetic input generator (no VV10 arithmetic here)."""
import numpy as np
import pytest

from paper_2208_14639_gb300 import synth


def test_water_grid_integrates_density():
    g = synth.config_water()
    assert g.n == 9900
    assert float(g.weights @ g.rho) == pytest.approx(10.0, rel=1e-3)
    assert np.all(g.weights >= 0)
    assert np.all(np.diff(g.atom_of_point) >= 0)


def test_radial_and_angular_rules():
    r, w = synth.radial_grid(60, 1.3)
    # int_0^inf r^2 exp(-r^2) dr = sqrt(pi)/4
    assert float(w @ np.exp(-r ** 2)) == pytest.approx(np.sqrt(np.pi) / 4, rel=1e-8)
    u, wa = synth.fibonacci_sphere(302)
    np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, rtol=1e-14)
    assert wa.sum() == pytest.approx(4 * np.pi)


def test_density_gradient_and_trials_by_finite_differences():
    g = synth.random_points(6, seed=1, n_atom=2)
    mol = g.molecule
    h = 1e-6
    rho0, grad0 = synth.density(mol, g.coords)
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (synth.density(mol, g.coords + e)[0] - synth.density(mol, g.coords - e)[0]) / (2 * h)
        np.testing.assert_allclose(grad0[:, d], fd, rtol=1e-6, atol=1e-12)
    rt, gt = synth.trial_densities(mol, g.coords)
    for A in range(mol.n_atom):
        for c in range(3):
            m_p = synth.Molecule(mol.symbols, mol.coords.copy())
            m_m = synth.Molecule(mol.symbols, mol.coords.copy())
            m_p.coords[A, c] += h
            m_m.coords[A, c] -= h
            rp, gp = synth.density(m_p, g.coords)
            rm, gm = synth.density(m_m, g.coords)
            np.testing.assert_allclose(rt[3 * A + c], (rp - rm) / (2 * h), rtol=1e-6, atol=1e-12)
            np.testing.assert_allclose(gt[3 * A + c], (gp - gm) / (2 * h), rtol=1e-6, atol=1e-11)


def test_configs_are_seeded():
    a = synth.config_cluster24(n_rad=6, n_ang=14)
    b = synth.config_cluster24(n_rad=6, n_ang=14)
    np.testing.assert_array_equal(a.coords, b.coords)
    assert a.molecule.n_atom == 24
    batch = synth.config_batch(n_mol=3, n_rad=4, n_ang=6)
    assert all(3 <= m.molecule.n_atom <= 30 for m in batch)


def test_trial_densities_torch_matches_numpy():
    import torch
    g = synth.random_points(500, seed=71, n_atom=3)
    rt, gt = synth.trial_densities(g.molecule, g.coords)
    rt2, gt2 = synth.trial_densities_torch(g.molecule, torch.from_numpy(g.coords))
    assert np.allclose(rt2.numpy(), rt, rtol=1e-13, atol=1e-13 * np.abs(rt).max())
    assert np.allclose(gt2.numpy(), gt, rtol=1e-13, atol=1e-13 * np.abs(gt).max())
    # into preallocated views of a larger buffer
    buf = torch.zeros(rt.size + 4, dtype=torch.float64)
    gbuf = torch.zeros(gt.size + 12, dtype=torch.float64)
    synth.trial_densities_torch(g.molecule, torch.from_numpy(g.coords),
                                out_rho=buf[4:].view(rt.shape), out_grad=gbuf[12:].view(gt.shape))
    assert np.array_equal(buf[4:].view(rt.shape).numpy(), rt2.numpy())
    assert np.array_equal(gbuf[12:].view(gt.shape).numpy(), gt2.numpy())


def test_config_batch_parallel_is_identical():
    a = synth.config_batch(n_mol=3, n_rad=4, n_ang=6, atom_range=(2, 4))
    b = synth.config_batch(n_mol=3, n_rad=4, n_ang=6, atom_range=(2, 4), workers=2)
    for x, y in zip(a, b):
        for f in ("coords", "weights", "rho", "grad_rho", "atom_of_point"):
            assert np.array_equal(getattr(x, f), getattr(y, f))


def test_weight_directions_are_becke_weight_derivatives():
    """The analytic nuclear derivatives of the Becke partition agree with central
    differences (the owner atom's points move with it) and sum to zero over the atoms."""
    mol = synth.random_chon(np.random.default_rng(0), 10)
    pts, _, own = synth.molecular_grid(mol, 6, 14)
    for a in (0, 4):
        p = pts[own == a][:120]
        f, gr = synth._becke_fraction_grad(p, a, mol.coords)
        np.testing.assert_array_equal(f, synth._becke_fraction(p, a, mol.coords))
        h = 1e-6
        for B in range(mol.n_atom):
            for c in range(3):
                ap, am = mol.coords.copy(), mol.coords.copy()
                ap[B, c] += h
                am[B, c] -= h
                pp, pm = p.copy(), p.copy()
                if B == a:
                    pp[:, c] += h
                    pm[:, c] -= h
                fd = (synth._becke_fraction(pp, a, ap) - synth._becke_fraction(pm, a, am)) / (2 * h)
                np.testing.assert_allclose(gr[:, B, c], fd, atol=1e-7)
        np.testing.assert_allclose(gr.sum(axis=1), 0.0, atol=1e-12)
    V = synth.weight_directions(mol, 6, 14)
    assert V.shape == (3 * mol.n_atom, pts.shape[0])
    np.testing.assert_allclose(V.reshape(mol.n_atom, 3, -1).sum(axis=0), 0.0,
                               atol=1e-12 * np.abs(V).max())


def test_ao_basis_values_gradients_and_density():
    """Basis functions normalised to unit self-overlap, analytic gradients against central
    differences, and the AO density's gradient against central differences."""
    mol = synth.water()
    b = synth.ao_basis(mol)
    rng = np.random.default_rng(3)
    pts = rng.normal(size=(40, 3)) * 1.5
    phi, dphi = synth.ao_values(b, pts)
    P = synth.density_matrix(b, 5, rng)
    rho, grad = synth.ao_density(phi, dphi, P)
    h = 1e-6
    for d in range(3):
        pp, pm = pts.copy(), pts.copy()
        pp[:, d] += h
        pm[:, d] -= h
        fp, fm = synth.ao_values(b, pp)[0], synth.ao_values(b, pm)[0]
        np.testing.assert_allclose(dphi[:, :, d], (fp - fm) / (2 * h), atol=1e-8)
        rp = synth.ao_density(fp, synth.ao_values(b, pp)[1], P)[0]
        rm = synth.ao_density(fm, synth.ao_values(b, pm)[1], P)[0]
        np.testing.assert_allclose(grad[:, d], (rp - rm) / (2 * h), atol=1e-8 * np.abs(grad).max())
    assert (rho >= 0).all()  # P is positive semi-definite
    g, phi, _, _, _, _, _ = synth.ao_system(mol, 30, 110, 1)
    np.testing.assert_allclose((g.weights[:, None] * phi ** 2).sum(axis=0), 1.0, atol=5e-3)


def test_nuclear_density_derivatives_at_moving_points():
    """The first and second derivatives of rho and grad rho at grid points that move with their
    atoms against central differences of the pipeline (grid and density rebuilt per geometry)."""
    mol, nr, na = synth.water(), 6, 14
    g = synth.make_system(mol, nr, na)
    rt, gt = synth.nuclear_density_derivatives(mol, g.coords, g.atom_of_point)
    r2, g2 = synth.nuclear_density_second_derivatives(mol, g.coords, g.atom_of_point)
    h = 1e-5
    for b in (0, 4, 8):
        out = []
        for sg in (1, -1):
            c = mol.coords.copy()
            c[b // 3, b % 3] += sg * h
            m2 = synth.Molecule(mol.symbols, c)
            gg = synth.make_system(m2, nr, na)
            out.append((gg.rho, gg.grad_rho) + synth.nuclear_density_derivatives(m2, gg.coords, gg.atom_of_point))
        np.testing.assert_allclose(rt[b], (out[0][0] - out[1][0]) / (2 * h), atol=1e-7 * np.abs(rt).max())
        np.testing.assert_allclose(gt[b], (out[0][1] - out[1][1]) / (2 * h), atol=1e-7 * np.abs(gt).max())
        np.testing.assert_allclose(r2[:, b], (out[0][2] - out[1][2]) / (2 * h), atol=1e-7 * np.abs(r2).max())
        np.testing.assert_allclose(g2[:, b], (out[0][3] - out[1][3]) / (2 * h), atol=1e-7 * np.abs(g2).max())


def test_ao_second_derivatives():
    """The basis-function Hessians: symmetric, and the central differences of the analytic
    gradients."""
    mol = synth.random_chon(np.random.default_rng(4), 3)
    b = synth.ao_basis(mol)
    pts = np.random.default_rng(5).normal(size=(40, 3)) * 1.5
    H = synth.ao_second_derivatives(b, pts)
    np.testing.assert_allclose(H, H.transpose(0, 1, 3, 2), rtol=0, atol=1e-14 * np.abs(H).max())
    h = 1e-5
    for d in range(3):
        pp, pm = pts.copy(), pts.copy()
        pp[:, d] += h
        pm[:, d] -= h
        fd = (synth.ao_values(b, pp)[1] - synth.ao_values(b, pm)[1]) / (2 * h)
        np.testing.assert_allclose(H[:, :, :, d], fd, atol=1e-8 * np.abs(H).max())


def test_ao_nuclear_density_derivatives_at_moving_points():
    """rho^a, grad rho^a of the AO density with the grid points and the basis moving with the
    atoms (density matrix fixed) against central differences of the rebuilt pipeline; their
    sum over the atoms vanishes (a rigid translation changes nothing at a moving point)."""
    mol, nr, na = synth.water(), 8, 14
    g, _, _, _, b, P, sel, rt, gt, _ = synth.ao_moving_system(mol, nr, na, seed=1)
    h = 1e-5
    for a in range(3 * mol.n_atom):
        out = []
        for sg in (1, -1):
            c = mol.coords.copy()
            c[a // 3, a % 3] += sg * h
            gg = synth.ao_moving_system(synth.Molecule(mol.symbols, c), nr, na, P=P, sel=sel)[0]
            out.append((gg.rho, gg.grad_rho))
        np.testing.assert_allclose(rt[a], (out[0][0] - out[1][0]) / (2 * h), atol=1e-7 * np.abs(rt).max())
        np.testing.assert_allclose(gt[a], (out[0][1] - out[1][1]) / (2 * h), atol=1e-7 * np.abs(gt).max())
    np.testing.assert_allclose(rt.reshape(mol.n_atom, 3, -1).sum(axis=0), 0.0, atol=1e-13 * np.abs(rt).max())
    np.testing.assert_allclose(gt.reshape(mol.n_atom, 3, -1, 3).sum(axis=0), 0.0, atol=1e-13 * np.abs(gt).max())
