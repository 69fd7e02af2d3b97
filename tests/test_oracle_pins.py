"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a value fixed
independently (a physical limit the paper states, an equivalent published definition,
a closed form, a finite difference of the oracle's own *energy*, an exact invariant).
A dropped term, a wrong sign or index, or a swapped g/g' in any oracle routine fails at
least one of them.  The paper prints no VV10 numbers for any system, so no test pins
against printed values.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2208_14639_gb300 import synth

B, C = 6.0, 0.01


def _sys(seed=3, n=9, n_atom=2):
    g = synth.random_points(n, seed=seed, n_atom=n_atom)
    return g, (g.coords, g.weights, g.rho, g.grad_rho)


# --------------------------------------------------------------------- point quantities

@pytest.mark.parametrize("rho", [1e-6, 1e-3, 0.1, 3.0, 200.0])
def test_beta_from_uniform_gas_limit(oracle_mod, rho):
    """Sec. II.A: beta makes E^VV10 vanish for a uniform density.

    For constant rho (gamma = 0) the energy per volume is rho*beta + 1/2 rho^2 * int Phi d^3R,
    so beta = -1/2 rho * int_0^inf Phi(R) 4 pi R^2 dR, independent of rho.  The integral is
    done by quadrature over the oracle's own omega, kappa and Phi; this pins beta, kappa,
    the gamma = 0 part of omega and the form of Phi at once.
    """
    p = oracle_mod.point_props([rho], [[0.0, 0.0, 0.0]], b=B, C=C)
    om, ka = p["omega"][0], p["kappa"][0]
    f = lambda R: oracle_mod.phi(om, ka, om, ka, R * R) * 4.0 * math.pi * R * R
    scale = math.sqrt(ka / om)
    val = integrate.quad(f, 0, scale, epsabs=0, epsrel=1e-13, limit=400)[0]
    val += integrate.quad(f, scale, np.inf, epsabs=0, epsrel=1e-13, limit=400)[0]
    beta_uniform = -0.5 * rho * val
    assert beta_uniform == pytest.approx(oracle_mod.beta(B), rel=1e-9)


def test_kappa_is_b_vF2_over_wp(oracle_mod):
    """kappa = b (3 pi/2)(rho/9pi)^(1/6) equals b v_F^2 / omega_p with v_F = (3 pi^2 rho)^(1/3)
    and omega_p = (4 pi rho)^(1/2), the original VV10 definition of kappa."""
    rho = np.logspace(-10, 3, 27)
    p = oracle_mod.point_props(rho, np.zeros((rho.size, 3)), b=B, C=C)
    vf = (3.0 * math.pi ** 2 * rho) ** (1.0 / 3.0)
    wp = np.sqrt(4.0 * math.pi * rho)
    np.testing.assert_allclose(p["kappa"], B * vf ** 2 / wp, rtol=1e-13)


def test_omega_is_sqrt_wg2_plus_wp2_over_3(oracle_mod):
    """omega = sqrt(omega_g^2 + omega_p^2/3) with omega_g^2 = C |grad rho / rho|^4 and
    omega_p^2 = 4 pi rho; gamma^2/rho^4 is |grad rho/rho|^4 when gamma = |grad rho|^2."""
    rng = np.random.default_rng(5)
    rho = 10.0 ** rng.uniform(-9, 2, 40)
    grad = rng.normal(size=(40, 3)) * rho[:, None] * 10.0 ** rng.uniform(-1, 1.3, (40, 1))
    p = oracle_mod.point_props(rho, grad, b=B, C=C)
    s = np.linalg.norm(grad, axis=1) / rho
    np.testing.assert_allclose(p["omega"], np.sqrt(C * s ** 4 + 4.0 * math.pi * rho / 3.0), rtol=1e-13)
    np.testing.assert_allclose(p["gamma"], np.linalg.norm(grad, axis=1) ** 2, rtol=1e-14)


def test_point_derivatives_by_finite_differences(oracle_mod):
    """d omega/d rho, d omega/d gamma, d kappa/d rho and the second derivatives used by the
    potential and the Hessian terms, against central differences of omega and kappa."""
    rng = np.random.default_rng(11)
    for _ in range(12):
        rho = 10.0 ** rng.uniform(-6, 1.5)
        gam = (rho * 10.0 ** rng.uniform(-0.5, 1.2)) ** 2

        def ok(r, gm):
            p = oracle_mod.point_props([r], [[math.sqrt(gm), 0.0, 0.0]], b=B, C=C)
            return np.array([p["omega"][0], p["kappa"][0], p["omega_rho"][0],
                             p["omega_gamma"][0], p["kappa_rho"][0]])

        base = oracle_mod.point_props([rho], [[math.sqrt(gam), 0.0, 0.0]], b=B, C=C)
        hr, hg = 1e-5 * rho, 1e-5 * gam
        dr = (ok(rho + hr, gam) - ok(rho - hr, gam)) / (2 * hr)
        dg = (ok(rho, gam + hg) - ok(rho, gam - hg)) / (2 * hg)
        assert dr[0] == pytest.approx(base["omega_rho"][0], rel=1e-7)
        assert dg[0] == pytest.approx(base["omega_gamma"][0], rel=1e-7)
        assert dr[1] == pytest.approx(base["kappa_rho"][0], rel=1e-7)
        # second derivatives: tolerance on the natural scale (first derivative / variable)
        s_rr = abs(base["omega_rho"][0]) / rho + abs(base["omega_rhorho"][0])
        s_rg = abs(base["omega_gamma"][0]) / rho + abs(base["omega_rhogamma"][0])
        s_gg = abs(base["omega_gamma"][0]) / gam + abs(base["omega_gammagamma"][0])
        assert abs(dr[2] - base["omega_rhorho"][0]) < 1e-6 * s_rr
        assert abs(dg[2] - base["omega_rhogamma"][0]) < 1e-6 * s_rg
        assert abs(dr[3] - base["omega_rhogamma"][0]) < 1e-6 * s_rg
        assert abs(dg[3] - base["omega_gammagamma"][0]) < 1e-6 * s_gg
        assert dr[4] == pytest.approx(base["kappa_rhorho"][0], rel=1e-7)


# --------------------------------------------------------------------- kernel Phi

def test_phi_symmetry_and_closed_forms(oracle_mod):
    """Phi_ij = Phi_ji (g'_ij = g_ji); Phi_ii = -3/(4 kappa^3) at R = 0; and the
    large-R limit -3 / (2 omega_i omega_j (omega_i + omega_j) R^6)."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        oi, oj = rng.uniform(0.1, 50, 2)
        ki, kj = rng.uniform(0.3, 20, 2)
        R2 = rng.uniform(0, 30)
        assert oracle_mod.phi(oi, ki, oj, kj, R2) == pytest.approx(oracle_mod.phi(oj, kj, oi, ki, R2), rel=1e-15)
        assert oracle_mod.phi(oi, ki, oj, ki, 0.0) == pytest.approx(-3.0 / (4.0 * ki ** 3), rel=1e-15)
        R2 = 1e8
        asym = -3.0 / (2.0 * oi * oj * (oi + oj) * R2 ** 3)
        assert oracle_mod.phi(oi, ki, oj, kj, R2) == pytest.approx(asym, rel=1e-5)


def test_one_and_two_point_energies(oracle_mod):
    """E = sum_i w_i rho_i (beta + 1/2 sum_j w_j rho_j Phi_ij) with j = i included,
    written out for one and for two points."""
    g, _ = _sys(seed=8, n=2)
    p = oracle_mod.point_props(g.rho, g.grad_rho)
    beta = oracle_mod.beta()
    c = g.weights * g.rho
    e1 = oracle_mod.energy(g.coords[:1], g.weights[:1], g.rho[:1], g.grad_rho[:1])
    assert e1 == pytest.approx(c[0] * beta + 0.5 * c[0] ** 2 * (-3.0 / (4.0 * p["kappa"][0] ** 3)), rel=1e-14)
    R2 = float(np.sum((g.coords[0] - g.coords[1]) ** 2))
    phi = lambda a, b_, r2: oracle_mod.phi(p["omega"][a], p["kappa"][a], p["omega"][b_], p["kappa"][b_], r2)
    expect = beta * c.sum() + 0.5 * (c[0] ** 2 * phi(0, 0, 0.0) + c[1] ** 2 * phi(1, 1, 0.0)
                                     + 2.0 * c[0] * c[1] * phi(0, 1, R2))
    assert oracle_mod.energy(*_sys(seed=8, n=2)[1]) == pytest.approx(expect, rel=1e-14)


def test_rotation_and_translation_invariance(oracle_mod):
    g, args = _sys(seed=4, n=12)
    e0 = oracle_mod.energy(*args)
    th = 0.7
    rot = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1.0]])
    rot = rot @ np.array([[1, 0, 0], [0, math.cos(0.3), -math.sin(0.3)], [0, math.sin(0.3), math.cos(0.3)]])
    e1 = oracle_mod.energy(g.coords @ rot.T + 1.7, g.weights, g.rho, g.grad_rho @ rot.T)
    assert e1 == pytest.approx(e0, rel=1e-13)


def test_cutoff_drops_points(oracle_mod):
    """Points below rho_cut take part in no sum and get zero outputs."""
    g, args = _sys(seed=9, n=10)
    rho = g.rho.copy()
    rho[3] = 1e-12
    full = oracle_mod.energy(g.coords, g.weights, rho, g.grad_rho)
    keep = np.arange(10) != 3
    sub = oracle_mod.energy(g.coords[keep], g.weights[keep], rho[keep], g.grad_rho[keep])
    assert full == pytest.approx(sub, rel=1e-15)
    _, vr, vg = oracle_mod.potential(g.coords, g.weights, rho, g.grad_rho)
    assert vr[3] == 0.0 and vg[3] == 0.0


# --------------------------------------------------------------------- first derivatives

def test_potential_is_energy_derivative(oracle_mod):
    """w_k f^rho_k = dE/d rho_k and 2 w_k f^gamma_k grad rho_k = dE/d grad rho_k
    (Sec. II.A), checked at every point by central differences of the energy."""
    g, args = _sys(seed=3, n=9)
    _, vr, vg = oracle_mod.potential(*args)
    for k in range(g.n):
        h = 1e-5 * g.rho[k]
        rp, rm = g.rho.copy(), g.rho.copy()
        rp[k] += h
        rm[k] -= h
        fd = (oracle_mod.energy(g.coords, g.weights, rp, g.grad_rho)
              - oracle_mod.energy(g.coords, g.weights, rm, g.grad_rho)) / (2 * h)
        assert fd == pytest.approx(g.weights[k] * vr[k], rel=1e-7)
        for d in range(3):
            hh = 1e-4 * np.linalg.norm(g.grad_rho[k])
            gp, gm = g.grad_rho.copy(), g.grad_rho.copy()
            gp[k, d] += hh
            gm[k, d] -= hh
            fd = (oracle_mod.energy(g.coords, g.weights, g.rho, gp)
                  - oracle_mod.energy(g.coords, g.weights, g.rho, gm)) / (2 * hh)
            an = 2 * g.weights[k] * vg[k] * g.grad_rho[k, d]
            assert fd == pytest.approx(an, rel=1e-5, abs=1e-9 * abs(g.weights[k] * vr[k]))


def test_weight_derivative(oracle_mod):
    """dE/dw_k = rho_k (beta + E_k) (the E^A_w term of Sec. II.A)."""
    g, args = _sys(seed=6, n=9)
    Ek = oracle_mod.pair_sums(*args)["E"]
    for k in range(g.n):
        h = 1e-6 * g.weights[k]
        wp, wm = g.weights.copy(), g.weights.copy()
        wp[k] += h
        wm[k] -= h
        fd = (oracle_mod.energy(g.coords, wp, g.rho, g.grad_rho)
              - oracle_mod.energy(g.coords, wm, g.rho, g.grad_rho)) / (2 * h)
        assert fd == pytest.approx(g.rho[k] * (oracle_mod.beta() + Ek[k]), rel=1e-8)


def test_point_gradient_is_energy_derivative(oracle_mod):
    g, args = _sys(seed=12, n=10)
    pg = oracle_mod.point_grad(*args)
    scale = np.abs(pg).max()
    for k in range(g.n):
        for d in range(3):
            h = 1e-5
            cp, cm = g.coords.copy(), g.coords.copy()
            cp[k, d] += h
            cm[k, d] -= h
            fd = (oracle_mod.energy(cp, g.weights, g.rho, g.grad_rho)
                  - oracle_mod.energy(cm, g.weights, g.rho, g.grad_rho)) / (2 * h)
            assert fd == pytest.approx(pg[k, d], rel=1e-6, abs=1e-8 * scale)
    np.testing.assert_allclose(pg.sum(axis=0), 0.0, atol=1e-15 * np.abs(pg).sum())


def test_atom_gradient_first_form(oracle_mod):
    """E^A_gr from the first form of Eq. grad_gr equals the derivative of E when all points
    of atom A move rigidly, equals the sum of the point gradients over i in A, and the
    atom terms sum to zero (translational invariance)."""
    g, args = _sys(seed=14, n=16, n_atom=3)
    ag = oracle_mod.atom_grad(*args, g.atom_of_point, 3)
    pg = oracle_mod.point_grad(*args)
    for A in range(3):
        np.testing.assert_allclose(ag[A], pg[g.atom_of_point == A].sum(axis=0), rtol=1e-11,
                                   atol=1e-14 * np.abs(ag).max())
        for d in range(3):
            h = 1e-5
            cp, cm = g.coords.copy(), g.coords.copy()
            cp[g.atom_of_point == A, d] += h
            cm[g.atom_of_point == A, d] -= h
            fd = (oracle_mod.energy(cp, g.weights, g.rho, g.grad_rho)
                  - oracle_mod.energy(cm, g.weights, g.rho, g.grad_rho)) / (2 * h)
            assert fd == pytest.approx(ag[A, d], rel=1e-6, abs=1e-8 * np.abs(ag).max())
    np.testing.assert_allclose(ag.sum(axis=0), 0.0, atol=1e-13 * np.abs(ag).max())


def test_simplified_gradient_form_disagrees(oracle_mod):
    """Reading of Eq. grad_gr: its second, 'simplified' form (keeping only the omega_i
    terms, times 2) is not the derivative of E; the oracle uses the first form."""
    g, args = _sys(seed=14, n=16, n_atom=3)
    p = oracle_mod.point_props(g.rho, g.grad_rho)
    c = g.weights * g.rho
    A = 0
    inA = g.atom_of_point == A
    simp = np.zeros(3)
    for i in range(g.n):
        for j in range(g.n):
            if inA[i] == inA[j]:
                continue
            R2 = float(np.sum((g.coords[i] - g.coords[j]) ** 2))
            gi = p["omega"][i] * R2 + p["kappa"][i]
            gj = p["omega"][j] * R2 + p["kappa"][j]
            phi = oracle_mod.phi(p["omega"][i], p["kappa"][i], p["omega"][j], p["kappa"][j], R2)
            if inA[i]:
                simp += -2 * c[i] * c[j] * phi * (p["omega"][i] / gi + p["omega"][i] / (gi + gj)) * (g.coords[i] - g.coords[j])
            else:
                simp += -2 * c[i] * c[j] * phi * (p["omega"][j] / gj + p["omega"][j] / (gi + gj)) * (g.coords[j] - g.coords[i])
    ag = oracle_mod.atom_grad(*args, g.atom_of_point, 3)
    assert np.abs(simp - ag[A]).max() > 1e-3 * np.abs(ag[A]).max()


def test_atom_resolved_terms_are_derivatives(oracle_mod):
    """E_i^{Bgr}, U_i^{Bgr}, W_i^{Bgr} are the derivatives of E_i, U_i, W_i when atom B's
    points move rigidly, for i not in B (the sums of Eq. EiBgr) and i in B (minus the
    other atoms' terms)."""
    g, args = _sys(seed=21, n=14, n_atom=3)
    oE, oU, oW = oracle_mod.atom_resolved(*args, g.atom_of_point, 3)
    h = 1e-5
    for B_ in range(3):
        for d in range(3):
            cp, cm = g.coords.copy(), g.coords.copy()
            cp[g.atom_of_point == B_, d] += h
            cm[g.atom_of_point == B_, d] -= h
            sp = oracle_mod.pair_sums(cp, g.weights, g.rho, g.grad_rho)
            sm = oracle_mod.pair_sums(cm, g.weights, g.rho, g.grad_rho)
            for key, arr in (("E", oE), ("U", oU), ("W", oW)):
                fd = (sp[key] - sm[key]) / (2 * h)
                scale = np.abs(arr[:, :, d]).max()
                np.testing.assert_allclose(arr[:, B_, d], fd, rtol=1e-5, atol=1e-8 * scale)


# --------------------------------------------------------------------- Hessian contraction

def _trials(g, P=None):
    rt, gt = synth.trial_densities(g.molecule, g.coords)
    return rt, gt


def test_hessian_contraction_is_potential_derivative(oracle_mod):
    """f^{rho,t}, f^{gamma,t} (Eq. frhot with the printed f^{rho rho} ... f^{gamma gamma},
    including their delta_ij/w_i parts) are the directional derivatives of f^rho, f^gamma
    along (rho^t, grad rho^t)."""
    g, args = _sys(seed=3, n=11, n_atom=2)
    rt, gt = _trials(g)
    fr, fg = oracle_mod.hessian_contract(*args, rt, gt)
    eps = 1e-5
    for t in range(rt.shape[0]):
        _, vrp, vgp = oracle_mod.potential(g.coords, g.weights, g.rho + eps * rt[t], g.grad_rho + eps * gt[t])
        _, vrm, vgm = oracle_mod.potential(g.coords, g.weights, g.rho - eps * rt[t], g.grad_rho - eps * gt[t])
        np.testing.assert_allclose(fr[t], (vrp - vrm) / (2 * eps), rtol=1e-6, atol=1e-7 * np.abs(fr[t]).max())
        np.testing.assert_allclose(fg[t], (vgp - vgm) / (2 * eps), rtol=1e-6, atol=1e-7 * np.abs(fg[t]).max())


def test_hessian_symmetry_and_linearity(oracle_mod):
    """<t1, H t2> = <t2, H t1> with <t, v> = sum_i w_i (rho^t_i v^rho_i + 2 gamma^t_i v^gamma_i),
    and the contraction is linear in the trial."""
    g, args = _sys(seed=5, n=15, n_atom=3)
    rng = np.random.default_rng(0)
    rt = rng.normal(size=(3, g.n)) * g.rho
    gt = rng.normal(size=(3, g.n, 3)) * np.linalg.norm(g.grad_rho, axis=1)[None, :, None]
    fr, fg = oracle_mod.hessian_contract(*args, rt, gt)
    gam_t = np.einsum("nd,tnd->tn", g.grad_rho, gt)
    ip = lambda a, b_: float(np.sum(g.weights * (rt[a] * fr[b_] + 2 * gam_t[a] * fg[b_])))
    for a, b_ in ((0, 1), (0, 2), (1, 2)):
        assert ip(a, b_) == pytest.approx(ip(b_, a), rel=1e-11)
    fr2, fg2 = oracle_mod.hessian_contract(*args, 2.0 * rt[:1] - 3.0 * rt[1:2], 2.0 * gt[:1] - 3.0 * gt[1:2])
    np.testing.assert_allclose(fr2[0], 2 * fr[0] - 3 * fr[1], rtol=1e-11, atol=1e-14 * np.abs(fr).max())
    np.testing.assert_allclose(fg2[0], 2 * fg[0] - 3 * fg[1], rtol=1e-11, atol=1e-14 * np.abs(fg).max())


def test_row_sampling_matches_full(oracle_mod):
    g, args = _sys(seed=7, n=20, n_atom=2)
    rows = np.array([17, 2, 9])
    full = oracle_mod.pair_sums(*args)
    part = oracle_mod.pair_sums(*args, rows=rows)
    for k in "EUWABC":
        np.testing.assert_array_equal(part[k], full[k][rows])
    rt, gt = _trials(g)
    fr, fg = oracle_mod.hessian_contract(*args, rt, gt)
    fr2, fg2 = oracle_mod.hessian_contract(*args, rt, gt, rows=rows)
    np.testing.assert_array_equal(fr2, fr[:, rows])
    np.testing.assert_array_equal(fg2, fg[:, rows])


# ----------------------------------------------------------------- grid-grid Hessian block

def _rigid(g, atom, d, h):
    c = g.coords.copy()
    c[g.atom_of_point == atom, d] += h
    return c


def test_coord_hessian_is_derivative_of_atom_gradient(oracle_mod):
    """E^{AB}_{gr,gr} (the D_i^B sums and the minus-sum diagonal) equals central finite
    differences of E^A_gr when the points of atom B move rigidly (rho, grad rho, w fixed)."""
    g = synth.random_points(70, seed=31, n_atom=3)
    na = 3
    H = oracle_mod.coord_hessian(g.coords, g.weights, g.rho, g.grad_rho, g.atom_of_point, na)
    h = 1e-4
    for B in range(na):
        for d in range(3):
            gp = oracle_mod.atom_grad(_rigid(g, B, d, h), g.weights, g.rho, g.grad_rho, g.atom_of_point, na)
            gm = oracle_mod.atom_grad(_rigid(g, B, d, -h), g.weights, g.rho, g.grad_rho, g.atom_of_point, na)
            fd = (gp - gm) / (2 * h)  # fd[A, c] = d E^A_{gr,c} / d R_{B,d}
            for A in range(na):
                np.testing.assert_allclose(H[A, B, :, d], fd[A], rtol=1e-6, atol=1e-9 * np.abs(H).max())


def test_coord_hessian_symmetry_and_invariances(oracle_mod):
    g = synth.random_points(80, seed=33, n_atom=4)
    na = 4
    args = (g.coords, g.weights, g.rho, g.grad_rho, g.atom_of_point, na)
    H = oracle_mod.coord_hessian(*args)
    scale = np.abs(H).max()
    # a symmetric Hessian: E^{AB} = (E^{BA})^T, each off-diagonal block itself symmetric
    np.testing.assert_allclose(H, H.transpose(1, 0, 3, 2), atol=1e-13 * scale)
    np.testing.assert_allclose(H, H.transpose(0, 1, 3, 2), atol=1e-13 * scale)
    # translational invariance: every block row sums to zero
    np.testing.assert_allclose(H.sum(axis=1), 0.0, atol=1e-12 * scale)
    # rotating the whole system (coordinates and density gradients) rotates every block
    th = 0.7
    Rm = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]]) @ \
        np.array([[1, 0, 0], [0, np.cos(0.3), -np.sin(0.3)], [0, np.sin(0.3), np.cos(0.3)]])
    Hr = oracle_mod.coord_hessian(g.coords @ Rm.T, g.weights, g.rho, g.grad_rho @ Rm.T,
                                  g.atom_of_point, na)
    np.testing.assert_allclose(Hr, np.einsum("uv,abvw,xw->abux", Rm, H, Rm), atol=1e-11 * scale)
    # the per-point matrices sum to the blocks: E^{AB} = sum_{i in A} w_i rho_i D_i^B
    Dp = oracle_mod.point_coord_hessian(*args)
    kept = g.rho >= 1e-10
    for A in range(na):
        m = (g.atom_of_point == A) & kept
        blk = np.einsum("i,ibuv->buv", (g.weights * g.rho)[m], Dp[m])
        for B in range(na):
            if B != A:
                np.testing.assert_allclose(blk[B], H[A, B], rtol=1e-10, atol=1e-13 * scale)
            else:
                assert not Dp[m][:, A].any()  # D_i^B is defined for i not in B only


# --------------------------------------------------------------------- weight-derivative sums

def _directions(g, P, seed):
    """P weight directions with the weights' scale and sign changes (like the components of
    w^B, which change sign across a Becke cell boundary)."""
    rng = np.random.default_rng(seed)
    return rng.normal(size=(P, g.n)) * g.weights[None, :]


def test_weight_sums_with_w_as_direction_are_row_sums(oracle_mod):
    """With w itself as the direction, E^{Bw}, U^{Bw}, W^{Bw} (Sec. II.B) are the row sums
    E_i, U_i, W_i of Sec. II.A."""
    g, args = _sys(seed=51, n=60, n_atom=3)
    ps = oracle_mod.pair_sums(*args)
    E, U, W = oracle_mod.weight_response(*args, g.weights[None, :])
    for got, key in ((E, "E"), (U, "U"), (W, "W")):
        np.testing.assert_allclose(got[0], ps[key], rtol=1e-12, atol=1e-14 * np.abs(ps[key]).max())


def test_weight_sums_are_second_weight_derivatives_of_energy(oracle_mod):
    """E is quadratic in w, with d^2E/dw_i dw_j = rho_i rho_j Phi_ij, so for directions a, b
    the mixed second difference of the energy is sum_i a_i rho_i E_i^{b} exactly (the
    E_i^{Bw} term of E^{AB}_{w,w}, Sec. II.B)."""
    g, args = _sys(seed=52, n=40, n_atom=3)
    V = _directions(g, 3, seed=1)
    E, _, _ = oracle_mod.weight_response(*args, V)
    h = 0.3
    en = lambda w: oracle_mod.energy(g.coords, w, g.rho, g.grad_rho)
    for a in range(3):
        for b in range(3):
            fd = (en(g.weights + h * V[a] + h * V[b]) - en(g.weights + h * V[a] - h * V[b])
                  - en(g.weights - h * V[a] + h * V[b]) + en(g.weights - h * V[a] - h * V[b])) / (4 * h * h)
            an = np.sum(V[a] * g.rho * E[b])
            assert fd == pytest.approx(an, rel=1e-8)
            # and the symmetry of the second derivative
            assert an == pytest.approx(np.sum(V[b] * g.rho * E[a]), rel=1e-12)


def test_weight_sums_are_potential_derivatives(oracle_mod):
    """f^rho_i = beta + E_i + rho_i (kappa'_i U_i + omega_rho,i W_i) and f^gamma_i =
    rho_i omega_gamma,i W_i are linear in w: their derivative along a weight direction v is
    the same expression in E_i^v, U_i^v, W_i^v.  f^gamma pins W^v, then f^rho pins U^v."""
    g, args = _sys(seed=53, n=40, n_atom=3)
    V = _directions(g, 2, seed=2)
    E, U, W = oracle_mod.weight_response(*args, V)
    pp = oracle_mod.point_props(g.rho, g.grad_rho)
    h = 0.5
    for p in range(2):
        _, vr_p, vg_p = oracle_mod.potential(g.coords, g.weights + h * V[p], g.rho, g.grad_rho)
        _, vr_m, vg_m = oracle_mod.potential(g.coords, g.weights - h * V[p], g.rho, g.grad_rho)
        dvr, dvg = (vr_p - vr_m) / (2 * h), (vg_p - vg_m) / (2 * h)
        np.testing.assert_allclose(g.rho * pp["omega_gamma"] * W[p], dvg, rtol=1e-8,
                                   atol=1e-12 * np.abs(dvg).max())
        an = E[p] + g.rho * (pp["kappa_rho"] * U[p] + pp["omega_rho"] * W[p])
        np.testing.assert_allclose(an, dvr, rtol=1e-8, atol=1e-12 * np.abs(dvr).max())
        # the three sums are independent: each term alone is far from the derivative
        assert np.abs(E[p] - dvr).max() > 1e-3 * np.abs(dvr).max()


# --------------------------------------------------------------------- AO-side assembly

def _ao_case(n_trials=0, seed=5):
    """A water grid with an AO-built density, restricted to points well above the cutoff so
    that finite differences of the density matrix move no point across it."""
    g, phi, dphi, P, Pt, rt, gt = synth.ao_system(synth.water(), 8, 14, seed, n_trials)
    m = g.rho > 1e-6
    h = synth.GridDensity(g.coords[m], g.weights[m], g.rho[m], g.grad_rho[m],
                          g.atom_of_point[m], g.molecule)
    return h, phi[m], dphi[m], P, Pt, rt[:, m], gt[:, m]


def test_fock_matrix_is_energy_derivative(oracle_mod):
    """F_mu_nu = dE/dP_mu_nu for rho = sum P_mu_nu phi_mu phi_nu (Sec. II.A): central
    differences of the oracle energy along the symmetric direction E_mu_nu + E_nu_mu."""
    g, phi, dphi, P, _, _, _ = _ao_case()
    _, vr, vg = oracle_mod.potential(g.coords, g.weights, g.rho, g.grad_rho)
    F = oracle_mod.fock_matrix(g.weights, g.grad_rho, vr, vg, phi, dphi)
    np.testing.assert_allclose(F, F.T, rtol=1e-12, atol=1e-14 * np.abs(F).max())
    nbf = P.shape[0]
    h = 1e-5
    for mu, nu in [(0, 0), (0, 3), (2, 7), (5, 5), (4, nbf - 1), (nbf - 1, nbf - 1)]:
        D = np.zeros_like(P)
        D[mu, nu] += 1.0
        D[nu, mu] += 1.0
        def energy(Pm):
            r, gr = synth.ao_density(phi, dphi, Pm)
            return oracle_mod.energy(g.coords, g.weights, r, gr)
        fd = (energy(P + h * D) - energy(P - h * D)) / (2 * h)
        assert fd == pytest.approx(2.0 * F[mu, nu], rel=1e-6, abs=1e-9 * np.abs(F).max())


def test_orbital_hessian_is_fock_derivative(oracle_mod):
    """G^t_mu_nu = dF_mu_nu/dP along P^t (Sec. II.B; the trial density is rho^t = sum P^t phi
    phi): central differences of the oracle Fock matrix, with the oracle potential at P +- h P^t,
    against the assembly of the oracle Hessian contraction."""
    g, phi, dphi, P, Pt, rt, gt = _ao_case(n_trials=2, seed=6)
    _, vr, vg = oracle_mod.potential(g.coords, g.weights, g.rho, g.grad_rho)
    fr, fg = oracle_mod.hessian_contract(g.coords, g.weights, g.rho, g.grad_rho, rt, gt)
    G = oracle_mod.orbital_hessian(g.weights, g.grad_rho, vg, fr, fg, gt, phi, dphi)
    h = 1e-5
    for t in range(2):
        np.testing.assert_allclose(G[t], G[t].T, rtol=1e-12, atol=1e-14 * np.abs(G[t]).max())
        Fs = []
        for sgn in (1, -1):
            r, gr = synth.ao_density(phi, dphi, P + sgn * h * Pt[t])
            _, vr2, vg2 = oracle_mod.potential(g.coords, g.weights, r, gr)
            Fs.append(oracle_mod.fock_matrix(g.weights, gr, vr2, vg2, phi, dphi))
        fd = (Fs[0] - Fs[1]) / (2 * h)
        np.testing.assert_allclose(G[t], fd, rtol=1e-5, atol=1e-8 * np.abs(G[t]).max())


# --------------------------------------------------------------------- nuclear gradient

NUCLEAR_CASES = [("water", lambda: synth.water(), 10, 26),
                 ("chon4", lambda: synth.random_chon(np.random.default_rng(2), 4), 8, 14)]


@pytest.mark.parametrize("name,make,nr,na", NUCLEAR_CASES, ids=[c[0] for c in NUCLEAR_CASES])
def test_nuclear_gradient_from_its_terms(oracle_mod, name, make, nr, na):
    """E^A = E^A_G + E^A_w + E^A_gr (Sec. II.A) against central differences of the energy of
    the whole synthetic pipeline (grid points, Becke weights and density all moving with the
    atoms): E^A_G from the potential and the density derivatives at the moving points, E^A_w
    from dE/dw_i = rho_i (beta + E_i) and the Becke weight derivatives, E^A_gr from the first
    form of the grid-position gradient."""
    mol = make()
    g = synth.make_system(mol, nr, na)
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    kept = g.rho >= 1e-10
    _, vr, vg = oracle_mod.potential(*args)
    E = oracle_mod.pair_sums(*args)["E"]
    rt, gt = synth.nuclear_density_derivatives(mol, g.coords, g.atom_of_point)
    W = synth.weight_directions(mol, nr, na)
    ga = oracle_mod.atom_grad(*args, g.atom_of_point, mol.n_atom)
    an = np.zeros(3 * mol.n_atom)
    for p in range(an.size):
        e_g = np.sum(g.weights * (vr * rt[p] + 2 * vg * np.einsum("nd,nd->n", g.grad_rho, gt[p])))
        e_w = np.sum((W[p] * g.rho * (oracle_mod.beta() + E))[kept])
        an[p] = e_g + e_w + ga[p // 3, p % 3]
    h = 1e-4
    for p in range(an.size):
        es = []
        for sg in (1, -1):
            c = mol.coords.copy()
            c[p // 3, p % 3] += sg * h
            g2 = synth.make_system(synth.Molecule(mol.symbols, c), nr, na)
            assert np.array_equal(g2.rho >= 1e-10, kept)  # no point crosses the cutoff
            es.append(oracle_mod.energy(g2.coords, g2.weights, g2.rho, g2.grad_rho))
        assert (es[0] - es[1]) / (2 * h) == pytest.approx(an[p], rel=1e-6, abs=1e-7 * np.abs(an).max())
    # translational invariance of the whole gradient
    assert np.abs(an.reshape(-1, 3).sum(axis=0)).max() <= 1e-6 * np.abs(an).max()


def _nuclear_case(mol, nr, na):
    g = synth.make_system(mol, nr, na)
    rt, gt = synth.nuclear_density_derivatives(mol, g.coords, g.atom_of_point)
    return g, rt, gt, synth.weight_directions(mol, nr, na)


def _nuclear_gradient(oracle_mod, g, rt, gt, W):
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    kept = g.rho >= 1e-10
    _, vr, vg = oracle_mod.potential(*args)
    E = oracle_mod.pair_sums(*args)["E"]
    ga = oracle_mod.atom_grad(*args, g.atom_of_point, g.molecule.n_atom).reshape(-1)
    return np.array([np.sum(g.weights * (vr * rt[p] + 2 * vg * np.einsum("nd,nd->n", g.grad_rho, gt[p])))
                     + np.sum((W[p] * g.rho * (oracle_mod.beta() + E))[kept]) + ga[p]
                     for p in range(rt.shape[0])])


@pytest.mark.parametrize("name,make,nr,na", NUCLEAR_CASES, ids=[c[0] for c in NUCLEAR_CASES])
def test_nuclear_hessian_from_its_nine_terms(oracle_mod, name, make, nr, na):
    """E^{AB} = E_GG + E_ww + E_grgr + (E_Gw + E_Ggr + E_wgr) + transposes (Sec. II.B, Eq. E_hess)
    from the oracle's pair sums (the Hessian contraction with the nuclear trials, the
    weight-derivative and atom-resolved sums, the grid-grid blocks) and the local derivatives,
    against central differences of the nuclear gradient (itself pinned to the pipeline's
    energy) with the whole synthetic pipeline moving with the atoms."""
    mol = make()
    g, rt, gt, W = _nuclear_case(mol, nr, na)
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    kept = g.rho >= 1e-10
    NA = mol.n_atom
    P = 3 * NA
    _, vr, vg = oracle_mod.potential(*args)
    E = oracle_mod.pair_sums(*args)["E"]
    pp = oracle_mod.point_props(g.rho, g.grad_rho)
    r2, g2 = synth.nuclear_density_second_derivatives(mol, g.coords, g.atom_of_point)
    Wab = synth.weight_second_derivatives(mol, nr, na)
    Ew, Uw, Ww = oracle_mod.weight_response(*args, W)
    Egr, Ugr, Wgr = (x.reshape(g.n, P).T for x in oracle_mod.atom_resolved(*args, g.atom_of_point, NA))
    fr, fg = oracle_mod.hessian_contract(*args, rt, gt)
    Hgg = oracle_mod.coord_hessian(*args, g.atom_of_point, NA).transpose(0, 2, 1, 3).reshape(P, P)
    H = oracle_mod.nuclear_hessian(g.weights, g.rho, g.grad_rho, kept, pp["kappa_rho"],
                                   pp["omega_rho"], pp["omega_gamma"], vr, vg, E, rt, gt, r2, g2,
                                   W, Wab, Ew, Uw, Ww, Egr, Ugr, Wgr, fr, fg, Hgg)
    h = 1e-4
    fd = np.zeros((P, P))
    for b in range(P):
        gs = []
        for sg in (1, -1):
            c = mol.coords.copy()
            c[b // 3, b % 3] += sg * h
            m2 = synth.Molecule(mol.symbols, c)
            g2s, rt2, gt2, W2 = _nuclear_case(m2, nr, na)
            assert np.array_equal(g2s.rho >= 1e-10, kept)
            gs.append(_nuclear_gradient(oracle_mod, g2s, rt2, gt2, W2))
        fd[:, b] = (gs[0] - gs[1]) / (2 * h)
    scale = np.abs(fd).max()
    assert np.abs(H - fd).max() <= 1e-6 * scale
    assert np.abs(H - H.T).max() <= 1e-8 * scale  # w^{ab} comes from central differences
    # translational invariance: every row sums to zero over the atoms (per component)
    assert np.abs(H.reshape(P, NA, 3).sum(axis=1)).max() <= 1e-6 * scale


def test_nuclear_hessian_pin_catches_planted_mistakes(oracle_mod):
    """Each input of the nine-term assembly zeroed in turn (a dropped term or pair sum: the
    potential, E_i, rho^a, grad rho^a, their second derivatives, w^a, w^{ab}, the
    weight-derivative and atom-resolved sums, the Hessian contraction, the grid-grid blocks)
    moves the nuclear Hessian at least 100 times the pin's tolerance away from the central
    differences of the gradient."""
    mol, nr, na = synth.water(), 10, 26
    g, rt, gt, W = _nuclear_case(mol, nr, na)
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    kept = g.rho >= 1e-10
    NA, P = mol.n_atom, 3 * mol.n_atom
    _, vr, vg = oracle_mod.potential(*args)
    pp = oracle_mod.point_props(g.rho, g.grad_rho)
    r2, g2 = synth.nuclear_density_second_derivatives(mol, g.coords, g.atom_of_point)
    Ew, Uw, Ww = oracle_mod.weight_response(*args, W)
    Egr, Ugr, Wgr = (x.reshape(g.n, P).T for x in oracle_mod.atom_resolved(*args, g.atom_of_point, NA))
    fr, fg = oracle_mod.hessian_contract(*args, rt, gt)
    base = dict(vr=vr, vg=vg, E=oracle_mod.pair_sums(*args)["E"], rt=rt, gt=gt, r2=r2, g2=g2, W=W,
                Wab=synth.weight_second_derivatives(mol, nr, na), Ew=Ew, Uw=Uw, Ww=Ww, Egr=Egr,
                Ugr=Ugr, Wgr=Wgr, fr=fr, fg=fg,
                Hgg=oracle_mod.coord_hessian(*args, g.atom_of_point, NA).transpose(0, 2, 1, 3).reshape(P, P))

    def assemble(**kw):
        q = dict(base, **kw)
        return oracle_mod.nuclear_hessian(g.weights, g.rho, g.grad_rho, kept, pp["kappa_rho"],
                                          pp["omega_rho"], pp["omega_gamma"], *(q[k] for k in (
                                              "vr", "vg", "E", "rt", "gt", "r2", "g2", "W", "Wab",
                                              "Ew", "Uw", "Ww", "Egr", "Ugr", "Wgr", "fr", "fg",
                                              "Hgg")))

    h = 1e-4
    fd = np.zeros((P, P))
    for b in range(P):
        gs = []
        for sg in (1, -1):
            c = mol.coords.copy()
            c[b // 3, b % 3] += sg * h
            gs.append(_nuclear_gradient(oracle_mod, *_nuclear_case(synth.Molecule(mol.symbols, c), nr, na)))
        fd[:, b] = (gs[0] - gs[1]) / (2 * h)
    scale = np.abs(fd).max()
    assert np.abs(assemble() - fd).max() <= 1e-6 * scale
    for k, v in base.items():
        assert np.abs(assemble(**{k: np.zeros_like(v)}) - fd).max() >= 1e-4 * scale, k


# ------------------------------------------------------ nuclear derivative of the Fock matrix

def _fock_derivative_terms(oracle_mod, g, phi, dphi, d2phi, basis, rt, gt, W):
    """The oracle's F^a from its pair sums: the potential, the Hessian contraction with the
    nuclear trials, the weight-derivative and the atom-resolved sums."""
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    NA = g.molecule.n_atom
    P = 3 * NA
    _, vr, vg = oracle_mod.potential(*args)
    Ew, Uw, Ww = oracle_mod.weight_response(*args, W)
    Egr, Ugr, Wgr = (x.reshape(g.n, P).T for x in oracle_mod.atom_resolved(*args, g.atom_of_point, NA))
    fr, fg = oracle_mod.hessian_contract(*args, rt, gt)
    pp = oracle_mod.point_props(g.rho, g.grad_rho)
    return oracle_mod.fock_derivative(g.weights, g.rho, g.grad_rho, g.rho >= 1e-10, pp["kappa_rho"],
                                      pp["omega_rho"], pp["omega_gamma"], vr, vg, phi, dphi, d2phi,
                                      basis.atom, g.atom_of_point, gt, W, Ew, Uw, Ww, Egr, Ugr, Wgr,
                                      fr, fg)


FOCK_NUCLEAR_CASES = [("water", lambda: synth.water(), 8, 14, 5),
                      ("chon4", lambda: synth.random_chon(np.random.default_rng(2), 4), 8, 14, 6)]


@pytest.mark.parametrize("name,make,nr,na,seed", FOCK_NUCLEAR_CASES,
                         ids=[c[0] for c in FOCK_NUCLEAR_CASES])
def test_fock_derivative_from_its_three_terms(oracle_mod, name, make, nr, na, seed):
    """F^A_mu_nu = F^A_G + F^A_gr + F^A_w (Sec. II.B) against central differences of the oracle
    Fock matrix of the whole moving pipeline (grid points, Becke weights, basis functions and
    the AO density of a fixed density matrix; the same subset of points at every geometry).
    Every term and both halves of the basis derivative (owner atom of the point, atom of the
    function) are needed to meet it; F^A is symmetric and sums to zero over the atoms."""
    mol = make()
    g, phi, dphi, d2phi, basis, Pm, sel, rt, gt, W = synth.ao_moving_system(mol, nr, na, seed=seed)
    FA = _fock_derivative_terms(oracle_mod, g, phi, dphi, d2phi, basis, rt, gt, W)
    scale = np.abs(FA).max()
    fd = _fock_differences(oracle_mod, mol, nr, na, Pm, sel)
    assert np.abs(FA - fd).max() <= 1e-6 * scale
    assert np.abs(FA - FA.transpose(0, 2, 1)).max() <= 1e-14 * scale
    assert np.abs(FA.reshape(mol.n_atom, 3, *FA.shape[1:]).sum(axis=0)).max() <= 1e-8 * scale


def _fock_differences(oracle_mod, mol, nr, na, Pm, sel, h=1e-4):
    """Central differences of the oracle Fock matrix of the moving pipeline, (3 N_atom, nbf, nbf)."""
    out = []
    for a in range(3 * mol.n_atom):
        Fs = []
        for sg in (1, -1):
            c = mol.coords.copy()
            c[a // 3, a % 3] += sg * h
            g2, f2, df2 = synth.ao_moving_system(synth.Molecule(mol.symbols, c), nr, na, P=Pm,
                                                 sel=sel)[:3]
            _, vr2, vg2 = oracle_mod.potential(g2.coords, g2.weights, g2.rho, g2.grad_rho)
            Fs.append(oracle_mod.fock_matrix(g2.weights, g2.grad_rho, vr2, vg2, f2, df2))
        out.append((Fs[0] - Fs[1]) / (2 * h))
    return np.array(out)


def test_fock_derivative_pin_catches_planted_mistakes(oracle_mod):
    """Each plausible mistake planted in the oracle's assembly (one term dropped by zeroing its
    input, or one half of the basis-function derivative dropped by relabelling the atoms) moves
    F^A at least 100 times the pin's tolerance away from the central differences."""
    mol, nr, na, seed = synth.water(), 8, 14, 5
    g, phi, dphi, d2phi, basis, Pm, sel, rt, gt, W = synth.ao_moving_system(mol, nr, na, seed=seed)
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    NA, P = mol.n_atom, 3 * mol.n_atom
    _, vr, vg = oracle_mod.potential(*args)
    Ew, Uw, Ww = oracle_mod.weight_response(*args, W)
    Egr, Ugr, Wgr = (x.reshape(g.n, P).T for x in oracle_mod.atom_resolved(*args, g.atom_of_point, NA))
    fr, fg = oracle_mod.hessian_contract(*args, rt, gt)
    pp = oracle_mod.point_props(g.rho, g.grad_rho)
    base = dict(vg=vg, d2phi=d2phi, bf_atom=basis.atom, own=g.atom_of_point, gt=gt, W=W, Ew=Ew,
                Uw=Uw, Ww=Ww, Egr=Egr, Ugr=Ugr, Wgr=Wgr, fr=fr, fg=fg)

    def assemble(**kw):
        q = dict(base, **kw)
        return oracle_mod.fock_derivative(g.weights, g.rho, g.grad_rho, g.rho >= 1e-10,
                                          pp["kappa_rho"], pp["omega_rho"], pp["omega_gamma"], vr,
                                          q["vg"], phi, dphi, q["d2phi"], q["bf_atom"], q["own"],
                                          q["gt"], q["W"], q["Ew"], q["Uw"], q["Ww"], q["Egr"],
                                          q["Ugr"], q["Wgr"], q["fr"], q["fg"])

    fd = _fock_differences(oracle_mod, mol, nr, na, Pm, sel)
    scale = np.abs(fd).max()
    assert np.abs(assemble() - fd).max() <= 1e-6 * scale
    planted = {k: {k: np.zeros_like(v)} for k, v in base.items()
               if k in ("d2phi", "gt", "W", "Ew", "Uw", "Ww", "Egr", "Ugr", "Wgr", "fr", "fg")}
    planted["owner half"] = {"own": np.full_like(g.atom_of_point, -1)}
    planted["centre half"] = {"bf_atom": np.full_like(basis.atom, -1)}
    for name, kw in planted.items():
        assert np.abs(assemble(**kw) - fd).max() >= 1e-4 * scale, name
