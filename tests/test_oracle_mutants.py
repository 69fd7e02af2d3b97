"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of the oracle's C source (a dropped term, a wrong sign
or factor, a dropped self pair) or of one of its numpy assemblies, and runs the named pins of
test_oracle_pins.py against it: every named pin must fail.  The unmodified oracle passes the
same pins in that module.  Planting happens on the CPU only; nothing here touches the CUDA path.
"""
import contextlib
import inspect
import os
import sys
import textwrap

import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import test_oracle_pins as pins  # noqa: E402

POT = pins.test_potential_is_energy_derivative
PTD = pins.test_point_derivatives_by_finite_differences
HES = pins.test_hessian_contraction_is_potential_derivative
ENE = pins.test_one_and_two_point_energies
PGR = pins.test_point_gradient_is_energy_derivative
AGR = pins.test_atom_gradient_first_form
ARS = pins.test_atom_resolved_terms_are_derivatives
CHS = pins.test_coord_hessian_is_derivative_of_atom_gradient
WPD = pins.test_weight_sums_are_potential_derivatives
WSD = pins.test_weight_sums_are_second_weight_derivatives_of_energy


def BETA(o):
    pins.test_beta_from_uniform_gas_limit(o, 0.1)


# (tag, text in vv10_oracle.c, its planted replacement, pins that must fail)
MUTANTS = [
    ("u_drops_1_over_g", "        double t1 = 1.0 / sg + 1.0 / g;\n        double t2",
     "        double t1 = 1.0 / sg;\n        double t2", [POT]),
    ("w_drops_r2", "nsum_add(&W, -cj * phi * R2 * t1);", "nsum_add(&W, -cj * phi * t1);", [POT]),
    ("omega_rho_sign", "double Qr = -4.0 * C", "double Qr = 4.0 * C", [PTD, POT]),
    ("kappa_rho_factor", "p.ka_r = p.kappa / (6.0 * rho);", "p.ka_r = p.kappa / (3.0 * rho);",
     [PTD, POT]),
    ("kappa_rr_sign", "p.ka_rr = -5.0 * p.kappa", "p.ka_rr = 5.0 * p.kappa", [PTD, HES]),
    ("energy_drops_half", "(s.beta + 0.5 * nsum_get(&Ei))", "(s.beta + nsum_get(&Ei))", [ENE, POT]),
    ("energy_drops_self_pair",
     "        for (int64_t j = 0; j < nk; ++j) {\n            double phi = orc_phi(",
     "        for (int64_t j = 0; j < nk; ++j) {\n            if (j == i) continue;\n"
     "            double phi = orc_phi(", [ENE]),
    ("beta_factor", "pow(3.0 / (b * b), 0.75) / 32.0", "pow(3.0 / (b * b), 0.75) / 16.0", [BETA]),
    ("contraction_drops_2_on_gamma_t",
     "nsum_add(&acc[t], wj * (f_rr * rtj[t] + 2.0 * f_rg * gtj[t]));",
     "nsum_add(&acc[t], wj * (f_rr * rtj[t] + f_rg * gtj[t]));", [HES]),
    ("contraction_diagonal_gg_term",
     "double d_gg = p->rho * (p->om_gg * W + p->om_g * p->om_g * Cc);",
     "double d_gg = p->rho * (p->om_gg * W);", [HES]),
    ("contraction_M_term", "double M = 2.0 / (sg * sg) + 2.0 / (g * gp);",
     "double M = 2.0 / (sg * sg);", [HES]),
    ("point_gradient_sign", "nsum_add(&acc[d], f * (s.xyz[3 * i + d] - s.xyz[3 * j + d]));",
     "nsum_add(&acc[d], f * (s.xyz[3 * j + d] - s.xyz[3 * i + d]));", [PGR]),
    ("bracket_drops_sum_term",
     "return pi->omega / g + pj->omega / gp + (pi->omega + pj->omega) / (g + gp);",
     "return pi->omega / g + pj->omega / gp;", [PGR, AGR]),
    ("atom_resolved_own_atom_sign", "nsum_add(&e[d], -oE[3 * B + d]);",
     "nsum_add(&e[d], oE[3 * B + d]);", [ARS]),
    ("atom_resolved_drops_t3_term",
     "double t3 = pi->omega / (g * g) + (pi->omega + pj->omega) / (sg * sg);",
     "double t3 = pi->omega / (g * g);", [ARS]),
    ("coord_hessian_identity_sign", "pre * (sq * dr[u] * dr[v] - (u == v ? D : 0.0))",
     "pre * (sq * dr[u] * dr[v] + (u == v ? D : 0.0))", [CHS]),
    ("coord_hessian_drops_a2", "double sq = 2.0 * (D * D + a * a + bb * bb + c * c);",
     "double sq = 2.0 * (D * D + bb * bb + c * c);", [CHS]),
    ("weight_sums_u_drops_1_over_g",
     "                    double t1 = 1.0 / sg + 1.0 / g;\n                    int64_t oj",
     "                    double t1 = 1.0 / sg;\n                    int64_t oj", [WPD]),
    ("weight_sums_use_w", "double vj = wt[(size_t)p * n + oj] * pj->rho;",
     "double vj = s.w[j] * pj->rho;", [WPD, WSD]),
]


@pytest.mark.parametrize("tag,old,new,catch", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pins(oracle_mod, tag, old, new, catch):
    with oracle_mod.planted(old, new, tag):
        for pin in catch:
            name = getattr(pin, "__name__", str(pin))
            try:
                pin(oracle_mod)
            except (AssertionError, FloatingPointError, ValueError):
                continue
            pytest.fail(f"{name} passed with the planted mistake {tag}")


def FOCK(o):
    pins.test_fock_matrix_is_energy_derivative(o)


def GT(o):
    pins.test_orbital_hessian_is_fock_derivative(o)


def FA(o):
    pins.test_fock_derivative_from_its_three_terms(o, *pins.FOCK_NUCLEAR_CASES[0])


def NH(o):
    pins.test_nuclear_hessian_from_its_nine_terms(o, *pins.NUCLEAR_CASES[0])


@contextlib.contextmanager
def planted_py(module, name, old, new):
    """The module's function `name` recompiled from its source with `old` (occurring once)
    replaced by `new`, until the block exits."""
    fn = getattr(module, name)
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, (name, old)
    ns = dict(module.__dict__)
    exec(compile(src.replace(old, new), f"<planted {name}>", "exec"), ns)
    setattr(module, name, ns[name])
    try:
        yield
    finally:
        setattr(module, name, fn)


# (tag, oracle function, text in its source, its planted replacement, pins that must fail)
PY_MUTANTS = [
    ("fock_drops_2_on_gamma_term", "fock_matrix", "v = 2.0 * (w * _f64(vgamma))[:, None]",
     "v = (w * _f64(vgamma))[:, None]", [FOCK]),
    ("fock_one_sided_gradient_term", "fock_matrix", "+ vdphi.T @ phi + phi.T @ vdphi",
     "+ 2.0 * vdphi.T @ phi", [FOCK]),
    ("orbital_hessian_drops_fgamma_grad_rho_t", "orbital_hessian",
     "(fg[t][:, None] * g + vg[:, None] * gt[t])", "(fg[t][:, None] * g)", [GT]),
    ("fock_derivative_drops_grad_rho_a_term", "fock_derivative",
     "+ D(2.0 * (w * vg)[:, None] * ga[a])", "", [FA]),
    ("fock_derivative_drops_basis_hessian_term", "fock_derivative",
     "+ bga.T @ phi + pa.T @ bdphi", "+ pa.T @ bdphi", [FA]),
    ("fock_derivative_drops_weight_derivative_term", "fock_derivative",
     "Fw = (S(wa[a] * m * vr) + ", "Fw = (", [FA]),
    ("nuclear_hessian_drops_a_transpose", "nuclear_hessian", "+ EGw + EGw.T +", "+ 2.0 * EGw +",
     [NH]),
    ("nuclear_hessian_gamma_ab_drops_first_product", "nuclear_hessian",
     'np.einsum("and,bnd->abn", ga, ga) + ', "", [NH]),
]


@pytest.mark.parametrize("tag,name,old,new,catch", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_planted_mistake_in_an_assembly_fails_its_pins(oracle_mod, tag, name, old, new, catch):
    with planted_py(oracle_mod, name, old, new):
        for pin in catch:
            try:
                pin(oracle_mod)
            except (AssertionError, FloatingPointError, ValueError):
                continue
            pytest.fail(f"{pin.__name__} passed with the planted mistake {tag}")
