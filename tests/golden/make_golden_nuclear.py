"""Write the stored expected values of the nuclear-derivative quantities under tests/golden/
(calls only oracle/ and the seeded input generator).  Run:
python tests/golden/make_golden_nuclear.py"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2208_14639_gb300 import synth  # noqa: E402

NR, NA = 10, 26
ROWS = [0, 100, 250, 400, 555, 779]


def quantities():
    """The values stored and re-checked: water on a 10 x 26 grid per atom (780 points)."""
    mol = synth.water()
    g = synth.make_system(mol, NR, NA)
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    kept = g.rho >= 1e-10
    P = 3 * mol.n_atom
    rt, gt = synth.nuclear_density_derivatives(mol, g.coords, g.atom_of_point)
    W = synth.weight_directions(mol, NR, NA)
    _, vr, vg = oracle.potential(*args)
    E = oracle.pair_sums(*args)["E"]
    ga = oracle.atom_grad(*args, g.atom_of_point, mol.n_atom).reshape(-1)
    grad = np.array([np.sum(g.weights * (vr * rt[p] + 2 * vg * np.einsum("nd,nd->n", g.grad_rho, gt[p])))
                     + np.sum((W[p] * g.rho * (oracle.beta() + E))[kept]) + ga[p] for p in range(P)])
    Ew, Uw, Ww = oracle.weight_response(*args, W)
    Egr, Ugr, Wgr = (x.reshape(g.n, P).T for x in oracle.atom_resolved(*args, g.atom_of_point, mol.n_atom))
    fr, fg = oracle.hessian_contract(*args, rt, gt)
    Hgg4 = oracle.coord_hessian(*args, g.atom_of_point, mol.n_atom)
    Hgg = Hgg4.transpose(0, 2, 1, 3).reshape(P, P)
    r2, g2 = synth.nuclear_density_second_derivatives(mol, g.coords, g.atom_of_point)
    Wab = synth.weight_second_derivatives(mol, NR, NA)
    pp = oracle.point_props(g.rho, g.grad_rho)
    H = oracle.nuclear_hessian(g.weights, g.rho, g.grad_rho, kept, pp["kappa_rho"], pp["omega_rho"],
                               pp["omega_gamma"], vr, vg, E, rt, gt, r2, g2, W, Wab, Ew, Uw, Ww,
                               Egr, Ugr, Wgr, fr, fg, Hgg)
    return dict(coord_hessian=Hgg4, weight_E=Ew[:, ROWS], weight_U=Uw[:, ROWS],
                weight_W=Ww[:, ROWS], nuclear_gradient=grad, nuclear_hessian=H)


AO_NR, AO_NA, AO_SEED = 8, 14, 5
AO_ROWS = [0, 4, 8, 12]


def fock_quantities():
    """The Fock matrix and its nuclear derivative for water with its AO basis (13 functions) on
    the 8 x 14 grid per atom, the points with rho > 1e-6: rows AO_ROWS of F and of every F^a."""
    mol = synth.water()
    g, phi, dphi, d2phi, basis, _, _, rt, gt, W = synth.ao_moving_system(mol, AO_NR, AO_NA, seed=AO_SEED)
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    P = 3 * mol.n_atom
    _, vr, vg = oracle.potential(*args)
    F = oracle.fock_matrix(g.weights, g.grad_rho, vr, vg, phi, dphi)
    Ew, Uw, Ww = oracle.weight_response(*args, W)
    Egr, Ugr, Wgr = (x.reshape(g.n, P).T for x in oracle.atom_resolved(*args, g.atom_of_point, mol.n_atom))
    fr, fg = oracle.hessian_contract(*args, rt, gt)
    pp = oracle.point_props(g.rho, g.grad_rho)
    FA = oracle.fock_derivative(g.weights, g.rho, g.grad_rho, g.rho >= 1e-10, pp["kappa_rho"],
                                pp["omega_rho"], pp["omega_gamma"], vr, vg, phi, dphi, d2phi,
                                basis.atom, g.atom_of_point, gt, W, Ew, Uw, Ww, Egr, Ugr, Wgr, fr, fg)
    return dict(fock_matrix=F[AO_ROWS], fock_derivative=FA[:, AO_ROWS])


def main():
    q = quantities()
    qf = fock_quantities()
    out = {"what": f"water, {NR}x{NA} points per atom, b=6, C=0.01, rho_cut=1e-10; Becke weight "
                   "directions; rows " + str(ROWS) + " of the weight-derivative sums; the Fock "
                   f"matrix and its nuclear derivative (rows {AO_ROWS}) on the {AO_NR}x{AO_NA} "
                   f"grid's points with rho > 1e-6, AO basis, density matrix seed {AO_SEED}",
           "source": "oracle/ (FP64 CPU) via tests/golden/make_golden_nuclear.py",
           "rows": ROWS, "ao_rows": AO_ROWS}
    out.update({k: np.asarray(v).tolist() for k, v in q.items()})
    out.update({k: np.asarray(v).tolist() for k, v in qf.items()})
    with open(os.path.join(HERE, "water_780_nuclear.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("nuclear gradient", q["nuclear_gradient"])


if __name__ == "__main__":
    main()
