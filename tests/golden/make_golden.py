"""Write the stored expected values under tests/golden/ (calls only oracle/ and the
seeded input generator).  Run: python tests/golden/make_golden.py"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2208_14639_gb300 import synth  # noqa: E402

ROWS = [0, 17, 1234, 3300, 5000, 7777, 9899]


def main():
    g = synth.config_water()
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    e, vr, vg = oracle.potential(*args)
    _, vr_s, vg_s = oracle.potential(*args, rows=ROWS)
    rt, gt = synth.trial_densities(g.molecule, g.coords)
    fr, fg = oracle.hessian_contract(*args, rt, gt, rows=ROWS)
    pg = oracle.point_grad(*args, rows=ROWS)
    out = {
        "what": "water, 30x110 points per atom (9,900 points), b=6, C=0.01, rho_cut=1e-10",
        "source": "oracle/ (FP64 CPU) via tests/golden/make_golden.py",
        "n_kept": int((g.rho >= 1e-10).sum()),
        "energy": e,
        "rows": ROWS,
        "vrho": vr_s.tolist(),
        "vgamma": vg_s.tolist(),
        "f_rho_t": fr.tolist(),
        "f_gamma_t": fg.tolist(),
        "point_grad": pg.tolist(),
        "beta_b6": oracle.beta(6.0),
    }
    assert np.allclose(vr[ROWS], vr_s, rtol=0, atol=0)
    with open(os.path.join(HERE, "water_9900.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("energy", e)


if __name__ == "__main__":
    main()
