"""The oracle reproduces its stored water values (written by tests/golden/make_golden.py,
which calls only oracle/); this catches a change in the oracle's arithmetic or a
machine-dependent build (x86 here, aarch64 on the GPU host)."""
import json
import os

import numpy as np

from paper_2208_14639_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def test_water_golden(oracle_mod):
    with open(os.path.join(HERE, "golden", "water_9900.json")) as f:
        gold = json.load(f)
    g = synth.config_water()
    args = (g.coords, g.weights, g.rho, g.grad_rho)
    assert int((g.rho >= 1e-10).sum()) == gold["n_kept"]
    e, _, _ = oracle_mod.potential(*args)
    assert abs(e - gold["energy"]) <= 1e-12 * abs(gold["energy"])
    rows = gold["rows"]
    _, vr, vg = oracle_mod.potential(*args, rows=rows)
    np.testing.assert_allclose(vr, gold["vrho"], rtol=1e-11)
    np.testing.assert_allclose(vg, gold["vgamma"], rtol=1e-11)
    rt, gt = synth.trial_densities(g.molecule, g.coords)
    fr, fg = oracle_mod.hessian_contract(*args, rt, gt, rows=rows)
    np.testing.assert_allclose(fr, gold["f_rho_t"], rtol=1e-10, atol=1e-13 * np.abs(fr).max())
    np.testing.assert_allclose(fg, gold["f_gamma_t"], rtol=1e-10, atol=1e-13 * np.abs(fg).max())
    pg = oracle_mod.point_grad(*args, rows=rows)
    np.testing.assert_allclose(pg, gold["point_grad"], rtol=1e-10, atol=1e-14)


def test_water_nuclear_golden(oracle_mod):
    """The nuclear-derivative quantities (grid-grid Hessian blocks, weight-derivative sums, the
    nuclear gradient, the nine-term nuclear Hessian, the Fock matrix and its nuclear derivative)
    reproduce their stored values (written
    by tests/golden/make_golden_nuclear.py, which calls only oracle/)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden_nuclear",
                                                  os.path.join(HERE, "golden", "make_golden_nuclear.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    with open(os.path.join(HERE, "golden", "water_780_nuclear.json")) as f:
        gold = json.load(f)
    assert gold["rows"] == mk.ROWS and gold["ao_rows"] == mk.AO_ROWS
    q = mk.quantities()
    q.update(mk.fock_quantities())
    for key, val in q.items():
        ref = np.asarray(gold[key])
        np.testing.assert_allclose(val, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max(), err_msg=key)
