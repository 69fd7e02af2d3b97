"""vv10_energy_potential_noalloc, the entry point for callers that cannot allocate device
memory, against vv10_energy_potential on the same inputs.  Collected last on purpose.

Two calls in a row for each precision, on different inputs, through the C ABI: the second
call must not see anything the first left in the shared static scratch array.
Tolerances are those of the parity tests: FP64 |dE|/|E| <= 1e-11 and potential <= 1e-10
relative; mixed |dE| <= 1e-7 and potential <= 1e-6 relative.
"""
import numpy as np
import pytest
import torch

from paper_2208_14639_gb300 import synth, vv10

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _dev(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev, torch.float64)


def _reference(g, prec, dev):
    eng = vv10.VV10(0)
    eng.prepare(_dev(g.coords, dev), _dev(g.weights, dev), _dev(g.rho, dev), _dev(g.grad_rho, dev))
    e, vr, vg = eng.energy_potential(prec)
    eng.close()
    return e, vr.cpu().numpy(), vg.cpu().numpy()


def test_noalloc_matches_energy_potential():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    vv10.load(build_if_missing=True)
    dev = torch.device("cuda", 0)
    systems = [synth.config_water(), synth.random_points(5000, seed=31, n_atom=3)]
    for prec, tol_e, tol_v in ((vv10.VV10_FP64, None, 1e-10), (vv10.VV10_MIXED_TF32X3, 1e-7, 1e-6)):
        for g in systems:  # two calls in a row sharing the static scratch
            e_ref, vr_ref, vg_ref = _reference(g, prec, dev)
            energy = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
            vrho = torch.full((g.n,), np.nan, dtype=torch.float64, device=dev)
            vgamma = torch.full((g.n,), np.nan, dtype=torch.float64, device=dev)
            vv10.vv10_energy_potential_noalloc(_dev(g.coords, dev), _dev(g.weights, dev),
                                               _dev(g.rho, dev), _dev(g.grad_rho, dev), prec,
                                               energy, vrho, vgamma)
            torch.cuda.synchronize()
            e = float(energy.item())
            if tol_e is None:
                assert abs(e - e_ref) <= 1e-11 * abs(e_ref)
            else:
                assert abs(e - e_ref) <= tol_e
            assert _rel(vrho.cpu().numpy(), vr_ref) <= tol_v
            assert _rel(vgamma.cpu().numpy(), vg_ref) <= tol_v
            kept = g.rho >= 1e-10
            assert np.all(vrho.cpu().numpy()[~kept] == 0.0)


def test_noalloc_rejects_too_many_points():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dev = torch.device("cuda", 0)
    n = vv10.VV10_NOALLOC_MAX_POINTS + 1
    z = torch.zeros(n, dtype=torch.float64, device=dev)
    z3 = torch.zeros(n, 3, dtype=torch.float64, device=dev)
    e = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(vv10.VV10Error) as ei:
        vv10.vv10_energy_potential_noalloc(z3, z, z, z3, vv10.VV10_FP64, e)
    assert ei.value.status == vv10.VV10_ERR_UNSUPPORTED
