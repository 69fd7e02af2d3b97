"""vv10_energy_potential_noalloc, the entry point for callers that cannot allocate device
memory (a runtime that took the device memory up front for its own allocator, a plug-in
that is only handed buffers), checked against the FP64 CPU oracle.  Collected last on
purpose, so that a run stopping at the first failure has run every other test first.

Two calls in a row for each precision, on different inputs, through the C ABI: the second
call must not see anything the first left in the shared static scratch array.  Sizes: the
water grid (9,900 points) and a 4-atom molecule's grid of the documented maximum,
VV10_NOALLOC_MAX_POINTS = 32,768 points.
Tolerances are those of the parity tests, against the oracle: FP64 |dE|/|E| <= 1e-11 and
potential <= 1e-10 relative L2; mixed |dE| <= 1e-7 Eh and potential <= 1e-6 relative L2;
each potential element also within tol * (|ref_i| + rms(ref)), with tol = 1e-10 (FP64) and
1e-5 (mixed, ten times the L2 tolerance, as in the parity tests).
"""
import numpy as np
import pytest
import torch

from paper_2208_14639_gb300 import synth, vv10

pytestmark = pytest.mark.gpu

PRECS = [(vv10.VV10_FP64, None, 1e-10), (vv10.VV10_MIXED_TF32X3, 1e-7, 1e-6),
         (vv10.VV10_MIXED_BF16X3, 1e-7, 1e-6), (vv10.VV10_FP64_TC, None, 1e-10)]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _elementwise_ok(a, b, tol):
    s = np.sqrt(np.mean(b * b))
    return bool(np.all(np.abs(a - b) <= tol * (np.abs(b) + s)))


def _dev(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev, torch.float64)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    vv10.load(build_if_missing=True)
    return torch.device("cuda", 0)


@pytest.fixture(scope="module")
def systems(oracle_mod):
    """(grid, oracle energy, vrho, vgamma) for the water grid and a grid of the maximum size."""
    out = []
    # a 4-atom CHON molecule on 64 x 128 points per atom: exactly the maximum, 32,768 points
    chon4 = synth.make_system(synth.random_chon(np.random.default_rng(31), 4), 64, 128)
    for g in (synth.config_water(), chon4):
        out.append((g, *oracle_mod.potential(g.coords, g.weights, g.rho, g.grad_rho)))
    assert out[1][0].n == vv10.VV10_NOALLOC_MAX_POINTS
    return out


def _call(g, prec, dev, d=None):
    d = d or [_dev(x, dev) for x in (g.coords, g.weights, g.rho, g.grad_rho)]
    energy = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
    vrho = torch.full((g.n,), np.nan, dtype=torch.float64, device=dev)
    vgamma = torch.full((g.n,), np.nan, dtype=torch.float64, device=dev)
    vv10.vv10_energy_potential_noalloc(*d, prec, energy, vrho, vgamma)
    torch.cuda.synchronize()
    return float(energy.item()), vrho.cpu().numpy(), vgamma.cpu().numpy()


@pytest.mark.parametrize("prec,tol_e,tol_v", PRECS, ids=["fp64", "tf32x3", "bf16x3", "fp64tc"])
def test_noalloc_matches_oracle(dev, systems, prec, tol_e, tol_v):
    for g, e_ref, vr_ref, vg_ref in systems:  # two calls in a row sharing the static scratch
        e, vr, vg = _call(g, prec, dev)
        if tol_e is None:
            assert abs(e - e_ref) <= 1e-11 * abs(e_ref)
        else:
            assert abs(e - e_ref) <= tol_e
        assert _rel(vr, vr_ref) <= tol_v and _rel(vg, vg_ref) <= tol_v
        el = tol_v if tol_e is None else 10.0 * tol_v
        assert _elementwise_ok(vr, vr_ref, el) and _elementwise_ok(vg, vg_ref, el)
        dropped = g.rho < 1e-10
        assert np.all(vr[dropped] == 0.0) and np.all(vg[dropped] == 0.0)


def test_noalloc_allocates_nothing(dev, systems):
    """After one warm-up call per precision (which may load the kernels), further calls
    leave the device's free memory and the torch allocator's counters unchanged."""
    g = systems[1][0]
    d = [_dev(x, dev) for x in (g.coords, g.weights, g.rho, g.grad_rho)]
    energy = torch.empty(1, dtype=torch.float64, device=dev)
    vrho = torch.empty(g.n, dtype=torch.float64, device=dev)
    vgamma = torch.empty_like(vrho)
    for prec, _, _ in PRECS:
        vv10.vv10_energy_potential_noalloc(*d, prec, energy, vrho, vgamma)
    torch.cuda.synchronize()
    before = (torch.cuda.mem_get_info(dev)[0], torch.cuda.memory_allocated(dev),
              torch.cuda.memory_reserved(dev))
    for _ in range(2):
        for prec, _, _ in PRECS:
            vv10.vv10_energy_potential_noalloc(*d, prec, energy, vrho, vgamma)
    torch.cuda.synchronize()
    after = (torch.cuda.mem_get_info(dev)[0], torch.cuda.memory_allocated(dev),
             torch.cuda.memory_reserved(dev))
    assert after == before


def test_noalloc_nonfinite_input_gives_nan(dev, systems):
    """A device-side failure cannot be returned by this entry point: a non-finite input
    makes it write NaN to the energy and every potential value; the next call is clean."""
    g = systems[0][0]
    w = g.weights.copy()
    w[7] = np.nan
    d = [_dev(x, dev) for x in (g.coords, w, g.rho, g.grad_rho)]
    e, vr, vg = _call(g, vv10.VV10_MIXED_TF32X3, dev, d)
    assert np.isnan(e) and np.all(np.isnan(vr)) and np.all(np.isnan(vg))
    e2, _, _ = _call(g, vv10.VV10_MIXED_TF32X3, dev)
    assert abs(e2 - systems[0][1]) <= 1e-7


def test_noalloc_rejects_too_many_points(dev):
    n = vv10.VV10_NOALLOC_MAX_POINTS + 1
    z = torch.zeros(n, dtype=torch.float64, device=dev)
    z3 = torch.zeros(n, 3, dtype=torch.float64, device=dev)
    e = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(vv10.VV10Error) as ei:
        vv10.vv10_energy_potential_noalloc(z3, z, z, z3, vv10.VV10_FP64, e)
    assert ei.value.status == vv10.VV10_ERR_UNSUPPORTED
