"""Two handles used at the same time on two CUDA streams (one handle per stream or thread,
as the header prescribes) give the same results as one handle used alone, and argument
errors of the newer entry points leave the handle usable."""
import threading

import numpy as np
import pytest
import torch

from paper_2208_14639_gb300 import synth, vv10

pytestmark = pytest.mark.gpu

MIXED = vv10.VV10_MIXED_TF32X3


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    vv10.load(build_if_missing=True)
    return torch.device("cuda", 0)


def T(a, dev, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)


def run(g, rt, gt, dev, stream=None):
    eng = vv10.VV10(0)
    s = stream if stream is not None else torch.cuda.current_stream()
    with torch.cuda.stream(s):
        eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                    T(g.atom_of_point, dev, torch.int32), g.molecule.n_atom, stream=s)
        f64 = dict(dtype=torch.float64, device=dev)
        out = dict(vrho=torch.empty(g.n, **f64), f_rho_t=torch.empty(rt.shape, **f64),
                   f_gamma_t=torch.empty(rt.shape, **f64), grad_points=torch.empty(g.n, 3, **f64))
        e = vv10.vv10_evaluate(eng.h, MIXED, T(rt, dev), T(gt, dev), stream=s, **out)
        s.synchronize()
    res = [e] + [t.cpu().numpy() for t in out.values()]
    eng.close()
    return res


def test_two_handles_on_two_streams_concurrently(dev):
    gs = [synth.random_points(3000, seed=201, n_atom=3), synth.random_points(2500, seed=202, n_atom=2)]
    trials = []
    for k, g in enumerate(gs):
        rng = np.random.default_rng(k)
        trials.append((rng.normal(size=(7, g.n)) * g.rho, rng.normal(size=(7, g.n, 3)) * np.abs(g.grad_rho)))
    alone = [run(g, rt, gt, dev) for g, (rt, gt) in zip(gs, trials)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    together = [None, None]

    def worker(k):
        together[k] = run(gs[k], *trials[k], dev, streams[k])

    th = [threading.Thread(target=worker, args=(k,)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for a, b in zip(alone, together):
        assert a[0] == b[0]  # same kernels, same order: identical results
        for x, y in zip(a[1:], b[1:]):
            assert np.array_equal(x, y)


def test_argument_errors_leave_the_handle_usable(dev):
    g = synth.random_points(400, seed=203, n_atom=2)
    eng = vv10.VV10(0)
    eng.prepare(T(g.coords, dev), T(g.weights, dev), T(g.rho, dev), T(g.grad_rho, dev),
                T(g.atom_of_point, dev, torch.int32), g.molecule.n_atom)
    rt = torch.zeros(2, g.n, dtype=torch.float64, device=dev)
    gt = torch.zeros(2, g.n, 3, dtype=torch.float64, device=dev)
    fr = torch.empty(2, g.n, dtype=torch.float64, device=dev)
    fg = torch.empty_like(fr)
    with pytest.raises(vv10.VV10Error) as ei:  # BF16x3 Hessian contraction
        vv10.vv10_evaluate(eng.h, vv10.VV10_MIXED_BF16X3, rt, gt, fr, fg)
    assert ei.value.status == vv10.VV10_ERR_UNSUPPORTED
    with pytest.raises(vv10.VV10Error):  # unknown precision
        vv10.vv10_evaluate(eng.h, 7, rt, gt, fr, fg)
    with pytest.raises(vv10.VV10Error):  # unknown option flag
        vv10.vv10_set_options(eng.h, 64)
    with pytest.raises(vv10.VV10Error):  # unknown tuning flag
        vv10.vv10_set_autotune(eng.h, 64)
    e = vv10.vv10_evaluate(eng.h, MIXED, rt, gt, fr, fg)
    assert np.isfinite(e)
    assert not fr.any() and not fg.any()  # zero trials give zero contractions
    eng.close()
