"""The operand splits of the tensor-core contraction, modelled on the CPU (no GPU): the pair
part of Eq. frhot (Sec. II.B) as kernel tiles times the trial matrix, with the operands
rounded as the kernels round them, against the same product in FP64.

  split TF32: hi = TF32(x) (round to nearest), lo = TF32(x - hi) (truncated, as the tensor
              core reads FP32 operands); products hi*hi + hi*lo + lo*hi;
  split FP16: trials scaled per column by a power of two s_t (the column's largest |u'|,
              |c_y y'| into [2^14, 2^15)), y by one global power of two c_y; kernel tiles
              scaled per row and 32-j stage by a power of two (the stage's largest |T| of the
              row into [2^14, 2^15)); hi = FP16(x), lo = FP16(x - hi); the same three
              products, each stage unscaled before it is summed.

Both must carry the product to well inside the mixed path's 1e-6 relative Frobenius
tolerance (the FP32 accumulation of the kernels is not modelled), and the FP16 split must
not be worse than the TF32 one by more than a small factor.  A mistake in the scaling (a
factor not undone, a range overflow, a flushed column) shows up as an error of order 1.
"""
import numpy as np
import pytest

from paper_2208_14639_gb300 import synth


def tf32_rn(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    return ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32).astype(np.float64)


def tf32_trunc(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    return (b & np.uint32(0xFFFFE000)).view(np.float32).astype(np.float64)


def split_tf32(x):
    x32 = np.asarray(x, dtype=np.float32)
    h = tf32_rn(x32)
    return h, tf32_trunc(x32.astype(np.float64) - h)


def split_f16(x):
    x32 = np.asarray(x, dtype=np.float32)
    h = x32.astype(np.float16)
    lo = (x32 - h.astype(np.float32)).astype(np.float16)
    return h.astype(np.float64), lo.astype(np.float64)


def pow2_into_range(m):
    """2^(14 - floor(log2 m)) (1 where m = 0): maps m into [2^14, 2^15)."""
    e = np.floor(np.log2(np.where(m > 0, m, 1.0)))
    return np.where(m > 0, 2.0 ** (14 - e), 1.0)


def tiles_and_trials(g, oracle_mod):
    """Kernel tiles T1..T4 (the pair part of f^rho rho, f^rho gamma, f^gamma rho, f^gamma
    gamma, divided by sigma where the paper multiplies by it) and u' = -3/2 w rho^t,
    y' = 3/2 sigma 2 w grad rho . grad rho^t, at the kept points."""
    rt, gt = synth.trial_densities(g.molecule, g.coords)
    keep = g.rho >= 1e-10
    x, w, rho, grad = g.coords[keep], g.weights[keep], g.rho[keep], g.grad_rho[keep]
    pp = oracle_mod.point_props(rho, grad)
    om, ka = pp["omega"], pp["kappa"]
    p, q, sig = rho * pp["kappa_rho"], rho * pp["omega_rho"], rho * pp["omega_gamma"]
    u = -1.5 * w[None] * rt[:, keep]
    y = 1.5 * sig[None] * 2 * w[None] * np.einsum("pnc,nc->pn", gt[:, keep], grad)
    d = x[:, None, :] - x[None, :, :]
    R2 = (d * d).sum(-1)
    gi, gj = om[:, None] * R2 + ka[:, None], om[None] * R2 + ka[None]
    s = gi + gj
    inv = 1.0 / (gi * gj * s)
    L, Gi, Gj = 1.0 / s, 1.0 / gi, 1.0 / gj
    M = 2.0 * (L * L + Gi * Gj)
    nAi, nAj = -(p[:, None] + q[:, None] * R2), -(p[None] + q[None] * R2)
    rp = R2 * inv
    T = [inv * (1 + nAi * (L + Gi) + nAj * (L + Gj) + nAi * nAj * M), rp * (nAi * M + L + Gj),
         rp * (nAj * M + L + Gi), rp * R2 * M]
    return T, u, y


def contract_f16(Ta, Tb, u, y, J=32, undo_row=True, undo_col=True, fold_cy=True):
    """The split-FP16 product; the flags plant mistakes (a factor not undone)."""
    cy = 2.0 ** np.round(np.log2(np.abs(u).max() / np.abs(y).max()))
    s_t = pow2_into_range(np.maximum(np.abs(u).max(1), cy * np.abs(y).max(1)))
    uh, ul = split_f16(u * s_t[:, None])
    yh, yl = split_f16(cy * y * s_t[:, None])
    if fold_cy:
        Tb = Tb / cy
    out = np.zeros((Ta.shape[0], u.shape[0]))
    for j0 in range(0, Ta.shape[1], J):
        a, b = Ta[:, j0:j0 + J], Tb[:, j0:j0 + J]
        r = pow2_into_range(np.maximum(np.abs(a).max(1), np.abs(b).max(1)))
        ah, al = split_f16(a * r[:, None])
        bh, bl = split_f16(b * r[:, None])
        sl = slice(j0, j0 + J)
        st = (ah @ uh[:, sl].T + ah @ ul[:, sl].T + al @ uh[:, sl].T +
              bh @ yh[:, sl].T + bh @ yl[:, sl].T + bl @ yh[:, sl].T)
        assert np.all(np.abs(np.concatenate([ah, bh])) <= 32768.0)  # rounded, well inside FP16
        out += st / r[:, None] if undo_row else st
    return out / s_t[None, :] if undo_col else out


def contract_tf32(Ta, Tb, u, y):
    ah, al = split_tf32(Ta)
    bh, bl = split_tf32(Tb)
    uh, ul = split_tf32(u)
    yh, yl = split_tf32(y)
    return ah @ uh.T + ah @ ul.T + al @ uh.T + bh @ yh.T + bh @ yl.T + bl @ yh.T


@pytest.mark.parametrize("case", ["water_small", "chon4"])
def test_fp16_split_as_accurate_as_tf32(oracle_mod, case):
    if case == "water_small":
        g = synth.config_water(n_rad=16, n_ang=38)
    else:
        g = synth.make_system(synth.random_chon(np.random.default_rng(7), 4), 12, 38)
    T, u, y = tiles_and_trials(g, oracle_mod)
    for Ta, Tb in ((T[0], T[1]), (T[2], T[3])):
        exact = Ta @ u.T + Tb @ y.T
        nrm = np.linalg.norm(exact)
        e16 = np.linalg.norm(contract_f16(Ta, Tb, u, y) - exact) / nrm
        e32 = np.linalg.norm(contract_tf32(Ta, Tb, u, y) - exact) / nrm
        assert e16 <= 2e-7 and e32 <= 2e-7, (e16, e32)
        assert e16 <= 3.0 * e32 + 1e-9, (e16, e32)


def test_scaling_mistakes_are_caught(oracle_mod):
    """Each factor left in place (the row-and-stage factor, the column factor, the y
    balance) moves the modelled product by far more than the tolerance the test above
    applies."""
    g = synth.config_water(n_rad=10, n_ang=26)
    T, u, y = tiles_and_trials(g, oracle_mod)
    Ta, Tb = T[0], T[1]
    exact = Ta @ u.T + Tb @ y.T
    nrm = np.linalg.norm(exact)
    err = lambda **kw: np.linalg.norm(contract_f16(Ta, Tb, u, y, **kw) - exact) / nrm
    assert err() <= 2e-7
    assert np.abs(np.log2(np.abs(u).max() / np.abs(y).max())) > 1  # c_y is not 1 here
    for planted in (dict(undo_row=False), dict(undo_col=False), dict(fold_cy=False)):
        assert err(**planted) > 1e-2, planted
