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


# ------------------------------------------------------------ FP64 accuracy from integer slices
#
# The FP64 tensor-core contraction: kernel tiles as FP32 pairs (hi, lo) cut into seven 8-bit
# integer slices in FP32 arithmetic, trials cut into seven slices in FP64; per 16-j stage one
# factor per tile row and one per trial column (powers of two into [2^6, 2^7)); the 28
# products with p + q <= 6 summed per level.

F32 = np.float32


def two_sum32(a, b):
    s = (a + b).astype(F32)
    bp = (s - a).astype(F32)
    return s, ((a - (s - bp)).astype(F32) + (b - bp).astype(F32)).astype(F32)


def tile_slices7(hi, lo, carry=True):
    """Seven slices of x = hi + lo (|x| < 2^7) in FP32: three from hi, whose remainder joins lo
    in an error-free sum w + e (dropped with carry=False), three from w, the last from what is
    left and e."""
    hi, lo = np.asarray(hi, F32), np.asarray(lo, F32)
    s0 = np.rint(hi)
    r0 = (hi - s0) * F32(256)
    s1 = np.rint(r0)
    r1 = (r0 - s1) * F32(256)
    s2 = np.rint(r1)
    w, e = two_sum32(((r1 - s2) * F32(2.0 ** -16)).astype(F32) if carry else np.zeros_like(lo), lo)
    u3 = (w * F32(2.0 ** 24)).astype(F32)
    s3 = np.rint(u3)
    u4 = ((u3 - s3) * F32(256)).astype(F32)
    s4 = np.rint(u4)
    u5 = ((u4 - s4) * F32(256)).astype(F32)
    s5 = np.rint(u5)
    s6 = np.rint((e.astype(np.float64) * 2.0 ** 48 + (u5 - s5).astype(np.float64) * 256).astype(F32))
    return [s.astype(np.float64) for s in (s0, s1, s2, s3, s4, s5, s6)]


def pair32(x):
    hi = np.asarray(x).astype(F32)
    return hi, (np.asarray(x) - hi.astype(np.float64)).astype(F32)


def trial_slices7(x):
    out, r = [], np.asarray(x, dtype=np.float64).copy()
    for _ in range(7):
        s = np.rint(r)
        out.append(s)
        r = (r - s) * 256.0
    return out


def pow2_into(m, lo_exp):
    e = np.floor(np.log2(np.where(m > 0, m, 1.0)))
    return np.where(m > 0, 2.0 ** (lo_exp - e), 1.0)


def contract_o64(Ta, Tb, u, y, J=16, levels=7, carry=True, weight=8, col_per_stage=True):
    """The seven-slice product over 16-j stages; level sums asserted to be integers below 2^23
    (exact in the tensor cores' FP32 accumulation; the bound is 7 x 32 x 2^14.6 = 2^22.4).  The
    flags plant mistakes."""
    cy = 2.0 ** np.round(np.log2(np.abs(u).max() / np.abs(y).max()))
    Tb = Tb / cy
    s_all = pow2_into(np.maximum(np.abs(u).max(1), cy * np.abs(y).max(1)), 6)
    out = np.zeros((Ta.shape[0], u.shape[0]))
    for j0 in range(0, Ta.shape[1], J):
        sl = slice(j0, j0 + J)
        a, b, us, ys = Ta[:, sl], Tb[:, sl], u[:, sl], cy * y[:, sl]
        s_t = pow2_into(np.maximum(np.abs(us).max(1), np.abs(ys).max(1)), 6) if col_per_stage \
            else s_all
        U, Y = trial_slices7(us * s_t[:, None]), trial_slices7(ys * s_t[:, None])
        r = pow2_into(np.maximum(np.abs(a).max(1), np.abs(b).max(1)), 6)
        A = tile_slices7(*pair32(a * r[:, None]), carry=carry)
        B = tile_slices7(*pair32(b * r[:, None]), carry=carry)
        st = np.zeros_like(out)
        for lev in range(levels):
            L = sum(A[p] @ U[lev - p].T + B[p] @ Y[lev - p].T for p in range(lev + 1))
            assert np.all(L == np.rint(L)) and np.abs(L).max() < 2.0 ** 23
            st += L * 2.0 ** (-weight * lev)
        out += st / r[:, None] / s_t[None, :]
    return out


def test_seven_slices_reconstruct():
    """Tile slices are integers of at most 8 bits (|s3|, |s6| <= 192), exact in FP16, and
    rebuild the FP32 pair hi + lo to within 2^-49 for |x| < 2^7 across the whole range (the
    pair itself carries x to 2^-48 relative); trial slices rebuild an FP64 value to within
    2^-49, exactly when all its bits lie above 2^-48 (|x| >= 2^4)."""
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-128, 128, 20000),
                        rng.uniform(-1, 1, 20000) * 10.0 ** rng.uniform(-15, 2, 20000),
                        [0.0, 127.99999999, -127.99999999, 2.0 ** -20, 3.0 ** -15]])
    hi, lo = pair32(x)
    s = tile_slices7(hi, lo)
    for k, sk in enumerate(s):
        assert np.all(sk == np.rint(sk)) and np.all(np.abs(sk) <= (192 if k in (3, 6) else 128))
        assert np.all(sk.astype(np.float16).astype(np.float64) == sk)
    pair = hi.astype(np.float64) + lo.astype(np.float64)
    assert np.abs(sum(sk * 2.0 ** (-8 * k) for k, sk in enumerate(s)) - pair).max() <= 2.0 ** -49
    t = trial_slices7(x)
    assert all(np.abs(tk).max() <= 128 for tk in t)
    rebuilt = sum(tk * 2.0 ** (-8 * k) for k, tk in enumerate(t))
    assert np.abs(rebuilt - x).max() <= 2.0 ** -49
    big = np.abs(x) >= 16.0  # all 53 bits above 2^-48: exact
    assert np.array_equal(rebuilt[big], x[big])
    # without the third slice's remainder carried into the low half, the bits of hi between
    # 2^-16 and 2^-24 of the scale are lost
    s_nc = tile_slices7(hi, lo, carry=False)
    assert np.abs(sum(sk * 2.0 ** (-8 * k) for k, sk in enumerate(s_nc)) - pair).max() > 2.0 ** -25


SLICE_CASES = [("water_small", lambda: synth.config_water(n_rad=16, n_ang=38)),
               ("chon4", lambda: synth.make_system(synth.random_chon(np.random.default_rng(7), 4), 12, 38)),
               ("rand255", lambda: synth.random_points(255, seed=4, n_atom=3))]


@pytest.mark.parametrize("case,make", SLICE_CASES, ids=[c[0] for c in SLICE_CASES])
def test_seven_slice_product_fp64_accuracy(oracle_mod, case, make):
    """Relative Frobenius error <= 1e-12 and every element within 1e-11 (|ref| + rms): inside
    the 1e-10 bound the GPU parity tests apply to the FP64 paths.  Random points (no shell
    structure) give the largest ranges inside a stage."""
    T, u, y = tiles_and_trials(make(), oracle_mod)
    for Ta, Tb in ((T[0], T[1]), (T[2], T[3])):
        exact = Ta @ u.T + Tb @ y.T
        nrm = np.linalg.norm(exact)
        got = contract_o64(Ta, Tb, u, y)
        assert np.linalg.norm(got - exact) / nrm <= 1e-12
        assert np.all(np.abs(got - exact) <= 1e-11 * (np.abs(exact) + np.sqrt(np.mean(exact ** 2))))


def test_seven_slice_mistakes_are_caught(oracle_mod):
    """A dropped level, the remainder carry left out or a wrong level weight each move the
    product well past the bounds above; one column factor for all of j (instead of one per
    stage) at least doubles the error."""
    T, u, y = tiles_and_trials(synth.random_points(255, seed=4, n_atom=3), oracle_mod)
    Ta, Tb = T[2], T[3]
    exact = Ta @ u.T + Tb @ y.T
    nrm = np.linalg.norm(exact)
    err = lambda **kw: np.linalg.norm(contract_o64(Ta, Tb, u, y, **kw) - exact) / nrm
    base = err()
    assert base <= 1e-12
    assert err(levels=6) > 1e-11
    assert err(carry=False) > 1e-11
    assert err(weight=7) > 1e-3
    assert err(col_per_stage=False) > 2 * base
