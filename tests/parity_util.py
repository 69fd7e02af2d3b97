"""Comparison helpers of the GPU parity tests.

Every check bounds both the whole-output error and every element:
    ||a - ref||_2 <= tol * ||ref||_2                    (relative L2 / Frobenius)
    |a_i - ref_i| <= el_tol * (|ref_i| + rms(ref))      for every element i
with el_tol = tol for FP64 results and el_tol = 10 tol for the mixed path (the worst
elements measured on the small systems reach 3.1e-6 of |ref_i| + rms there, against
relative L2 errors of 2e-7 to 9e-7: rows where the pair part and the delta_ij/w_i terms
nearly cancel keep the FP32 pair sums' absolute error).  The second bound keeps a wrong
value at a few points (e.g. low-density tail points, where the FP32 pair arithmetic is most
fragile) from hiding in a norm over 10^5 elements; rms(ref) is the scale below which an
element counts as zero.  The assertion message reports the relative L2 error, the largest
absolute error and the worst element's ratio to its bound.
"""

MIXED_EL_FACTOR = 10.0
import numpy as np


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def errors(a, ref):
    """(relative L2 error, max |a - ref|, max over i of |a_i - ref_i| / (|ref_i| + rms))."""
    a = np.asarray(a, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    d = np.abs(a - ref)
    s = float(np.sqrt(np.mean(ref * ref))) if ref.size else 0.0
    den = np.abs(ref) + s
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(den > 0, d / np.where(den > 0, den, 1.0), np.where(d > 0, np.inf, 0.0))
    return rel(a, ref), float(d.max()) if d.size else 0.0, float(ratio.max()) if ratio.size else 0.0


def check(a, ref, tol, el_tol=None, what=""):
    """tol <= 1e-8 is an FP64 tolerance (el_tol = tol), larger ones mixed (el_tol = 10 tol)."""
    if el_tol is None:
        el_tol = tol if tol <= 1e-8 else MIXED_EL_FACTOR * tol
    r, mx, worst = errors(a, ref)
    assert np.all(np.isfinite(np.asarray(a))), f"{what}: non-finite values"
    assert r <= tol and worst <= el_tol, (
        f"{what}: rel L2 {r:.3e} (tol {tol:.0e}), max abs {mx:.3e}, "
        f"worst element {worst:.3e} of |ref_i| + rms (tol {el_tol:.0e})")
    return r, mx
