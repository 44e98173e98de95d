"""Tolerances of the FP64 parity tests (CUDA path against the oracle, same inputs).

Two bounds per variable and step:
- relative L1 over the compared cells <= 1e-10: the target for the FP64 path; the
  denominator has a floor of 1e-3 per cell for variables that are identically ~0;
- per element, max |a - b| <= 1e-8 of the variable's largest magnitude (same floor):
  a localised mistake that an L1 over ~10^5 cells would dilute below 1e-10 (a single
  wrong cell of relative size 1e-6, say) still fails it.  The Newton solves of both
  sides agree to ~1e-13 of the momentum scale, far inside it."""
import numpy as np

TOL_L1 = 1e-10
TOL_MAX = 1e-8


def rel_l1(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = max(np.abs(b).sum(), 1e-3 * b.size)
    return np.abs(a - b).sum() / den


def rel_max(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if b.size == 0:
        return 0.0
    den = max(np.abs(b).max(), 1e-3)
    return float(np.abs(a - b).max() / den)


def check(a, b, tag="", tol=TOL_L1, tol_max=TOL_MAX):
    """Assert both bounds; returns the relative L1."""
    r = rel_l1(a, b)
    m = rel_max(a, b)
    assert r <= tol, f"{tag}: relative L1 {r:.3e} > {tol:.0e}"
    assert m <= tol_max, f"{tag}: largest element error {m:.3e} of the field scale > {tol_max:.0e}"
    return r
