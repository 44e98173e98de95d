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


# ---------------------------------------------------------------------------
# windows of a large problem: oracle parity at sizes the oracle cannot step whole
# ---------------------------------------------------------------------------

# Cells whose value after one IMEX-SSP2 step can depend on a given cell: per stage the
# face states reach two cells (MC), the edge EMFs one more across, the cell-centred B
# and the Gauss-law charge one more (radius 3); two stages make 6 per step.
RADIUS_PER_STEP = 6


def window(pr, start, size):
    """The sub-problem of ``pr`` made of the interior cells ``start[d] ..
    start[d] + size[d] - 1`` (with the two ghost layers around them cut from the same
    padded arrays).  Its boundaries are outflow; where a window side lies on the
    problem's own boundary, that boundary must be outflow too.  The window keeps the
    problem's cell widths exactly (``dx``), whatever the rounding of its ``lo``/``hi``."""
    import dataclasses
    from paper_2110_03732_gb300.problems import Problem

    @dataclasses.dataclass
    class Window(Problem):
        dx_fixed: list = None

        @property
        def dx(self):
            return list(self.dx_fixed)

    ng = pr.ng
    sl = tuple(slice(start[d], start[d] + size[d] + 2 * ng[d]) for d in (2, 1, 0))

    def crop(a):
        return None if a is None else np.ascontiguousarray(np.asarray(a)[sl])

    dx = pr.dx
    for d in range(pr.ndim):
        assert 0 <= start[d] and start[d] + size[d] <= pr.n[d], "window outside the problem"
        if pr.bc[d] != "outflow":
            assert 0 < start[d] and start[d] + size[d] < pr.n[d], \
                "a window may touch the problem's boundary only where that boundary is outflow"
    kw = {f.name: getattr(pr, f.name) for f in dataclasses.fields(pr)}
    kw.update(n=list(size), lo=[pr.lo[d] + start[d] * dx[d] for d in range(3)],
              hi=[pr.lo[d] + (start[d] + size[d]) * dx[d] for d in range(3)],
              bc=["outflow" if d < pr.ndim else pr.bc[d] for d in range(3)],
              prim=[crop(p) for p in pr.prim],
              bface=None if pr.bface is None else [crop(b) for b in pr.bface],
              A_edge=None if pr.A_edge is None else [crop(a) for a in pr.A_edge],
              alpha=crop(pr.alpha), psi=crop(pr.psi), eta=crop(pr.eta), dx_fixed=list(dx))
    return Window(**kw)


def window_core(pr, start, size, nsteps):
    """Per direction the slice of the window's interior (window-local interior
    indices) that its own cut boundaries cannot reach within ``nsteps`` steps, and the
    same cells as problem interior indices.  A side on the problem's boundary needs no
    margin (the window has the same boundary there)."""
    m = RADIUS_PER_STEP * nsteps + 2
    loc, glob = [], []
    for d in range(3):
        if d >= pr.ndim:
            loc.append(slice(0, 1))
            glob.append(slice(0, 1))
            continue
        a = 0 if start[d] == 0 else m
        b = size[d] if start[d] + size[d] == pr.n[d] else size[d] - m
        assert b > a, "window too small for its margin"
        loc.append(slice(a, b))
        glob.append(slice(start[d] + a, start[d] + b))
    return loc, glob


def padded(sl, ng):
    """Interior-index slices (x, y, z order) as a padded (z, y, x) index tuple."""
    return tuple(slice(sl[d].start + ng[d], sl[d].stop + ng[d]) for d in (2, 1, 0))
