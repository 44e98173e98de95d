"""Elliptic divergence cleaning (arXiv 2110.03732 Sec. 3.3) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline leg may use
this module.  It shares no code with the CUDA path.

The cleaning solves the Poisson equation  lap(Phi) = div(q_B)  and replaces
q_B  by  q_B - grad(Phi)  (Sec. 3.3, Eqs. poisson and update_bfield; the reference
metric is Cartesian, so the operators are the flat ones).  The paper solves it by
multigrid; the oracle instead takes its plain definition: the exact solution of the
assembled discrete linear system, by a sparse direct solve (scipy), with every
operator written out below.

Discretisation (a reading; the paper gives none):
  * staggered fields (faces, the CT layout): div on cells from face differences,
    grad on faces from the two adjacent cells, so lap = div(grad) is the compact
    (2 ndim + 1)-point Laplacian and the cleaned field is divergence-free to the
    round-off of the solve;
  * cell-centred fields (the GLM layout): div and grad by central differences, lap
    the same compact Laplacian, so the projection is approximate (the difference
    between the wide and the compact Laplacian is left over);
  * boundaries: periodic directions wrap; in the others Phi has zero normal gradient
    (no flux through the boundary face, which is therefore not corrected).  The
    system is then singular with constant null space: the right-hand side is made
    mean-free, one cell is pinned, and Phi is returned mean-free.  With zero-gradient
    boundaries the mean divergence (the net flux through the kept boundary faces)
    therefore stays; with periodic ones it is zero.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _interior(grid):
    return grid.interior()


def _cell_index(grid):
    n = grid.n
    return np.arange(n[0] * n[1] * n[2]).reshape(n[2], n[1], n[0])


def laplacian(grid):
    """Compact Laplacian over the interior cells (x fastest), with the boundary rules
    above, as a sparse matrix."""
    n, dx = grid.n, grid.dx
    idx = _cell_index(grid)
    N = idx.size
    rows, cols, vals = [], [], []
    for d in range(grid.ndim):
        ax = 2 - d
        h2 = 1.0 / dx[d] ** 2
        for s in (-1, 1):
            nb = np.roll(idx, -s, axis=ax)           # neighbour index in direction s
            valid = np.ones(idx.shape, dtype=bool)
            if grid.bc[d] != 0:                        # not periodic: no neighbour past the boundary
                sl = [slice(None)] * 3
                sl[ax] = -1 if s == 1 else 0
                valid[tuple(sl)] = False
            r = idx[valid]
            rows += [r, r]
            cols += [nb[valid], r]
            vals += [np.full(r.size, h2), np.full(r.size, -h2)]
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def solve_poisson(grid, rhs):
    """Mean-free Phi with lap(Phi) = rhs - mean(rhs) (interior arrays, shape (n2, n1, n0))."""
    L = laplacian(grid).tolil()
    b = (rhs - rhs.mean()).ravel()
    # pin the first cell (the null space is the constants)
    L[0, :] = 0.0
    L[0, 0] = 1.0
    b = b.copy()
    b[0] = 0.0
    phi = spla.spsolve(L.tocsc(), b).reshape(rhs.shape)
    return phi - phi.mean()


def _pad_phi(grid, phi):
    """Phi on the padded grid with one layer of ghosts by the boundary rule (wrap or
    copy = zero normal gradient)."""
    pads = [(1, 1) if grid.ndim > d else (0, 0) for d in (2, 1, 0)]
    out = phi
    for d in range(grid.ndim):
        ax = 2 - d
        pw = [(0, 0)] * 3
        pw[ax] = (1, 1)
        out = np.pad(out, pw, mode="wrap" if grid.bc[d] == 0 else "edge")
    return out, pads


def div_faces(grid, bf):
    """Cell divergence of staggered q_B over the interior (face differences)."""
    I = _interior(grid)
    out = np.zeros(tuple(grid.n[d] for d in (2, 1, 0)))
    for d in range(grid.ndim):
        up = [slice(s.start, s.stop) for s in I]
        ax = 2 - d
        up[ax] = slice(I[ax].start + 1, I[ax].stop + 1)
        hi = bf[d][tuple(up)].copy()
        if grid.bc[d] == 0:
            # periodic: the upper face of the last cell is the lower face of the first
            first = [slice(s.start, s.stop) for s in I]
            first[ax] = slice(I[ax].start, I[ax].start + 1)
            last = [slice(None)] * 3
            last[ax] = slice(-1, None)
            hi[tuple(last)] = bf[d][tuple(first)]
        out += (hi - bf[d][I]) / grid.dx[d]
    return out


def div_central(grid, qB):
    """Cell divergence of cell-centred q_B by central differences (ghosts by the
    boundary rule of the solver's grid: wrap or copy)."""
    I = _interior(grid)
    out = np.zeros(tuple(grid.n[d] for d in (2, 1, 0)))
    for d in range(grid.ndim):
        ax = 2 - d
        a = qB[d][I]
        pw = [(0, 0)] * 3
        pw[ax] = (1, 1)
        ap = np.pad(a, pw, mode="wrap" if grid.bc[d] == 0 else "edge")
        sl_p = [slice(None)] * 3
        sl_m = [slice(None)] * 3
        sl_p[ax] = slice(2, None)
        sl_m[ax] = slice(0, -2)
        out += (ap[tuple(sl_p)] - ap[tuple(sl_m)]) / (2.0 * grid.dx[d])
    return out


def clean_faces(grid, bf):
    """Staggered cleaning: returns (cleaned face arrays, Phi).  Faces between two
    interior cells (and the wrapped lower face of a periodic direction) get
    q_B -= (Phi_c - Phi_{c-1})/dx; boundary faces of other directions are kept."""
    phi = solve_poisson(grid, div_faces(grid, bf))
    pp, _ = _pad_phi(grid, phi)
    out = [b.copy() for b in bf]
    I = _interior(grid)
    for d in range(grid.ndim):
        ax = 2 - d
        # interior-shaped view of Phi and of its lower neighbour along d
        c = [slice(1, -1) if grid.ndim > e else slice(None) for e in (2, 1, 0)]
        m = list(c)
        m[ax] = slice(0, -2)
        grad = (pp[tuple(c)] - pp[tuple(m)]) / grid.dx[d]
        if grid.bc[d] != 0:
            sl = [slice(None)] * 3
            sl[ax] = 0
            grad[tuple(sl)] = 0.0             # lower boundary face: no flux
        out[d][I] = bf[d][I] - grad
    return out, phi


def clean_cells(grid, qB):
    """Cell-centred cleaning: q_B -= central grad(Phi) with Phi from the compact
    Laplacian and the central divergence.  Returns (cleaned arrays, Phi)."""
    phi = solve_poisson(grid, div_central(grid, qB))
    pp, _ = _pad_phi(grid, phi)
    out = [b.copy() for b in qB]
    I = _interior(grid)
    for d in range(grid.ndim):
        ax = 2 - d
        c = [slice(1, -1) if grid.ndim > e else slice(None) for e in (2, 1, 0)]
        p_ = list(c)
        m_ = list(c)
        p_[ax] = slice(2, None)
        m_[ax] = slice(0, -2)
        out[d][I] = qB[d][I] - (pp[tuple(p_)] - pp[tuple(m_)]) / (2.0 * grid.dx[d])
    return out, phi
