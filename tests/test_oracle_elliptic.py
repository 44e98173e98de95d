"""Pins of the oracle's elliptic divergence cleaning (Sec. 3.3): lap(Phi) = div q_B,
q_B -= grad(Phi).

* Staggered fields: the discrete Helmholtz decomposition is exact, so a field built
  as curl(A) + grad(chi) (operators written out here, independently of the oracle)
  is cleaned back to curl(A) to round-off, for periodic and for zero-gradient
  boundaries; a random field ends divergence-free; cleaning is idempotent; the
  removed part is orthogonal to every divergence-free field (periodic).
* Cell-centred fields: a central curl is left unchanged; for a smooth gradient part the
  left-over central divergence (wide minus compact Laplacian) falls at second order."""
import math

import numpy as np
import pytest

import oracle
from oracle import elliptic as E


def _grid(ndim, n, bc):
    dx = [0.7 / n[0], 0.5 / n[1] if ndim > 1 else 1.0, 0.9 / n[2] if ndim > 2 else 1.0][:3]
    return oracle.Grid(ndim, n, dx, [bc] * 3, 5.0 / 3.0)


def _periodic_pad(core, ndim):
    pads = [(2, 2) if ndim > d else (0, 0) for d in (2, 1, 0)]
    return np.pad(core, pads, mode="wrap")


def _edge_potential(g, rng, periodic):
    core_shape = tuple(g.n[d] for d in (2, 1, 0))
    A = []
    for _ in range(3):
        core = rng.normal(size=core_shape)
        A.append(np.ascontiguousarray(_periodic_pad(core, g.ndim) if periodic else
                                      rng.normal(size=g.shape)))
    return A


def _face_gradient(g, chi):
    """(chi_c - chi_{c-1})/dx on the lower face of every interior cell; across a
    non-periodic boundary the lower face of the first cell gets 0 (no flux)."""
    out = [np.zeros(g.shape) for _ in range(3)]
    I = g.interior()
    for d in range(g.ndim):
        ax = 2 - d
        lower = np.roll(chi, 1, axis=ax)
        gr = (chi - lower) / g.dx[d]
        if g.bc[d] != 0:
            sl = [slice(None)] * 3
            sl[ax] = 0
            gr[tuple(sl)] = 0.0
        out[d][I] = gr
    return out


@pytest.mark.parametrize("ndim,n,bc", [(1, [40], "periodic"), (2, [16, 12], "periodic"), (2, [14, 10], "outflow"),
                                       (3, [8, 6, 7], "periodic"), (3, [7, 6, 5], "outflow")])
def test_staggered_helmholtz_decomposition(ndim, n, bc):
    g = _grid(ndim, n, bc)
    rng = np.random.default_rng(11 + ndim)
    if ndim == 1:
        curl = [np.full(g.shape, 0.37), np.zeros(g.shape), np.zeros(g.shape)]   # 1-D: B^x constant
    else:
        curl = oracle.curl_A(g, _edge_potential(g, rng, bc == "periodic"))
    chi = rng.normal(size=tuple(g.n[d] for d in (2, 1, 0)))
    grad = _face_gradient(g, chi)
    bf = [c + gr for c, gr in zip(curl, grad)]
    clean, phi = E.clean_faces(g, bf)
    I = g.interior()
    for d in range(3):
        scale = max(np.abs(bf[d][I]).max(), 1e-300)
        np.testing.assert_allclose(clean[d][I], curl[d][I], rtol=0, atol=1e-11 * scale, err_msg=str(d))
    np.testing.assert_allclose(phi, chi - chi.mean(), rtol=0, atol=1e-11 * np.abs(chi).max())


@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_staggered_cleaning_is_a_projection(bc):
    g = _grid(3, [9, 8, 6], bc)
    rng = np.random.default_rng(5)
    bf = [rng.normal(size=g.shape) for _ in range(3)]
    div0 = E.div_faces(g, bf)
    d0 = np.abs(div0).max()
    c1, _ = E.clean_faces(g, bf)
    # what is left is the mean divergence, the net flux through the boundary faces
    # that zero-gradient boundaries keep (zero when periodic)
    left = E.div_faces(g, c1)
    assert np.abs(left - div0.mean()).max() < 1e-12 * d0
    if bc == "periodic":
        assert abs(div0.mean()) < 1e-13 * d0
    c2, phi2 = E.clean_faces(g, c1)
    I = g.interior()
    for d in range(3):
        np.testing.assert_allclose(c2[d][I], c1[d][I], rtol=0, atol=1e-12 * np.abs(bf[d]).max())
    if bc == "periodic":
        # the removed gradient is orthogonal to the divergence-free part (sum over faces)
        dot = sum(((bf[d] - c1[d])[I] * c1[d][I]).sum() for d in range(3))
        assert abs(dot) < 1e-10 * sum((c1[d][I] ** 2).sum() for d in range(3))


def test_cell_centred_cleaning():
    # a central curl of a cell potential is left alone
    g = _grid(2, [20, 16], "periodic")
    rng = np.random.default_rng(8)
    A = [np.ascontiguousarray(_periodic_pad(rng.normal(size=(1, 16, 20)), 2)) for _ in range(3)]
    qB = oracle.curl_A_cc(g, A)
    c, phi = E.clean_cells(g, qB)
    I = g.interior()
    assert np.abs(phi).max() < 1e-12 * max(np.abs(qB[0][I]).max(), 1.0)
    # a smooth gradient part is removed up to the wide-minus-compact Laplacian, O(h^2)
    res = []
    for n in (32, 64):
        g = oracle.Grid(2, [n, n], [2 * math.pi / n] * 2, ["periodic"] * 2, 5.0 / 3.0)
        x = (np.arange(n) + 0.5) * 2 * math.pi / n
        X, Y = np.meshgrid(x, x, indexing="xy")
        qB = [np.zeros(g.shape) for _ in range(3)]
        qB[0][g.interior()] = (np.cos(X) * np.sin(2 * Y))[None]        # grad of sin x sin 2y
        qB[1][g.interior()] = (2 * np.sin(X) * np.cos(2 * Y))[None]
        d0 = np.abs(E.div_central(g, qB)).max()
        c, _ = E.clean_cells(g, qB)
        res.append(np.abs(E.div_central(g, c)).max() / d0)
    assert res[0] < 0.05 and res[1] < 0.3 * res[0], res
