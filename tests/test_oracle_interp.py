"""Pins of the oracle's interpolation over mesh elements (Section 3.5) and
of the staggered-mesh effect (Section 4.3).  No GPU needed.

* Koornwinder polynomials (Section 2.1) are orthonormal on the standard
  simplex: Gram matrix = I under a collapsed Gauss rule exact for the degree.
* The interpolation nodes: dim P_N of them (Table "ord_len_interp"), inside
  the simplex, invariant under the simplex's symmetries, unisolvent with a
  stated condition number.
* Interpolation reproduces polynomials of degree <= N to rounding, on
  straight elements, at points located anywhere in the mesh.
* Staggering the interpolation mesh against the quadrature mesh lowers the
  sub-triangles (s_n) and self panels (s_l) per target, the trends of Tables
  "near_corr" and "self_stag".
"""
import numpy as np
import pytest

from oracle.interp import Interpolator, dim_p, interp_nodes, koornwinder
from oracle.oracle import Oracle
from paper_2205_04401_gb300 import inputs


def collapsed_gauss(n):
    g, w = np.polynomial.legendre.leggauss(n)
    u, wu = 0.5 * (g + 1), 0.5 * w
    U, V = np.meshgrid(u, u, indexing="ij")
    WU, WV = np.meshgrid(wu, wu, indexing="ij")
    return U.ravel(), ((1 - U) * V).ravel(), (WU * WV * (1 - U)).ravel()


@pytest.mark.parametrize("N", [1, 4, 12, 20])
def test_koornwinder_orthonormal(N):
    x, y, w = collapsed_gauss(N + 2)
    K = koornwinder(N, x, y)
    G = (K * w[:, None]).T @ K
    assert np.abs(G - np.eye(dim_p(N))).max() <= 1e-12


def test_koornwinder_first_members():
    """K_00 = sqrt(2), K_01 = 2 sqrt(3)... written out from the definition at
    random points: n = 1 gives c_01 P_1^{(1,0)}(2x-1) = 2 (3x - 1) and
    c_11 (2y + x - 1) = 2 sqrt(3) (2y + x - 1)."""
    rng = np.random.default_rng(1)
    x, y = rng.random(50) * 0.5, rng.random(50) * 0.5
    K = koornwinder(1, x, y)
    assert np.allclose(K[:, 0], np.sqrt(2.0), rtol=0, atol=1e-15)
    assert np.allclose(K[:, 1], 2.0 * (3.0 * x - 1.0), rtol=0, atol=1e-14)
    assert np.allclose(K[:, 2], 2.0 * np.sqrt(3.0) * (2.0 * y + x - 1.0), rtol=0, atol=1e-14)


@pytest.mark.parametrize("N,kmax", [(12, 30.0), (20, 700.0)])
def test_interpolation_nodes(N, kmax):
    x, y = interp_nodes(N)
    assert len(x) == dim_p(N)
    assert min(x.min(), y.min(), (1 - x - y).min()) > 1e-3
    P = np.stack([x, y], 1)
    for Q in (np.stack([y, x], 1), np.stack([1 - x - y, x], 1), np.stack([y, 1 - x - y], 1)):
        d = np.linalg.norm(P[:, None, :] - Q[None, :, :], axis=2).min(axis=1)
        assert d.max() <= 1e-14
    assert np.linalg.cond(koornwinder(N, x, y)) <= kmax


@pytest.mark.parametrize("N", [4, 12])
def test_interpolation_reproduces_polynomials(tables, N):
    mesh = inputs.disk_mesh()
    it = Interpolator(Oracle("far16", tables=tables), mesh.vxy, mesh.tri, N)
    rng = np.random.default_rng(N)
    c = rng.normal(size=(N + 1, N + 1))

    def poly(p):
        out = np.zeros(len(p))
        for a in range(N + 1):
            for b in range(N + 1 - a):
                out += c[a, b] * p[:, 0] ** a * p[:, 1] ** b
        return out

    nodes = it.nodes()
    coef = it.coeffs(poly(nodes)[None, :])
    pts = inputs.random_interior_points(mesh, 500, 3)
    u, T = it.evaluate(coef, pts)
    assert (T >= 0).all()
    ref = poly(pts)
    assert np.abs(u[0] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_staggered_mesh_lowers_subdivisions(tables):
    """Curved unit disk (both meshes represent the circle exactly, so every
    interpolation node is inside the quadrature mesh), 256 triangles,
    19-node rule, N_s = 12: the sub-triangles and self panels per target
    fall when the interpolation mesh is staggered (Tables "near_corr" and
    "self_stag": s_n*/s_n+ 26-45%, s_l*/s_l0 86-88% in the paper)."""
    circ = [(0.0, 0.0, 1.0)]
    q = inputs.disk_mesh()
    tq, cq = inputs.curved_boundary(q, circ)
    st = inputs.disk_mesh(stagger=True)
    ts, cs = inputs.curved_boundary(st, circ)
    o = Oracle("far19", tables=tables)
    out = {}
    for name, (vxy, tri, cur) in (("same", (q.vxy, tq, cq)), ("staggered", (st.vxy, ts, cs))):
        nodes = Interpolator(o, vxy, tri, 12, curves=cur).nodes()
        s = o.setup(q.vxy, tq, node_targets=False, extra=nodes, curves=cq)
        assert (s["tself"] >= 0).all()
        _, info = o.potential(s, np.ones((1, s["N"])))
        near = info["pkind"] == 0
        M = len(nodes)
        out[name] = (info["stats"][near].sum() / M, info["stats"][~near].sum() / M)
    sn = out["staggered"][0] / out["same"][0]
    sl = out["staggered"][1] / out["same"][1]
    assert sn < 0.95 and sl < 0.95, (out, sn, sl)
