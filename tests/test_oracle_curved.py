"""Pins of the oracle's curved elements (blending map of Section 3.1).

With curved boundary elements the unit disk is represented exactly, so the
closed forms of Section 5.1 become tests at full accuracy:
    f = 1:    u(x) = (|x|^2 - 1) / 4
    f = r^2:  u(x) = (|x|^4 - 1) / 16
(u = -int_r^1 s^-1 int_0^s f(t) t dt ds for a radial density on the unit
disk, zero on the circle), the node weights sum to pi, and the curved
routines with a straight curve (D = 0) reproduce the straight ones.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2205_04401_gb300 import inputs


@pytest.fixture(scope="module")
def disk_curved():
    mesh = inputs.disk_mesh()
    tri, cur = inputs.curved_boundary(mesh, [(0.0, 0.0, 1.0)])
    return mesh, tri, cur


@pytest.mark.parametrize("rule", ["far16", "far19"])
def test_curved_disk_area_is_pi(tables, disk_curved, rule):
    mesh, tri, cur = disk_curved
    o = Oracle(rule, tables=tables)
    _, _, W, _ = o.nodes_curved(mesh.vxy, tri, cur)
    assert abs(W.sum() - math.pi) <= 1e-13
    assert (W > 0).all()


def test_blend_map_vertices_sides_and_jacobian(tables, disk_curved):
    mesh, tri, cur = disk_curved
    o = Oracle("far16", tables=tables)
    tri_ccw, _, _, _ = o.nodes_curved(mesh.vxy, tri, cur)
    curved = np.where(cur["cidx"] >= 0)[0]
    assert len(curved) == 32
    rng = np.random.default_rng(3)
    for T in curved[:8]:
        v = mesh.vxy[tri_ccw[T]]
        # vertices
        y, _ = o.map_curved(mesh.vxy, tri_ccw, cur, [T] * 3, [0.0, 1.0, 0.0], [0.0, 0.0, 1.0])
        assert np.abs(y - v).max() <= 1e-15
        # the curved side eta = 0 lies on the unit circle, the others on their chords
        t = rng.random(50)
        y0, _ = o.map_curved(mesh.vxy, tri_ccw, cur, [T] * 50, t, np.zeros(50))
        assert np.abs(np.hypot(y0[:, 0], y0[:, 1]) - 1.0).max() <= 1e-14
        y1, _ = o.map_curved(mesh.vxy, tri_ccw, cur, [T] * 50, t, 1.0 - t)
        y2, _ = o.map_curved(mesh.vxy, tri_ccw, cur, [T] * 50, np.zeros(50), t)
        for Y, P, Q in ((y1, v[1], v[2]), (y2, v[0], v[2])):
            cr = (Q[0] - P[0]) * (Y[:, 1] - P[1]) - (Q[1] - P[1]) * (Y[:, 0] - P[0])
            assert np.abs(cr).max() <= 1e-15
        # positive Jacobian determinant inside, matching a finite difference of the map
        a, b = rng.random(40), rng.random(40)
        keep = a + b < 1
        a, b = a[keep], b[keep]
        _, det = o.map_curved(mesh.vxy, tri_ccw, cur, [T] * len(a), a, b)
        assert (det > 0).all()
        h = 1e-6
        ya, _ = o.map_curved(mesh.vxy, tri_ccw, cur, [T] * len(a), a + h, b)
        yam, _ = o.map_curved(mesh.vxy, tri_ccw, cur, [T] * len(a), a - h, b)
        yb, _ = o.map_curved(mesh.vxy, tri_ccw, cur, [T] * len(a), a, b + h)
        ybm, _ = o.map_curved(mesh.vxy, tri_ccw, cur, [T] * len(a), a, b - h)
        da, db = (ya - yam) / (2 * h), (yb - ybm) / (2 * h)
        fd = da[:, 0] * db[:, 1] - da[:, 1] * db[:, 0]
        assert np.abs(fd - det).max() <= 1e-8 * np.abs(det).max()


def test_newton_preimage_round_trip(tables, disk_curved):
    mesh, tri, cur = disk_curved
    o = Oracle("far16", tables=tables)
    tri_ccw, _, _, _ = o.nodes_curved(mesh.vxy, tri, cur)
    curved = np.where(cur["cidx"] >= 0)[0]
    rng = np.random.default_rng(4)
    a, b = rng.random(200), rng.random(200)
    keep = a + b < 1
    T = rng.choice(curved, keep.sum())
    y, _ = o.map_curved(mesh.vxy, tri_ccw, cur, T, a[keep], b[keep])
    ref, it = o.inverse_curved(mesh.vxy, tri_ccw, cur, T, y)
    assert (it > 0).all()
    assert np.abs(ref[:, 0] - a[keep]).max() <= 1e-13 and np.abs(ref[:, 1] - b[keep]).max() <= 1e-13


def test_point_location_in_the_bulge(tables, disk_curved):
    """Points between the chord polygon and the circle belong to the curved
    element; points outside the circle to none."""
    mesh, tri, cur = disk_curved
    o = Oracle("far16", tables=tables)
    tri_ccw, _, _, _ = o.nodes_curved(mesh.vxy, tri, cur)
    th = np.linspace(0, 2 * np.pi, 2000, endpoint=False) + 0.001
    for gap in (1e-3, 1e-6, 1e-9):
        inside = np.stack([(1 - gap) * np.cos(th), (1 - gap) * np.sin(th)], 1)
        outside = np.stack([(1 + gap) * np.cos(th), (1 + gap) * np.sin(th)], 1)
        li = o.locate_curved(mesh.vxy, tri_ccw, cur, inside)
        lo = o.locate_curved(mesh.vxy, tri_ccw, cur, outside)
        assert (li >= 0).all() and (lo < 0).all()
    # away from the boundary the curved and straight locations agree
    p = inputs.random_interior_points(mesh, 300, 5)
    p = p[np.hypot(p[:, 0], p[:, 1]) < 0.8]
    assert np.array_equal(o.locate_curved(mesh.vxy, tri_ccw, cur, p), o.locate(mesh.vxy, tri_ccw, p))


def test_curved_routines_reduce_to_straight(tables):
    """A zero curve (D = 0) makes the blending map affine: identical nodes and
    near moments, self moments equal to rounding (reference-coordinate fans
    versus physical fans)."""
    mesh = inputs.disk_mesh()
    o = Oracle("far19", tables=tables)
    cur0 = {"cidx": np.zeros(mesh.nt, np.int32), "coef": np.zeros((1, 2, 4))}
    s0 = o.setup(mesh.vxy, mesh.tri, node_targets=True, curves=cur0)
    s1 = o.setup(mesh.vxy, mesh.tri, node_targets=True)
    assert np.array_equal(s0["yxy"], s1["yxy"]) and np.array_equal(s0["W"], s1["W"])
    rng = np.random.default_rng(1)
    for T in rng.choice(mesh.nt, 12, replace=False):
        A, B, Cv = [s1["vxy"][s1["tri"][T, i]] for i in range(3)]
        x_self = (A + B + Cv) / 3 + 0.2 * rng.random() * (A - Cv)
        x_near = 0.5 * (A + B) - 0.05 * (Cv - 0.5 * (A + B))
        m_c, n_c = o.pair_moments_curved(s0, T, x_near, 0)
        m_s, n_s = o.pair_moments(A, B, Cv, s1["J"][T], x_near, 0)
        assert n_c == n_s and np.array_equal(m_c, m_s)
        m_c, _ = o.pair_moments_curved(s0, T, x_self, 1)
        m_s, _ = o.pair_moments(A, B, Cv, s1["J"][T], x_self, 1)
        assert np.abs(m_c - m_s).max() <= 1e-13 * np.abs(m_s).max()


@pytest.mark.parametrize("rule", ["far16", "far19"])
def test_curved_disk_constant_density_closed_form(tables, disk_curved, rule):
    mesh, tri, cur = disk_curved
    o = Oracle(rule, tables=tables)
    rng = np.random.default_rng(7)
    th = rng.random(60) * 2 * np.pi
    r = 1 - 10.0 ** rng.uniform(-6, -1, 60)                # down to 1e-6 from the circle
    extra = np.stack([r * np.cos(th), r * np.sin(th)], 1)
    s = o.setup(mesh.vxy, tri, node_targets=True, extra=extra, curves=cur)
    assert (s["tself"] >= 0).all()
    u, info = o.potential(s, np.ones((1, s["N"])))
    ex = (np.sum(s["txy"] ** 2, 1) - 1) / 4
    assert np.abs(u[0] - ex).max() / np.abs(ex).max() <= 1e-11
    assert info["capped"] == 0


def test_curved_disk_quadratic_density_converges(tables):
    """f = |x|^2 is not a polynomial on the curved elements' reference
    simplex, so the P_4 projection leaves an error that falls with h."""
    o = Oracle("far19", tables=tables)
    errs = []
    for nb, ni in ((32, 113), (64, 480)):
        m = inputs.disk_mesh(n_b=nb, n_i=ni)
        t2, cur = inputs.curved_boundary(m, [(0.0, 0.0, 1.0)])
        s = o.setup(m.vxy, t2, node_targets=True, curves=cur)
        u, _ = o.potential(s, np.sum(s["yxy"] ** 2, 1)[None, :])
        ex = (np.sum(s["txy"] ** 2, 1) ** 2 - 1) / 16
        errs.append(np.abs(u[0] - ex).max() / np.abs(ex).max())
    assert errs[0] <= 1e-10 and errs[1] <= errs[0] / 3


def test_curved_annulus_location_and_closed_form(tables):
    """Annulus with both circles curved.  Points that lie in the wedge of a
    hole element's two straight sides, beyond its curved side (seen through
    the hole), belong to the straight elements that hold them: away from the
    curved sides the curved and straight locations agree.  With f = 1 the
    potential is the unit disk's minus the hole's,
        u(x) = (|x|^2 - 1)/4 - (r0^2/2) log|x|,   r0 < |x| < 1,
    (outside a disk of radius a and unit density, (a^2/2) log|x|), at the
    nodes and at points down to 1e-6 from both circles."""
    r0 = 0.45
    circles = [(0.0, 0.0, 1.0), (0.0, 0.0, r0)]
    mesh = inputs.snap_to_circles(inputs.annulus_mesh(600, 21, r0), circles)
    tri, cur = inputs.curved_boundary(mesh, circles)
    assert (cur["cidx"] >= 0).sum() > 60
    o = Oracle("far19", tables=tables)
    tri_ccw, _, W, _ = o.nodes_curved(mesh.vxy, tri, cur)
    assert abs(W.sum() - math.pi * (1 - r0 ** 2)) <= 1e-13
    rng = np.random.default_rng(8)
    r = np.sqrt(rng.uniform((r0 + 0.05) ** 2, 0.95 ** 2, 3000))
    th = rng.random(3000) * 2 * np.pi
    p = np.stack([r * np.cos(th), r * np.sin(th)], 1)
    lc = o.locate_curved(mesh.vxy, tri_ccw, cur, p)
    assert (lc >= 0).all() and np.array_equal(lc, o.locate(mesh.vxy, tri_ccw, p))
    gaps = 10.0 ** rng.uniform(-6, -1, 80)
    th = rng.random(80) * 2 * np.pi
    rr = np.where(np.arange(80) % 2 == 0, 1 - gaps, r0 * (1 + gaps))
    extra = np.stack([rr * np.cos(th), rr * np.sin(th)], 1)
    s = o.setup(mesh.vxy, tri, node_targets=True, extra=extra, curves=cur)
    assert (s["tself"] >= 0).all()
    u, info = o.potential(s, np.ones((1, s["N"])))
    rt = np.hypot(s["txy"][:, 0], s["txy"][:, 1])
    ex = (rt ** 2 - 1) / 4 - 0.5 * r0 ** 2 * np.log(rt)
    assert np.abs(u[0] - ex).max() / np.abs(ex).max() <= 1e-11
    assert info["capped"] == 0
