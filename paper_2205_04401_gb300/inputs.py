"""Seeded synthetic inputs: triangle meshes, densities and target points.

This module only *makes inputs*. It holds none of the volume-potential
arithmetic (no quadrature, no kernel, no near-field test), so both the CUDA
path and the CPU oracle can be fed from it without sharing any of the method.

The paper meshes its domains with a modified Distmesh (Appendix A.3-A.4) and
uses a "wobbly ellipse" given only as a figure (Section 5.2). The fixtures
here stand in for those: a polygonal boundary sampled from a parametrised
curve, interior points drawn from a size function and relaxed by a few
spring iterations (the truss analogy of Appendix A.3), then a Delaunay
triangulation restricted to the polygon.  A triangulation of a polygon with
n_b boundary vertices, n_i interior vertices and k holes has exactly
T = 2 n_i + n_b - 2 + 2k triangles, which is how exact triangle counts are
reached.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.spatial import Delaunay, cKDTree


@dataclasses.dataclass
class Mesh:
    """Straight-sided triangle mesh: vertices (nv, 2) float64 and CCW
    triangles (nt, 3) int32, plus the boundary loops it was built from."""
    vxy: np.ndarray
    tri: np.ndarray
    loops: list            # list of (n, 2) arrays, outer CCW, holes CW
    name: str = ""

    @property
    def nt(self) -> int:
        return int(self.tri.shape[0])

    @property
    def nv(self) -> int:
        return int(self.vxy.shape[0])


# ----------------------------------------------------------------- geometry
def _point_in_loops(p: np.ndarray, loops) -> np.ndarray:
    """Even-odd crossing test of points p (m, 2) against closed polylines."""
    inside = np.zeros(len(p), dtype=bool)
    x, y = p[:, 0][:, None], p[:, 1][:, None]
    for lp in loops:
        a = lp
        b = np.roll(lp, -1, axis=0)
        ay, by = a[:, 1][None, :], b[:, 1][None, :]
        ax, bx = a[:, 0][None, :], b[:, 0][None, :]
        cond = (ay > y) != (by > y)
        with np.errstate(divide="ignore", invalid="ignore"):
            xint = ax + (y - ay) * (bx - ax) / (by - ay)
        cross = cond & (x < xint)
        inside ^= (np.count_nonzero(cross, axis=1) % 2).astype(bool)
    return inside


def _polygon_area(lp: np.ndarray) -> float:
    x, y = lp[:, 0], lp[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def _resample_closed(curve: np.ndarray, n: int) -> np.ndarray:
    """n points equally spaced in arc length along a densely sampled closed curve."""
    seg = np.linalg.norm(np.diff(np.vstack([curve, curve[:1]]), axis=0), axis=1)
    s = np.concatenate([[0.0], np.cumsum(seg)])
    t = np.arange(n) * (s[-1] / n)
    cx = np.interp(t, s, np.concatenate([curve[:, 0], curve[:1, 0]]))
    cy = np.interp(t, s, np.concatenate([curve[:, 1], curve[:1, 1]]))
    return np.stack([cx, cy], axis=1)


def _curve_length(curve: np.ndarray) -> float:
    return float(np.sum(np.linalg.norm(np.diff(np.vstack([curve, curve[:1]]), axis=0), axis=1)))


class _Domain:
    """A planar domain given by dense closed curves (outer CCW, holes CW)."""

    def __init__(self, curves, corners=None, inside=None):
        self.curves = curves
        dense = np.vstack(curves)
        self.tree = cKDTree(dense)
        self.corners = corners or []
        self._inside = inside

    def inside(self, p):
        if self._inside is not None:
            return self._inside(p)
        return _point_in_loops(p, self.curves)

    def dist(self, p):
        return self.tree.query(p)[0]

    def area(self):
        return sum(_polygon_area(c) for c in self.curves)

    def bbox(self):
        d = np.vstack(self.curves)
        return d.min(0), d.max(0)


def _star_curve(n, lobes, amp, r0=1.0, center=(0.0, 0.0), phase=0.0, cw=False):
    th = np.linspace(0.0, 2 * np.pi, n, endpoint=False)
    r = r0 * (1.0 + amp * np.cos(lobes * th + phase))
    c = np.stack([center[0] + r * np.cos(th), center[1] + r * np.sin(th)], axis=1)
    return c[::-1].copy() if cw else c


def _star_inside(lobes, amp, r0=1.0):
    def f(p):
        r = np.hypot(p[:, 0], p[:, 1])
        th = np.arctan2(p[:, 1], p[:, 0])
        return r < r0 * (1.0 + amp * np.cos(lobes * th))
    return f


def _lshape_inside(p):
    x, y = p[:, 0], p[:, 1]
    box = (x > -1) & (x < 1) & (y > -1) & (y < 1)
    return box & ~((x > 0) & (y > 0))


def _lshape_curve(n_per_unit=2000):
    pts = [(-1, -1), (1, -1), (1, 0), (0, 0), (0, 1), (-1, 1)]
    out = []
    for a, b in zip(pts, pts[1:] + pts[:1]):
        a = np.array(a, float)
        b = np.array(b, float)
        m = max(2, int(np.linalg.norm(b - a) * n_per_unit))
        t = np.arange(m) / m
        out.append(a[None, :] + t[:, None] * (b - a)[None, :])
    return np.vstack(out), [np.array(p, float) for p in pts]


# ------------------------------------------------------------ mesh builder
def _sample_loop(curve, h_b, corners):
    """Boundary vertices at spacing about h_b, keeping polygon corners."""
    if not corners:
        n = max(8, int(round(_curve_length(curve) / h_b)))
        return _resample_closed(curve, n)
    # split the curve at corners and sample each straight piece
    cidx = [int(np.argmin(np.linalg.norm(curve - c, axis=1))) for c in corners]
    order = np.argsort(cidx)
    cidx = [cidx[i] for i in order]
    out = []
    for k in range(len(cidx)):
        a = curve[cidx[k]]
        b = curve[cidx[(k + 1) % len(cidx)]]
        m = max(1, int(round(np.linalg.norm(b - a) / h_b)))
        t = np.arange(m) / m
        out.append(a[None, :] + t[:, None] * (b - a)[None, :])
    return np.vstack(out)


def _triangulate(bpts, ipts, loops, hole_count):
    pts = np.vstack([bpts, ipts])
    simp = Delaunay(pts).simplices
    cen = pts[simp].mean(axis=1)
    keep = _point_in_loops(cen, loops)
    tri = simp[keep].astype(np.int64)
    a, b, c = pts[tri[:, 0]], pts[tri[:, 1]], pts[tri[:, 2]]
    o = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    flip = o < 0
    tri[flip, 1], tri[flip, 2] = tri[flip, 2].copy(), tri[flip, 1].copy()
    n_b, n_i = len(bpts), len(ipts)
    ok = len(tri) == 2 * n_i + n_b - 2 + 2 * hole_count
    if ok:
        area = 0.5 * np.abs(o).sum()
        ok = abs(area - sum(_polygon_area(lp) for lp in loops)) < 1e-9 * max(1.0, area)
        ok = ok and np.abs(o).min() > 0
    return pts, tri.astype(np.int32), ok


def _relax(dom, bpts, ipts, hfun, iters, rng):
    """A few truss-relaxation steps (the spring analogy of Distmesh)."""
    nb = len(bpts)
    for _ in range(iters):
        pts = np.vstack([bpts, ipts])
        simp = Delaunay(pts).simplices
        cen = pts[simp].mean(axis=1)
        simp = simp[dom.inside(cen)]
        e = np.vstack([simp[:, [0, 1]], simp[:, [1, 2]], simp[:, [2, 0]]])
        e = np.unique(np.sort(e, axis=1), axis=0)
        vec = pts[e[:, 0]] - pts[e[:, 1]]
        L = np.linalg.norm(vec, axis=1)
        hb = hfun(0.5 * (pts[e[:, 0]] + pts[e[:, 1]]))
        L0 = hb * 1.2 * math.sqrt(np.sum(L ** 2) / np.sum(hb ** 2))
        F = np.maximum(L0 - L, 0.0)
        Fv = (F / np.maximum(L, 1e-300))[:, None] * vec
        acc = np.zeros_like(pts)
        np.add.at(acc, e[:, 0], Fv)
        np.add.at(acc, e[:, 1], -Fv)
        ipts = ipts + 0.2 * acc[nb:]
        # keep interior points inside and away from the boundary
        d = dom.dist(ipts)
        bad = (~dom.inside(ipts)) | (d < 0.35 * hfun(ipts))
        if np.any(bad):
            ipts[bad] = _pull_inside(dom, ipts[bad], hfun)
    return ipts


def _pull_inside(dom, p, hfun):
    # move toward the nearest boundary point's inward side
    _, idx = dom.tree.query(p)
    q = dom.tree.data[idx]
    out = p.copy()
    for k in range(len(p)):
        best = None
        for s in (0.5, 1.0, 1.5, 2.0, 3.0):
            # step inward along the direction away from the boundary point
            dvec = p[k] - q[k]
            n = np.linalg.norm(dvec)
            if n == 0:
                dvec = -q[k]
                n = np.linalg.norm(dvec)
            cand = q[k] + dvec / n * s * hfun(q[k:k + 1])[0]
            cand2 = q[k] - dvec / n * s * hfun(q[k:k + 1])[0]
            for c in (cand, cand2):
                if dom.inside(c[None, :])[0] and dom.dist(c[None, :])[0] >= 0.35 * hfun(c[None, :])[0]:
                    best = c
                    break
            if best is not None:
                break
        out[k] = best if best is not None else p[k]
    return out


def _build(dom: _Domain, n_tri: int, hfun_rel, seed: int, relax_iters: int = 12, name: str = "",
           max_tries: int = 12) -> Mesh:
    """Mesh `dom` with exactly n_tri triangles.

    hfun_rel(p) is the relative size function (1 on the boundary).  The
    boundary spacing h_b is solved so that the interior count implied by the
    size function matches T = 2 n_i + n_b - 2 + 2 holes.
    """
    holes = len(dom.curves) - 1
    area = dom.area()
    lo, hi = dom.bbox()
    rng0 = np.random.default_rng(seed)
    probe = lo + (hi - lo) * rng0.random((20000, 2))
    probe = probe[dom.inside(probe)]
    inv_h2 = np.mean(1.0 / hfun_rel(probe) ** 2)
    perim = sum(_curve_length(c) for c in dom.curves)
    c_hex = math.sqrt(3.0) / 2.0
    for attempt in range(max_tries):
        rng = np.random.default_rng(seed * 1000 + attempt)
        # solve n_b + 2 n_i = n_tri + 2 - 2 holes for h_b
        def count(hb):
            return perim / hb + 2.0 * area * inv_h2 / (c_hex * hb * hb)
        a_, b_ = 1e-4, 10.0
        for _ in range(200):
            m_ = math.sqrt(a_ * b_)
            if count(m_) > n_tri + 2 - 2 * holes:
                a_ = m_
            else:
                b_ = m_
        h_b = math.sqrt(a_ * b_)
        bl = [_sample_loop(c, h_b, dom.corners if i == 0 else None) for i, c in enumerate(dom.curves)]
        bpts = np.vstack(bl)
        n_b = len(bpts)
        if (n_tri - n_b + 2 - 2 * holes) % 2:
            # drop one boundary vertex from the longest loop to fix parity
            i = int(np.argmax([len(x) for x in bl]))
            bl[i] = np.delete(bl[i], 0 if not (i == 0 and dom.corners) else 1, axis=0)
            bpts = np.vstack(bl)
            n_b = len(bpts)
        n_i = (n_tri - n_b + 2 - 2 * holes) // 2
        hfun = lambda p: h_b * hfun_rel(p)
        # rejection-sample n_i interior points with density ~ h^-2
        pts = []
        need = n_i
        hmin = h_b
        while need > 0:
            c = lo + (hi - lo) * rng.random((max(4 * need, 1000), 2))
            c = c[dom.inside(c)]
            c = c[dom.dist(c) > 0.5 * hfun(c)]
            acc = rng.random(len(c)) < (hmin / hfun(c)) ** 2
            c = c[acc][:need]
            pts.append(c)
            need -= len(c)
        ipts = np.vstack(pts)
        ipts = _relax(dom, bpts, ipts, hfun, relax_iters, rng)
        loops = [b for b in bl]
        vxy, tri, ok = _triangulate(bpts, ipts, loops, holes)
        if ok and len(tri) == n_tri:
            return Mesh(vxy=np.ascontiguousarray(vxy, dtype=np.float64),
                        tri=np.ascontiguousarray(tri, dtype=np.int32), loops=loops, name=name)
    raise RuntimeError(f"mesh generation failed for {name} after {max_tries} tries")


# ----------------------------------------------------------------- fixtures
def disk_mesh(seed: int = 2205044011, n_b: int = 32, n_i: int = 113, stagger: bool = False) -> Mesh:
    """Unit disk: n_b vertices on the circle, n_i jittered-hex interior
    points, Delaunay.  The default gives 2*113 + 32 - 2 = 256 triangles.
    stagger=True shifts the initial tiling to the centroids of its triangles
    (by (h/2, h sqrt(3)/6)) and the boundary vertices by half a spacing, so
    that the mesh's edges avoid those of the unshifted mesh (the staggered
    interpolation mesh of Section 4.3)."""
    rng = np.random.default_rng(seed)
    th = 2 * np.pi * (np.arange(n_b) + (0.5 if stagger else 0.0)) / n_b
    bpts = np.stack([np.cos(th), np.sin(th)], axis=1)
    h_b = 2 * math.sin(math.pi / n_b)
    r_keep = math.cos(math.pi / n_b) - 0.45 * h_b

    def lattice(h, jit):
        nx = int(2.5 / h) + 2
        ii, jj = np.meshgrid(np.arange(-nx, nx + 1), np.arange(-nx, nx + 1), indexing="ij")
        x = (ii + 0.5 * (jj % 2) + (0.5 if stagger else 0.0)) * h
        y = (jj * math.sqrt(3) / 2 + (math.sqrt(3) / 6 if stagger else 0.0)) * h
        p = np.stack([x.ravel(), y.ravel()], axis=1)
        return p + jit[: len(p)] * h

    jit = (rng.random((200000, 2)) - 0.5) * 0.3
    a, b = 0.01, 1.0
    for _ in range(100):
        m = 0.5 * (a + b)
        p = lattice(m, jit)
        if np.count_nonzero(np.linalg.norm(p, axis=1) < r_keep) >= n_i:
            a = m
        else:
            b = m
    p = lattice(a, jit)
    p = p[np.linalg.norm(p, axis=1) < r_keep]
    p = p[np.argsort(np.linalg.norm(p, axis=1), kind="stable")[:n_i]]
    vxy, tri, ok = _triangulate(bpts, p, [bpts], 0)
    if not ok:
        raise RuntimeError("disk mesh invalid")
    return Mesh(vxy=vxy, tri=tri, loops=[bpts], name=f"disk{len(tri)}" + ("_staggered" if stagger else ""))


def star_mesh(n_tri: int = 16384, seed: int = 2205044012, lobes: int = 5, amp: float = 0.3,
              grading: float = 8.0, grade_width: float = 0.5, relax_iters: int = 12) -> Mesh:
    """Star r(t) = 1 + amp cos(lobes t), graded toward the boundary with size
    h(delta) = h_b min(grading, 1 + (grading - 1) delta / grade_width)."""
    curve = _star_curve(20000, lobes, amp)
    dom = _Domain([curve], inside=_star_inside(lobes, amp))
    hrel = lambda p: np.minimum(grading, 1.0 + (grading - 1.0) * dom.dist(p) / grade_width)
    return _build(dom, n_tri, hrel, seed, relax_iters, name=f"star{lobes}_{n_tri}")


def annulus_mesh(n_tri: int, seed: int, r_in: float, relax_iters: int = 8) -> Mesh:
    outer = _star_curve(8000, 0, 0.0)
    inner = _star_curve(max(2000, int(8000 * r_in)), 0, 0.0, r0=r_in, cw=True)
    dom = _Domain([outer, inner], inside=lambda p: (np.hypot(p[:, 0], p[:, 1]) < 1.0)
                  & (np.hypot(p[:, 0], p[:, 1]) > r_in))
    return _build(dom, n_tri, lambda p: np.ones(len(p)), seed, relax_iters, name=f"annulus_{n_tri}")


def lshape_mesh(n_tri: int, seed: int, relax_iters: int = 8) -> Mesh:
    curve, corners = _lshape_curve()
    dom = _Domain([curve], corners=corners, inside=_lshape_inside)
    return _build(dom, n_tri, lambda p: np.ones(len(p)), seed, relax_iters, name=f"lshape_{n_tri}")


def lobed_mesh(n_tri: int, seed: int, lobes: int, amp: float, relax_iters: int = 8) -> Mesh:
    dom = _Domain([_star_curve(12000, lobes, amp)], inside=_star_inside(lobes, amp))
    return _build(dom, n_tri, lambda p: np.ones(len(p)), seed, relax_iters, name=f"star{lobes}_{n_tri}")


def disk_uniform_mesh(n_tri: int, seed: int, relax_iters: int = 8) -> Mesh:
    dom = _Domain([_star_curve(8000, 0, 0.0)], inside=_star_inside(0, 0.0))
    return _build(dom, n_tri, lambda p: np.ones(len(p)), seed, relax_iters, name=f"disk_{n_tri}")


def curved_boundary(mesh: Mesh, circles, K=None, tol: float = 1e-15):
    """Curved boundary elements for a mesh whose boundary edges lie on circles.

    circles: list of (cx, cy, R).  Every triangle with a boundary edge on one
    of the circles is rotated (orientation kept) so that the edge is
    v0 -> v1, and its curved side is the arc from v0 to v1 (the short way
    round), given as the deviation from the chord,
        c(xi) - (1 - xi) v0 - xi v1 = xi (1 - xi) D(xi),
    with D interpolated at K+1 Chebyshev points of [0, 1]
    (D = sum_k a_k T_k(2 xi - 1)).  K=None takes the smallest K (2..15) whose
    curves stay within tol R of their circles on 401 points of every arc
    (higher coefficients would only carry rounding noise).  Returns
    (tri, {"cidx", "coef"}): the rotated triangles, the curve index of every
    triangle (-1 straight) and the coefficients [ncurve][2][K+1].
    """
    if K is None:
        for k in range(2, 16):
            tri, cur = curved_boundary(mesh, circles, K=k)
            if _curve_deviation(mesh.vxy, tri, cur, circles) <= tol:
                return tri, cur
        return tri, cur
    tri = mesh.tri.copy()
    vxy = mesh.vxy
    edges = {}
    for t in range(len(tri)):
        for e in range(3):
            a, b = int(tri[t, e]), int(tri[t, (e + 1) % 3])
            edges.setdefault((min(a, b), max(a, b)), []).append((t, e))
    cidx = np.full(len(tri), -1, np.int32)
    coefs = []
    z = np.cos(np.pi * (np.arange(K + 1) + 0.5) / (K + 1))       # Chebyshev points of the first kind
    xs = 0.5 * (z + 1.0)
    V = np.polynomial.chebyshev.chebvander(z, K)
    for (a, b), owners in edges.items():
        if len(owners) != 1:
            continue
        t, e = owners[0]
        va, vb = vxy[tri[t, e]], vxy[tri[t, (e + 1) % 3]]
        circ = None
        for cx, cy, R in circles:
            ra, rb = math.hypot(va[0] - cx, va[1] - cy), math.hypot(vb[0] - cx, vb[1] - cy)
            if abs(ra - R) < 1e-9 * R and abs(rb - R) < 1e-9 * R:
                circ = (cx, cy, R)
                break
        if circ is None or cidx[t] >= 0:
            continue
        tri[t] = np.roll(tri[t], -e)                                 # boundary edge first, orientation kept
        v0, v1 = vxy[tri[t, 0]], vxy[tri[t, 1]]
        cx, cy, R = circ
        th0 = math.atan2(v0[1] - cy, v0[0] - cx)
        dth = math.atan2(v1[1] - cy, v1[0] - cx) - th0
        dth = (dth + math.pi) % (2 * math.pi) - math.pi
        th = th0 + xs * dth
        c = np.stack([cx + R * np.cos(th), cy + R * np.sin(th)], axis=1)
        # endpoints exactly at v0, v1
        c += (1 - xs)[:, None] * (v0 - [cx + R * math.cos(th0), cy + R * math.sin(th0)])
        c += xs[:, None] * (v1 - [cx + R * math.cos(th0 + dth), cy + R * math.sin(th0 + dth)])
        Dv = (c - (1 - xs)[:, None] * v0 - xs[:, None] * v1) / (xs * (1 - xs))[:, None]
        coefs.append(np.linalg.solve(V, Dv).T)                       # [2][K+1]
        cidx[t] = len(coefs) - 1
    return tri, {"cidx": cidx, "coef": np.ascontiguousarray(np.array(coefs).reshape(-1, 2, K + 1))}


def _curve_deviation(vxy, tri, cur, circles) -> float:
    """Largest |distance to the circle - R| / R over 401 points of every curved side."""
    xs = np.linspace(0.0, 1.0, 401)
    t = 2.0 * xs - 1.0
    worst = 0.0
    for T in np.where(cur["cidx"] >= 0)[0]:
        a = cur["coef"][cur["cidx"][T]]
        v0, v1 = vxy[tri[T, 0]], vxy[tri[T, 1]]
        D = np.stack([np.polynomial.chebyshev.chebval(t, a[0]), np.polynomial.chebyshev.chebval(t, a[1])], 1)
        c = (1 - xs)[:, None] * v0 + xs[:, None] * v1 + (xs * (1 - xs))[:, None] * D
        best = np.inf
        for cx, cy, R in circles:
            best = min(best, np.abs(np.hypot(c[:, 0] - cx, c[:, 1] - cy) - R).max() / R)
        worst = max(worst, best)
    return worst


def snap_to_circles(mesh: Mesh, circles, tol: float = 1e-6) -> Mesh:
    """A copy of the mesh whose vertices within tol (relative) of one of the
    circles (cx, cy, R) are moved radially onto it, so that boundary edges
    sampled from a circle as a fine polyline become chords of the circle
    (what curved_boundary expects)."""
    vxy = mesh.vxy.copy()
    for cx, cy, R in circles:
        d = vxy - [cx, cy]
        r = np.hypot(d[:, 0], d[:, 1])
        on = np.abs(r - R) < tol * R
        vxy[on] = np.array([cx, cy]) + d[on] * (R / r[on])[:, None]
    return Mesh(vxy, mesh.tri.copy(), mesh.loops, mesh.name)


def random_interior_points(mesh: Mesh, m: int, seed: int) -> np.ndarray:
    """m points uniform in the meshed polygon (rejection sampling)."""
    rng = np.random.default_rng(seed)
    lo, hi = mesh.vxy.min(0), mesh.vxy.max(0)
    out = []
    need = m
    while need > 0:
        c = lo + (hi - lo) * rng.random((max(2 * need, 256), 2))
        c = c[_point_in_loops(c, mesh.loops)][:need]
        out.append(c)
        need -= len(c)
    return np.ascontiguousarray(np.vstack(out), dtype=np.float64)


# --------------------------------------------------------------- densities
@dataclasses.dataclass
class GaussianMix:
    """f(x) = sum_i a_i exp(-|x - c_i|^2 / s_i)."""
    a: np.ndarray
    c: np.ndarray
    s: np.ndarray

    def __call__(self, p: np.ndarray) -> np.ndarray:
        d2 = ((p[:, None, :] - self.c[None, :, :]) ** 2).sum(-1)
        return (self.a[None, :] * np.exp(-d2 / self.s[None, :])).sum(1)


def gaussian_mix(mesh: Mesh, seed: int, k: int = 4, s_lo: float = 0.05, s_hi: float = 0.2) -> GaussianMix:
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.5, 1.5, k)
    s = rng.uniform(s_lo, s_hi, k)
    c = random_interior_points(mesh, k, seed + 7)
    return GaussianMix(a=a, c=c, s=s)


def manufactured_sin_cos(k: float):
    """f = Laplacian of u = sin(kx) cos(ky), i.e. -2 k^2 sin(kx) cos(ky)."""
    return lambda p: -2.0 * k * k * np.sin(k * p[:, 0]) * np.cos(k * p[:, 1])


def gaussian_bump(seed: int, width: float = 0.05, r: float = 0.5):
    """f = exp(-|x - x0|^2 / width) with x0 uniform in the disk of radius r."""
    rng = np.random.default_rng(seed)
    while True:
        x0 = rng.uniform(-r, r, 2)
        if x0 @ x0 < r * r:
            break
    return lambda p: np.exp(-((p - x0[None, :]) ** 2).sum(1) / width), x0


def two_gaussian_poly(p: np.ndarray) -> np.ndarray:
    """The two-Gaussian polynomial density of the paper's Section 5.2 experiment."""
    x, y = p[:, 0], p[:, 1]
    return (4 * np.exp(-(x + 1.6) ** 2 - (y + 0.2) ** 2) * (x * x + y * y + 3.2 * x + 0.4 * y + 1.6)
            + 4 * np.exp(-(x - 0.2) ** 2 - (y - 1) ** 2) * (x * x + y * y - 0.4 * x - 2 * y + 0.04))


# ---------------------------------------------------------- config recipes
SEED0 = 2205044010


def config1():
    """Unit disk, 256 triangles; densities f = 1 and a Gaussian bump."""
    mesh = disk_mesh(seed=SEED0 + 1)
    bump, x0 = gaussian_bump(SEED0 + 1)
    return mesh, [lambda p: np.ones(len(p)), bump]


def config2(n_tri: int = 16384, m_extra: int = 10000, relax_iters: int = 12):
    """Graded star, n_tri triangles, 4-Gaussian density, m_extra random targets."""
    mesh = star_mesh(n_tri=n_tri, seed=SEED0 + 2, relax_iters=relax_iters)
    f = gaussian_mix(mesh, SEED0 + 2)
    extra = random_interior_points(mesh, m_extra, SEED0 + 20)
    return mesh, f, extra


def config3_densities(mesh: Mesh, n_gauss: int = 56, n_sin: int = 8):
    fs = [gaussian_mix(mesh, SEED0 + 300 + i) for i in range(n_gauss)]
    fs += [manufactured_sin_cos(float(k)) for k in range(1, n_sin + 1)]
    return fs


def batch_meshes(n_mesh: int = 200, t_lo: int = 500, t_hi: int = 20000, seed: int = SEED0 + 4,
                 relax_iters: int = 4):
    """Seeded mix of disks, annuli, 3-7-lobed stars and L-shapes with
    log-uniform triangle counts in [t_lo, t_hi] (even counts for parity of
    the triangle-count identity), and 1-8 densities each."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_mesh):
        t = int(round(math.exp(rng.uniform(math.log(t_lo), math.log(t_hi)))))
        kind = int(rng.integers(0, 4))
        d = int(rng.integers(1, 9))
        s = seed * 1000 + i
        if kind == 0:
            m = disk_uniform_mesh(t, s, relax_iters)
        elif kind == 1:
            m = annulus_mesh(t + (t % 2), s, float(rng.uniform(0.3, 0.6)), relax_iters)
        elif kind == 2:
            m = lobed_mesh(t, s, int(rng.integers(3, 8)), float(rng.uniform(0.1, 0.35)), relax_iters)
        else:
            m = lshape_mesh(t, s, relax_iters)
        out.append((m, d, s))
    return out
