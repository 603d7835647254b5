"""Independent integrators used to pin the oracle (test-side only).

Nothing here shares code with the oracle or with the library:
* ``polygon_f1``: int_T log|x-y| dA in closed form from the divergence
  theorem, div[(y-x)(2 log r - 1)/4] = log r, with the textbook
  antiderivative of log sqrt(u^2 + h^2) along each edge.
* ``fan_poly``: int_T log|x-y| q(y) dA for a polynomial q of degree <= 4, by
  a signed fan decomposition of T seen from x, exact radial moments
  int_0^R r^(k+1) log r dr, and adaptive Gauss-Kronrod in the angle.
* ``green_volume``: V[lap u](x) = u(x) - oint (u dG/dn - G du/dn) ds
  (Green's third identity) by adaptive quadrature along boundary edges.
"""
import math

import numpy as np
from scipy import integrate

TWO_PI = 2.0 * math.pi


def seg_log_int(x, P, Q):
    """int over the segment PQ of log|y - x| ds."""
    d = Q - P
    L = np.linalg.norm(d)
    u = d / L
    n = np.array([u[1], -u[0]])
    h = float((x - P) @ n)
    u0, u1 = float((P - x) @ u), float((Q - x) @ u)
    ah = abs(h)

    def F(t):
        if ah == 0.0:
            return t * math.log(abs(t)) - t if t != 0 else 0.0
        return 0.5 * (t * math.log(t * t + h * h) - 2 * t + 2 * ah * math.atan(t / ah))

    return F(u1) - F(u0)


def tri_f1(x, A, B, C):
    """int_T log|x - y| dA for a CCW triangle (any x)."""
    s = 0.0
    for P, Q in ((A, B), (B, C), (C, A)):
        d = Q - P
        L = np.linalg.norm(d)
        n = np.array([d[1], -d[0]]) / L          # outward for CCW
        h = float((P - x) @ n)
        s += h / 4.0 * (2.0 * seg_log_int(x, P, Q) - L)
    return s


def polygon_f1(vxy, tri, x):
    """(1/2pi) int_Omega log|x - y| dA over the triangulated polygon."""
    return sum(tri_f1(x, vxy[t[0]], vxy[t[1]], vxy[t[2]]) for t in tri) / TWO_PI


def _radial_moment(k, R):
    # int_0^R r^(k+1) log r dr
    return R ** (k + 2) * (math.log(R) / (k + 2) - 1.0 / (k + 2) ** 2)


def _poly_along_ray(qfun, x, e, deg, scale):
    """Coefficients c_k of q(x + r e) = sum_k c_k r^k (exact for deg <= 4),
    from samples at r = scale * (0..deg) / deg (Chebyshev-free but well
    scaled to the triangle)."""
    t = np.arange(deg + 1, dtype=float) / deg
    vals = np.array([qfun(x + scale * ti * e) for ti in t])
    V = np.vander(t, deg + 1, increasing=True)
    c = np.linalg.solve(V, vals)
    return c / scale ** np.arange(deg + 1)


def fan_poly(x, A, B, C, qfun, deg=4, epsabs=3e-15, epsrel=3e-14):
    """int_T log|x - y| q(y) dA, q a polynomial of degree <= deg.

    Each fan (x, P, Q) is integrated along its edge: the ray to P + t (Q - P)
    has length R(t) = |a + t d| (a = P - x, d = Q - P) and sweeps the angle
    at the rate cross(a, d) / R(t)^2, so the fan is
        int_0^1 [int_0^R(t) r log r q(x + r e(t)) dr] cross(a, d) / R(t)^2 dt.
    The t-integrand peaks at the foot of the perpendicular from x with a width
    of about the distance h from x to the line; the interval is cut there and
    at geometric offsets h 10^j on either side."""
    x = np.asarray(x, float)
    total = 0.0
    scale = max(np.linalg.norm(v - x) for v in (A, B, C))
    for P, Q in ((A, B), (B, C), (C, A)):
        a, d = P - x, Q - P
        cross = a[0] * d[1] - a[1] * d[0]
        if abs(cross) < 1e-300:
            continue
        dd = float(d @ d)

        def g(t):
            v = a + t * d
            R = math.sqrt(float(v @ v))
            c = _poly_along_ray(qfun, x, v / R, deg, scale)
            return sum(c[k] * _radial_moment(k, R) for k in range(deg + 1)) * cross / (R * R)
        t_foot = float(-(a @ d) / dd)
        width = abs(cross) / dd            # h / |d|
        cuts = {0.0, 1.0}
        for j in range(6):
            for sgn in (-1.0, 1.0):
                c = t_foot + sgn * width * 10.0 ** j
                if 0.0 < c < 1.0:
                    cuts.add(c)
        if 0.0 < t_foot < 1.0:
            cuts.add(t_foot)
        cuts = sorted(cuts)
        for lo, hi in zip(cuts, cuts[1:]):
            val, _ = integrate.quad(g, lo, hi, epsabs=epsabs, epsrel=epsrel, limit=400)
            total += val
    return total


def green_volume(x, loops_edges, u, gradu, epsabs=1e-14, epsrel=1e-13):
    """V[lap u](x) = u(x) - oint (u dG/dn - G du/dn) ds for x inside.

    loops_edges: list of (P, Q) boundary edges oriented with the domain on
    the left (outward normal = (dy, -dx)/L)."""
    x = np.asarray(x, float)
    s = 0.0
    for P, Q in loops_edges:
        d = Q - P
        L = np.linalg.norm(d)
        n = np.array([d[1], -d[0]]) / L

        def g(t):
            y = P + t * d
            v = y - x
            r2 = v @ v
            G = 0.5 * math.log(r2) / TWO_PI
            dGdn = (v @ n) / r2 / TWO_PI
            return (u(y) * dGdn - G * (gradu(y) @ n)) * L
        val, _ = integrate.quad(g, 0.0, 1.0, epsabs=epsabs, epsrel=epsrel, limit=400)
        s += val
    return u(x) - s


def boundary_edges(tri):
    """Boundary edges of a CCW triangulation, oriented with the interior on the left."""
    from collections import Counter
    cnt = Counter()
    for t in tri:
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            cnt[(min(a, b), max(a, b))] += 1
    out = []
    for t in tri:
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            if cnt[(min(a, b), max(a, b))] == 1:
                out.append((int(a), int(b)))
    return out
