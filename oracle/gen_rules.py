"""Quadrature tables for the CPU oracle (test infrastructure only).

The paper takes its triangle rules from published tables (Section 5, the
Xiao-Gimbutas and Vioreanu-Rokhlin tables) and uses a generalized Gaussian
rule in the radial direction of the self-interaction scheme (Section 3.4,
Table "orders and lengths of the quadrature rules": GGQ of order 8 has 8
nodes).  None of those tables is available here, so this script *derives*
every rule from its defining moment equations in 60-digit arithmetic
(mpmath) and rounds each value once to double:

* gl16 / gl7 : Gauss-Legendre on [0,1] (Newton on the Legendre recurrence).
* near33     : the S3-symmetric 33-point rule of degree 12 (the order-12
               near rule of Section 5.1), the same rule as sym12 below.
* far16      : S3-symmetric, degree 8, orbits [centroid, 3 x S21, 1 x S111].
* far19      : S3-symmetric, degree 9, orbits [centroid, 4 x S21, 1 x S111].
               Both solved by Gauss-Newton on all monomial moments
               x^i y^j (i+j <= degree), from the starting orbit parameters
               listed in FAR_START below (they define which root is meant).
* sym<n>     : S3-symmetric far rules of degree n = 12, 20, 25, 30, 40, 50
               (Section 4.2), Newton's method on the S3-invariant moment
               equations from the orbit definitions in far_sym_defs.py
               (90 digits; see symmetric_far_rule).
* ggq8       : 8 nodes r_j, weights om_j on [0,1] with
               sum_j om_j r_j^k = int_0^1 r r^k dr and
               sum_j om_j r_j^k log r_j = int_0^1 r r^k log r dr, k = 0..7,
               reached by continuation from the Gauss rule for the weight r
               through the functions r^k (r^t - 1)/t, t = 8 -> 0.
* what       : the weight w of Section 4.1 (Eq. rho0): the largest weight
               among the ceil((N+1)/2) nodes closest to an edge of the
               reference simplex, maximised over the three edges.
* basis      : an orthonormal basis of P_4 on the reference simplex, made
               from products of shifted Legendre polynomials
               P_a(2x-1) P_b(2y-1), a+b <= 4, orthonormalised by the
               Cholesky factor of their exact Gram matrix.

Reference simplex: {(x, y): x >= 0, y >= 0, x + y <= 1}, area 1/2.
Barycentric (l1, l2, l3) of the vertices (0,0), (1,0), (0,1) maps to
(x, y) = (l2, l3).  Orbit point order: S21(a): (a, 1-2a), (1-2a, a), (a, a);
S111(a, b), c = 1-a-b: (l2, l3) from the permutations
(a,b,c),(a,c,b),(b,a,c),(b,c,a),(c,a,b),(c,b,a) of (l1,l2,l3).

Run:  python oracle/gen_rules.py   (writes oracle/rules_oracle.json)
"""
from __future__ import annotations

import json
import math
import os
from fractions import Fraction

import mpmath as mp

mp.mp.dps = 60

# Starting orbit parameters that single out the positive-interior roots.
# centroid weight; S21 (a, w) pairs; S111 (a, b, w) triples.
FAR_START = {
    "far16": dict(degree=8, w0=0.0722, s21=[(0.0505, 0.0162), (0.4593, 0.0475), (0.1706, 0.0516)],
                  s111=[(0.0084, 0.2631, 0.0136)]),
    "far19": dict(degree=9, w0=0.0486, s21=[(0.0447, 0.0128), (0.1882, 0.0398), (0.4371, 0.0389),
                                           (0.4897, 0.0157)],
                  s111=[(0.0368, 0.2220, 0.0216)]),
}


def _legendre_and_deriv(n, x):
    p0, p1 = mp.mpf(1), x
    if n == 0:
        return p0, mp.mpf(0)
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    dp = n * (x * p1 - p0) / (x * x - 1)
    return p1, dp


def gauss_legendre01(n):
    """Gauss-Legendre nodes/weights on [0,1], ascending."""
    xs, ws = [], []
    for i in range(1, n + 1):
        x = mp.cos(mp.pi * (i - mp.mpf(1) / 4) / (n + mp.mpf(1) / 2))
        for _ in range(100):
            p, dp = _legendre_and_deriv(n, x)
            dx = p / dp
            x -= dx
            if abs(dx) < mp.mpf(10) ** (-55):
                break
        p, dp = _legendre_and_deriv(n, x)
        xs.append((1 - x) / 2)           # ascending on [0,1]
        ws.append(1 / ((1 - x * x) * dp * dp))
    return xs, ws


def duffy_rule(n):
    u, a = gauss_legendre01(n)
    X, Y, W = [], [], []
    for i in range(n):
        for j in range(n):
            X.append(u[i])
            Y.append((1 - u[i]) * u[j])
            W.append(a[i] * a[j] * (1 - u[i]))
    return X, Y, W


def _monos(d):
    return [(i, n - i) for n in range(d + 1) for i in range(n + 1)]


def _simplex_moment(i, j):
    return mp.mpf(math.factorial(i) * math.factorial(j)) / math.factorial(i + j + 2)


def _expand(params, n21, n111):
    X, Y, W = [mp.mpf(1) / 3], [mp.mpf(1) / 3], [params[0]]
    k = 1
    for _ in range(n21):
        a, w = params[k], params[k + 1]
        k += 2
        for (l2, l3) in [(a, 1 - 2 * a), (1 - 2 * a, a), (a, a)]:
            X.append(l2)
            Y.append(l3)
            W.append(w)
    for _ in range(n111):
        a, b, w = params[k], params[k + 1], params[k + 2]
        k += 3
        c = 1 - a - b
        for (l1, l2, l3) in [(a, b, c), (a, c, b), (b, a, c), (b, c, a), (c, a, b), (c, b, a)]:
            X.append(l2)
            Y.append(l3)
            W.append(w)
    return X, Y, W


def _moment_residual(params, deg, n21, n111):
    X, Y, W = _expand(params, n21, n111)
    return [mp.fsum(w * x ** i * y ** j for x, y, w in zip(X, Y, W)) - _simplex_moment(i, j)
            for i, j in _monos(deg)]


def symmetric_rule(spec):
    deg = spec["degree"]
    n21, n111 = len(spec["s21"]), len(spec["s111"])
    p = [mp.mpf(spec["w0"])]
    for a, w in spec["s21"]:
        p += [mp.mpf(a), mp.mpf(w)]
    for a, b, w in spec["s111"]:
        p += [mp.mpf(a), mp.mpf(b), mp.mpf(w)]
    h = mp.mpf(10) ** (-30)
    for it in range(60):
        r = mp.matrix(_moment_residual(p, deg, n21, n111))
        J = mp.matrix(len(r), len(p))
        for c in range(len(p)):
            pp = list(p)
            pm = list(p)
            pp[c] += h
            pm[c] -= h
            rp = _moment_residual(pp, deg, n21, n111)
            rm = _moment_residual(pm, deg, n21, n111)
            for rr in range(len(r)):
                J[rr, c] = (rp[rr] - rm[rr]) / (2 * h)
        step = mp.lu_solve(J.T * J, J.T * r)
        p = [p[c] - step[c] for c in range(len(p))]
        if mp.norm(step) < mp.mpf(10) ** (-50):
            break
    res = max(abs(x) for x in _moment_residual(p, deg, n21, n111))
    assert res < mp.mpf(10) ** (-45), res
    return _expand(p, n21, n111)


# --------------------------------------------------- S3-symmetric far rules
# Far rules of degree 12-50 for the order sweep of Section 4.2 (the paper
# takes Xiao-Gimbutas rules; none is available here).  Each rule is named by
# its orbit structure and approximate orbit parameters in far_sym_defs.py;
# the exact rule is the root of its moment equations next to them, reached
# here by Newton's method in 90-digit arithmetic.  The moment equations are
# taken on the S3-invariant polynomials, which for a symmetric rule are all
# the conditions there are: with the centred barycentric coordinates
# u_i = l_i - 1/3 and the power sums p2 = sum u_i^2, p3 = sum u_i^3, the
# products p2^i p3^j, 2i + 3j <= degree, span the invariant polynomials of
# that degree, and one node per orbit gives the orbit's sum.  Their exact
# integrals come from the collapsed Gauss rule of degree // 2 + 2 points
# (exact to total degree >= degree + 2).  A parameter listed in `fixed` is
# held at its listed value, which makes the system square where the orbit
# structure has one parameter more than there are equations.

def _far_sym_defs():
    try:
        from .far_sym_defs import FAR_SYM
    except ImportError:          # run as a script from this folder
        from far_sym_defs import FAR_SYM
    return FAR_SYM


def _sym_pairs(deg):
    return [(i, j) for j in range(deg // 3 + 1) for i in range((deg - 3 * j) // 2 + 1)]


def _p2p3(l1, l2, l3):
    t = mp.mpf(1) / 3
    u = (l1 - t, l2 - t, l3 - t)
    return u[0] ** 2 + u[1] ** 2 + u[2] ** 2, u[0] ** 3 + u[1] ** 3 + u[2] ** 3, u


def _sym_exact(deg):
    X, Y, W = duffy_rule(deg // 2 + 2)
    pairs = _sym_pairs(deg)
    out = [mp.mpf(0)] * len(pairs)
    for x, y, w in zip(X, Y, W):
        p2, p3, _ = _p2p3(1 - x - y, x, y)
        for k, (i, j) in enumerate(pairs):
            out[k] += w * p2 ** i * p3 ** j
    return out


def _sym_params(spec):
    p = [] if spec["w0"] is None else [mp.mpf(spec["w0"])]
    for a, w in spec["s21"]:
        p += [mp.mpf(a), mp.mpf(w)]
    for a, b, w in spec["s111"]:
        p += [mp.mpf(a), mp.mpf(b), mp.mpf(w)]
    return p


def _sym_system(p, spec, pairs, exact):
    """Residuals sum_orbits |orbit| w p2^i p3^j - exact and their Jacobian."""
    R = [-v for v in exact]
    J = [[mp.mpf(0)] * len(p) for _ in pairs]
    c = 0
    kinds = ([0] if spec["w0"] is not None else []) + [1] * len(spec["s21"]) + [2] * len(spec["s111"])
    for kind in kinds:
        if kind == 0:                 # centroid: p2 = p3 = 0
            R[0] += p[c]
            J[0][c] += 1
            c += 1
            continue
        if kind == 1:                 # S21(a): barycentric (a, a, 1 - 2a)
            a, w = p[c], p[c + 1]
            lam, dirs, mult = (a, a, 1 - 2 * a), [(1, 1, -2)], 3
        else:                         # S111(a, b): (a, b, 1 - a - b)
            a, b, w = p[c], p[c + 1], p[c + 2]
            lam, dirs, mult = (a, b, 1 - a - b), [(1, 0, -1), (0, 1, -1)], 6
        p2, p3, u = _p2p3(*lam)
        dp2 = [sum(2 * u[q] * d[q] for q in range(3)) for d in dirs]
        dp3 = [sum(3 * u[q] ** 2 * d[q] for q in range(3)) for d in dirs]
        for k, (i, j) in enumerate(pairs):
            psi = p2 ** i * p3 ** j
            R[k] += mult * w * psi
            gi = i * p2 ** (i - 1) * p3 ** j if i > 0 else 0
            gj = j * p2 ** i * p3 ** (j - 1) if j > 0 else 0
            for s, _ in enumerate(dirs):
                J[k][c + s] += mult * w * (gi * dp2[s] + gj * dp3[s])
            J[k][c + len(dirs)] += mult * psi
        c += len(dirs) + 1
    return R, J


def symmetric_far_rule(degree):
    """The S3-symmetric far rule of the given degree (far_sym_defs.FAR_SYM):
    dict of floats x, y, w, degree, what, with the nodes in orbit order."""
    spec = _far_sym_defs()[degree]
    with mp.workdps(90):
        pairs = _sym_pairs(degree)
        exact = _sym_exact(degree)
        p = _sym_params(spec)
        free = [c for c in range(len(p)) if c not in spec["fixed"]]
        assert len(free) == len(pairs), (len(free), len(pairs))
        for _ in range(40):
            R, J = _sym_system(p, spec, pairs, exact)
            step = mp.lu_solve(mp.matrix([[J[k][c] for c in free] for k in range(len(pairs))]), mp.matrix(R))
            for s, c in enumerate(free):
                p[c] -= step[s]
            if max(abs(v) for v in step) < mp.mpf(10) ** -60:   # far below double precision
                break
        R, _ = _sym_system(p, spec, pairs, exact)
        assert max(abs(v) for v in R) < mp.mpf(10) ** -60
        n21, n111 = len(spec["s21"]), len(spec["s111"])
        X, Y, W = [], [], []
        c = 0
        if spec["w0"] is not None:
            X.append(mp.mpf(1) / 3)
            Y.append(mp.mpf(1) / 3)
            W.append(p[0])
            c = 1
        for _ in range(n21):
            a, w = p[c], p[c + 1]
            c += 2
            for (l2, l3) in [(a, 1 - 2 * a), (1 - 2 * a, a), (a, a)]:
                X.append(l2)
                Y.append(l3)
                W.append(w)
        for _ in range(n111):
            a, b, w = p[c], p[c + 1], p[c + 2]
            c += 3
            cc = 1 - a - b
            for (l1, l2, l3) in [(a, b, cc), (a, cc, b), (b, a, cc), (b, cc, a), (cc, a, b), (cc, b, a)]:
                X.append(l2)
                Y.append(l3)
                W.append(w)
        assert all(w > 0 for w in W) and all(x > 0 and y > 0 and 1 - x - y > 0 for x, y in zip(X, Y))
        return dict(degree=degree, x=[float(v) for v in X], y=[float(v) for v in Y], w=[float(v) for v in W],
                    what=float(what_for(X, Y, W, degree)))


def _ggq_residual(z, t):
    r, om = z[:8], z[8:]
    out = []
    for k in range(8):
        out.append(mp.fsum(om[j] * r[j] ** k for j in range(8)) - mp.mpf(1) / (k + 2))
    for k in range(8):
        if t == 0:
            f = [r[j] ** k * mp.log(r[j]) for j in range(8)]
            mom = -mp.mpf(1) / (k + 2) ** 2
        else:
            f = [r[j] ** k * (r[j] ** t - 1) / t for j in range(8)]
            mom = -mp.mpf(1) / ((k + 2) * (k + 2 + t))
        out.append(mp.fsum(om[j] * f[j] for j in range(8)) - mom)
    return out


def _newton(fun, z, tol=mp.mpf(10) ** (-50), maxit=80):
    h = mp.mpf(10) ** (-30)
    for _ in range(maxit):
        r = mp.matrix(fun(z))
        n = len(z)
        J = mp.matrix(n, n)
        for c in range(n):
            zp, zm = list(z), list(z)
            zp[c] += h
            zm[c] -= h
            fp, fm = fun(zp), fun(zm)
            for rr in range(n):
                J[rr, c] = (fp[rr] - fm[rr]) / (2 * h)
        step = mp.lu_solve(J, r)
        z = [z[c] - step[c] for c in range(n)]
        if mp.norm(step) < tol:
            return z
    raise RuntimeError("Newton did not converge")


def ggq8():
    # Gauss rule for the weight r on [0,1] (8 nodes) = the t = 8 system.
    # Start from Gauss-Legendre nodes, polish with Newton on that system.
    x0, w0 = gauss_legendre01(8)
    z = [x for x in x0] + [w * x for w, x in zip(w0, x0)]
    z = _newton(lambda q: _ggq_residual(q, mp.mpf(8)), z)
    # For integer t <= 7 the two families overlap (r^(k+t) is already a
    # polynomial of degree <= 7), so the path is sampled between integers.
    steps = 64
    for i in range(1, steps + 1):
        t = mp.mpf(8) * (steps - i + mp.mpf(1) / 2) / steps
        z = _newton(lambda q: _ggq_residual(q, t), z)
    z = _newton(lambda q: _ggq_residual(q, 0), z)
    return z[:8], z[8:]


def what_for(X, Y, W, degree):
    """Largest weight among the ceil((N+1)/2) nodes nearest each edge; max over edges."""
    k = (degree + 2) // 2
    best = mp.mpf(0)
    n = len(X)
    for e in range(3):
        if e == 0:
            dist = [Y[i] for i in range(n)]                         # edge y = 0
        elif e == 1:
            dist = [X[i] for i in range(n)]                         # edge x = 0
        else:
            dist = [(1 - X[i] - Y[i]) / mp.sqrt(2) for i in range(n)]  # edge x + y = 1
        order = sorted(range(n), key=lambda i: (dist[i], i))[:k]
        best = max(best, max(W[i] for i in order))
    return best


def conical_rule(degree):
    """Conical-product Gauss far rule of total degree `degree` (Section 4.2's
    higher far orders): m = (degree + 3) // 2 Gauss-Legendre points u_i with
    weights a_i on [0, 1]; node k = i m + j at (u_i, (1 - u_i) u_j) with weight
    a_i a_j (1 - u_i), the collapse (u, v) -> (u, (1 - u) v) of the square onto
    the simplex, exact for total degree 2m - 2.

    w-hat (Eq. rho0): over the three edges, the largest weight among the
    (degree + 2) // 2 nodes nearest the edge, nodes whose distance equals that
    of the last of them to 1e-9 relative included (the product structure ties
    distances exactly, so an index tie-break would depend on rounding).
    Returns a dict of floats: x, y, w, degree, what."""
    m = (degree + 3) // 2
    X, Y, W = duffy_rule(m)
    k = (degree + 2) // 2
    best = mp.mpf(0)
    n = len(X)
    for e in range(3):
        if e == 0:
            dist = list(Y)
        elif e == 1:
            dist = list(X)
        else:
            dist = [(1 - X[i] - Y[i]) / mp.sqrt(2) for i in range(n)]
        cut = sorted(dist)[k - 1] * (1 + mp.mpf(10) ** -9)
        best = max(best, max(W[i] for i in range(n) if dist[i] <= cut))
    return dict(degree=degree, x=[float(v) for v in X], y=[float(v) for v in Y], w=[float(v) for v in W],
                what=float(best))


def _shifted_legendre_coeffs(n):
    # P_n(2x-1) = sum_k (-1)^(n+k) C(n,k) C(n+k,k) x^k
    return [Fraction((-1) ** (n + k) * math.comb(n, k) * math.comb(n + k, k)) for k in range(n + 1)]


def oracle_basis(deg=4):
    idx = [(a, n - a) for n in range(deg + 1) for a in range(n, -1, -1)]
    coef = {n: _shifted_legendre_coeffs(n) for n in range(deg + 1)}

    def integ(a, b, c, e):
        px = [Fraction(0)] * (a + c + 1)
        for i, ci in enumerate(coef[a]):
            for j, cj in enumerate(coef[c]):
                px[i + j] += ci * cj
        py = [Fraction(0)] * (b + e + 1)
        for i, ci in enumerate(coef[b]):
            for j, cj in enumerate(coef[e]):
                py[i + j] += ci * cj
        s = Fraction(0)
        for i, ci in enumerate(px):
            if ci == 0:
                continue
            for j, cj in enumerate(py):
                if cj == 0:
                    continue
                s += ci * cj * Fraction(math.factorial(i) * math.factorial(j), math.factorial(i + j + 2))
        return s

    n = len(idx)
    G = mp.matrix(n, n)
    for r in range(n):
        for c in range(n):
            a, b = idx[r]
            cc, e = idx[c]
            v = integ(a, b, cc, e)
            G[r, c] = mp.mpf(v.numerator) / v.denominator
    L = mp.cholesky(G)
    Linv = mp.inverse(L)
    return idx, [[Linv[r, c] if c <= r else mp.mpf(0) for c in range(n)] for r in range(n)]


def _hx(v):
    return float(v).hex()


def main(path=None):
    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "rules_oracle.json")
    out = {}
    for name, n in [("gl16", 16), ("gl7", 7)]:
        x, w = gauss_legendre01(n)
        out[name] = dict(x=[_hx(v) for v in x], w=[_hx(v) for v in w])
    r = symmetric_far_rule(12)
    out["near33"] = dict(degree=12, x=[_hx(v) for v in r["x"]], y=[_hx(v) for v in r["y"]],
                         w=[_hx(v) for v in r["w"]], what=_hx(r["what"]))
    for name, spec in FAR_START.items():
        X, Y, W = symmetric_rule(spec)
        out[name] = dict(degree=spec["degree"], x=[_hx(v) for v in X], y=[_hx(v) for v in Y],
                         w=[_hx(v) for v in W], what=_hx(what_for(X, Y, W, spec["degree"])))
    for d in sorted(_far_sym_defs()):
        r = symmetric_far_rule(d)
        out[f"sym{d}"] = dict(degree=d, x=[_hx(v) for v in r["x"]], y=[_hx(v) for v in r["y"]],
                              w=[_hx(v) for v in r["w"]], what=_hx(r["what"]))
    r, om = ggq8()
    out["ggq8"] = dict(r=[_hx(v) for v in r], w=[_hx(v) for v in om])
    idx, Linv = oracle_basis(4)
    out["basis"] = dict(index=idx, Linv=[[_hx(v) for v in row] for row in Linv])
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    return path


if __name__ == "__main__":
    print(main())
