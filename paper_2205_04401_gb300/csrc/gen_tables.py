"""Writes vp_tables.h: the quadrature constants compiled into libvp.

The rules are the ones the method needs (Sections 3.2-3.4 and 5.1 of Shen &
Serkh, arXiv 2205.04401), derived here from their moment equations in
50-digit arithmetic and rounded once to double:

  far16   S3-symmetric 16-point rule of degree 8 on the reference simplex
  far19   S3-symmetric 19-point rule of degree 9
  near33  the S3-symmetric 33-point rule of degree 12 (the near rule, Section 5.1)
  sym<n>  S3-symmetric far rules of degree n = 12, 20, 25, 30, 40, 50 (Section 4.2),
          from the orbit definitions in sym_rule_defs.py
  ggq8    8-point generalized Gaussian rule on [0,1] for r p(r), r log(r) p(r), p in P_7
  gl16    16-point Gauss-Legendre rule on [0,1]
  what    largest weight among the ceil((N+1)/2) nodes nearest an edge (max over edges)

Symmetric orbits are listed centroid first, then S21(a) as (a,1-2a),
(1-2a,a), (a,a), then S111(a,b,c=1-a-b) as the (l2,l3) entries of the
barycentric permutations abc, acb, bac, bca, cab, cba.  The start values
below select the positive-interior root of each system.

Run once when a rule changes:  python paper_2205_04401_gb300/csrc/gen_tables.py
(needs mpmath; the generated header is committed).
"""
import math
from fractions import Fraction
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 50

START = {
    "far16": (8, 0.0722, [(0.0505, 0.0162), (0.4593, 0.0475), (0.1706, 0.0516)], [(0.0084, 0.2631, 0.0136)]),
    "far19": (9, 0.0486, [(0.0447, 0.0128), (0.1882, 0.0398), (0.4371, 0.0389), (0.4897, 0.0157)],
              [(0.0368, 0.2220, 0.0216)]),
}


def shifted_legendre(n, t):
    """P~_n(t) = P_n(2t-1) and its t-derivative by the three-term recurrences."""
    x = 2 * t - 1
    p_prev, p = mp.mpf(1), x
    d_prev, d = mp.mpf(0), mp.mpf(2)
    if n == 0:
        return mp.mpf(1), mp.mpf(0)
    for k in range(1, n):
        p_next = ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
        d_next = d_prev + 2 * (2 * k + 1) * p
        p_prev, p = p, p_next
        d_prev, d = d, d_next
    return p, d


def gl01(n):
    # Golub-Welsch guess in double, Newton polish in mpmath
    beta = np.array([k / math.sqrt(4.0 * k * k - 1.0) for k in range(1, n)])
    guess = np.sort(np.linalg.eigvalsh(np.diag(beta, 1) + np.diag(beta, -1)))
    ts, ws = [], []
    for g in guess:
        t = mp.mpf((g + 1) / 2)
        for _ in range(60):
            p, d = shifted_legendre(n, t)
            step = p / d
            t -= step
            if abs(step) < mp.mpf(10) ** -45:
                break
        p, d = shifted_legendre(n, t)
        ts.append(t)
        ws.append(1 / (t * (1 - t) * d * d))
    return ts, ws


def duffy(n):
    u, a = gl01(n)
    pts = []
    for i in range(n):
        for j in range(n):
            pts.append((u[i], (1 - u[i]) * u[j], a[i] * a[j] * (1 - u[i])))
    return pts


def orbit_points(c0, s21, s111):
    third = mp.mpf(1) / 3
    pts = [(third, third, c0)]
    for a, w in s21:
        b = 1 - 2 * a
        pts += [(a, b, w), (b, a, w), (a, a, w)]
    for a, b, w in s111:
        c = 1 - a - b
        for l1, l2, l3 in ((a, b, c), (a, c, b), (b, a, c), (b, c, a), (c, a, b), (c, b, a)):
            pts.append((l2, l3, w))
    return pts


def solve_symmetric(deg, c0, s21, s111):
    """Levenberg-Marquardt on all moments x^i y^j, i + j <= deg, with the
    Jacobian taken analytically from the orbit parametrisation."""
    mono = [(i, n - i) for n in range(deg + 1) for i in range(n + 1)]
    exact = [mp.mpf(math.factorial(i) * math.factorial(j)) / math.factorial(i + j + 2) for i, j in mono]
    n21, n111 = len(s21), len(s111)
    p = [mp.mpf(c0)] + [mp.mpf(v) for a, w in s21 for v in (a, w)] + [mp.mpf(v) for a, b, w in s111 for v in (a, b, w)]

    def unpack(p):
        s2 = [(p[1 + 2 * i], p[2 + 2 * i]) for i in range(n21)]
        o = 1 + 2 * n21
        s3 = [(p[o + 3 * i], p[o + 3 * i + 1], p[o + 3 * i + 2]) for i in range(n111)]
        return p[0], s2, s3

    def mom(x, y, i, j):
        return x ** i * y ** j

    def dmom(x, y, i, j):
        dx = i * x ** (i - 1) * y ** j if i > 0 else mp.mpf(0)
        dy = j * x ** i * y ** (j - 1) if j > 0 else mp.mpf(0)
        return dx, dy

    def resid_jac(p):
        c0_, s2, s3 = unpack(p)
        R = []
        Jm = []
        for (i, j), ex in zip(mono, exact):
            row = [mp.mpf(0)] * len(p)
            third = mp.mpf(1) / 3
            val = c0_ * mom(third, third, i, j)
            row[0] = mom(third, third, i, j)
            for k, (a, w) in enumerate(s2):
                b = 1 - 2 * a
                for (x, y, dxa, dya) in ((a, b, 1, -2), (b, a, -2, 1), (a, a, 1, 1)):
                    m = mom(x, y, i, j)
                    dx, dy = dmom(x, y, i, j)
                    val += w * m
                    row[1 + 2 * k] += w * (dx * dxa + dy * dya)
                    row[2 + 2 * k] += m
            o = 1 + 2 * n21
            for k, (a, b_, w) in enumerate(s3):
                c = 1 - a - b_
                # (l2, l3) and their derivatives w.r.t. a and b (c = 1 - a - b)
                perms = (((b_, c), (0, -1), (1, -1)), ((c, b_), (-1, 0), (-1, 1)), ((a, c), (1, -1), (0, -1)),
                         ((c, a), (-1, 1), (-1, 0)), ((a, b_), (1, 0), (0, 1)), ((b_, a), (0, 1), (1, 0)))
                for (x, y), (dxa, dya), (dxb, dyb) in perms:
                    m = mom(x, y, i, j)
                    dx, dy = dmom(x, y, i, j)
                    val += w * m
                    row[o + 3 * k] += w * (dx * dxa + dy * dya)
                    row[o + 3 * k + 1] += w * (dx * dxb + dy * dyb)
                    row[o + 3 * k + 2] += m
            R.append(val - ex)
            Jm.append(row)
        return mp.matrix(R), mp.matrix(Jm)

    lam = mp.mpf(10) ** -3
    for _ in range(200):
        R, Jm = resid_jac(p)
        A = Jm.T * Jm
        g = Jm.T * R
        for d in range(A.rows):
            A[d, d] *= (1 + lam)
        step = mp.lu_solve(A, g)
        trial = [p[c] - step[c] for c in range(len(p))]
        R2, _ = resid_jac(trial)
        if mp.norm(R2) < mp.norm(R):
            p = trial
            lam = max(lam / 10, mp.mpf(10) ** -40)
        else:
            lam *= 10
        if mp.norm(step) < mp.mpf(10) ** -40:
            break
    R, _ = resid_jac(p)
    assert mp.norm(R) < mp.mpf(10) ** -40
    c0_, s2, s3 = unpack(p)
    return orbit_points(c0_, s2, s3)


def _sym_defs():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "sym_rule_defs", os.path.join(os.path.dirname(os.path.abspath(__file__)), "sym_rule_defs.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.SYM_RULES


def e23_moment(i, j):
    """Exact integral over the reference simplex of e2^i e3^j, e2 = l1 l2 +
    l1 l3 + l2 l3 and e3 = l1 l2 l3 of the barycentric coordinates, from
    int l1^a l2^b l3^c = a! b! c! / (a + b + c + 2)! and the multinomial
    expansion of e2^i."""
    f = math.factorial
    tot = Fraction(0)
    for p1 in range(i + 1):
        for p2 in range(i - p1 + 1):
            p3 = i - p1 - p2
            mult = f(i) // (f(p1) * f(p2) * f(p3))
            tot += Fraction(mult * f(p1 + p2 + j) * f(p1 + p3 + j) * f(p2 + p3 + j), f(2 * i + 3 * j + 2))
    return tot


def solve_sym_e23(deg, rule):
    """S3-symmetric rule of degree deg from its orbit definition (sym_rule_defs):
    Newton's method in 90-digit arithmetic on the moment equations of the
    invariant basis e2^i e3^j, 2i + 3j <= deg (on the plane l1 + l2 + l3 = 1
    these span the S3-invariant polynomials of degree <= deg, so they are all
    the conditions of a symmetric rule).  Orbit sums by one representative:
    centroid (weight w0), S21(a) = (a, a, 1 - 2a) x 3, S111(a, b) =
    (a, b, 1 - a - b) x 6.  Parameters listed in rule["fixed"] keep their
    listed values.  Returns [(x, y, w)] in orbit order."""
    with mp.workdps(90):
        idx = [(i, j) for i in range(deg // 2 + 1) for j in range((deg - 2 * i) // 3 + 1)]
        exact = []
        for i, j in idx:
            q = e23_moment(i, j)
            exact.append(mp.mpf(q.numerator) / q.denominator)
        kinds = ([0] if rule["w0"] is not None else []) + [1] * len(rule["s21"]) + [2] * len(rule["s111"])
        p = ([mp.mpf(rule["w0"])] if rule["w0"] is not None else []) + \
            [mp.mpf(v) for o in rule["s21"] for v in o] + [mp.mpf(v) for o in rule["s111"] for v in o]
        free = [c for c in range(len(p)) if c not in rule["fixed"]]
        assert len(free) == len(idx), (deg, len(free), len(idx))

        def orbit(c, k):
            if k == 0:
                t = mp.mpf(1) / 3
                return (t, t, t), [], 1, p[c], 1
            if k == 1:
                a = p[c]
                return (a, a, 1 - 2 * a), [(1, 1, -2)], 3, p[c + 1], 2
            a, b = p[c], p[c + 1]
            return (a, b, 1 - a - b), [(1, 0, -1), (0, 1, -1)], 6, p[c + 2], 3

        def system():
            R = [-v for v in exact]
            J = [[mp.mpf(0)] * len(p) for _ in idx]
            c = 0
            for k in kinds:
                lam, dirs, mult, w, n = orbit(c, k)
                e2 = lam[0] * lam[1] + lam[0] * lam[2] + lam[1] * lam[2]
                e3 = lam[0] * lam[1] * lam[2]
                de2 = (lam[1] + lam[2], lam[0] + lam[2], lam[0] + lam[1])
                de3 = (lam[1] * lam[2], lam[0] * lam[2], lam[0] * lam[1])
                g2 = [sum(de2[q] * d[q] for q in range(3)) for d in dirs]
                g3 = [sum(de3[q] * d[q] for q in range(3)) for d in dirs]
                for r, (i, j) in enumerate(idx):
                    v = e2 ** i * e3 ** j
                    R[r] += mult * w * v
                    di = i * e2 ** (i - 1) * e3 ** j if i else 0
                    dj = j * e2 ** i * e3 ** (j - 1) if j else 0
                    for s_, _ in enumerate(dirs):
                        J[r][c + s_] += mult * w * (di * g2[s_] + dj * g3[s_])
                    J[r][c + n - 1] += mult * v
                c += n
            return R, J

        for _ in range(40):
            R, J = system()
            dx = mp.lu_solve(mp.matrix([[J[r][c] for c in free] for r in range(len(idx))]), mp.matrix(R))
            for s_, c in enumerate(free):
                p[c] -= dx[s_]
            if max(abs(v) for v in dx) < mp.mpf(10) ** -60:   # far below double precision
                break
        R, _ = system()
        assert max(abs(v) for v in R) < mp.mpf(10) ** -60, deg
        pts = []
        c = 0
        for k in kinds:
            lam, _, _, w, n = orbit(c, k)
            if k == 0:
                pts.append((lam[1], lam[2], w))
            elif k == 1:
                a = lam[0]
                pts += [(a, 1 - 2 * a, w), (1 - 2 * a, a, w), (a, a, w)]
            else:
                a, b, cc = lam
                for l1, l2, l3 in ((a, b, cc), (a, cc, b), (b, a, cc), (b, cc, a), (cc, a, b), (cc, b, a)):
                    pts.append((l2, l3, w))
            c += n
        assert all(w > 0 and x > 0 and y > 0 and 1 - x - y > 0 for x, y, w in pts), deg
        return pts


def radial5():
    """Interpolatory radial rule of the self-interaction on the 5 Gauss-Legendre
    nodes r_i of [0, 1]: weights a_i, b_i with sum_i a_i p(r_i) = int_0^1 r p(r) dr
    and sum_i b_i p(r_i) = int_0^1 r log(r) p(r) dr for every p of degree <= 4
    (moments 1 / (k + 2) and -1 / (k + 2)^2).  Along a ray the P_4 moments of
    Section 3.4 need no more: the integrand is r log(r r0) times a polynomial of
    degree <= 4 in r, for which this rule and the GGQ rule of order 8 are both
    exact."""
    r, _ = gl01(5)
    V = mp.matrix([[ri ** k for ri in r] for k in range(5)])
    a = mp.lu_solve(V, mp.matrix([mp.mpf(1) / (k + 2) for k in range(5)]))
    b = mp.lu_solve(V, mp.matrix([-mp.mpf(1) / (k + 2) ** 2 for k in range(5)]))
    return r, [a[i] for i in range(5)], [b[i] for i in range(5)]


def ggq8():
    """8-node generalized Gaussian rule for {r^k, r^k log r}, k = 0..7, with
    the weight r on [0,1].  Unknowns are log r_j and log w_j (positivity is
    kept by construction).  Continuation from the Gauss rule for the weight
    r (t = 8) through the Muntz-type family r^k (r^t - 1)/t on the geometric
    schedule t = 8 exp(-i/10), which never lands on an integer, to t = 0."""
    def funcs(r, k, t):
        if t == 0:
            return r ** k * mp.log(r), k * r ** (k - 1) * mp.log(r) + r ** (k - 1) if k > 0 else 1 / r
        f = r ** k * (r ** t - 1) / t
        df = (((k + t) * r ** (k + t - 1)) - (k * r ** (k - 1) if k > 0 else 0)) / t
        return f, df

    def moments(k, t):
        return mp.mpf(1) / (k + 2), (-1 / (mp.mpf(k + 2) ** 2) if t == 0 else -1 / ((k + 2) * (k + 2 + t)))

    def system(u, t):
        r = [mp.exp(v) for v in u[:8]]
        w = [mp.exp(v) for v in u[8:]]
        F = mp.matrix(16, 1)
        J = mp.matrix(16, 16)
        for k in range(8):
            m1, m2 = moments(k, t)
            F[k] = mp.fsum(w[j] * r[j] ** k for j in range(8)) - m1
            F[8 + k] = mp.fsum(w[j] * funcs(r[j], k, t)[0] for j in range(8)) - m2
            for j in range(8):
                dpk = k * r[j] ** (k - 1) if k > 0 else mp.mpf(0)
                f, df = funcs(r[j], k, t)
                J[k, j] = w[j] * dpk * r[j]           # d/du_j with r = e^u
                J[k, 8 + j] = w[j] * r[j] ** k        # d/dv_j with w = e^v
                J[8 + k, j] = w[j] * df * r[j]
                J[8 + k, 8 + j] = w[j] * f
        return F, J

    def solve(u, t, tol=mp.mpf(10) ** -20):
        for _ in range(100):
            F, J = system(u, t)
            du = mp.lu_solve(J, F)
            u = [u[c] - du[c] for c in range(16)]
            if mp.norm(du) < tol:
                return u
        raise RuntimeError("ggq continuation failed at t=%s" % t)

    # Gauss rule for the weight r on [0,1] from the Jacobi(0,1) Golub-Welsch matrix
    n = 8
    diag = [1.0 / ((2 * k + 1) * (2 * k + 3)) for k in range(n)]
    off = [2.0 / (2 * k + 1) * math.sqrt(k * k * (k + 1) * (k + 1) / ((2 * k + 1) ** 2 - 1)) for k in range(1, n)]
    ev, V = np.linalg.eigh(np.diag(diag) + np.diag(off, 1) + np.diag(off, -1))
    u = [mp.log(mp.mpf((e + 1) / 2)) for e in ev] + [mp.log(mp.mpf(0.5 * V[0, i] ** 2)) for i in range(n)]
    u = solve(u, mp.mpf(8))
    for i in range(1, 91):
        u = solve(u, 8 * mp.exp(-mp.mpf(i) / 10))
    u = solve(u, 0, mp.mpf(10) ** -42)
    return [mp.exp(v) for v in u[:8]], [mp.exp(v) for v in u[8:]]


def what(pts, degree):
    k = (degree + 2) // 2
    best = mp.mpf(0)
    for e in range(3):
        key = []
        for idx, (x, y, w) in enumerate(pts):
            d = y if e == 0 else (x if e == 1 else (1 - x - y) / mp.sqrt(2))
            key.append((d, idx, w))
        key.sort(key=lambda t: (t[0], t[1]))
        best = max(best, max(t[2] for t in key[:k]))
    return best


def legendre_tensor_index():
    """Basis of P_4 used on the device: L_ab(x, y) = P_a(3x - 1) P_b(3y - 1), a + b <= 4,
    ordered by total degree n = a + b, then a from n down to 0."""
    return [(a, n - a) for n in range(5) for a in range(n, -1, -1)]


def _legendre_poly_coeffs(n):
    """Monomial coefficients of P_n(t) (Bonnet recurrence, exact rationals)."""
    from fractions import Fraction
    p0, p1 = [Fraction(1)], [Fraction(0), Fraction(1)]
    if n == 0:
        return p0
    for k in range(1, n):
        nxt = [Fraction(0)] * (k + 2)
        for i, c in enumerate(p1):
            nxt[i + 1] += Fraction(2 * k + 1, k + 1) * c
        for i, c in enumerate(p0):
            nxt[i] -= Fraction(k, k + 1) * c
        p0, p1 = p1, nxt
    return p1


def leg15_gram_inverse():
    """Inverse of the Gram matrix H_ij = int L_i L_j dA of the tensor-Legendre
    basis over the reference simplex (exact rationals, then inverted)."""
    from fractions import Fraction
    idx = legendre_tensor_index()
    # L_ab as polynomials in (x, y): P_a(3x - 1) expanded to monomials
    def shifted(n):
        c = _legendre_poly_coeffs(n)
        out = [Fraction(0)] * (n + 1)
        for k, ck in enumerate(c):          # ck (3x - 1)^k
            for j in range(k + 1):
                out[j] += ck * math.comb(k, j) * Fraction(3) ** j * Fraction(-1) ** (k - j)
        return out
    sp = {n: shifted(n) for n in range(5)}
    def gram(i, j):
        (a, b), (c, d) = idx[i], idx[j]
        px = [Fraction(0)] * (a + c + 1)
        for u, cu in enumerate(sp[a]):
            for v, cv in enumerate(sp[c]):
                px[u + v] += cu * cv
        py = [Fraction(0)] * (b + d + 1)
        for u, cu in enumerate(sp[b]):
            for v, cv in enumerate(sp[d]):
                py[u + v] += cu * cv
        tot = Fraction(0)
        for u, cu in enumerate(px):
            for v, cv in enumerate(py):
                tot += cu * cv * Fraction(math.factorial(u) * math.factorial(v), math.factorial(u + v + 2))
        return tot
    n = len(idx)
    H = mp.matrix(n, n)
    for i in range(n):
        for j in range(n):
            g = gram(i, j)
            H[i, j] = mp.mpf(g.numerator) / g.denominator
    Hinv = mp.inverse(H)
    return Hinv


def mon15_gram_inverse():
    """Inverse of the Gram matrix of the monomial basis M_ab(x, y) = u^a v^b,
    u = 3x - 1, v = 3y - 1, a + b <= 4, in the order of the tensor-Legendre
    basis (exact rationals, then inverted).  The float-float weight kernels
    accumulate their moments in this basis (cheaper products, smaller values
    on the simplex and a better-conditioned Gram matrix than L_ab)."""
    from fractions import Fraction
    idx = legendre_tensor_index()

    def expand(a):      # (3x - 1)^a = sum_j C(a, j) 3^j (-1)^(a - j) x^j
        return [Fraction(math.comb(a, j) * 3 ** j * (-1) ** (a - j)) for j in range(a + 1)]

    ex = {a: expand(a) for a in range(5)}

    def gram(i, j):
        (a, b), (c, d) = idx[i], idx[j]
        px = [Fraction(0)] * (a + c + 1)
        for p1, c1 in enumerate(ex[a]):
            for p2, c2 in enumerate(ex[c]):
                px[p1 + p2] += c1 * c2
        py = [Fraction(0)] * (b + d + 1)
        for p1, c1 in enumerate(ex[b]):
            for p2, c2 in enumerate(ex[d]):
                py[p1 + p2] += c1 * c2
        tot = Fraction(0)
        for u, cu in enumerate(px):
            for v, cv in enumerate(py):
                tot += cu * cv * Fraction(math.factorial(u) * math.factorial(v), math.factorial(u + v + 2))
        return tot
    n = len(idx)
    H = mp.matrix(n, n)
    for i in range(n):
        for j in range(n):
            g = gram(i, j)
            H[i, j] = mp.mpf(g.numerator) / g.denominator
    return mp.inverse(H)


def projection_matrix_mon(pts):
    """QM[k][i] = w_k sum_j HMinv[i][j] M_j(x_k, y_k): the map of
    projection_matrix for moments in the monomial basis M_ab."""
    idx = legendre_tensor_index()
    n = len(idx)
    Hinv = mon15_gram_inverse()
    Q = []
    for x, y, w in pts:
        m = [(3 * x - 1) ** a * (3 * y - 1) ** b for a, b in idx]
        Q.append([w * mp.fsum(Hinv[i, j] * m[j] for j in range(n)) for i in range(n)])
    return Q


def projection_matrix(pts):
    """Q[k][i] = w_k sum_j Hinv[i][j] L_j(x_k, y_k): maps the moments
    mu_i = int_T G L_i(rho_T^-1 y) dA to the nodal correction weights of the
    discrete L2 projection onto P_4 with the far rule (exact Gram H, since
    the rule has degree >= 8)."""
    idx = legendre_tensor_index()
    n = len(idx)
    Hinv = leg15_gram_inverse()
    def L(x, y):
        def P(k, t):
            return sum(c * t ** e for e, c in enumerate(_legendre_poly_coeffs(k)))
        return [P(a, 3 * x - 1) * P(b, 3 * y - 1) for a, b in idx]
    Q = []
    for x, y, w in pts:
        l = L(x, y)
        Q.append([w * mp.fsum(Hinv[i, j] * l[j] for j in range(n)) for i in range(n)])
    return Q


def cdbl(v):
    return float(v).hex()


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    out = ["/* Generated by gen_tables.py - quadrature constants of the method. Do not edit. */",
           "#pragma once", ""]

    def arr(name, vals):
        out.append(f"static const double {name}[{len(vals)}] = {{")
        for i in range(0, len(vals), 4):
            out.append("  " + ", ".join(cdbl(v) for v in vals[i:i + 4]) + ",")
        out.append("};")

    for name in ("far16", "far19"):
        deg, c0, s21, s111 = START[name]
        pts = solve_symmetric(deg, c0, s21, s111)
        Q = projection_matrix(pts)
        arr(f"VP_{name.upper()}_Q", [v for row in Q for v in row])
        QM = projection_matrix_mon(pts)
        arr(f"VP_{name.upper()}_QM", [v for row in QM for v in row])
        arr(f"VP_{name.upper()}_X", [p[0] for p in pts])
        arr(f"VP_{name.upper()}_Y", [p[1] for p in pts])
        arr(f"VP_{name.upper()}_W", [p[2] for p in pts])
        out.append(f"static const double VP_{name.upper()}_WHAT = {cdbl(what(pts, deg))};")
        out.append(f"static const int VP_{name.upper()}_DEGREE = {deg};")
    sym = _sym_defs()
    for deg in sorted(sym):
        pts = solve_sym_e23(deg, sym[deg])
        arr(f"VP_SYM{deg}_X", [q[0] for q in pts])
        arr(f"VP_SYM{deg}_Y", [q[1] for q in pts])
        arr(f"VP_SYM{deg}_W", [q[2] for q in pts])
        out.append(f"static const double VP_SYM{deg}_WHAT = {cdbl(what(pts, deg))};")
    out.append("struct VpSymRule { int degree, n; const double *x, *y, *w; double what; };")
    out.append(f"static const VpSymRule VP_SYM_RULES[{len(sym)}] = {{")
    for deg in sorted(sym):
        n = (1 if sym[deg]["w0"] is not None else 0) + 3 * len(sym[deg]["s21"]) + 6 * len(sym[deg]["s111"])
        out.append(f"  {{{deg}, {n}, VP_SYM{deg}_X, VP_SYM{deg}_Y, VP_SYM{deg}_W, VP_SYM{deg}_WHAT}},")
    out.append("};")
    Hinv = leg15_gram_inverse()
    arr("VP_LEG15_HINV", [Hinv[i, j] for i in range(Hinv.rows) for j in range(Hinv.cols)])
    Hinv = mon15_gram_inverse()
    arr("VP_MON15_HINV", [Hinv[i, j] for i in range(Hinv.rows) for j in range(Hinv.cols)])
    pts = solve_sym_e23(12, sym[12])        # the near rule: the symmetric rule of degree 12
    arr("VP_NEAR33_X", [p[0] for p in pts])
    arr("VP_NEAR33_Y", [p[1] for p in pts])
    arr("VP_NEAR33_W", [p[2] for p in pts])
    out.append(f"static const double VP_NEAR33_WHAT = {cdbl(what(pts, 12))};")
    out.append("static const int VP_NEAR33_DEGREE = 12;")
    r, w = ggq8()
    arr("VP_GGQ8_R", r)
    arr("VP_GGQ8_W", w)
    r, a, b = radial5()
    arr("VP_RAD5_R", r)
    arr("VP_RAD5_A", a)
    arr("VP_RAD5_B", b)
    t, w = gl01(16)
    arr("VP_GL16_X", t)
    arr("VP_GL16_W", w)
    # FP64 logarithm table: c_i = 1 + (i + 1/2)/128, 1/c_i and log c_i
    cs = [1 + (mp.mpf(i) + mp.mpf(1) / 2) / 128 for i in range(128)]
    arr("VP_LOG128_RC", [1 / c for c in cs])
    arr("VP_LOG128_L", [mp.log(c) for c in cs])
    out.append(f"static const double VP_LN2 = {cdbl(mp.log(2))};")
    path = os.path.join(here, "vp_tables.h")
    with open(path, "w") as fh:
        fh.write("\n".join(out) + "\n")
    print(path)


if __name__ == "__main__":
    main()
