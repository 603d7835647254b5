"""Pins for the oracle's quadrature tables against exact moments.

Every rule is checked against integrals computed here in exact rational
arithmetic (monomials on the reference simplex: i! j! / (i+j+2)!; on [0,1]:
1/(k+1) and -1/(k+1)^2), not against the generator's own equations.
"""
import math
from fractions import Fraction

import numpy as np
import pytest


def simplex_moment(i, j):
    return Fraction(math.factorial(i) * math.factorial(j), math.factorial(i + j + 2))


def max_moment_error(x, y, w, degree):
    err = 0.0
    for n in range(degree + 1):
        for i in range(n + 1):
            j = n - i
            q = float(np.sum(w * x ** i * y ** j))
            err = max(err, abs(q - float(simplex_moment(i, j))))
    return err


@pytest.mark.parametrize("name,n,degree", [("far16", 16, 8), ("far19", 19, 9), ("near33", 33, 12)])
def test_triangle_rule_exact(tables, name, n, degree):
    r = tables[name]
    x, y, w = r["x"], r["y"], r["w"]
    assert len(w) == n and r["degree"] == degree
    assert max_moment_error(x, y, w, degree) < 2e-16 * 8
    # positive weights, interior nodes (paper's X-G rules are positive-interior)
    assert np.all(w > 0)
    assert np.all(x > 0) and np.all(y > 0) and np.all(x + y < 1)
    # the rule is not exact one degree higher (it is a genuine degree-d rule)
    assert max_moment_error(x, y, w, degree + 1) > 1e-10


@pytest.mark.parametrize("name", ["far16", "far19", "near33"] + [f"sym{d}" for d in (12, 20, 25, 30, 40, 50)])
def test_far_rule_symmetric(tables, name):
    r = tables[name]
    pts = np.c_[1 - r["x"] - r["y"], r["x"], r["y"]]
    key = lambda b, w: (tuple(np.round(np.sort(b), 12)), round(w, 14))
    base = sorted(key(b, w) for b, w in zip(pts, r["w"]))
    for perm in [(1, 2, 0), (0, 2, 1)]:
        moved = sorted(key(b[list(perm)], w) for b, w in zip(pts, r["w"]))
        assert moved == base


@pytest.mark.parametrize("name,n", [("gl16", 16), ("gl7", 7)])
def test_gauss_legendre(tables, name, n):
    x, w = tables[name]["x"], tables[name]["w"]
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 4e-16


def test_ggq8(tables):
    """Eight nodes integrate r P_7 and r log r P_7 on [0,1] (Section 3.4)."""
    r, w = tables["ggq8"]["r"], tables["ggq8"]["w"]
    assert len(r) == 8 and np.all((r > 0) & (r < 1)) and np.all(w > 0)
    for k in range(8):
        assert abs(np.sum(w * r ** k) - 1.0 / (k + 2)) < 4e-16
        assert abs(np.sum(w * r ** k * np.log(r)) + 1.0 / (k + 2) ** 2) < 4e-16
    # a Gauss-Legendre rule of the same length cannot do the log family
    g = np.polynomial.legendre.leggauss(8)
    gx, gw = (g[0] + 1) / 2, g[1] / 2
    assert abs(np.sum(gw * gx * np.log(gx)) + 0.25) > 1e-6


def test_what(tables):
    """w of Eq. rho0: largest weight among the ceil((N+1)/2) nodes closest to
    an edge, max over edges (reading of the '~n/2 nodes' passage)."""
    for name in ["far16", "far19", "near33"]:
        r = tables[name]
        k = (r["degree"] + 2) // 2
        dists = [r["y"], r["x"], (1 - r["x"] - r["y"]) / np.sqrt(2)]
        best = 0.0
        for d in dists:
            order = np.lexsort((np.arange(len(d)), d))[:k]
            best = max(best, r["w"][order].max())
        assert r["what"] == best
        assert r["what"] <= r["w"].max() and 10 * r["what"] >= r["w"].max()


def test_oracle_basis_orthonormal(tables):
    """The oracle's P_4 basis is orthonormal on the reference simplex (degree
    8 products, integrated exactly by the degree-12 rule) and spans P_4."""
    from oracle.oracle import Oracle
    o = Oracle("far19", tables=tables)
    nr = tables["near33"]
    K = o.basis(nr["x"], nr["y"])
    Gm = (K * nr["w"][:, None]).T @ K
    assert np.abs(Gm - np.eye(15)).max() < 1e-13
    # spans P_4: every monomial of degree <= 4 is reproduced by its projection
    for n in range(5):
        for i in range(n + 1):
            mono = nr["x"] ** i * nr["y"] ** (n - i)
            c = K.T @ (nr["w"] * mono)
            assert np.abs(K @ c - mono).max() < 1e-12


def test_far_rule_projection_exact(tables):
    """The discrete L2 projection with the far rule has an identity Gram
    matrix (rule degree >= 8 = 2*4), so it reproduces P_4 exactly."""
    from oracle.oracle import Oracle
    o = Oracle("far19", tables=tables)
    fr = tables["far19"]
    K = o.basis(fr["x"], fr["y"])
    assert np.abs((K * fr["w"][:, None]).T @ K - np.eye(15)).max() < 1e-13


CONICAL = [8, 12, 20, 25, 30, 40, 50]


@pytest.mark.parametrize("degree", CONICAL)
def test_conical_rule_exact(degree):
    """Higher far orders for the offloading of Section 4.2: the conical-product
    rule of total degree n integrates every monomial of degree <= n exactly
    (closed form i! j! / (i + j + 2)!), has positive weights, interior nodes
    and m^2 nodes, m = (n + 3) // 2, in the documented order (k = i m + j)."""
    from oracle import gen_rules
    r = gen_rules.conical_rule(degree)
    x, y, w = (np.array(r[k]) for k in "xyw")
    m = (degree + 3) // 2
    assert len(w) == m * m and r["degree"] == degree
    assert np.all(w > 0) and np.all(x > 0) and np.all(y > 0) and np.all(x + y < 1)
    assert max_moment_error(x, y, w, degree) < 1e-15
    # the row structure: x constant along j, y / (1 - x) the same along i
    X, Y = x.reshape(m, m), y.reshape(m, m)
    assert np.all(X == X[:, :1]) and np.all(np.diff(X[:, 0]) > 0)
    assert np.abs(Y / (1 - X) - Y[0] / (1 - X[0])).max() < 1e-13


@pytest.mark.parametrize("degree", CONICAL)
def test_conical_what(degree):
    """w-hat of a conical rule is one of its weights and at least the largest
    weight of the row nearest the edge x = 0 (its (n + 2) // 2 nearest nodes
    all lie on that row, at the same distance u_0)."""
    from oracle import gen_rules
    r = gen_rules.conical_rule(degree)
    w = np.array(r["w"])
    m = (degree + 3) // 2
    assert r["what"] in set(w.tolist())
    assert r["what"] >= w[:m].max()
    assert r["what"] <= w.max()


def test_conical_projection_exact():
    """The P_4 projection with a conical far rule has an identity Gram matrix."""
    from oracle import gen_rules
    from oracle.oracle import Oracle
    r = gen_rules.conical_rule(20)
    o = Oracle(r)
    x, y, w = (np.array(r[k]) for k in "xyw")
    K = o.basis(x, y)
    assert np.abs((K * w[:, None]).T @ K - np.eye(15)).max() < 1e-13


# S3-symmetric far rules of Section 4.2's orders, with the node counts of the
# orbit structures (the paper's Xiao-Gimbutas rules: 32 at degree 12, 290 at
# 40, 444 at 50; the conical rules of the same degrees have 49 ... 676).
SYM = {12: 33, 20: 81, 25: 124, 30: 175, 40: 295, 50: 453}


def exact_moment_error(x, y, w, degree):
    """max over x^i y^j, i + j <= degree, of |sum w x^i y^j - i! j! / (i+j+2)!|
    relative to the moment, the sum taken exactly from the stored doubles."""
    X = [Fraction(v) for v in x]
    Y = [Fraction(v) for v in y]
    W = [Fraction(v) for v in w]
    err = 0.0
    px = [[Fraction(1)] * len(X)]
    for _ in range(degree):
        px.append([a * b for a, b in zip(px[-1], X)])
    py = [[Fraction(1)] * len(Y)]
    for _ in range(degree):
        py.append([a * b for a, b in zip(py[-1], Y)])
    for n in range(degree + 1):
        for i in range(n + 1):
            j = n - i
            q = sum(wk * a * b for wk, a, b in zip(W, px[i], py[j]))
            ex = simplex_moment(i, j)
            err = max(err, float(abs(q - ex) / ex))
    return err


@pytest.mark.parametrize("degree", sorted(SYM))
def test_symmetric_rule_exact(tables, degree):
    """The S3-symmetric far rule of each sweep degree: every monomial of degree
    <= n integrated to rounding (the sum of the stored doubles in exact
    arithmetic against i! j! / (i + j + 2)!), positive weights, nodes strictly
    inside, the stated node count, and not exact one degree higher."""
    r = tables[f"sym{degree}"]
    x, y, w = r["x"], r["y"], r["w"]
    assert len(w) == SYM[degree] and r["degree"] == degree
    assert np.all(w > 0) and np.all(x > 0) and np.all(y > 0) and np.all(x + y < 1)
    # positive terms: the rounding of the stored nodes moves each moment by a
    # few units of 1e-16 relative, whatever its size
    assert exact_moment_error(x, y, w, degree) < 1e-13
    assert max_moment_error(x, y, w, degree + 1) > 1e-17


def test_near_rule_is_sym12(tables):
    """The near rule (order 12, Section 5.1) is the degree-12 symmetric rule."""
    a, b = tables["near33"], tables["sym12"]
    for k in "xyw":
        assert np.array_equal(a[k], b[k])
    assert a["what"] == b["what"]


@pytest.mark.parametrize("degree", sorted(SYM))
def test_symmetric_what(tables, degree):
    """w-hat (Eq. rho0) of a symmetric rule is one of its weights: the largest
    among the (n + 2) // 2 nodes nearest the edge y = 0 (all three edges give
    the same by symmetry), found here by sorting the distances directly."""
    r = tables[f"sym{degree}"]
    k = (degree + 2) // 2
    order = np.lexsort((np.arange(len(r["y"])), r["y"]))[:k]
    assert r["what"] == r["w"][order].max()
