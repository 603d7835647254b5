"""CPU oracle for interpolating the volume potential over a mesh (Section 3.5)
and for the staggered-mesh experiment of Section 4.3.

TEST INFRASTRUCTURE ONLY: the tests and bench.py's CPU-baseline leg call
this; the library never does.  Plain numpy/scipy, FP64, no code shared with
the CUDA path.

Section 3.5: on an element Delta with map rho from the standard simplex, the
Koornwinder expansion of u o rho of degree N_s is obtained from the values
of u at N_s-th order interpolation nodes of Delta (their number is
dim P_{N_s} = (N_s + 1)(N_s + 2)/2, Table "ord_len_interp") by the inverse
of the interpolation (Vandermonde) matrix, and u(x) = I(rho^{-1}(x)).

The paper's Vioreanu-Rokhlin nodes come from tables that are not available;
the nodes here are the Blyth-Pozrikidis construction applied to the N + 1
Gauss-Legendre points (an explicit, S3-symmetric set with the same count,
all inside the element like the Vioreanu-Rokhlin nodes): with
v_0 < ... < v_N those points mapped to [0, 1], node (i, j, k),
i + j + k = N, sits at
    x = (1 + 2 v_i - v_j - v_k) / 3,   y = (1 + 2 v_j - v_i - v_k) / 3,
which is (i/N, j/N) for equispaced v.  The condition numbers of their
interpolation matrices are 26.9 (N = 12) and 677 (N = 20), against 19.2 and
194 for the paper's rules (Table "ord_len_interp").
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import eval_jacobi


def dim_p(n: int) -> int:
    return (n + 1) * (n + 2) // 2


def koornwinder(N: int, x, y) -> np.ndarray:
    """K_mn(x, y) of Section 2.1 for 0 <= m <= n <= N at the points (x, y)
    of the standard simplex, column a = n (n + 1) / 2 + m:
        K_mn = c_mn (1 - x)^m P_{n-m}^{(2m+1, 0)}(2x - 1) P_m(2y / (1 - x) - 1),
    with c_mn = sqrt(2 (2m + 1)(n + 1)) (unit L2 norm on the simplex, pinned
    by the Gram-matrix test).  (1 - x)^m P_m(2y/(1 - x) - 1) is evaluated by
    Legendre's three-term recurrence in homogeneous form, which is defined at
    x = 1 as well."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    w = 1.0 - x
    s = 2.0 * y - w                    # (1 - x) (2y/(1 - x) - 1)
    H = [np.ones_like(x), s]           # (1 - x)^m P_m(...), m = 0, 1, ...
    for m in range(1, N):
        H.append(((2 * m + 1) * s * H[m] - m * w * w * H[m - 1]) / (m + 1))
    out = np.empty(x.shape + (dim_p(N),))
    for n in range(N + 1):
        for m in range(n + 1):
            c = math.sqrt(2.0 * (2 * m + 1) * (n + 1))
            out[..., n * (n + 1) // 2 + m] = c * H[m] * eval_jacobi(n - m, 2 * m + 1, 0, 2.0 * x - 1.0)
    return out


def gauss_points(n: int) -> np.ndarray:
    """The n Gauss-Legendre points on [-1, 1], ascending (roots of P_n)."""
    return np.sort(np.polynomial.legendre.legroots(np.eye(n + 1)[n]).real)


def interp_nodes(N: int):
    """The interpolation nodes of order N on the standard simplex, ordered
    by (j, i) with k = N - i - j: arrays x, y of length dim P_N."""
    v = 0.5 * (gauss_points(N + 1) + 1.0)
    xs, ys = [], []
    for j in range(N + 1):
        for i in range(N + 1 - j):
            k = N - i - j
            xs.append((1.0 + 2.0 * v[i] - v[j] - v[k]) / 3.0)
            ys.append((1.0 + 2.0 * v[j] - v[i] - v[k]) / 3.0)
    return np.array(xs), np.array(ys)


class Interpolator:
    """Section 3.5 on every element of an interpolation mesh (straight, or
    curved through the oracle's blending map)."""

    def __init__(self, oracle, vxy, tri, N: int, curves=None):
        from oracle.oracle import Oracle  # noqa: F401  (type only)
        self.o = oracle
        self.N = N
        self.nn = dim_p(N)
        self.vxy = np.ascontiguousarray(vxy, np.float64)
        self.curves = curves
        if curves is not None:
            self.tri, _, _, _ = oracle.nodes_curved(self.vxy, tri, curves)
        else:
            self.tri, _, _, _ = oracle.nodes(self.vxy, tri)
        self.nt = len(self.tri)
        self.zx, self.zy = interp_nodes(N)
        self.V = koornwinder(N, self.zx, self.zy)          # [node][basis]

    def nodes(self) -> np.ndarray:
        """Interpolation nodes of every element, [nt * nn][2], element-major."""
        T = np.repeat(np.arange(self.nt), self.nn)
        xi = np.tile(self.zx, self.nt)
        eta = np.tile(self.zy, self.nt)
        return self.map(T, xi, eta)

    def map(self, T, xi, eta) -> np.ndarray:
        if self.curves is not None:
            y, _ = self.o.map_curved(self.vxy, self.tri, self.curves, T, xi, eta)
            return y
        A = self.vxy[self.tri[T, 0]]
        B = self.vxy[self.tri[T, 1]]
        Cv = self.vxy[self.tri[T, 2]]
        return A + xi[:, None] * (B - A) + eta[:, None] * (Cv - A)

    def coeffs(self, u_nodes) -> np.ndarray:
        """Koornwinder coefficients [d][nt][nn] from node values [d][nt*nn]."""
        u = np.atleast_2d(np.asarray(u_nodes, np.float64))
        d = u.shape[0]
        U = u.reshape(d * self.nt, self.nn).T              # [nn][d*nt]
        c = np.linalg.solve(self.V, U)                     # [nn][d*nt]
        return c.T.reshape(d, self.nt, self.nn)

    def locate(self, pts):
        pts = np.ascontiguousarray(pts, np.float64)
        if self.curves is not None:
            return self.o.locate_curved(self.vxy, self.tri, self.curves, pts)
        return self.o.locate(self.vxy, self.tri, pts)

    def reference(self, T, pts):
        """rho_T^{-1}(x): the affine inverse, or Newton on curved elements."""
        T = np.asarray(T, np.int64)
        pts = np.asarray(pts, np.float64)
        if self.curves is not None:
            ref, _ = self.o.inverse_curved(self.vxy, self.tri, self.curves, T, pts)
            return ref[:, 0], ref[:, 1]
        A = self.vxy[self.tri[T, 0]]
        B = self.vxy[self.tri[T, 1]]
        Cv = self.vxy[self.tri[T, 2]]
        e, f, q = B - A, Cv - A, pts - A
        J = e[:, 0] * f[:, 1] - e[:, 1] * f[:, 0]
        xi = (q[:, 0] * f[:, 1] - q[:, 1] * f[:, 0]) / J
        eta = (e[:, 0] * q[:, 1] - e[:, 1] * q[:, 0]) / J
        return xi, eta

    def evaluate(self, coef, pts):
        """u at points [m][2] from coefficients [d][nt][nn]: ([d][m], element
        of each point, -1 outside with NaN values)."""
        coef = np.asarray(coef)
        T = self.locate(pts)
        out = np.full((coef.shape[0], len(pts)), np.nan)
        ok = T >= 0
        if ok.any():
            xi, eta = self.reference(T[ok], np.asarray(pts)[ok])
            B = koornwinder(self.N, xi, eta)                # [m][nn]
            out[:, ok] = np.einsum("ma,dma->dm", B, coef[:, T[ok], :])
        return out, T
