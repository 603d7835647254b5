// Curved elements (Section 3.1, blending map of Eq. for:blend), device side.
//
// A curved element is a counter-clockwise triangle (v0, v1, v2) whose side
// v0 -> v1 is a curve c(xi), xi in [0, 1], c(0) = v0, c(1) = v1, given by its
// deviation from the chord,
//     c(xi) - (1 - xi) v0 - xi v1 = xi (1 - xi) D(xi),
//     D(xi) = sum_{k<=K} a_k T_k(2 xi - 1)          (Chebyshev, per coordinate).
// With the opposite vertex v2 the blending map becomes
//     rho(xi, eta) = v0 + xi (v1 - v0) + eta (v2 - v0) + xi (1 - xi - eta) D(xi),
// which is affine when D = 0 and maps the three sides of the reference
// simplex onto the curve and the two straight sides.  Every function here
// uses explicit round-to-nearest operations in a fixed order, so that the
// decisions taken from them (point location, subdivision stop tests, panel
// counts) are those of an IEEE FP64 evaluation of the same formulas.
#pragma once
#include "vp_device.cuh"

#define VP_MAX_CHEB 64   // largest Chebyshev degree K accepted

// Curves of a mesh on the device: cidx[T] = curve of triangle T (-1:
// straight), coef[c][2][K+1] = Chebyshev coefficients of D (x, then y).
struct CurveDev {
    const int32_t* cidx;
    const double* coef;
    const double* dcoef;   // [c][2][K+1]: Chebyshev coefficients of dD/dt (d/dxi = 2 d/dt)
    int K;
};

// D(xi) and dD/dxi for one coordinate (three-term recurrences of T_k and T_k').
__device__ __forceinline__ void cheb_eval_rn(const double* __restrict__ a, int K, double xi, double* v, double* dv) {
    const double t = rn_sub(rn_mul(2.0, xi), 1.0);
    double T0 = 1.0, T1 = t, dT0 = 0.0, dT1 = 1.0;
    double s = a[0], ds = 0.0;
    if (K >= 1) {
        s = rn_add(s, rn_mul(a[1], T1));
        ds = rn_add(ds, rn_mul(a[1], dT1));
    }
    for (int k = 2; k <= K; k++) {
        const double T2 = rn_sub(rn_mul(rn_mul(2.0, t), T1), T0);
        const double dT2 = rn_sub(rn_add(rn_mul(2.0, T1), rn_mul(rn_mul(2.0, t), dT1)), dT0);
        s = rn_add(s, rn_mul(a[k], T2));
        ds = rn_add(ds, rn_mul(a[k], dT2));
        T0 = T1;
        T1 = T2;
        dT0 = dT1;
        dT1 = dT2;
    }
    *v = s;
    *dv = rn_mul(2.0, ds);
}

// y = rho_T(xi, eta), the Jacobian matrix (columns d/dxi, d/deta: Jm[0..3] =
// a11, a21, a12, a22) and its determinant.  v: the triangle's six vertex
// coordinates; ax: the curve's coefficients (x then y), nullptr if straight.
__device__ __forceinline__ void geom_map_rn(const double* v, const double* __restrict__ ax, int K, double xi,
                                            double eta, double* y, double* Jm, double* det) {
    const double Ax = v[0], Ay = v[1];
    const double ex = rn_sub(v[2], Ax), ey = rn_sub(v[3], Ay);
    const double fx = rn_sub(v[4], Ax), fy = rn_sub(v[5], Ay);
    double yx = rn_add(Ax, rn_add(rn_mul(xi, ex), rn_mul(eta, fx)));
    double yy = rn_add(Ay, rn_add(rn_mul(xi, ey), rn_mul(eta, fy)));
    double a11 = ex, a21 = ey, a12 = fx, a22 = fy;
    if (ax) {
        double Dx, dDx, Dy, dDy;
        cheb_eval_rn(ax, K, xi, &Dx, &dDx);
        cheb_eval_rn(ax + (K + 1), K, xi, &Dy, &dDy);
        const double b = rn_mul(xi, rn_sub(rn_sub(1.0, xi), eta));
        const double bx = rn_sub(rn_sub(1.0, rn_mul(2.0, xi)), eta);   // d b / d xi
        yx = rn_add(yx, rn_mul(b, Dx));
        yy = rn_add(yy, rn_mul(b, Dy));
        a11 = rn_add(a11, rn_add(rn_mul(bx, Dx), rn_mul(b, dDx)));
        a21 = rn_add(a21, rn_add(rn_mul(bx, Dy), rn_mul(b, dDy)));
        a12 = rn_sub(a12, rn_mul(xi, Dx));                               // d b / d eta = -xi
        a22 = rn_sub(a22, rn_mul(xi, Dy));
    }
    y[0] = yx;
    y[1] = yy;
    if (Jm) {
        Jm[0] = a11;
        Jm[1] = a21;
        Jm[2] = a12;
        Jm[3] = a22;
    }
    if (det) *det = rn_sub(rn_mul(a11, a22), rn_mul(a12, a21));
}

// Sum_k a_k T_k(t) by Clenshaw's recurrence (fused multiply-adds).
__device__ __forceinline__ double cheb_clenshaw(const double* __restrict__ a, int K, double t) {
    const double t2 = 2.0 * t;
    double b1 = 0.0, b2 = 0.0;
    for (int k = K; k >= 1; k--) {
        const double b0 = fma(t2, b1, a[k] - b2);
        b2 = b1;
        b1 = b0;
    }
    return fma(t, b1, a[0] - b2);
}

// rho_T(xi, eta) and det J_rho for quadrature nodes, where no decision
// depends on the last bit: Clenshaw sums of D and of its derivative series
// (dcoef) with fused multiply-adds, about a third of the operations of
// geom_map_rn.  The results agree with geom_map_rn to rounding.
__device__ __forceinline__ void geom_map_fast(const double* v, const double* __restrict__ ax,
                                              const double* __restrict__ dax, int K, double xi, double eta, double* y,
                                              double* det) {
    const double Ax = v[0], Ay = v[1];
    const double ex = v[2] - Ax, ey = v[3] - Ay;
    const double fx = v[4] - Ax, fy = v[5] - Ay;
    double yx = fma(eta, fx, fma(xi, ex, Ax)), yy = fma(eta, fy, fma(xi, ey, Ay));
    double a11 = ex, a21 = ey, a12 = fx, a22 = fy;
    if (ax) {
        const double t = fma(2.0, xi, -1.0);
        const double Dx = cheb_clenshaw(ax, K, t), Dy = cheb_clenshaw(ax + (K + 1), K, t);
        const double dDx = 2.0 * cheb_clenshaw(dax, K, t), dDy = 2.0 * cheb_clenshaw(dax + (K + 1), K, t);
        const double b = xi * (1.0 - xi - eta);
        const double bx = 1.0 - 2.0 * xi - eta;
        yx = fma(b, Dx, yx);
        yy = fma(b, Dy, yy);
        a11 = fma(bx, Dx, fma(b, dDx, a11));
        a21 = fma(bx, Dy, fma(b, dDy, a21));
        a12 = fma(-xi, Dx, a12);
        a22 = fma(-xi, Dy, a22);
    }
    y[0] = yx;
    y[1] = yy;
    *det = a11 * a22 - a12 * a21;
}

// rho_T^{-1}(x) by Newton's method started from the chord triangle's affine
// inverse.  Stops when a step is below 1e-14 (relative to 1 + |xi| + |eta|),
// or when it no longer shrinks and is below 1e-12; returns the number of
// iterations, or -1 after 60 without convergence.
__device__ __forceinline__ int geom_inverse_rn(const double* v, const double* __restrict__ ax, int K, double x, double y,
                                               double* xi, double* eta) {
    const double Ax = v[0], Ay = v[1];
    const double ex = rn_sub(v[2], Ax), ey = rn_sub(v[3], Ay);
    const double fx = rn_sub(v[4], Ax), fy = rn_sub(v[5], Ay);
    const double J = rn_sub(rn_mul(ex, fy), rn_mul(ey, fx));
    const double qx = rn_sub(x, Ax), qy = rn_sub(y, Ay);
    double a = rn_div(rn_sub(rn_mul(qx, fy), rn_mul(qy, fx)), J);
    double b = rn_div(rn_sub(rn_mul(ex, qy), rn_mul(ey, qx)), J);
    double prev = 1e300;
    for (int it = 0; it < 60; it++) {
        double p[2], M[4], det;
        geom_map_rn(v, ax, K, a, b, p, M, &det);
        const double rx = rn_sub(p[0], x), ry = rn_sub(p[1], y);
        const double da = rn_div(rn_sub(rn_mul(M[3], rx), rn_mul(M[2], ry)), det);
        const double db = rn_div(rn_add(rn_mul(-M[1], rx), rn_mul(M[0], ry)), det);
        const double step = rn_add(fabs(da), fabs(db));
        if (step >= prev && step <= rn_mul(1e-12, rn_add(rn_add(1.0, fabs(a)), fabs(b)))) {
            *xi = a;
            *eta = b;
            return it + 1;
        }
        a = rn_sub(a, da);
        b = rn_sub(b, db);
        if (step <= rn_mul(1e-14, rn_add(rn_add(1.0, fabs(a)), fabs(b)))) {
            *xi = a;
            *eta = b;
            return it + 1;
        }
        prev = step;
    }
    *xi = a;
    *eta = b;
    return -1;
}

// Point location in one element (Appendix A.5): a straight triangle holds x
// when its three orientation tests are >= 0; a curved one when x is on the
// inner side of its two straight sides (v1 -> v2, v2 -> v0) and the Newton
// preimage converged inside the reference simplex: eta >= 0 (inner side of
// the curve), xi >= -1e-9 and xi + eta <= 1 + 1e-9 (the straight sides are
// decided by the orientation tests; the slack absorbs the preimage's
// rounding, and the bounds reject the map's other roots far from T).
__device__ __forceinline__ bool elem_contains_rn(const double* v, const double* __restrict__ ax, int K, double xx,
                                                 double xy) {
    if (!ax) return tri_contains_rn(v, xx, xy);
    if (!(orient_rn(v[2], v[3], v[4], v[5], xx, xy) >= 0.0 && orient_rn(v[4], v[5], v[0], v[1], xx, xy) >= 0.0))
        return false;
    double xi, eta;
    return geom_inverse_rn(v, ax, K, xx, xy, &xi, &eta) > 0 && eta >= 0.0 && xi >= -1e-9 &&
           rn_add(xi, eta) <= 1.0 + 1e-9;
}

__device__ __forceinline__ const double* curve_coef(const CurveDev& c, int64_t T) {
    if (!c.cidx) return nullptr;
    const int k = c.cidx[T];
    return k >= 0 ? c.coef + (int64_t)k * 2 * (c.K + 1) : nullptr;
}
__device__ __forceinline__ const double* curve_dcoef(const CurveDev& c, int64_t T) {
    if (!c.cidx) return nullptr;
    const int k = c.cidx[T];
    return k >= 0 ? c.dcoef + (int64_t)k * 2 * (c.K + 1) : nullptr;
}
