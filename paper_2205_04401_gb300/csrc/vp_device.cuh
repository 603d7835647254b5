// Device helpers of libvp: exact-rounding geometric predicates, the kernel G,
// and the Koornwinder basis of P_4 on the reference simplex.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define VP_NB 15            // dim P_4
#define VP_MAXQ 19          // largest far rule
#define VP_NNEAR 33         // near rule length
#define VP_NGGQ 8
#define VP_NGL 16
#define VP_NRAD 5           // radial rule of the float-float self weights
#define VP_INV_TWO_PI 0.15915494309189533576888376337251
#define VP_INV_FOUR_PI 0.079577471545947667884441881686257

// Quadrature tables in device global memory (read through L1).
struct VpTables {
    double fx[2][VP_MAXQ], fy[2][VP_MAXQ], fw[2][VP_MAXQ];   // [0] = 16-point, [1] = 19-point
    double far_what[2];
    int nq[2], far_degree[2];
    double nx[VP_NNEAR], ny[VP_NNEAR], nw[VP_NNEAR];
    double near_what;
    int near_degree;
    double gr[VP_NGGQ], gw[VP_NGGQ], glogr[VP_NGGQ];
    double lx[VP_NGL], lw[VP_NGL];
    // projection rows: Pk[rule][k][a] = w_k K_a(xi_k) (Koornwinder basis)
    double Pk[2][VP_MAXQ][VP_NB];
    // Q[rule][k][i]: moments of the tensor-Legendre basis leg15 -> nodal weights
    double Q[2][VP_MAXQ][VP_NB];
    // FP64 logarithm table: 1/c_i and log c_i, c_i = 1 + (i + 1/2)/128
    double log_rc[128], log_lc[128];
    double ln2;
    // the same constants as pairs of FP32 values (h, l = fl(x - h)) for the
    // float-float quadratures
    float4 nz2[VP_NNEAR];               // near-rule nodes x (h, l), y (h, l)
    float4 nz3[VP_NNEAR];               // 3 x, 3 y of the near-rule nodes (h, l)
    float2 nw2[VP_NNEAR];               // near-rule weights
    float2 Q2[2][VP_MAXQ][VP_NB];       // Q for moments in the monomial basis (f2_mon15_acc)
    // root-leaf map of rule r: a near pair whose triangle is a leaf has
    // C_k = sum_j B[j nq + k] g_j over the near-rule nodes j (B = QM M^T)
    float2 B2[2][VP_NNEAR * VP_MAXQ];
    float2 lx2[VP_NGL], lw2[VP_NGL];    // Gauss-Legendre nodes and weights on [0, 1]
    float2 gr2[VP_NGGQ], glr2[VP_NGGQ], gwl2[VP_NGGQ];   // GGQ nodes, their logs, weights / 2pi
    float2 rr2[VP_NRAD], ra2[VP_NRAD], rb2[VP_NRAD];     // radial nodes, weights / 2pi of r p and r log(r) p
};

// Tensor-Legendre basis of P_4 used to accumulate moments on the device:
// L_ab(x, y) = P_a(3x - 1) P_b(3y - 1), a + b <= 4, ordered by n = a + b and
// then a from n down to 0 (the order of the Q table).
__host__ __device__ __forceinline__ void leg15(double x, double y, double* L) {
    const double u = fma(3.0, x, -1.0), v = fma(3.0, y, -1.0);
    const double u2 = u * u, v2 = v * v;
    const double pu2 = fma(1.5, u2, -0.5), pv2 = fma(1.5, v2, -0.5);
    const double pu3 = u * fma(2.5, u2, -1.5), pv3 = v * fma(2.5, v2, -1.5);
    const double pu4 = fma(u2, fma(4.375, u2, -3.75), 0.375), pv4 = fma(v2, fma(4.375, v2, -3.75), 0.375);
    L[0] = 1.0;
    L[1] = u;        L[2] = v;
    L[3] = pu2;      L[4] = u * v;      L[5] = pv2;
    L[6] = pu3;      L[7] = pu2 * v;    L[8] = u * pv2;    L[9] = pv3;
    L[10] = pu4;     L[11] = pu3 * v;   L[12] = pu2 * pv2; L[13] = u * pv3;  L[14] = pv4;
}

// log(x) for normal x > 0: x = 2^E m, m in [1,2), c = 1 + (i + 1/2)/128 the
// centre of m's bucket, z = (m - c)/c (m - c exact), |z| < 2^-8, and
// log x = E ln 2 + log c + log(1 + z) with the series of log(1 + z) to z^7.
__device__ __forceinline__ double vp_logd(double x, const double* __restrict__ rc, const double* __restrict__ lc,
                                          double ln2) {
    const long long b = __double_as_longlong(x);
    const int E = (int)(b >> 52) - 1023;
    const int i = (int)((b >> 45) & 127);
    const double m = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    const double c = fma((double)i + 0.5, 0.0078125, 1.0);
    const double z = (m - c) * rc[i];
    double p = fma(z, 1.0 / 7.0, -1.0 / 6.0);
    p = fma(z, p, 0.2);
    p = fma(z, p, -0.25);
    p = fma(z, p, 1.0 / 3.0);
    p = fma(z, p, -0.5);
    return fma((double)E, ln2, lc[i] + fma(z * z, p, z));
}

// ------------------------------------------------------------------------
// Predicates evaluated with explicit round-to-nearest operations (no fused
// multiply-add), in the operation order of the definitions, so that every
// decision is the one an IEEE FP64 evaluation of the formula makes.
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rn_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double rn_sqrt(double a) { return __dsqrt_rn(a); }

// o_PQ(X) = (Q - P) x (X - P) = (qx-px)(xy-py) - (qy-py)(xx-px)
__device__ __forceinline__ double orient_rn(double px, double py, double qx, double qy, double xx, double xy) {
    double a = rn_mul(rn_sub(qx, px), rn_sub(xy, py));
    double b = rn_mul(rn_sub(qy, py), rn_sub(xx, px));
    return rn_sub(a, b);
}

// Membership of X in the open Bernstein ellipse of the edge PQ with
// parameter R^(1/N) (Section 4.1): rho_X^N < R, with s = (|X-P|+|X-Q|)/|Q-P|,
// rho_X = s + sqrt(max(s^2 - 1, 0)), rho_X^N a left-to-right product.
__device__ __forceinline__ bool edge_near_rn(double px, double py, double qx, double qy, double xx, double xy, int N,
                                             double R) {
    double ex = rn_sub(qx, px), ey = rn_sub(qy, py);
    double L = rn_sqrt(rn_add(rn_mul(ex, ex), rn_mul(ey, ey)));
    double ax = rn_sub(xx, px), ay = rn_sub(xy, py), bx = rn_sub(xx, qx), by = rn_sub(xy, qy);
    double s = rn_div(rn_add(rn_sqrt(rn_add(rn_mul(ax, ax), rn_mul(ay, ay))),
                             rn_sqrt(rn_add(rn_mul(bx, bx), rn_mul(by, by)))), L);
    double t = rn_sub(rn_mul(s, s), 1.0);
    if (t < 0.0) t = 0.0;
    double rho = rn_add(s, rn_sqrt(t));
    double p = rho;
    for (int i = 1; i < N; i++) p = rn_mul(p, rho);
    return p < R;
}

__device__ __forceinline__ bool tri_near_rn(const double* v, double xx, double xy, int N, double R) {
    return edge_near_rn(v[0], v[1], v[2], v[3], xx, xy, N, R) || edge_near_rn(v[2], v[3], v[4], v[5], xx, xy, N, R) ||
           edge_near_rn(v[4], v[5], v[0], v[1], xx, xy, N, R);
}

__device__ __forceinline__ bool tri_contains_rn(const double* v, double xx, double xy) {
    return orient_rn(v[0], v[1], v[2], v[3], xx, xy) >= 0.0 && orient_rn(v[2], v[3], v[4], v[5], xx, xy) >= 0.0 &&
           orient_rn(v[4], v[5], v[0], v[1], xx, xy) >= 0.0;
}

// Fast pre-test of edge_near_rn in FP32, with P and Q given relative to X
// (px = P - X, ...).  Returns 1 (near) or 0 (far) when the FP32 value of
// rho^N is more than 10% away from R, and 2 when the exact FP64 test must
// decide.  For every case that does not overflow, the FP32 evaluation of
// rho^N is within 1% of the FP64 one (s, the chord L and rho carry relative
// errors of order 2^-24 s and sqrt(10 * 2^-24); times N <= 50), and an
// overflow to +inf means rho^N far above any admissible R: both give the
// exact decision.
__device__ __forceinline__ int edge_near_f32(float px, float py, float qx, float qy, int N, float R) {
    const float ex = qx - px, ey = qy - py;
    const float L = sqrtf(ex * ex + ey * ey);
    const float s = (sqrtf(px * px + py * py) + sqrtf(qx * qx + qy * qy)) / L;
    const float t = fmaxf(s * s - 1.0f, 0.0f);
    const float rho = s + sqrtf(t);
    float p = rho;
    for (int i = 1; i < N; i++) p *= rho;
    if (p < 0.9f * R) return 1;
    if (p > 1.1f * R) return 0;
    return 2;
}

// Ellipse membership of X for the triangle with vertices v (FP64): the FP32
// pre-test per edge, the exact FP64 test only for undecided edges.
__device__ __forceinline__ bool tri_near_fast(const double* v, double xx, double xy, int N, double R) {
    const float Rf = (float)R;
    float d[6];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        d[2 * i] = (float)(v[2 * i] - xx);
        d[2 * i + 1] = (float)(v[2 * i + 1] - xy);
    }
#pragma unroll
    for (int e = 0; e < 3; e++) {
        const int a = e, b = (e + 1) % 3;
        const int r = edge_near_f32(d[2 * a], d[2 * a + 1], d[2 * b], d[2 * b + 1], N, Rf);
        if (r == 1) return true;
        if (r == 2 && edge_near_rn(v[2 * a], v[2 * a + 1], v[2 * b], v[2 * b + 1], xx, xy, N, R)) return true;
    }
    return false;
}

// R = (w J) / (eps C_N)   (Eq. rho0 raised to the power N)
__device__ __forceinline__ double ellipse_R_rn(double what, double J, double eps, double cn) {
    return rn_div(rn_mul(what, J), rn_mul(eps, cn));
}

// G(x, y) = log|x - y| / 2pi, from the squared distance.
__device__ __forceinline__ double kernel_G(double dx, double dy) {
    return log(dx * dx + dy * dy) * (0.5 * VP_INV_TWO_PI);
}

// ------------------------------------------------------------------------
// Koornwinder polynomials (Section 2.1), orthonormal on the reference
// simplex: K_mn(x,y) = c_mn (1-x)^m P_{n-m}^{(2m+1,0)}(2x-1) P_m(2y/(1-x) - 1),
// c_mn = sqrt(2 (n+1) (2m+1)), index a = n(n+1)/2 + m, 0 <= m <= n <= 4.
// (1-x)^m P_m(2y/(1-x) - 1) is evaluated by the homogeneous Legendre
// recurrence Q_{m+1} = ((2m+1) Q_1 Q_m - m (1-x)^2 Q_{m-1}) / (m+1),
// Q_0 = 1, Q_1 = 2y + x - 1, which needs no division by 1 - x.
__host__ __device__ __forceinline__ void koornwinder4(double x, double y, double* K) {
    const double omx = 1.0 - x;
    const double omx2 = omx * omx;
    const double z = 2.0 * x - 1.0;
    double Q[5];
    Q[0] = 1.0;
    Q[1] = 2.0 * y + x - 1.0;
    Q[2] = (3.0 * Q[1] * Q[1] - omx2) * 0.5;
    Q[3] = (5.0 * Q[1] * Q[2] - 2.0 * omx2 * Q[1]) * (1.0 / 3.0);
    Q[4] = (7.0 * Q[1] * Q[3] - 3.0 * omx2 * Q[2]) * 0.25;
#pragma unroll
    for (int m = 0; m <= 4; m++) {
        const double a = 2.0 * m + 1.0;
        // Jacobi P_k^{(a,0)}(z), k = 0..4-m
        double pkm1 = 1.0, pk = 0.5 * ((a + 2.0) * z + a);
#pragma unroll
        for (int n = m; n <= 4; n++) {
            const int k = n - m;
            double Pj;
            if (k == 0) Pj = 1.0;
            else if (k == 1) Pj = pk;
            else {
                // advance from (P_{k-2}, P_{k-1}) to P_k
                const double kk = k - 1.0;  // recurrence index
                const double c1 = 2.0 * kk + a;
                const double num = (c1 + 1.0) * ((c1 + 2.0) * c1 * z + a * a) * pk - 2.0 * kk * (kk + a) * (c1 + 2.0) * pkm1;
                const double den = 2.0 * (kk + 1.0) * (kk + a + 1.0) * c1;
                const double pn = num / den;
                pkm1 = pk;
                pk = pn;
                Pj = pn;
            }
            const double c = sqrt(2.0 * (n + 1.0) * (2.0 * m + 1.0));
            K[n * (n + 1) / 2 + m] = c * Q[m] * Pj;
        }
    }
}

// ------------------------------------------------------------------------
// Bounded-wait helpers: status flags live in device memory and are read by
// the host after synchronisation.
#define VP_DEV_ERR_STACK 1
#define VP_DEV_ERR_BADIDX 2
#define VP_DEV_ERR_DEGEN 4
#define VP_DEV_ERR_NONFINITE 8
#define VP_DEV_ERR_CELL 16
#define VP_DEV_ERR_TIMEOUT 32   // a bounded wait of a pipelined kernel gave up
#define VP_DEV_ERR_CURVED_CW 64 // a curved element given clockwise
#define VP_DEV_ERR_ALLOC 128    // a device allocation inside a pipelined step failed
